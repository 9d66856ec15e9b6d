// Finite-difference-sieve terms of the loop hafnian on sm_103a (arXiv:2108.01622, App. B.4,
// Eq. fdsieve, with the repeated pairs of App. B.2-B.4).
//
// One term: for the sign/repeat vector delta' (delta'_i = eta_i - 2 k_i) the working matrix is the
// bordered matrix K = [[0, v X], [v^T, C X]] with X = X_delta' (App. B.4). With
//   d_M(t) = det(I - t C X),   d_K(t) = det(I - t K),
// the coefficients g_k of Eq. ET_poly are
//   sum_k Tr((C X)^k) t^k / k = -log d_M(t)            (power sums by Newton's identities)
//   sum_k v X (C X)^(k-1) v^T t^(k+1) = 1 - d_K(t) / d_M(t)
// and f = [t^h] exp(sum_k g_k t^k). Both determinants come from one Hessenberg form of K: the
// reduction fixes index 0, so its trailing block is a Hessenberg form of C X, and one reverse
// La Budde sweep gives the characteristic polynomials of all trailing blocks, d_K and d_M among
// them. The Hessenberg reduction uses stabilised elementary similarity transforms (Gaussian
// elimination with partial pivoting): half the multiply-adds of Householder reflectors.
//
// A team of G lanes evaluates one term at a time with its working matrix in shared memory; a CTA
// holds 128 / G teams (G < 32) or one team of G lanes (G >= 32). Every FP64 instruction issues at
// one warp instruction per ~64 cycles per SM sub-partition on this part, and idle lanes cost the
// same as busy ones, so each phase spreads its independent multiply-adds over all G lanes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lhaf_internal.h"

namespace lhafgpu {

template <typename R> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };

__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }

template <typename V> __device__ __forceinline__ V cmake(decltype(V::x) a, decltype(V::x) b) {
  V r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmake<V>(rfma(a.x, b.x, -(a.y * b.y)), rfma(a.x, b.y, a.y * b.x));
}
// acc += a * b
template <typename V> __device__ __forceinline__ void cmac(V& acc, V a, V b) {
  acc.x = rfma(a.x, b.x, acc.x);
  acc.x = rfma(-a.y, b.y, acc.x);
  acc.y = rfma(a.x, b.y, acc.y);
  acc.y = rfma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename V> __device__ __forceinline__ void cmsub(V& acc, V a, V b) {
  acc.x = rfma(-a.x, b.x, acc.x);
  acc.x = rfma(a.y, b.y, acc.x);
  acc.y = rfma(-a.x, b.y, acc.y);
  acc.y = rfma(-a.y, b.x, acc.y);
}

// Sign flip and magnitude keys with integer instructions only (no FP64 issue slot).
__device__ __forceinline__ double flip(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ float flip(float x) { return __int_as_float(__float_as_int(x) ^ (int)0x80000000u); }
__device__ __forceinline__ unsigned long long mag_key(double2 z) {
  unsigned long long a = (unsigned long long)__double_as_longlong(z.x) & 0x7fffffffffffffffull;
  unsigned long long b = (unsigned long long)__double_as_longlong(z.y) & 0x7fffffffffffffffull;
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long mag_key(float2 z) {
  unsigned a = (unsigned)__float_as_int(z.x) & 0x7fffffffu;
  unsigned b = (unsigned)__float_as_int(z.y) & 0x7fffffffu;
  return a > b ? a : b;
}

// 1 / z with the exponent of max(|re|, |im|) scaled out first (exact power-of-two scaling), so
// neither |z|^2 nor its reciprocal leaves the representable range. Returns 0 for z == 0.
__device__ __forceinline__ double2 crecip(double2 z) {
  unsigned long long k = mag_key(z);
  if (k == 0ull) return make_double2(0.0, 0.0);
  int e = (int)(k >> 52);          // biased exponent of the larger part (0 for subnormals)
  if (e < 1) e = 1;
  if (e > 2045) e = 2045;
  double sc = __longlong_as_double((long long)(2046 - e) << 52);  // 2^(1023 - (e - 1023))
  double xs = z.x * sc, ys = z.y * sc;
  double d = fma(xs, xs, ys * ys);
  double rd = __drcp_rn(d);
  return make_double2(xs * rd * sc, flip(ys) * rd * sc);
}
__device__ __forceinline__ float2 crecip(float2 z) {
  unsigned k = (unsigned)mag_key(z);
  if (k == 0u) return make_float2(0.f, 0.f);
  int e = (int)(k >> 23);
  if (e < 1) e = 1;
  if (e > 253) e = 253;
  float sc = __int_as_float((253 - e + 1) << 23);  // 2^(127 - (e - 127)) clamped
  float xs = z.x * sc, ys = z.y * sc;
  float d = fmaf(xs, xs, ys * ys);
  float rd = __frcp_rn(d);
  return make_float2(xs * rd * sc, flip(ys) * rd * sc);
}

// Double-double accumulation (Knuth's TwoSum).
__device__ __forceinline__ void dd_add(double& hi, double& lo, double x) {
  double s = hi + x;
  double bb = s - hi;
  double err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err;
}
__device__ __forceinline__ void dd_add_dd(double& hi, double& lo, double bh, double bl) {
  double s = hi + bh;
  double bb = s - hi;
  double err = (hi - (s - bb)) + (bh - bb);
  err += lo + bl;
  double t = s + err;  // FastTwoSum renormalisation
  lo = err - (t - s);
  hi = t;
}

template <int G> __device__ __forceinline__ void team_sync() {
  if constexpr (G <= 32) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

__host__ __device__ constexpr int cta_of(int G) { return G < 32 ? 128 : G; }

// C(n, k): exact in 64-bit integers for n <= 62, else rounded (the weight only feeds a product).
__device__ __forceinline__ double binom_d(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  if (k > n - k) k = n - k;
  if (k == 0) return 1.0;
  if (k == 1) return (double)n;
  if (n <= 62) {
    unsigned long long c = 1ull;
    for (int i = 1; i <= k; i++) c = c * (unsigned long long)(n - k + i) / (unsigned long long)i;
    return (double)c;
  }
  double c = 1.0;
  for (int i = 1; i <= k; i++) c = c * (double)(n - k + i) / (double)i;
  return c;
}

struct TeamScratch {  // small per-team area
  unsigned long long key[4];
  int row[4];
  double weight;
  int delta[kMaxPairs];
};

template <typename R, int G>
__global__ void __launch_bounds__(cta_of(G))
terms_kernel(const typename Cx<R>::t* __restrict__ chat, const TermParams p, double* __restrict__ partials) {
  using V = typename Cx<R>::t;
  constexpr int CTA = cta_of(G);
  constexpr int TEAMS = CTA / G;
  constexpr int SG = G < 32 ? G : 32;  // lanes that run the series recurrences
  extern __shared__ __align__(16) unsigned char smem[];

  const int nd = p.nd, ld = p.ld, bord = p.bord, h = p.h, H = p.H, Hl = p.Hl, P = p.P;
  const int tid = threadIdx.x;
  const int team = tid / G;
  const int lt = tid - team * G;

  uint16_t* items = reinterpret_cast<uint16_t*>(smem);
  R* invk = reinterpret_cast<R*>(smem + ((p.n_items * 2 + 15) & ~15));
  unsigned char* tb = smem + p.items_bytes + (size_t)team * p.team_bytes;
  V* W = reinterpret_cast<V*>(tb);
  V* Sa = W + nd * ld;  // series arrays, H + 2 entries each
  V* Sc = Sa + (H + 2);
  V* SR = Sc + (H + 2);
  V* Sp = SR + (H + 2);
  V* Sz = Sp + (H + 2);
  V* Se = Sz + (H + 2);
  TeamScratch* ts = reinterpret_cast<TeamScratch*>(Se + (H + 2));

  // Push items (d, e) of La Budde's recurrence, sorted by e then d: 2 <= d, d + e <= Hl.
  for (int w = tid; w < p.n_items; w += CTA) {
    int e = 0, base = 0;
    while (base + (Hl - 1 - e) <= w) {
      base += Hl - 1 - e;
      e++;
    }
    items[w] = (uint16_t)(((2 + (w - base)) << 8) | e);
  }
  for (int k = tid; k <= H + 1; k += CTA) invk[k] = k ? (R)1 / (R)k : (R)0;
  __syncthreads();

  const V zero = cmake<V>((R)0, (R)0);
  const V one = cmake<V>((R)1, (R)0);
  const unsigned long long team_global = (unsigned long long)blockIdx.x * TEAMS + team;
  double acc_re = 0.0, acc_re_lo = 0.0, acc_im = 0.0, acc_im_lo = 0.0;

  for (unsigned long long rnd = 0; rnd < p.rounds; rnd++) {
    unsigned long long t = p.t_begin + team_global + rnd * p.total_teams;
    const bool valid = t < p.t_end;
    if (!valid) t = p.t_begin;

    // ---- digits k_i of the term, delta'_i = eta_i - 2 k_i, and the weight (App. B.4) ----
    if (lt == 0) {
      unsigned long long x = t;
      double w = valid ? 1.0 : 0.0;
      int parity = 0;
      for (int q = 0; q < P; q++) {
        const unsigned long long rad = (unsigned long long)p.radix[q];
        const int k = (int)(x % rad);
        x /= rad;
        const int eta = p.eta[q];
        w *= binom_d(eta, k);
        parity ^= (k & 1);
        ts->delta[q] = eta - 2 * k;
        if (q == p.hp && !(p.hp_even && 2 * k == eta)) w *= 2.0;  // sign-symmetry halving
      }
      ts->weight = parity ? -w : w;
    }
    team_sync<G>();

    // ---- working matrix K[i][j] = Chat[i][partner(j)] * delta_hat(j) ----
    for (int w = lt; w < nd * nd; w += G) {
      const int i = w / nd, j = w - i * nd;
      int jj = j, dl = 1;
      if (j >= bord) {
        const int s = j - bord;
        jj = bord + (s ^ 1);
        dl = ts->delta[s >> 1];
      }
      V c = chat[i * nd + jj];
      if (dl == -1) {
        c.x = flip(c.x);
        c.y = flip(c.y);
      } else if (dl != 1) {
        const R f = (R)dl;
        c.x *= f;
        c.y *= f;
      }
      W[i * ld + j] = c;
    }
    team_sync<G>();

    // ---- Hessenberg form by elimination with partial pivoting (fixes index 0) ----
    for (int k = 0; k < nd - 2; k++) {
      unsigned long long key = 0ull;
      int row = k + 1;
      for (int i = k + 1 + lt; i < nd; i += G) {
        const unsigned long long kk = mag_key(W[i * ld + k]);
        if (kk > key) {
          key = kk;
          row = i;
        }
      }
      if constexpr (G <= 32) {
#pragma unroll
        for (int off = G / 2; off >= 1; off >>= 1) {
          const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, off);
          const int orow = __shfl_xor_sync(0xffffffffu, row, off);
          if (ok > key || (ok == key && orow < row)) {
            key = ok;
            row = orow;
          }
        }
      } else {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, off);
          const int orow = __shfl_xor_sync(0xffffffffu, row, off);
          if (ok > key || (ok == key && orow < row)) {
            key = ok;
            row = orow;
          }
        }
        if ((lt & 31) == 0) {
          ts->key[lt >> 5] = key;
          ts->row[lt >> 5] = row;
        }
        __syncthreads();
        key = ts->key[0];
        row = ts->row[0];
        for (int q = 1; q < G / 32; q++) {
          if (ts->key[q] > key || (ts->key[q] == key && ts->row[q] < row)) {
            key = ts->key[q];
            row = ts->row[q];
          }
        }
      }
      const int r = row;
      // swap rows r and k+1 (columns k..nd-1), then columns r and k+1: a similarity transform
      for (int j = k + lt; j < nd; j += G) {
        const V a = W[r * ld + j], b = W[(k + 1) * ld + j];
        W[r * ld + j] = b;
        W[(k + 1) * ld + j] = a;
      }
      team_sync<G>();
      for (int i = lt; i < nd; i += G) {
        const V a = W[i * ld + r], b = W[i * ld + k + 1];
        W[i * ld + r] = b;
        W[i * ld + k + 1] = a;
      }
      team_sync<G>();
      // multipliers l_i = K[i][k] / K[k+1][k], kept in column k below the subdiagonal
      const V ip = crecip(W[(k + 1) * ld + k]);
      for (int i = k + 2 + lt; i < nd; i += G) W[i * ld + k] = cmul(W[i * ld + k], ip);
      team_sync<G>();
      // rows: K[i][j] -= l_i K[k+1][j] for i >= k+2, j >= k+1
      const int cols = nd - k - 1;
      const int nrc = (cols - 1) * cols;
      for (int w = lt; w < nrc; w += G) {
        const int ii = w / cols;
        const int i = k + 2 + ii, j = k + 1 + (w - ii * cols);
        V a = W[i * ld + j];
        cmsub(a, W[i * ld + k], W[(k + 1) * ld + j]);
        W[i * ld + j] = a;
      }
      team_sync<G>();
      // columns: K[i][k+1] += sum_{j >= k+2} K[i][j] l_j
      for (int i = lt; i < nd; i += G) {
        V a = W[i * ld + k + 1];
        for (int j = k + 2; j < nd; j++) cmac(a, W[i * ld + j], W[j * ld + k]);
        W[i * ld + k + 1] = a;
      }
      team_sync<G>();
    }

    // ---- La Budde's recurrence, reverse (trailing blocks), truncated at degree Hl ----
    // q_j(t) = det(I - t K[j.., j..]) = (1 - t K_jj) q_{j+1} - sum_{l > j} c_{j,l} t^(l-j+1) q_{l+1}
    // with c_{j,l} = K_jl prod_{r=j+1..l} K_{r,r-1}, stored over K_jl (l - j <= Hl - 1).
    for (int j = lt; j < nd - 1; j += G) {
      V pi = one;
      const int dmax = min(Hl - 1, nd - 1 - j);
      for (int dp = 1; dp <= dmax; dp++) {
        const int l = j + dp;
        pi = cmul(pi, W[l * ld + l - 1]);
        W[j * ld + l] = cmul(W[j * ld + l], pi);
      }
    }
    team_sync<G>();
    // q_l[m] lives at K[l+m-1][l] (m >= 1); its push accumulator shares the slots (m >= 2).
    for (int l = lt; l < nd; l += G) {
      const int mm = min(Hl, nd - l);
      for (int m = 2; m <= mm; m++) W[(l + m - 1) * ld + l] = zero;
    }
    V hll = W[(nd - 1) * ld + nd - 1];
    team_sync<G>();
    for (int l = nd - 1; l >= 0; l--) {
      const int deg = nd - l - 1;  // degree of q_{l+1}
      const int E = min(deg, Hl - 2);
      const int np = (E >= 0) ? (E + 1) * (Hl - 1) - E * (E + 1) / 2 : 0;
      const int nq = min(Hl, nd - l);
      for (int w = lt; w < np + nq; w += G) {
        if (w < np) {
          // push q_{l+1} into the accumulator of q_j, j = l - d + 1
          const int it = items[w];
          const int d = it >> 8, e = it & 255;
          const int j = l - d + 1;
          if (j >= 0) {
            const V Pe = (e == 0) ? one : W[(l + e) * ld + l + 1];
            V a = W[(l + e) * ld + j];
            cmsub(a, W[j * ld + l], Pe);
            W[(l + e) * ld + j] = a;
          }
        } else {
          // q_l[m] = q_{l+1}[m] - K_ll q_{l+1}[m-1] + acc_l[m]
          const int m = w - np + 1;
          const V Pm = (m <= deg) ? W[(l + m) * ld + l + 1] : zero;
          const V Pm1 = (m == 1) ? one : ((m - 1 <= deg) ? W[(l + m - 1) * ld + l + 1] : zero);
          V v = Pm;
          if (m >= 2) {
            const V a = W[(l + m - 1) * ld + l];
            v.x += a.x;
            v.y += a.y;
          }
          cmsub(v, hll, Pm1);
          W[(l + m - 1) * ld + l] = v;
        }
      }
      V hnext = zero;
      if (l > 0) hnext = W[(l - 1) * ld + l - 1];
      team_sync<G>();
      hll = hnext;
    }

    // ---- series: a = d_M, c = d_M - d_K, then Newton, division and exp (Eq. ET_poly) ----
    for (int m = lt; m <= H + 1; m += G) {
      V am = zero, bm = zero;
      if (m == 0) {
        am = one;
        bm = one;
      } else if (m <= Hl) {
        if (bord) {
          if (m <= nd - 1) am = W[m * ld + 1];
          if (m <= nd) bm = W[(m - 1) * ld];
        } else {
          if (m <= nd) am = W[(m - 1) * ld];
          bm = am;
        }
      }
      Sa[m] = am;
      Sc[m] = cmake<V>(am.x - bm.x, am.y - bm.y);
    }
    team_sync<G>();

    if (G <= 32 || lt < 32) {
      const int sl = lt;  // < SG
      if (sl == 0) {
        SR[0] = zero;
        SR[1] = Sc[1];
        Se[0] = one;
        Sp[0] = zero;
        Sz[0] = zero;
      }
      __syncwarp();
      for (int k = 1; k <= h; k++) {
        V sR = zero, sp = zero;
        for (int i = 1 + sl; i <= k; i += SG) {
          cmac(sR, Sa[i], SR[k + 1 - i]);
          if (i < k) cmac(sp, Sa[i], Sp[k - i]);
        }
#pragma unroll
        for (int off = SG / 2; off >= 1; off >>= 1) {
          sR.x += __shfl_xor_sync(0xffffffffu, sR.x, off);
          sR.y += __shfl_xor_sync(0xffffffffu, sR.y, off);
          sp.x += __shfl_xor_sync(0xffffffffu, sp.x, off);
          sp.y += __shfl_xor_sync(0xffffffffu, sp.y, off);
        }
        const V ck = Sc[k + 1], ak = Sa[k];
        const R kk = (R)k;
        const V Rk = cmake<V>(ck.x - sR.x, ck.y - sR.y);            // R_{k+1}
        const V pk = cmake<V>(-rfma(kk, ak.x, sp.x), -rfma(kk, ak.y, sp.y));  // power sum p_k
        const V zk = cmake<V>((R)0.5 * rfma(kk, Rk.x, pk.x), (R)0.5 * rfma(kk, Rk.y, pk.y));
        __syncwarp();
        if (sl == 0) {
          SR[k + 1] = Rk;
          Sp[k] = pk;
          Sz[k] = zk;
        }
        __syncwarp();
        V se = zero;
        for (int j = 1 + sl; j <= k; j += SG) cmac(se, Sz[j], Se[k - j]);
#pragma unroll
        for (int off = SG / 2; off >= 1; off >>= 1) {
          se.x += __shfl_xor_sync(0xffffffffu, se.x, off);
          se.y += __shfl_xor_sync(0xffffffffu, se.y, off);
        }
        if (sl == 0) Se[k] = cmake<V>(se.x * invk[k], se.y * invk[k]);
        __syncwarp();
      }
      if (lt == 0) {
        const V f = Se[h];
        const double w = ts->weight;
        const double fr = (double)f.x * w, fi = (double)f.y * w;
        if (p.plain) {
          acc_re += fr;
          acc_im += fi;
        } else {
          dd_add(acc_re, acc_re_lo, fr);
          dd_add(acc_im, acc_im_lo, fi);
        }
      }
    }
    team_sync<G>();
  }

  if (lt == 0) {
    double* o = partials + 4ull * team_global;
    o[0] = acc_re;
    o[1] = acc_re_lo;
    o[2] = acc_im;
    o[3] = acc_im_lo;
  }
}

// ---------------------------------------------------------------------------------------------
// Double-double reduction of per-team partials, then the exact 2^-h scaling of Eq. fdsieve.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
reduce_kernel(const double* __restrict__ partials, long long count, int h, double* out_dd, double2* out_val) {
  __shared__ double s[4][256];
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
  for (long long i = threadIdx.x; i < count; i += 256) {
    dd_add_dd(rh, rl, partials[4 * i + 0], partials[4 * i + 1]);
    dd_add_dd(ih, il, partials[4 * i + 2], partials[4 * i + 3]);
  }
  s[0][threadIdx.x] = rh;
  s[1][threadIdx.x] = rl;
  s[2][threadIdx.x] = ih;
  s[3][threadIdx.x] = il;
  __syncthreads();
  for (int off = 128; off >= 1; off >>= 1) {
    if (threadIdx.x < off) {
      double a = s[0][threadIdx.x], b = s[1][threadIdx.x];
      dd_add_dd(a, b, s[0][threadIdx.x + off], s[1][threadIdx.x + off]);
      s[0][threadIdx.x] = a;
      s[1][threadIdx.x] = b;
      double c = s[2][threadIdx.x], d = s[3][threadIdx.x];
      dd_add_dd(c, d, s[2][threadIdx.x + off], s[3][threadIdx.x + off]);
      s[2][threadIdx.x] = c;
      s[3][threadIdx.x] = d;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (out_dd) {
      out_dd[0] = s[0][0];
      out_dd[1] = s[1][0];
      out_dd[2] = s[2][0];
      out_dd[3] = s[3][0];
    }
    if (out_val) {
      // 2^-h as an exact power of two, applied in up to two steps to stay in range
      int e1 = h > 1000 ? 1000 : h;
      int e2 = h - e1;
      const double s1 = __longlong_as_double((long long)(1023 - e1) << 52);
      const double s2 = __longlong_as_double((long long)(1023 - e2) << 52);
      out_val[0] = make_double2((s[0][0] + s[1][0]) * s1 * s2, (s[2][0] + s[3][0]) * s1 * s2);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Slot-matrix gather from device inputs (for device-pointer calls).
// ---------------------------------------------------------------------------------------------
struct SlotModes {
  int mode[kMaxDim];
};

__global__ void gather_kernel(const double2* __restrict__ B, const double2* __restrict__ gamma, int M,
                              SlotModes sm, int n, int bord, double2* chat, float2* chat32) {
  const int nd = n + bord;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nd * nd; w += gridDim.x * blockDim.x) {
    const int i = w / nd, j = w - i * nd;
    double2 c = make_double2(0.0, 0.0);
    if (bord && i == 0 && j == 0) {
      c = make_double2(0.0, 0.0);
    } else if (bord && (i == 0 || j == 0)) {
      const int s = (i == 0 ? j : i) - 1;
      const int m = sm.mode[s];
      if (m < 0) {
        c = make_double2(1.0, 0.0);
      } else {
        c = gamma ? gamma[m] : B[(size_t)m * M + m];
      }
    } else {
      const int a = sm.mode[i - bord], b = sm.mode[j - bord];
      if (a >= 0 && b >= 0) {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        c = B[(size_t)lo * M + hi];
      }
    }
    if (chat) chat[w] = c;
    if (chat32) chat32[w] = make_float2((float)c.x, (float)c.y);
  }
}

// ---------------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------------
int cta_threads(int team) { return cta_of(team); }
int teams_per_cta(int team) { return cta_of(team) / team; }

size_t team_shared_bytes(bool fp32, int nd, int H, int P) {
  (void)P;
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  const int ld = nd | 1;
  size_t b = (size_t)nd * ld * cs + 6 * (size_t)(H + 2) * cs + sizeof(TeamScratch);
  return (b + 15) & ~(size_t)15;
}

static size_t items_bytes_of(bool fp32, int Hl, int H) {
  const int n_items = Hl * (Hl - 1) / 2;
  size_t b = ((size_t)n_items * 2 + 15) & ~(size_t)15;
  b += (size_t)(H + 2) * (fp32 ? sizeof(float) : sizeof(double));
  return (b + 15) & ~(size_t)15;
}

size_t cta_shared_bytes(bool fp32, int team, int nd, int H, int Hl, int P) {
  return items_bytes_of(fp32, Hl, H) + (size_t)teams_per_cta(team) * team_shared_bytes(fp32, nd, H, P);
}

template <typename R, int G> static const void* kernel_ptr() { return (const void*)terms_kernel<R, G>; }

static const void* pick_kernel(bool fp32, int team) {
  if (fp32) {
    switch (team) {
      case 8: return kernel_ptr<float, 8>();
      case 16: return kernel_ptr<float, 16>();
      case 32: return kernel_ptr<float, 32>();
      case 64: return kernel_ptr<float, 64>();
      case 128: return kernel_ptr<float, 128>();
    }
  } else {
    switch (team) {
      case 8: return kernel_ptr<double, 8>();
      case 16: return kernel_ptr<double, 16>();
      case 32: return kernel_ptr<double, 32>();
      case 64: return kernel_ptr<double, 64>();
      case 128: return kernel_ptr<double, 128>();
    }
  }
  return nullptr;
}

int max_ctas_per_sm(bool fp32, int team, size_t smem_bytes) {
  const void* k = pick_kernel(fp32, team);
  if (!k) return 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, cta_of(team), smem_bytes) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_terms(bool fp32, int team, const void* chat, const TermParams& p, int grid, double* partials,
                         cudaStream_t stream) {
  const void* k = pick_kernel(fp32, team);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = (size_t)p.items_bytes + (size_t)teams_per_cta(team) * p.team_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&chat, (void*)&p, (void*)&partials};
  return cudaLaunchKernel(k, dim3(grid), dim3(cta_of(team)), args, smem, stream);
}

cudaError_t launch_reduce(const double* partials, long long count, int h, double* out_dd, double2* out_val,
                          cudaStream_t stream) {
  reduce_kernel<<<1, 256, 0, stream>>>(partials, count, h, out_dd, out_val);
  return cudaGetLastError();
}

cudaError_t launch_gather(const double2* B, const double2* gamma, int M, const int* slot_mode_host, int P, int bord,
                          double2* chat, float2* chat32, cudaStream_t stream) {
  SlotModes sm;
  for (int i = 0; i < kMaxDim; i++) sm.mode[i] = (i < 2 * P) ? slot_mode_host[i] : -1;
  const int n = 2 * P;
  const int nd = n + bord;
  const int threads = 256;
  int blocks = (nd * nd + threads - 1) / threads;
  if (blocks < 1) blocks = 1;
  gather_kernel<<<blocks, threads, 0, stream>>>(B, gamma, M, sm, n, bord, chat, chat32);
  return cudaGetLastError();
}

}  // namespace lhafgpu
