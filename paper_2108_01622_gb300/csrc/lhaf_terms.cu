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
// is one warp holding 32 / G teams (G <= 32) or one team of G lanes (G > 32). Every FP64
// instruction issues at one warp instruction per ~64 cycles per SM sub-partition on this part,
// and idle lanes cost the same as busy ones, so each phase spreads its independent multiply-adds
// over all G lanes. The last step (three short sequential recurrences per term) either runs in
// the team (inline) or is staged to global memory and run one term per thread by series_kernel,
// where it needs no cross-lane reductions.
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

// x * 2^k by exponent arithmetic (integer instructions, no FP64 issue slot): exact for normal x
// and normal results; zero and subnormal x, and results below the normal range, give a signed
// zero; results above it give a signed infinity.
__device__ __forceinline__ double scale2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  const int ne = ex + k;
  const long long sign = b & (long long)0x8000000000000000ull;
  if (ex == 0 || ne <= 0) return __longlong_as_double(sign);
  if (ne >= 2047) return __longlong_as_double(sign | (long long)0x7ff0000000000000ull);
  return __longlong_as_double((b & ~(long long)0x7ff0000000000000ull) | ((long long)ne << 52));
}

// 1 / z = conj(z) / |z|^2. The exponent of max(|re|, |im|) is scaled out first (by exponent
// arithmetic), so d = |z s|^2 lies in [1, 8). 1/d: an FP32 reciprocal of d's leading bits (moved
// between the formats with integer instructions) refined by two Newton-Raphson steps
// r <- r (2 - d r) (relative error ~2^-23 -> ~2^-46 -> below 2^-53); the result is scaled back the
// same way. Returns 0 for z == 0.
__device__ __forceinline__ double2 crecip(double2 z) {
  const unsigned long long k = mag_key(z);
  if (k == 0ull) return make_double2(0.0, 0.0);
  int e = (int)(k >> 52);  // biased exponent of the larger part (0 for subnormals)
  if (e < 1) e = 1;
  if (e > 2045) e = 2045;
  const int sh = 1023 - e;  // s = 2^sh brings the larger part into [1, 2)
  const double xs = scale2(z.x, sh), ys = scale2(z.y, sh);
  const double d = fma(xs, xs, ys * ys);
  // float with d's exponent and its 23 leading mantissa bits (d in [1, 8): exponent 0..2)
  const long long db = __double_as_longlong(d);
  if (db == 0) return make_double2(0.0, 0.0);  // both parts subnormal: treated as a zero pivot
  const int de = (int)((db >> 52) & 0x7ff) - 1023;
  const unsigned fm = (unsigned)((db >> 29) & 0x7fffff);
  const float rf = __frcp_rn(__int_as_float(((de + 127) << 23) | (int)fm));
  const int fb = __float_as_int(rf);
  double r = __longlong_as_double(((long long)(((fb >> 23) & 0xff) - 127 + 1023) << 52) |
                                  ((long long)(fb & 0x7fffff) << 29));
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  // 1/z = (xs, -ys) * r * s
  return make_double2(scale2(xs * r, sh), scale2(flip(ys) * r, sh));
}
__device__ __forceinline__ float2 crecip(float2 z) {
  const unsigned k = (unsigned)mag_key(z);
  if (k == 0u) return make_float2(0.f, 0.f);
  int e = (int)(k >> 23);
  if (e < 1) e = 1;
  if (e > 253) e = 253;
  const float sc = __int_as_float((254 - e) << 23);  // 2^(127 - (e - 127))
  const float xs = z.x * sc, ys = z.y * sc;
  const float d = fmaf(xs, xs, ys * ys);
  const float rs = __frcp_rn(d) * sc;
  return make_float2(xs * rs, flip(ys) * rs);
}

// Double-double accumulation (Knuth's TwoSum).
__device__ __forceinline__ void dd_add(double& hi, double& lo, double x) {
  const double s = hi + x;
  const double bb = s - hi;
  const double err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err;
}
__device__ __forceinline__ void dd_add_dd(double& hi, double& lo, double bh, double bl) {
  const double s = hi + bh;
  const double bb = s - hi;
  double err = (hi - (s - bb)) + (bh - bb);
  err += lo + bl;
  const double t = s + err;  // FastTwoSum renormalisation
  lo = err - (t - s);
  hi = t;
}

// acc += sum_{j0 <= j < j1} row[j] * col[j * ld], with running pointers. Long sums keep two
// partial sums (even and odd j) so that two independent multiply-add chains per component are in
// flight; short sums keep one (merging costs two adds).
template <typename V>
__device__ __forceinline__ void dot_accumulate(V& acc, const V* row, const V* col, int ld, int j0, int j1) {
  const V* pr = row + j0;
  const V* pc = col + j0 * ld;
  int n = j1 - j0;
  if (n >= 8) {
    V b = cmake<V>(0, 0);
    for (; n >= 2; n -= 2) {
      cmac(acc, pr[0], pc[0]);
      cmac(b, pr[1], pc[ld]);
      pr += 2;
      pc += 2 * ld;
    }
    if (n) cmac(acc, pr[0], pc[0]);
    acc.x += b.x;
    acc.y += b.y;
  } else {
    for (; n > 0; n--) {
      cmac(acc, *pr, *pc);
      pr++;
      pc += ld;
    }
  }
}

template <int G> __device__ __forceinline__ void team_sync() {
  if constexpr (G <= 32) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

__host__ __device__ constexpr int cta_of(int G) { return G < 32 ? 32 : G; }

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
  double pvx[4], pvy[4];
  double weight;
  int delta[kMaxPairs];
  double fdelta[kMaxPairs];  // delta as a double (converted once per pair and term)
  int dself;                 // batched-mode self-pair delta' of the term
  int pad_;
};

// ---------------------------------------------------------------------------------------------
// CTA tables shared by the teams: the push items (d, e) of La Budde's recurrence (2 <= d,
// d + e <= Hl) twice, sorted by e then d (a level's items with e <= E are a prefix) and sorted by d
// then e (its items with d <= l + 1 are a prefix), and 1/k for k <= H + 1.
// ---------------------------------------------------------------------------------------------
__host__ __device__ constexpr int item_table_bytes(int n_items) { return (n_items * 4 + 15) & ~15; }

template <typename R, int CTA>
__device__ __forceinline__ void build_cta_tables(const TermParams& p, unsigned char* smem) {
  uint16_t* items = reinterpret_cast<uint16_t*>(smem);
  uint16_t* items_d = items + p.n_items;
  R* invk = reinterpret_cast<R*>(smem + item_table_bytes(p.n_items));
  const int Hl = p.Hl;
  for (int w = threadIdx.x; w < p.n_items; w += CTA) {
    int e = 0, base = 0;
    while (e < Hl - 2 && base + (Hl - 1 - e) <= w) {
      base += Hl - 1 - e;
      e++;
    }
    items[w] = (uint16_t)(((2 + (w - base)) << 8) | e);
    int d = 2;
    base = 0;
    while (d < Hl && base + (Hl - d + 1) <= w) {
      base += Hl - d + 1;
      d++;
    }
    items_d[w] = (uint16_t)((d << 8) | (w - base));
  }
  for (int k = threadIdx.x; k <= p.H + 1; k += CTA) invk[k] = k ? (R)1 / (R)k : (R)0;
}

#include "lhaf_adjoint.cuh"

// ---------------------------------------------------------------------------------------------
// The sieve terms t = p.t_begin + team_global + r * p.total_teams (r < p.rounds, t < p.t_end)
// of one loop hafnian, for the team of the calling thread. acc (lane 0 of the team) receives the
// double-double sum (re_hi, re_lo, im_hi, im_lo) of weight * f. STAGE: instead of finishing a
// term, write d_M and d_M - d_K to `stage` (coefficient-major, stage_ld terms per row, column
// t - p.t_begin) and its weight to `wstage`.
// ---------------------------------------------------------------------------------------------
template <typename R, int G, bool STAGE, bool GRAD = false>
__device__ __forceinline__ void sieve_terms(const typename Cx<R>::t* __restrict__ chat, const TermParams& p,
                                            unsigned char* smem, unsigned long long team_global,
                                            typename Cx<R>::t* __restrict__ stage, double* __restrict__ wstage,
                                            long long stage_ld, double* acc,
                                            typename Cx<R>::t* __restrict__ gslice = nullptr,
                                            const int* __restrict__ smap = nullptr, int n_full = 0) {
  using V = typename Cx<R>::t;
  constexpr int SG = G < 32 ? G : 32;  // lanes of the first warp of a team

  const int nd = p.nd, ld = p.ld, bord = p.bord, h = p.h, H = p.H, Hl = p.Hl, P = p.P;
  const int team = threadIdx.x / G;
  const int lt = threadIdx.x - team * G;

  const uint16_t* items = reinterpret_cast<const uint16_t*>(smem);
  const R* invk = reinterpret_cast<const R*>(smem + item_table_bytes(p.n_items));
  unsigned char* tb = smem + p.items_bytes + (size_t)team * p.team_bytes;
  V* W = reinterpret_cast<V*>(tb);
  V* Sa = W + nd * ld;  // inline series arrays, H + 2 entries each (absent when staging)
  V* Sc = Sa + (H + 2);
  V* SR = Sc + (H + 2);
  V* Sp = SR + (H + 2);
  V* Sz = Sp + (H + 2);
  V* Se = Sz + (H + 2);
  TeamScratch* ts = reinterpret_cast<TeamScratch*>(STAGE ? (void*)(W + nd * ld) : (void*)(Se + (H + 2)));

  const V zero = cmake<V>((R)0, (R)0);
  const V one = cmake<V>((R)1, (R)0);
  double acc_re = 0.0, acc_re_lo = 0.0, acc_im = 0.0, acc_im_lo = 0.0;

  // adjoint buffers (GRAD): S and Kb (nd x ld each), q_bar ((nd + 1) x (Hl + 1)), the region that
  // the adjoint's phases share (series adjoints, then c_bar, then multipliers, their adjoints and
  // dot-product partials: adjoint_union entries) and the pivot rows (nd ints) in shared memory; the
  // gradient sums Ga (n x n) and Gv (n), or n_full x n_full and n_full through the slot map smap, in
  // the team's own zeroed slice gslice of global memory (which leaves shared memory for a fourth
  // CTA on an SM at n = 27)
  const int ng = nd - bord;
  V* gS = reinterpret_cast<V*>(reinterpret_cast<unsigned char*>(ts) + ((sizeof(TeamScratch) + 15) & ~(size_t)15));
  V* gK = gS + nd * ld;
  V* gQ = gK + nd * ld;
  V* gU = gQ + (nd + 1) * (Hl + 1);
  int* gpiv = reinterpret_cast<int*>(gU + adjoint_union(nd, H, Hl, G));
  const int gn = smap ? n_full : ng;
  V* gA = GRAD ? gslice : nullptr;
  V* gV = GRAD ? gA + gn * gn : nullptr;

  for (unsigned long long rnd = 0; rnd < p.rounds; rnd++) {
    const unsigned long long t_raw = p.t_begin + team_global + rnd * p.total_teams;
    const bool valid = t_raw >= p.t_lo && t_raw < p.t_end;
    const unsigned long long t = valid ? t_raw : p.t_begin;  // an idle team repeats a valid term

    if (p.et_P > 0) {
      // ---- eigenvalue-trace term (App. B.1 Eq. ET_loop, repeated pairs as in App. B.2) ----
      // The term is one choice of P kept pairs out of et_P with z_q in 1..eta_q copies each; its
      // rank t is unranked pair by pair from the last with the table W[i][k] = e_k(eta_0..
      // eta_{i-1}), the number of such choices of k pairs among the first i (pair i-1 left out:
      // ranks below W[i-1][k]; kept: z - 1 = quotient by W[i-1][k-1]). Kept pairs take compacted
      // positions in ascending order: delta[c] = the pair's index, fdelta[c] = z. Weight
      // prod C(eta_q, z_q) (-1)^(h - sum z) (the sign reading of Eq. ET_loop) times wscale.
      if (lt == 0) {
        const int PF = p.et_P;
        const unsigned long long* Wt = p.et_table;
        unsigned long long r = t;
        int kk = P;
        double wq = 1.0;
        int zsum = 0;
        for (int i = PF; i >= 1 && kk > 0; i--) {
          const unsigned long long ex = Wt[(i - 1) * (PF + 1) + kk];
          if (r < ex) continue;
          r -= ex;
          const unsigned long long w1 = Wt[(i - 1) * (PF + 1) + kk - 1];
          if (w1 == 0ull) break;  // only for a rank out of range
          unsigned long long zq;
          if (r <= 0xffffffffull && w1 <= 0xffffffffull) {
            zq = (unsigned)r / (unsigned)w1;
          } else {
            zq = r / w1;
          }
          r -= zq * w1;
          const int z = 1 + (int)zq;
          kk--;
          ts->delta[kk] = i - 1;
          ts->fdelta[kk] = (double)z;
          wq *= binom_d(p.eta[i - 1], z);  // 0 when z > eta (only for a rank out of range)
          zsum += z;
        }
        for (int c = 0; c < kk; c++) {  // unreachable for ranks in range; keeps indices valid
          ts->delta[c] = c;
          ts->fdelta[c] = 0.0;
          wq = 0.0;
        }
        ts->weight = valid ? (((h - zsum) & 1) ? -wq : wq) * p.wscale : 0.0;
      }
    } else if (G <= 32 || lt < 32) {
      // ---- digits k_i of the term, delta'_i = eta_i - 2 k_i, and the weight (App. B.4) ----
      // Lane q of the first warp of the team decodes digit q; the weight is a product over lanes.
      double wq = 1.0;
      int par = 0;
      for (int q = lt; q < P; q += SG) {
        unsigned long long st = 1ull;
        for (int u = 0; u < q; u++) st *= (unsigned long long)p.radix[u];
        const unsigned rad = (unsigned)p.radix[q];
        unsigned long long qt;
        if (t <= 0xffffffffull && st <= 0xffffffffull) {
          qt = (unsigned)t / (unsigned)st;
        } else {
          qt = t / st;
        }
        const int eta = p.eta[q];
        int k = (int)(qt % rad);
        if (q == p.bq) {
          // batched-mode self pair: delta' runs over bA, bA - 1, ..., -bA (or bA..0 when this is
          // the halved digit); its binomial weight depends on the outcome and is applied later
          const int dlt = p.bA - k;
          ts->delta[q] = dlt;
          ts->fdelta[q] = (double)dlt;
          ts->dself = dlt;
          if (q == p.hp && dlt != 0) wq *= 2.0;
          continue;
        }
        if (((p.skip_mask >> q) & 1u) && 2 * k >= eta) k++;  // zero-digit group: no middle digit
        wq *= binom_d(eta, k);
        par ^= (k & 1);
        ts->delta[q] = eta - 2 * k;
        ts->fdelta[q] = (double)(eta - 2 * k);
        if (q == p.hp && !(p.hp_even && 2 * k == eta)) wq *= 2.0;  // sign-symmetry halving
      }
#pragma unroll
      for (int off = SG / 2; off >= 1; off >>= 1) {
        wq *= __shfl_xor_sync(0xffffffffu, wq, off);
        par ^= __shfl_xor_sync(0xffffffffu, par, off);
      }
      if (lt == 0) ts->weight = valid ? (par ? -wq : wq) * p.wscale : 0.0;
    }
    team_sync<G>();

    // ---- working matrix K[i][j] = Chat[i][partner(j)] * delta_hat(j) ----
    // Column by column, so that the lanes of a team mostly share one column's factor and the FP64
    // multiplies issue only for columns whose |delta'| > 1 in some team of the warp.
    if (p.et_P > 0) {
      // eigenvalue-trace term: the kept pairs' slots of the full slot matrix (et_ndf x et_ndf at
      // chat + et_off), columns scaled by the copies z (X_z of App. B.2)
      const int ndf = p.et_ndf;
      const V* fc = chat + p.et_off;
      for (int w = lt; w < nd * nd; w += G) {
        const int i = w / nd, j = w - (w / nd) * nd;
        int fi = i, fj = j;
        R f = (R)1;
        if (i >= bord) {
          const int s = i - bord;
          fi = bord + 2 * ts->delta[s >> 1] + (s & 1);
        }
        if (j >= bord) {
          const int s = j - bord;
          fj = bord + 2 * ts->delta[s >> 1] + ((s & 1) ^ 1);
          f = (R)ts->fdelta[s >> 1];
        }
        V c = fc[fi * ndf + fj];
        c.x *= f;
        c.y *= f;
        W[i * ld + j] = c;
      }
    } else {
      const int sj = G / nd, si = G - (G / nd) * nd;
      int j = lt / nd, i = lt - (lt / nd) * nd;
      for (int w = lt; w < nd * nd; w += G) {
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
          const R f = (R)ts->fdelta[(j - bord) >> 1];
          c.x *= f;
          c.y *= f;
        }
        W[i * ld + j] = c;
        j += sj;
        i += si;
        if (i >= nd) {
          i -= nd;
          j++;
        }
      }
    }
    team_sync<G>();

    // ---- Hessenberg form by elimination with partial pivoting (fixes index 0) ----
    for (int k = 0; k < nd - 2; k++) {
      // pivot: largest max(|re|, |im|) in column k below the diagonal (ties: lowest row); its
      // value travels with the reduction
      unsigned long long key = 0ull;
      int row = k + 1;
      V pv = zero;
      for (int i = k + 1 + lt; i < nd; i += G) {
        const V z = W[i * ld + k];
        const unsigned long long kk = mag_key(z);
        if (kk > key) {
          key = kk;
          row = i;
          pv = z;
        }
      }
#pragma unroll
      for (int off = SG / 2; off >= 1; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int orow = __shfl_xor_sync(0xffffffffu, row, off);
        const R ox = __shfl_xor_sync(0xffffffffu, pv.x, off);
        const R oy = __shfl_xor_sync(0xffffffffu, pv.y, off);
        if (ok > key || (ok == key && orow < row)) {
          key = ok;
          row = orow;
          pv.x = ox;
          pv.y = oy;
        }
      }
      if constexpr (G > 32) {
        if ((lt & 31) == 0) {
          ts->key[lt >> 5] = key;
          ts->row[lt >> 5] = row;
          ts->pvx[lt >> 5] = (double)pv.x;
          ts->pvy[lt >> 5] = (double)pv.y;
        }
        __syncthreads();
        key = ts->key[0];
        row = ts->row[0];
        pv.x = (R)ts->pvx[0];
        pv.y = (R)ts->pvy[0];
        for (int q = 1; q < G / 32; q++) {
          if (ts->key[q] > key || (ts->key[q] == key && ts->row[q] < row)) {
            key = ts->key[q];
            row = ts->row[q];
            pv.x = (R)ts->pvx[q];
            pv.y = (R)ts->pvy[q];
          }
        }
      }
      const int r = row;
      if constexpr (GRAD) {
        if (lt == 0) gpiv[k] = r;
      }
      const V ip = crecip(pv);  // issued before the swaps, so its latency overlaps them
      if (STAGE && p.ng > 0 && ld > nd && lt == 0) W[k * ld + nd].x = (R)r;  // for the loop vectors
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
      for (int i = k + 2 + lt; i < nd; i += G) W[i * ld + k] = cmul(W[i * ld + k], ip);
      team_sync<G>();
      // rows: K[i][j] -= l_i K[k+1][j] for i >= k+2, j >= k+1. Flattened over the team: passes of
      // four items per lane while every lane has four (loads of all before any store), then one
      // item per lane; indices advanced without division.
      const int cols = nd - k - 1;
      const int nrc = (cols - 1) * cols;
      {
        const int si = G / cols, sj = G - (G / cols) * cols;
        int ii = lt / cols, jj = lt - (lt / cols) * cols;
        int w = 0;
        for (; w + 4 * G <= nrc; w += 4 * G) {
          V* pa[4];
          V a[4], l[4], r[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            pa[u] = W + (k + 2 + ii) * ld + (k + 1 + jj);
            a[u] = *pa[u];
            l[u] = W[(k + 2 + ii) * ld + k];
            r[u] = W[(k + 1) * ld + k + 1 + jj];
            ii += si;
            jj += sj;
            if (jj >= cols) {
              jj -= cols;
              ii++;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; u++) cmsub(a[u], l[u], r[u]);
#pragma unroll
          for (int u = 0; u < 4; u++) *pa[u] = a[u];
        }
        for (; w < nrc; w += G) {
          if (w + lt < nrc) {
            V* p1 = W + (k + 2 + ii) * ld + (k + 1 + jj);
            V a1 = *p1;
            cmsub(a1, W[(k + 2 + ii) * ld + k], W[(k + 1) * ld + k + 1 + jj]);
            *p1 = a1;
          }
          ii += si;
          jj += sj;
          if (jj >= cols) {
            jj -= cols;
            ii++;
          }
        }
      }
      team_sync<G>();
      // columns: K[i][k+1] += sum_{j >= k+2} K[i][j] l_j. One lane per row, or, when it fills the
      // team better, two lanes per row (halves of the dot product, combined by one shuffle).
      {
        const int L = nd - k - 2;
        const int half = (L + 1) >> 1;
        const int slots1 = ((nd + G - 1) / G) * L;
        const int slots2 = ((2 * nd + G - 1) / G) * (half + 1);
        if (L >= 4 && slots2 < slots1) {
          for (int base = 0; base < nd; base += G / 2) {
            const int i = base + (lt >> 1);
            const int sgm = lt & 1;
            V acc = zero;
            if (i < nd) {
              const int j0 = k + 2 + sgm * half;
              const int j1 = sgm ? nd : k + 2 + half;
              dot_accumulate(acc, W + i * ld, W + k, ld, j0, j1);
            }
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
            if (i < nd && sgm == 0) {
              V a = W[i * ld + k + 1];
              a.x += acc.x;
              a.y += acc.y;
              W[i * ld + k + 1] = a;
            }
          }
        } else {
          for (int i = lt; i < nd; i += G) {
            V a = W[i * ld + k + 1];
            dot_accumulate(a, W + i * ld, W + k, ld, k + 2, nd);
            W[i * ld + k + 1] = a;
          }
        }
      }
      team_sync<G>();
    }

    if constexpr (STAGE) {
      if (G <= 32 && p.ng > 0 && bord == 0 && ld > nd) {
        // ---- loop sequences of several loop-weight vectors on one Hessenberg form (App. B.5) ----
        // M = C X_delta' = Q H Q^-1 with Q = P_0 L_0 P_1 L_1 ... (the swaps r_k recorded in the
        // padding column, the multipliers l_i below the subdiagonal). For loop weights v (on the
        // slots) and u = v X_delta', s_k = u M^(k-1) v^T = (u Q) H^(k-1) (Q^-1 v^T), k = 1..min(h, n),
        // staged in rows h + g h + k - 1; the series kernel extends s_k past n with the
        // characteristic polynomial (they are R_{k+1} of the bordered form).
        // Two vectors per pass (nv = 2, or 1 for the last of an odd count): the swaps and
        // multipliers, and each H entry of the products, are loaded once for both.
        V* xu = gS;           // u' of the pass's vectors, nd each
        V* xa = xu + 2 * nd;  // Krylov vectors
        V* xb = xa + 2 * nd;  // next Krylov vectors
        const V* gvs = reinterpret_cast<const V*>(p.gv);
        const int kr = h < nd ? h : nd;
        const bool st_col = valid || p.stage_pad;
        const long long col = (long long)(t_raw - p.t_begin);
        for (int g0 = 0; g0 < p.ng; g0 += 2) {
          const int nv = (p.ng - g0 >= 2) ? 2 : 1;
          for (int w = lt; w < nv * nd; w += G) {
            const int c = w >= nd ? 1 : 0;
            const int i = w - c * nd;
            const V* vg = gvs + (size_t)(g0 + c) * nd;
            xa[c * nd + i] = vg[i];
            V z = vg[i ^ 1];
            const int dl = ts->delta[i >> 1];
            if (dl == -1) {
              z.x = flip(z.x);
              z.y = flip(z.y);
            } else if (dl != 1) {
              const R f = (R)ts->fdelta[i >> 1];
              z.x *= f;
              z.y *= f;
            }
            xu[c * nd + i] = z;
          }
          team_sync<G>();
          for (int k = 0; k < nd - 2; k++) {
            const int r = (int)W[k * ld + nd].x;
            if (lt < nv && r > k + 1 && r < nd) {  // lane c swaps vector c
              V* a = xa + lt * nd;
              V* b = xu + lt * nd;
              const V ta = a[r];
              a[r] = a[k + 1];
              a[k + 1] = ta;
              const V tb = b[r];
              b[r] = b[k + 1];
              b[k + 1] = tb;
            }
            team_sync<G>();
            const V vk0 = xa[k + 1];
            const V vk1 = xa[nd + k + 1];
            V su0 = zero, su1 = zero;
            for (int i = k + 2 + lt; i < nd; i += G) {
              const V l = W[i * ld + k];
              V a0 = xa[i];
              cmsub(a0, l, vk0);
              xa[i] = a0;
              cmac(su0, xu[i], l);
              if (nv == 2) {
                V a1 = xa[nd + i];
                cmsub(a1, l, vk1);
                xa[nd + i] = a1;
                cmac(su1, xu[nd + i], l);
              }
            }
#pragma unroll
            for (int off = SG / 2; off >= 1; off >>= 1) {
              su0.x += __shfl_xor_sync(0xffffffffu, su0.x, off);
              su0.y += __shfl_xor_sync(0xffffffffu, su0.y, off);
              su1.x += __shfl_xor_sync(0xffffffffu, su1.x, off);
              su1.y += __shfl_xor_sync(0xffffffffu, su1.y, off);
            }
            if (lt == 0) {
              V a = xu[k + 1];
              a.x += su0.x;
              a.y += su0.y;
              xu[k + 1] = a;
              if (nv == 2) {
                V b = xu[nd + k + 1];
                b.x += su1.x;
                b.y += su1.y;
                xu[nd + k + 1] = b;
              }
            }
            team_sync<G>();
          }
          V* x = xa;
          V* y = xb;
          for (int k = 1; k <= kr; k++) {
            V d0 = zero, d1 = zero;
            for (int i = lt; i < nd; i += G) {
              cmac(d0, xu[i], x[i]);
              if (nv == 2) cmac(d1, xu[nd + i], x[nd + i]);
            }
#pragma unroll
            for (int off = SG / 2; off >= 1; off >>= 1) {
              d0.x += __shfl_xor_sync(0xffffffffu, d0.x, off);
              d0.y += __shfl_xor_sync(0xffffffffu, d0.y, off);
              d1.x += __shfl_xor_sync(0xffffffffu, d1.x, off);
              d1.y += __shfl_xor_sync(0xffffffffu, d1.y, off);
            }
            if (lt == 0 && st_col) {
              stage[(long long)(h + g0 * h + k - 1) * stage_ld + col] = d0;
              if (nv == 2) stage[(long long)(h + (g0 + 1) * h + k - 1) * stage_ld + col] = d1;
            }
            if (k < kr) {
              for (int i = lt; i < nd; i += G) {
                V a0 = zero, a1 = zero;
                for (int j = (i > 0 ? i - 1 : 0); j < nd; j++) {
                  const V hij = W[i * ld + j];
                  cmac(a0, hij, x[j]);
                  if (nv == 2) cmac(a1, hij, x[nd + j]);
                }
                y[i] = a0;
                if (nv == 2) y[nd + i] = a1;
              }
              team_sync<G>();
              V* tmp = x;
              x = y;
              y = tmp;
            }
          }
          team_sync<G>();
        }
      }
    }

    if constexpr (GRAD) {  // the Hessenberg form with its multipliers, for the adjoint
      for (int w = lt; w < nd * ld; w += G) gS[w] = W[w];
      team_sync<G>();
    }

    // ---- La Budde's recurrence, reverse (trailing blocks), truncated at degree Hl ----
    // q_j(t) = det(I - t K[j.., j..]) = (1 - t K_jj) q_{j+1} - sum_{l > j} c_{j,l} t^(l-j+1) q_{l+1}
    // with c_{j,l} = K_jl prod_{r=j+1..l} K_{r,r-1}, stored over K_jl (l - j <= Hl - 1).
    // Each lane runs the product chains of up to four of its rows j side by side.
    for (int j0 = lt; j0 < nd - 1; j0 += 4 * G) {
      V pi[4];
      int dm[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int j = j0 + u * G;
        dm[u] = (j < nd - 1) ? min(Hl - 1, nd - 1 - j) : 0;
        pi[u] = one;
      }
      for (int dp = 1; dp <= dm[0]; dp++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (dp <= dm[u]) {
            const int j = j0 + u * G, l = j + dp;
            pi[u] = cmul(pi[u], W[l * ld + l - 1]);
            W[j * ld + l] = cmul(W[j * ld + l], pi[u]);
          }
        }
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
      // valid pushes have e <= E and d <= l + 1: walk the shorter of the two sorted prefixes
      const int npe = (E >= 0) ? (E + 1) * (Hl - 1) - E * (E + 1) / 2 : 0;
      const int dmx = min(Hl, l + 1);
      const int npd = (dmx >= 2) ? (dmx - 1) * (2 * Hl - dmx) / 2 : 0;
      const bool by_d = npd < npe;
      const uint16_t* tab = by_d ? items + p.n_items : items;
      const int np = by_d ? npd : npe;
      const int nq = min(Hl, nd - l);
      // Every item is dst <- a - b c: a push into acc_j, or the update of q_l[m]; the items of one
      // level are independent. Passes of four items per lane while every lane has four (loads
      // first), then one item per lane.
      auto load_item = [&](int x, V*& dst, V& a, V& b, V& c) -> bool {
        if (x < np) {
          // push q_{l+1} into the accumulator of q_j, j = l - d + 1
          const int it = tab[x];
          const int d = it >> 8, e = it & 255;
          const int j = l - d + 1;
          if (j >= 0 && e <= E) {
            dst = W + (l + e) * ld + j;
            a = *dst;
            b = W[j * ld + l];
            c = (e == 0) ? one : W[(l + e) * ld + l + 1];
            return true;
          }
          return false;
        }
        // q_l[m] = q_{l+1}[m] - K_ll q_{l+1}[m-1] + acc_l[m]
        const int m = x - np + 1;
        dst = W + (l + m - 1) * ld + l;
        V v = (m <= deg) ? W[(l + m) * ld + l + 1] : zero;
        if (m >= 2) {
          const V acc = *dst;
          v.x += acc.x;
          v.y += acc.y;
        }
        a = v;
        b = hll;
        c = (m == 1) ? one : ((m - 1 <= deg) ? W[(l + m - 1) * ld + l + 1] : zero);
        return true;
      };
      const int nitems = np + nq;
      int w = 0;
      for (; w + 4 * G <= nitems; w += 4 * G) {
        V* dst[4];
        V a[4], b[4], c[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          dst[u] = W;
          a[u] = zero;
          b[u] = zero;
          c[u] = zero;
          ok[u] = load_item(w + u * G + lt, dst[u], a[u], b[u], c[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) cmsub(a[u], b[u], c[u]);
#pragma unroll
        for (int u = 0; u < 4; u++)
          if (ok[u]) *dst[u] = a[u];
      }
      for (; w < nitems; w += G) {
        const int x = w + lt;
        if (x < nitems) {
          V* dst = W;
          V a = zero, b = zero, c = zero;
          if (load_item(x, dst, a, b, c)) {
            cmsub(a, b, c);
            *dst = a;
          }
        }
      }
      V hnext = zero;
      if (l > 0) hnext = W[(l - 1) * ld + l - 1];
      team_sync<G>();
      hll = hnext;
    }

    if constexpr (STAGE) {
      // ---- stage a_m = [t^m] d_M (m = 1..h) and c_m = [t^m](d_M - d_K) (m = 1..h+1) ----
      if (valid || p.stage_pad) {
        const long long col = (long long)(t_raw - p.t_begin);
        const int nc = bord ? 2 * h + 1 : h;
        for (int x = lt; x < nc; x += G) {
          const int m = x < h ? x + 1 : x - h + 1;
          V am = zero, bm = zero;
          if (m <= Hl) {
            if (bord) {
              if (m <= nd - 1) am = W[m * ld + 1];
              if (m <= nd) bm = W[(m - 1) * ld];
            } else {
              if (m <= nd) am = W[(m - 1) * ld];
            }
          }
          stage[(long long)x * stage_ld + col] = (x < h) ? am : cmake<V>(am.x - bm.x, am.y - bm.y);
        }
        if (lt == 0) {
          wstage[col] = ts->weight;
          if (p.bq >= 0) wstage[stage_ld + col] = (double)ts->dself;  // second row: the self delta'
        }
      }
      team_sync<G>();
    } else {
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
        // Step k: R_{k+1}, p_k, z_k = (p_k + k R_{k+1}) / 2 and e_{k-1} = sum_j z_j e_{k-1-j}/(k-1)
        // from one reduction round (e lags one step, so its dot product needs no z_k).
        // With 16 or more lanes the three dot products run side by side on three groups of SG / 4
        // lanes (the fourth idle), each with a short shuffle tree: the trees' FP64 adds, not the
        // products, dominate a step of a degree <= 32 series.
        constexpr int GW = SG >= 16 ? SG / 4 : SG;
        const int grp = sl / GW, gl = sl - grp * GW;
        for (int k = 1; k <= h + 1; k++) {
          const bool rp = k <= h;
          V sR = zero, sp = zero, se = zero;
          if constexpr (SG >= 16) {
            // group 0: sum_(i<=k) a_i R_(k+1-i); group 1: sum_(i<k) a_i p_(k-i); group 2: sum_(i<k) z_i e_(k-1-i)
            const int top = grp == 0 ? k : k - 1;
            const bool on = grp < 3 && (grp == 2 || rp);
            V sg = zero;
            for (int i = 1 + gl; i <= k; i += GW) {
              const bool v = on && i <= top;
              const int iy = v ? (grp == 0 ? k + 1 - i : (grp == 1 ? k - i : k - 1 - i)) : 0;
              const V x = grp == 2 ? Sz[i] : Sa[i];
              const V y = grp == 0 ? SR[iy] : (grp == 1 ? Sp[iy] : Se[iy]);
              cmac(sg, v ? x : zero, y);
            }
#pragma unroll
            for (int off = GW / 2; off >= 1; off >>= 1) {
              sg.x += __shfl_xor_sync(0xffffffffu, sg.x, off);
              sg.y += __shfl_xor_sync(0xffffffffu, sg.y, off);
            }
            sR = cmake<V>(__shfl_sync(0xffffffffu, sg.x, 0, SG), __shfl_sync(0xffffffffu, sg.y, 0, SG));
            sp = cmake<V>(__shfl_sync(0xffffffffu, sg.x, GW, SG), __shfl_sync(0xffffffffu, sg.y, GW, SG));
            se = cmake<V>(__shfl_sync(0xffffffffu, sg.x, 2 * GW, SG), __shfl_sync(0xffffffffu, sg.y, 2 * GW, SG));
          } else {
            for (int i = 1 + sl; i <= k; i += SG) {
              if (rp) cmac(sR, Sa[i], SR[k + 1 - i]);
              if (i < k) {
                if (rp) cmac(sp, Sa[i], Sp[k - i]);
                cmac(se, Sz[i], Se[k - 1 - i]);
              }
            }
#pragma unroll
            for (int off = SG / 2; off >= 1; off >>= 1) {
              sR.x += __shfl_xor_sync(0xffffffffu, sR.x, off);
              sR.y += __shfl_xor_sync(0xffffffffu, sR.y, off);
              sp.x += __shfl_xor_sync(0xffffffffu, sp.x, off);
              sp.y += __shfl_xor_sync(0xffffffffu, sp.y, off);
              se.x += __shfl_xor_sync(0xffffffffu, se.x, off);
              se.y += __shfl_xor_sync(0xffffffffu, se.y, off);
            }
          }
          if (sl == 0) {
            if (rp) {
              const V ck = Sc[k + 1], ak = Sa[k];
              const R kk = (R)k;
              const V Rk = cmake<V>(ck.x - sR.x, ck.y - sR.y);                        // R_{k+1}
              const V pk = cmake<V>(-rfma(kk, ak.x, sp.x), -rfma(kk, ak.y, sp.y));  // power sum p_k
              SR[k + 1] = Rk;
              Sp[k] = pk;
              Sz[k] = cmake<V>((R)0.5 * rfma(kk, Rk.x, pk.x), (R)0.5 * rfma(kk, Rk.y, pk.y));
            }
            if (k >= 2) Se[k - 1] = cmake<V>(se.x * invk[k - 1], se.y * invk[k - 1]);
          }
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
      if constexpr (GRAD) {
        adjoint_series_labudde<R, G>(W, gS, gK, gQ, gU, Sa, Sc, SR, Sp, Sz, Se, nd, ld, bord, h, H, Hl, lt);
        adjoint_elimination<R, G>(gS, gK, gU, gpiv, nd, ld, lt);
        adjoint_accumulate<R, G>(gK, nd, ld, bord, ts->delta, ts->weight, gA, gV, smap, gn, lt);
      }
    }
  }


  acc[0] = acc_re;
  acc[1] = acc_re_lo;
  acc[2] = acc_im;
  acc[3] = acc_im_lo;
}

// One loop hafnian over a grid of CTAs: team tg of the grid takes terms tg, tg + teams, ...
template <typename R, int G, bool STAGE>
__global__ void __launch_bounds__(cta_of(G))
terms_kernel(const typename Cx<R>::t* __restrict__ chat, const __grid_constant__ TermParams p,
             double* __restrict__ partials, typename Cx<R>::t* __restrict__ stage, double* __restrict__ wstage,
             long long stage_ld) {
  constexpr int CTA = cta_of(G);
  constexpr int TEAMS = CTA / G;
  extern __shared__ __align__(16) unsigned char smem[];
  build_cta_tables<R, CTA>(p, smem);
  __syncthreads();
  const int team = threadIdx.x / G;
  const int lt = threadIdx.x - team * G;
  const unsigned long long team_global = (unsigned long long)blockIdx.x * TEAMS + team;
  double acc[4];
  sieve_terms<R, G, STAGE>(chat, p, smem, team_global, stage, wstage, stage_ld, acc);
  if constexpr (!STAGE) {
    if (lt == 0) {
      double* o = partials + 4ull * team_global;
      o[0] = acc[0];
      o[1] = acc[1];
      o[2] = acc[2];
      o[3] = acc[3];
    }
  }
}

// One loop hafnian over several sieves (zero-digit groups): chunks of TEAMS terms that stay inside
// one sieve, taken grid-strided so that each round the CTAs work on neighbouring chunks (similar
// cost). The CTA copies its chunk's sieve description into shared memory and rebuilds the La Budde
// tables when the truncation changes.
template <typename R, int G, bool STAGE>
__global__ void __launch_bounds__(cta_of(G))
grouped_terms_kernel(const typename Cx<R>::t* __restrict__ chat_pool, const BatchItem* __restrict__ jobs, int n_jobs,
                     const long long* __restrict__ chunk_off, long long k_begin, long long k_end, int rounds,
                     unsigned long long tb, unsigned long long te, int team_bytes, int items_bytes,
                     double* __restrict__ partials, typename Cx<R>::t* __restrict__ stage,
                     double* __restrict__ wstage, long long stage_ld, int per_chunk,
                     unsigned long long* __restrict__ next_chunk) {
  using V = typename Cx<R>::t;
  constexpr int CTA = cta_of(G);
  constexpr int TEAMS = CTA / G;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TermParams sp;
  __shared__ int s_job, s_Hl;
  __shared__ long long s_k;
  const int team = threadIdx.x / G;
  const int lt = threadIdx.x - team * G;
  if (threadIdx.x == 0) {
    s_job = -1;
    s_Hl = -1;
  }
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
  for (int r = 0;; r++) {
    // chunk of this round: taken from the shared counter (CTAs whose SM sub-partitions share a
    // less loaded FP64 unit take more chunks), or grid-strided without one
    long long k;
    if (next_chunk) {
      __syncthreads();  // the previous s_k has been read by every thread
      if (threadIdx.x == 0) s_k = k_begin + (long long)atomicAdd(next_chunk, 1ull);
      __syncthreads();
      k = s_k;
    } else {
      if (r >= rounds) break;
      k = k_begin + blockIdx.x + (long long)r * gridDim.x;
    }
    if (k >= k_end) break;  // uniform over the CTA
    // sieve of chunk k: the last j with chunk_off[j] <= k
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_off[mid] <= k) {
        lo = mid;
      } else {
        hi = mid - 1;
      }
    }
    const int j = lo;
    __syncthreads();  // the previous chunk is done with sp and the tables
    if (j != s_job) {
      // copy the description (a POD of 8-byte words) with all threads
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&jobs[j].p);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sp);
      for (int w = threadIdx.x; w < (int)(sizeof(TermParams) / 8); w += CTA) dst[w] = src[w];
    }
    __syncthreads();
    const bool valid_desc = sp.nd >= 2 && sp.nd <= kMaxDim && sp.P <= kMaxPairs && sp.h <= kMaxDegree &&
                            sp.Hl <= sp.nd && sp.n_items == sp.Hl * (sp.Hl - 1) / 2;
    if (!valid_desc) {  // a description outside the compiled limits is skipped (its slots read 0)
      if (!STAGE && per_chunk && lt == 0) {
        double* o = partials + 4ll * ((k - k_begin) * TEAMS + team);
        o[0] = o[1] = o[2] = o[3] = 0.0;
      }
      continue;
    }
    if (j != s_job || sp.Hl != s_Hl) {
      build_cta_tables<R, CTA>(sp, smem);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      // chunk terms t0 .. t0 + TEAMS - 1 of sieve j; valid below its term count (jobs[j].p.t_end)
      // and inside [tb, te) of the loop hafnian's numbering
      const unsigned long long t0 = (unsigned long long)(k - chunk_off[j]) * TEAMS;
      const unsigned long long base = jobs[j].base, T = jobs[j].p.t_end;
      unsigned long long hi = T < t0 + TEAMS ? T : t0 + TEAMS;
      if (te <= base) {
        hi = t0;
      } else if (te - base < hi) {
        hi = te - base;
      }
      sp.t_begin = t0;
      sp.t_end = hi > t0 ? hi : t0;
      sp.t_lo = tb > base ? tb - base : 0ull;
      sp.rounds = 1;
      sp.total_teams = TEAMS;
      sp.team_bytes = team_bytes;
      sp.items_bytes = items_bytes;
      sp.stage_pad = STAGE ? 1 : 0;
      s_job = j;
      s_Hl = sp.Hl;
    }
    __syncthreads();
    double acc[4];
    const long long colbase = (k - k_begin) * TEAMS;
    sieve_terms<R, G, STAGE>(reinterpret_cast<const V*>(chat_pool) + jobs[j].chat_off, sp, smem,
                             (unsigned long long)team, STAGE ? stage + colbase : nullptr,
                             STAGE ? wstage + colbase : nullptr, stage_ld, acc);
    if constexpr (!STAGE) {
      if (per_chunk) {
        if (lt == 0) {
          double* o = partials + 4ll * (colbase + team);
          o[0] = acc[0];
          o[1] = acc[1];
          o[2] = acc[2];
          o[3] = acc[3];
        }
      } else {
        dd_add_dd(rh, rl, acc[0], acc[1]);
        dd_add_dd(ih, il, acc[2], acc[3]);
      }
    }
  }
  if constexpr (!STAGE) {
    if (lt == 0 && !per_chunk) {
      double* o = partials + 4ull * ((unsigned long long)blockIdx.x * TEAMS + team);
      o[0] = rh;
      o[1] = rl;
      o[2] = ih;
      o[3] = il;
    }
  }
}

// One block per item: the item's bordered slot matrix from device B (shared M x M, or one per
// item at B_stride) and gamma (M per item at gamma_stride; NULL: diag of B).
__global__ void batch_gather_kernel(const double2* __restrict__ B, long long B_stride, const double2* __restrict__ gamma,
                                    long long gamma_stride, int M, const BatchItem* __restrict__ items,
                                    double2* __restrict__ chat_pool, float2* __restrict__ chat32_pool) {
  const int item = blockIdx.x;
  const BatchItem& it = items[item];
  const int nd = it.p.nd, bord = it.p.bord;
  if (nd <= 0) return;
  const double2* Bi = B + (long long)it.src * B_stride;
  const double2* gi = gamma ? gamma + (long long)it.src * gamma_stride : nullptr;
  for (int w = threadIdx.x; w < nd * nd; w += blockDim.x) {
    const int i = w / nd, j = w - i * nd;
    double2 c = make_double2(0.0, 0.0);
    if (bord && i == 0 && j == 0) {
    } else if (bord && (i == 0 || j == 0)) {
      const int m = it.slot_mode[(i == 0 ? j : i) - 1];
      c = (m < 0) ? make_double2(1.0, 0.0) : (gi ? gi[m] : Bi[(size_t)m * M + m]);
    } else {
      const int a = it.slot_mode[i - bord], bm = it.slot_mode[j - bord];
      if (a >= 0 && bm >= 0) {
        const int lo = a < bm ? a : bm, hi = a < bm ? bm : a;
        c = Bi[(size_t)lo * M + hi];
      }
    }
    if (chat_pool) chat_pool[it.chat_off + w] = c;
    if (chat32_pool) chat32_pool[it.chat_off + w] = make_float2((float)c.x, (float)c.y);
  }
}

// ---------------------------------------------------------------------------------------------
// Value and adjoint of one loop hafnian: like terms_kernel (inline series), plus per-team gradient
// partials (n x n for the slot matrix, then n for the loop vector) in gpart.
// ---------------------------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(cta_of(G))
grad_kernel(const double2* __restrict__ chat, const __grid_constant__ TermParams p, double* __restrict__ partials,
            double2* __restrict__ gpart) {
  constexpr int CTA = cta_of(G);
  constexpr int TEAMS = CTA / G;
  extern __shared__ __align__(16) unsigned char smem[];
  build_cta_tables<double, CTA>(p, smem);
  __syncthreads();
  const int team = threadIdx.x / G;
  const int lt = threadIdx.x - team * G;
  const unsigned long long team_global = (unsigned long long)blockIdx.x * TEAMS + team;
  const int ng = p.nd - p.bord;
  double2* gslice = gpart + team_global * (unsigned long long)(ng * ng + ng);
  for (int w = lt; w < ng * ng + ng; w += G) gslice[w] = make_double2(0.0, 0.0);
  team_sync<G>();
  double acc[4];
  sieve_terms<double, G, false, true>(chat, p, smem, team_global, nullptr, nullptr, 0, acc, gslice);
  if (lt == 0) {
    double* o = partials + 4ull * team_global;
    o[0] = acc[0];
    o[1] = acc[1];
    o[2] = acc[2];
    o[3] = acc[3];
  }
}

// Value and adjoint over several sieves (a loop hafnian's zero-digit groups) in one launch: CTA c
// takes chunks c, c + grid, ... of TEAMS terms of one sieve each (a fixed assignment, so that the
// FP64 gradient sums of a team always add the same terms in the same order), the smaller groups'
// terms on their smaller matrices; each team's gradient sums stay in the full problem's slots
// (n_full) through each sieve's slot map, and its double-double value partial covers its chunks.
template <int G>
__global__ void __launch_bounds__(cta_of(G))
grad_grouped_kernel(const double2* __restrict__ chat_pool, const GradSieve* __restrict__ sieves, int n_sieves,
                    const long long* __restrict__ chunk_off, long long n_chunks, int n_full, int team_bytes,
                    int items_bytes, double* __restrict__ partials, double2* __restrict__ gpart) {
  constexpr int CTA = cta_of(G);
  constexpr int TEAMS = CTA / G;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TermParams sp;
  __shared__ int s_job, s_Hl;
  const int team = threadIdx.x / G;
  const int lt = threadIdx.x - team * G;
  const unsigned long long team_global = (unsigned long long)blockIdx.x * TEAMS + team;
  double2* gslice = gpart + team_global * (unsigned long long)(n_full * n_full + n_full);
  for (int w = lt; w < n_full * n_full + n_full; w += G) gslice[w] = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) {
    s_job = -1;
    s_Hl = -1;
  }
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
  for (long long k = blockIdx.x; k < n_chunks; k += gridDim.x) {
    __syncthreads();  // the previous chunk no longer reads sp and the tables
    int lo = 0, hi = n_sieves - 1;  // sieve of chunk k: the last j with chunk_off[j] <= k
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_off[mid] <= k) {
        lo = mid;
      } else {
        hi = mid - 1;
      }
    }
    const int j = lo;
    if (j != s_job) {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&sieves[j].p);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sp);
      for (int w = threadIdx.x; w < (int)(sizeof(TermParams) / 8); w += CTA) dst[w] = src[w];
    }
    __syncthreads();
    const bool valid_desc = sp.nd >= 2 && sp.nd <= kMaxDim && sp.P <= kMaxPairs && sp.h <= kMaxDegree &&
                            sp.Hl <= sp.nd && sp.n_items == sp.Hl * (sp.Hl - 1) / 2 &&
                            sp.nd - sp.bord <= n_full;
    if (!valid_desc) continue;  // a description outside the compiled limits adds nothing
    if (j != s_job || sp.Hl != s_Hl) {
      build_cta_tables<double, CTA>(sp, smem);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const unsigned long long t0 = (unsigned long long)(k - chunk_off[j]) * TEAMS;
      const unsigned long long T = sieves[j].p.t_end;
      const unsigned long long te = T < t0 + TEAMS ? T : t0 + TEAMS;
      sp.t_begin = t0;
      sp.t_end = te > t0 ? te : t0;
      sp.t_lo = 0ull;
      sp.rounds = 1;
      sp.total_teams = TEAMS;
      sp.team_bytes = team_bytes;
      sp.items_bytes = items_bytes;
      s_job = j;
      s_Hl = sp.Hl;
    }
    __syncthreads();
    double acc[4];
    sieve_terms<double, G, false, true>(chat_pool + sieves[j].chat_off, sp, smem, (unsigned long long)team, nullptr,
                                        nullptr, 0, acc, gslice, sieves[j].smap, n_full);
    dd_add_dd(rh, rl, acc[0], acc[1]);
    dd_add_dd(ih, il, acc[2], acc[3]);
  }
  if (lt == 0) {
    double* o = partials + 4ull * team_global;
    o[0] = rh;
    o[1] = rl;
    o[2] = ih;
    o[3] = il;
  }
}

// out[k] = 2^-h * sum over teams of gpart[team][k] (double-double), k < len.
__global__ void grad_reduce_kernel(const double2* __restrict__ gpart, long long teams, int len, int h,
                                   double2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= len) return;
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
  for (long long t = 0; t < teams; t++) {
    const double2 v = gpart[t * len + k];
    dd_add(rh, rl, v.x);
    dd_add(ih, il, v.y);
  }
  const double s1 = __longlong_as_double((long long)(1023 - h) << 52);
  out[k] = make_double2((rh + rl) * s1, (ih + il) * s1);
}

// ---------------------------------------------------------------------------------------------
// Staged series: one term per thread. From a_m = [t^m] d_M and c_m = [t^m](d_M - d_K):
//   R_{k+1} = c_{k+1} - sum_{i=1..k} a_i R_{k+1-i}           (R = (1 - d_K/d_M)/t, R_1 = c_1)
//   p_k     = -k a_k - sum_{i=1..k-1} a_i p_{k-i}             (Newton: power sums Tr((C X)^k))
//   z_k     = k g_k = (p_k + k R_{k+1}) / 2                   (g_k of Eq. ET_poly)
//   e_k     = (1/k) sum_{j=1..k} z_j e_{k-j},  e_0 = 1,  f = e_h
// Working arrays live in shared memory, [index][thread]. The weighted values are summed in
// double-double per block.
// ---------------------------------------------------------------------------------------------
constexpr int kSeriesThreads = 64;

template <typename R>
__global__ void __launch_bounds__(kSeriesThreads)
series_kernel(const typename Cx<R>::t* __restrict__ stage, const double* __restrict__ wstage, long long count,
              long long stage_ld, int h, int bord, int plain, double* __restrict__ partials) {
  using V = typename Cx<R>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  V* SR = reinterpret_cast<V*>(smem);             // (h + 2) x threads
  V* Sp = SR + (size_t)(h + 2) * kSeriesThreads;  // (h + 1) x threads
  V* Sz = Sp + (size_t)(h + 1) * kSeriesThreads;
  V* Se = Sz + (size_t)(h + 1) * kSeriesThreads;
  const int tid = threadIdx.x;
  const long long tt = (long long)blockIdx.x * kSeriesThreads + tid;
  const V zero = cmake<V>((R)0, (R)0);
  double fr = 0.0, fi = 0.0;
  if (tt < count) {
    auto A = [&](int m) -> V { return stage[(long long)(m - 1) * stage_ld + tt]; };
    auto C = [&](int m) -> V { return bord ? stage[(long long)(h + m - 1) * stage_ld + tt] : zero; };
#define SIDX(i) ((size_t)(i) * kSeriesThreads + tid)
    SR[SIDX(0)] = zero;
    SR[SIDX(1)] = C(1);
    Se[SIDX(0)] = cmake<V>((R)1, (R)0);
    for (int k = 1; k <= h; k++) {
      V sR = zero, sp = zero;
      for (int i = 1; i <= k; i++) {
        const V ai = A(i);
        if (bord) cmac(sR, ai, SR[SIDX(k + 1 - i)]);
        if (i < k) cmac(sp, ai, Sp[SIDX(k - i)]);
      }
      const V ck = C(k + 1), ak = A(k);
      const R kk = (R)k;
      const V Rk = cmake<V>(ck.x - sR.x, ck.y - sR.y);
      const V pk = cmake<V>(-rfma(kk, ak.x, sp.x), -rfma(kk, ak.y, sp.y));
      const V zk = cmake<V>((R)0.5 * rfma(kk, Rk.x, pk.x), (R)0.5 * rfma(kk, Rk.y, pk.y));
      SR[SIDX(k + 1)] = Rk;
      Sp[SIDX(k)] = pk;
      Sz[SIDX(k)] = zk;
      V se = zero;
      for (int j = 1; j <= k; j++) cmac(se, Sz[SIDX(j)], Se[SIDX(k - j)]);
      const R ik = (R)1 / kk;
      Se[SIDX(k)] = cmake<V>(se.x * ik, se.y * ik);
    }
    const V f = Se[SIDX(h)];
#undef SIDX
    const double w = wstage[tt];
    fr = (double)f.x * w;
    fi = (double)f.y * w;
  }
  // block sum in double-double
  __shared__ double red[4][kSeriesThreads];
  red[0][tid] = fr;
  red[1][tid] = 0.0;
  red[2][tid] = fi;
  red[3][tid] = 0.0;
  __syncthreads();
  for (int off = kSeriesThreads / 2; off >= 1; off >>= 1) {
    if (tid < off) {
      double a = red[0][tid], b = red[1][tid], c = red[2][tid], d = red[3][tid];
      if (plain) {
        a += red[0][tid + off];
        c += red[2][tid + off];
      } else {
        dd_add_dd(a, b, red[0][tid + off], red[1][tid + off]);
        dd_add_dd(c, d, red[2][tid + off], red[3][tid + off]);
      }
      red[0][tid] = a;
      red[1][tid] = b;
      red[2][tid] = c;
      red[3][tid] = d;
    }
    __syncthreads();
  }
  if (tid == 0) {
    double* o = partials + 4ll * blockIdx.x;
    o[0] = red[0][0];
    o[1] = red[1][0];
    o[2] = red[2][0];
    o[3] = red[3][0];
  }
}

// ---------------------------------------------------------------------------------------------
// Double-double reduction of partials, then the exact 2^-h scaling of Eq. fdsieve. With
// accumulate != 0 the sum is added to the dd value already in out_dd (chunked sums).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
reduce_kernel(const double* __restrict__ partials, long long count, int h, double* out_dd, double2* out_val,
              int accumulate) {
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
    double a = s[0][0], b = s[1][0], c = s[2][0], d = s[3][0];
    if (accumulate && out_dd) {
      dd_add_dd(a, b, out_dd[0], out_dd[1]);
      dd_add_dd(c, d, out_dd[2], out_dd[3]);
    }
    if (out_dd) {
      out_dd[0] = a;
      out_dd[1] = b;
      out_dd[2] = c;
      out_dd[3] = d;
    }
    if (out_val) {
      // 2^-h as an exact power of two, applied in up to two steps to stay in range
      const int e1 = h > 1000 ? 1000 : h;
      const int e2 = h - e1;
      const double s1 = __longlong_as_double((long long)(1023 - e1) << 52);
      const double s2 = __longlong_as_double((long long)(1023 - e2) << 52);
      out_val[0] = make_double2((a + b) * s1 * s2, (c + d) * s1 * s2);
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

size_t team_shared_bytes(bool fp32, int nd, int H, int P, bool staged) {
  (void)P;
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  const int ld = nd | 1;
  size_t b = (size_t)nd * ld * cs + (staged ? 0 : 6 * (size_t)(H + 2) * cs) + sizeof(TeamScratch);
  return (b + 15) & ~(size_t)15;
}

static size_t items_bytes_of(bool fp32, int Hl, int H) {
  const int n_items = Hl * (Hl - 1) / 2;
  size_t b = (size_t)item_table_bytes(n_items);
  b += (size_t)(H + 2) * (fp32 ? sizeof(float) : sizeof(double));
  return (b + 15) & ~(size_t)15;
}

size_t cta_shared_bytes(bool fp32, int team, int nd, int H, int Hl, int P, bool staged) {
  return items_bytes_of(fp32, Hl, H) + (size_t)teams_per_cta(team) * team_shared_bytes(fp32, nd, H, P, staged);
}

template <typename R, int G, bool S> static const void* kptr() { return (const void*)terms_kernel<R, G, S>; }

template <bool S> static const void* pick_kernel_s(bool fp32, int team) {
  if (fp32) {
    switch (team) {
      case 8: return kptr<float, 8, S>();
      case 16: return kptr<float, 16, S>();
      case 32: return kptr<float, 32, S>();
      case 64: return kptr<float, 64, S>();
      case 128: return kptr<float, 128, S>();
    }
  } else {
    switch (team) {
      case 8: return kptr<double, 8, S>();
      case 16: return kptr<double, 16, S>();
      case 32: return kptr<double, 32, S>();
      case 64: return kptr<double, 64, S>();
      case 128: return kptr<double, 128, S>();
    }
  }
  return nullptr;
}

static const void* pick_kernel(bool fp32, int team, bool staged) {
  return staged ? pick_kernel_s<true>(fp32, team) : pick_kernel_s<false>(fp32, team);
}

int max_ctas_per_sm(bool fp32, int team, size_t smem_bytes, bool staged) {
  const void* k = pick_kernel(fp32, team, staged);
  if (!k) return 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, cta_of(team), smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_terms(bool fp32, int team, const void* chat, const TermParams& p, int grid, double* partials,
                         cudaStream_t stream, void* stage, double* wstage, long long stage_ld) {
  const bool staged = stage != nullptr;
  const void* k = pick_kernel(fp32, team, staged);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = (size_t)p.items_bytes + (size_t)teams_per_cta(team) * p.team_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&chat, (void*)&p, (void*)&partials, (void*)&stage, (void*)&wstage, (void*)&stage_ld};
  return cudaLaunchKernel(k, dim3(grid), dim3(cta_of(team)), args, smem, stream);
}

// Series of the staged terms of a grouped launch, one term per thread, each with its own sieve's
// degree and border (column col belongs to chunk k_begin + col / tpc of sieve j, found in
// chunk_off): writes the weighted value (re, 0, im, 0) of every column to values, for a per-item
// reduction afterwards. Working arrays in shared memory for the largest degree h_max.
template <typename R>
__global__ void __launch_bounds__(kSeriesThreads)
series_values_kernel(const typename Cx<R>::t* __restrict__ stage, const double* __restrict__ wstage, long long count,
                     long long stage_ld, const BatchItem* __restrict__ jobs, int n_jobs,
                     const long long* __restrict__ chunk_off, long long k_begin, int tpc, int h_max,
                     double* __restrict__ values) {
  using V = typename Cx<R>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  V* SR = reinterpret_cast<V*>(smem);                 // (h_max + 2) x threads
  V* Sp = SR + (size_t)(h_max + 2) * kSeriesThreads;  // (h_max + 1) x threads
  V* Sz = Sp + (size_t)(h_max + 1) * kSeriesThreads;
  V* Se = Sz + (size_t)(h_max + 1) * kSeriesThreads;
  const int tid = threadIdx.x;
  const long long tt = (long long)blockIdx.x * kSeriesThreads + tid;
  if (tt >= count) return;
  const long long k = k_begin + tt / tpc;
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chunk_off[mid] <= k) {
      lo = mid;
    } else {
      hi = mid - 1;
    }
  }
  const int h = jobs[lo].p.h, bord = jobs[lo].p.bord;
  const V zero = cmake<V>((R)0, (R)0);
  double fr = 0.0, fi = 0.0;
  if (h >= 1 && h <= h_max) {
    auto A = [&](int m) -> V { return stage[(long long)(m - 1) * stage_ld + tt]; };
    auto C = [&](int m) -> V { return bord ? stage[(long long)(h + m - 1) * stage_ld + tt] : zero; };
#define SIDX(i) ((size_t)(i) * kSeriesThreads + tid)
    SR[SIDX(0)] = zero;
    SR[SIDX(1)] = C(1);
    Se[SIDX(0)] = cmake<V>((R)1, (R)0);
    for (int kk_ = 1; kk_ <= h; kk_++) {
      V sR = zero, sp = zero;
      for (int i = 1; i <= kk_; i++) {
        const V ai = A(i);
        if (bord) cmac(sR, ai, SR[SIDX(kk_ + 1 - i)]);
        if (i < kk_) cmac(sp, ai, Sp[SIDX(kk_ - i)]);
      }
      const V ck = C(kk_ + 1), ak = A(kk_);
      const R kk = (R)kk_;
      const V Rk = cmake<V>(ck.x - sR.x, ck.y - sR.y);
      const V pk = cmake<V>(-rfma(kk, ak.x, sp.x), -rfma(kk, ak.y, sp.y));
      const V zk = cmake<V>((R)0.5 * rfma(kk, Rk.x, pk.x), (R)0.5 * rfma(kk, Rk.y, pk.y));
      SR[SIDX(kk_ + 1)] = Rk;
      Sp[SIDX(kk_)] = pk;
      Sz[SIDX(kk_)] = zk;
      V se = zero;
      for (int j = 1; j <= kk_; j++) cmac(se, Sz[SIDX(j)], Se[SIDX(kk_ - j)]);
      const R ik = (R)1 / kk;
      Se[SIDX(kk_)] = cmake<V>(se.x * ik, se.y * ik);
    }
    const V f = Se[SIDX(h)];
#undef SIDX
    const double w = wstage[tt];
    fr = (double)f.x * w;
    fi = (double)f.y * w;
  }
  double* o = values + 4ll * tt;
  o[0] = fr;
  o[1] = 0.0;
  o[2] = fi;
  o[3] = 0.0;
}

// Batched mode (App. B.5): the staged terms of one parity class, one term per thread. The series
// runs to the class's largest degree h_max; outcome t (degree h_t) takes e_{h_t} with the weight
// coef[t][delta_self + A] (the self pair's binomial and sign for that outcome, 0 where the term
// does not occur). Per block and outcome the double-double sum goes to
// partials[4 * (t * gridDim.x + block)].
template <typename R>
__global__ void __launch_bounds__(kSeriesThreads)
series_modes_kernel(const typename Cx<R>::t* __restrict__ stage, const double* __restrict__ wstage, long long count,
                    long long stage_ld, int h_max, int bord, int n_out, const int* __restrict__ h_out,
                    const double* __restrict__ coef, int A, double* __restrict__ partials) {
  using V = typename Cx<R>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  V* SR = reinterpret_cast<V*>(smem);                 // (h_max + 2) x threads
  V* Sp = SR + (size_t)(h_max + 2) * kSeriesThreads;  // (h_max + 1) x threads
  V* Sz = Sp + (size_t)(h_max + 1) * kSeriesThreads;
  V* Se = Sz + (size_t)(h_max + 1) * kSeriesThreads;
  __shared__ double red[4][kSeriesThreads];
  const int tid = threadIdx.x;
  const long long tt = (long long)blockIdx.x * kSeriesThreads + tid;
  const V zero = cmake<V>((R)0, (R)0);
  const bool live = tt < count;
  double w = 0.0;
  int ds = 0;
#define SIDX(i) ((size_t)(i) * kSeriesThreads + tid)
  if (live) {
    const int h = h_max;
    auto A_ = [&](int m) -> V { return stage[(long long)(m - 1) * stage_ld + tt]; };
    auto C_ = [&](int m) -> V { return bord ? stage[(long long)(h + m - 1) * stage_ld + tt] : zero; };
    SR[SIDX(0)] = zero;
    SR[SIDX(1)] = C_(1);
    Se[SIDX(0)] = cmake<V>((R)1, (R)0);
    for (int k = 1; k <= h; k++) {
      V sR = zero, sp = zero;
      for (int i = 1; i <= k; i++) {
        const V ai = A_(i);
        if (bord) cmac(sR, ai, SR[SIDX(k + 1 - i)]);
        if (i < k) cmac(sp, ai, Sp[SIDX(k - i)]);
      }
      const V ck = C_(k + 1), ak = A_(k);
      const R kk = (R)k;
      const V Rk = cmake<V>(ck.x - sR.x, ck.y - sR.y);
      const V pk = cmake<V>(-rfma(kk, ak.x, sp.x), -rfma(kk, ak.y, sp.y));
      const V zk = cmake<V>((R)0.5 * rfma(kk, Rk.x, pk.x), (R)0.5 * rfma(kk, Rk.y, pk.y));
      SR[SIDX(k + 1)] = Rk;
      Sp[SIDX(k)] = pk;
      Sz[SIDX(k)] = zk;
      V se = zero;
      for (int j = 1; j <= k; j++) cmac(se, Sz[SIDX(j)], Se[SIDX(k - j)]);
      const R ik = (R)1 / kk;
      Se[SIDX(k)] = cmake<V>(se.x * ik, se.y * ik);
    }
    w = wstage[tt];
    ds = A > 0 ? (int)wstage[stage_ld + tt] : 0;  // without a self pair every delta' is 0
  }
  for (int t = 0; t < n_out; t++) {
    double fr = 0.0, fi = 0.0;
    if (live && ds >= -A && ds <= A) {
      const double c = coef[(size_t)t * (2 * A + 1) + (ds + A)];
      const int ht = h_out[t];
      if (c != 0.0 && ht >= 0 && ht <= h_max) {
        const V f = Se[SIDX(ht)];
        fr = (double)f.x * w * c;
        fi = (double)f.y * w * c;
      }
    }
    red[0][tid] = fr;
    red[1][tid] = 0.0;
    red[2][tid] = fi;
    red[3][tid] = 0.0;
    __syncthreads();
    for (int off = kSeriesThreads / 2; off >= 1; off >>= 1) {
      if (tid < off) {
        double a = red[0][tid], b = red[1][tid], cc = red[2][tid], d = red[3][tid];
        dd_add_dd(a, b, red[0][tid + off], red[1][tid + off]);
        dd_add_dd(cc, d, red[2][tid + off], red[3][tid + off]);
        red[0][tid] = a;
        red[1][tid] = b;
        red[2][tid] = cc;
        red[3][tid] = d;
      }
      __syncthreads();
    }
    if (tid == 0) {
      double* o = partials + 4ll * ((long long)t * gridDim.x + blockIdx.x);
      o[0] = red[0][0];
      o[1] = red[1][0];
      o[2] = red[2][0];
      o[3] = red[3][0];
    }
    __syncthreads();
  }
#undef SIDX
}

// Per segment s: double-double sum of entries seg_begin[s] .. seg_begin[s+1]-1 (4 doubles each),
// added to acc[4 * seg_item[s]] (one warp per segment; segments of one launch name distinct items).
__global__ void __launch_bounds__(128)
segment_reduce_kernel(const double* __restrict__ entries, const long long* __restrict__ seg_begin,
                      const int* __restrict__ seg_item, int n_seg, int plain, double* __restrict__ acc) {
  const int sg = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (sg >= n_seg) return;
  const long long b = seg_begin[sg], e = seg_begin[sg + 1];
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
  for (long long i = b + lane; i < e; i += 32) {
    if (plain) {
      rh += entries[4 * i + 0];
      ih += entries[4 * i + 2];
    } else {
      dd_add_dd(rh, rl, entries[4 * i + 0], entries[4 * i + 1]);
      dd_add_dd(ih, il, entries[4 * i + 2], entries[4 * i + 3]);
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const double a = __shfl_xor_sync(0xffffffffu, rh, off), bb = __shfl_xor_sync(0xffffffffu, rl, off);
    const double c = __shfl_xor_sync(0xffffffffu, ih, off), d = __shfl_xor_sync(0xffffffffu, il, off);
    dd_add_dd(rh, rl, a, bb);
    dd_add_dd(ih, il, c, d);
  }
  if (lane == 0) {
    double* o = acc + 4ll * seg_item[sg];
    double h0 = o[0], l0 = o[1], h1 = o[2], l1 = o[3];
    dd_add_dd(h0, l0, rh, rl);
    dd_add_dd(h1, l1, ih, il);
    o[0] = h0;
    o[1] = l0;
    o[2] = h1;
    o[3] = l1;
  }
}

// out[i] = 2^-h_i * acc[i] (h < 0: empty pattern, 1; h == INT_MAX: not computed, NaN).
__global__ void item_finalize_kernel(const double* __restrict__ acc, const int* __restrict__ item_h, int n_items,
                                     double2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  const int h = item_h[i];
  if (h < 0) {
    out[i] = make_double2(1.0, 0.0);
  } else if (h == 0x7fffffff) {
    out[i] = make_double2(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
  } else {
    const double s1 = __longlong_as_double((long long)(1023 - h) << 52);
    out[i] = make_double2((acc[4 * i] + acc[4 * i + 1]) * s1, (acc[4 * i + 2] + acc[4 * i + 3]) * s1);
  }
}

// Series of several loop-weight vectors on shared terms (App. B.5): thread (term tt, vector
// g = blockIdx.y). d_M's coefficients a_m (rows 0..h-1) are the term's; the loop sequence s_k of
// vector g (rows h + g h + k - 1, k <= kr = min(h, nd)) is R_{k+1} of the bordered form, continued
// past kr by the characteristic polynomial: R_{k+1} = -sum_{i=1..k} a_i R_{k+1-i}. Then Newton,
// z_k and e_k as in series_kernel; block partials at partials[4 (g blocks + block)].
__global__ void __launch_bounds__(kSeriesThreads)
series_multi_kernel(const double2* __restrict__ stage, const double* __restrict__ wstage, long long count,
                    long long stage_ld, int h, int kr, int plain, double* __restrict__ partials) {
  using V = double2;
  extern __shared__ __align__(16) unsigned char smem[];
  V* SR = reinterpret_cast<V*>(smem);             // (h + 2) x threads
  V* Sp = SR + (size_t)(h + 2) * kSeriesThreads;  // (h + 1) x threads
  V* Sz = Sp + (size_t)(h + 1) * kSeriesThreads;
  V* Se = Sz + (size_t)(h + 1) * kSeriesThreads;
  const int tid = threadIdx.x;
  const int g = blockIdx.y;
  const long long tt = (long long)blockIdx.x * kSeriesThreads + tid;
  const V zero = make_double2(0.0, 0.0);
  double fr = 0.0, fi = 0.0;
  if (tt < count) {
    auto A = [&](int m) -> V { return stage[(long long)(m - 1) * stage_ld + tt]; };
    auto S = [&](int k) -> V { return stage[(long long)(h + g * h + k - 1) * stage_ld + tt]; };
#define SIDX(i) ((size_t)(i) * kSeriesThreads + tid)
    SR[SIDX(0)] = zero;
    SR[SIDX(1)] = zero;  // R_1 = [t^1](d_M - d_K) = 0
    Se[SIDX(0)] = make_double2(1.0, 0.0);
    for (int k = 1; k <= h; k++) {
      V sR = zero, sp = zero;
      for (int i = 1; i <= k; i++) {
        const V ai = A(i);
        if (k > kr) cmac(sR, ai, SR[SIDX(k + 1 - i)]);
        if (i < k) cmac(sp, ai, Sp[SIDX(k - i)]);
      }
      const V ak = A(k);
      const double kk = (double)k;
      const V Rk = (k <= kr) ? S(k) : make_double2(-sR.x, -sR.y);
      const V pk = make_double2(-fma(kk, ak.x, sp.x), -fma(kk, ak.y, sp.y));
      const V zk = make_double2(0.5 * fma(kk, Rk.x, pk.x), 0.5 * fma(kk, Rk.y, pk.y));
      SR[SIDX(k + 1)] = Rk;
      Sp[SIDX(k)] = pk;
      Sz[SIDX(k)] = zk;
      V se = zero;
      for (int j = 1; j <= k; j++) cmac(se, Sz[SIDX(j)], Se[SIDX(k - j)]);
      const double ik = 1.0 / kk;
      Se[SIDX(k)] = make_double2(se.x * ik, se.y * ik);
    }
    const V f = Se[SIDX(h)];
#undef SIDX
    const double w = wstage[tt];
    fr = f.x * w;
    fi = f.y * w;
  }
  __shared__ double red[4][kSeriesThreads];
  red[0][tid] = fr;
  red[1][tid] = 0.0;
  red[2][tid] = fi;
  red[3][tid] = 0.0;
  __syncthreads();
  for (int off = kSeriesThreads / 2; off >= 1; off >>= 1) {
    if (tid < off) {
      double a = red[0][tid], b = red[1][tid], c = red[2][tid], d = red[3][tid];
      if (plain) {
        a += red[0][tid + off];
        c += red[2][tid + off];
      } else {
        dd_add_dd(a, b, red[0][tid + off], red[1][tid + off]);
        dd_add_dd(c, d, red[2][tid + off], red[3][tid + off]);
      }
      red[0][tid] = a;
      red[1][tid] = b;
      red[2][tid] = c;
      red[3][tid] = d;
    }
    __syncthreads();
  }
  if (tid == 0) {
    double* o = partials + 4ll * ((long long)g * gridDim.x + blockIdx.x);
    o[0] = red[0][0];
    o[1] = red[1][0];
    o[2] = red[2][0];
    o[3] = red[3][0];
  }
}

size_t series_shared_bytes(bool fp32, int h) {
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  return (size_t)(4 * h + 5) * kSeriesThreads * cs;
}

long long series_blocks(long long count) { return (count + kSeriesThreads - 1) / kSeriesThreads; }

cudaError_t launch_series(bool fp32, const void* stage, const double* wstage, long long count, long long stage_ld,
                          int h, int bord, int plain, double* partials, cudaStream_t stream) {
  const size_t smem = series_shared_bytes(fp32, h);
  const void* k = fp32 ? (const void*)series_kernel<float> : (const void*)series_kernel<double>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = series_blocks(count);
  void* args[] = {(void*)&stage, (void*)&wstage, (void*)&count, (void*)&stage_ld, (void*)&h,
                  (void*)&bord,  (void*)&plain,  (void*)&partials};
  return cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(kSeriesThreads), args, smem, stream);
}

cudaError_t launch_series_multi(const void* stage, const double* wstage, long long count, long long stage_ld, int h,
                                int kr, int ng, int plain, double* partials, cudaStream_t stream) {
  if (count <= 0 || ng <= 0) return cudaSuccess;
  const size_t smem = series_shared_bytes(false, h);
  const void* k = (const void*)series_multi_kernel;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = series_blocks(count);
  void* args[] = {(void*)&stage, (void*)&wstage, (void*)&count, (void*)&stage_ld,
                  (void*)&h,     (void*)&kr,     (void*)&plain, (void*)&partials};
  return cudaLaunchKernel(k, dim3((unsigned)blocks, (unsigned)ng), dim3(kSeriesThreads), args, smem, stream);
}

size_t multi_team_bytes(int nd, int H) {
  size_t b = team_shared_bytes(false, nd, H, 0, true) + ((sizeof(TeamScratch) + 15) & ~(size_t)15);
  b += 6 * (size_t)nd * sizeof(double2);  // u', Krylov and next Krylov vectors of two loop vectors
  return (b + 15) & ~(size_t)15;
}

cudaError_t launch_series_values(bool fp32, const void* stage, const double* wstage, long long count,
                                 long long stage_ld, const BatchItem* jobs, int n_jobs, const long long* chunk_off,
                                 long long k_begin, int tpc, int h_max, double* values, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = series_shared_bytes(fp32, h_max);
  const void* k = fp32 ? (const void*)series_values_kernel<float> : (const void*)series_values_kernel<double>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = series_blocks(count);
  void* args[] = {(void*)&stage,    (void*)&wstage,  (void*)&count, (void*)&stage_ld,
                  (void*)&jobs,     (void*)&n_jobs,  (void*)&chunk_off, (void*)&k_begin,
                  (void*)&tpc,      (void*)&h_max,   (void*)&values};
  return cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(kSeriesThreads), args, smem, stream);
}

cudaError_t launch_series_modes(bool fp32, const void* stage, const double* wstage, long long count,
                                long long stage_ld, int h_max, int bord, int n_out, const int* h_out,
                                const double* coef, int A, double* partials, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = series_shared_bytes(fp32, h_max);
  const void* k = fp32 ? (const void*)series_modes_kernel<float> : (const void*)series_modes_kernel<double>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long blocks = series_blocks(count);
  void* args[] = {(void*)&stage,  (void*)&wstage, (void*)&count, (void*)&stage_ld, (void*)&h_max, (void*)&bord,
                  (void*)&n_out,  (void*)&h_out,  (void*)&coef,  (void*)&A,        (void*)&partials};
  return cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(kSeriesThreads), args, smem, stream);
}

cudaError_t launch_segment_reduce(const double* entries, const long long* seg_begin, const int* seg_item, int n_seg,
                                  int plain, double* acc, cudaStream_t stream) {
  if (n_seg <= 0) return cudaSuccess;
  segment_reduce_kernel<<<(n_seg + 3) / 4, 128, 0, stream>>>(entries, seg_begin, seg_item, n_seg, plain, acc);
  return cudaGetLastError();
}

cudaError_t launch_item_finalize(const double* acc, const int* item_h, int n_items, double2* out,
                                 cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
  item_finalize_kernel<<<(n_items + 127) / 128, 128, 0, stream>>>(acc, item_h, n_items, out);
  return cudaGetLastError();
}

size_t cta_table_bytes(bool fp32, int Hl, int H) { return items_bytes_of(fp32, Hl, H); }

size_t grad_team_bytes(int nd, int H, int h, int bord, int team) {
  (void)h;
  (void)bord;
  const int ld = nd | 1, Hl = H < nd ? H : nd;
  // team_shared_bytes covers the working matrix, the series arrays and the team scratch (ending
  // 16-byte aligned, where the adjoint's buffers start): then S, Kb, q_bar and the phase-shared
  // region of the adjoint, and the pivot rows
  size_t b = team_shared_bytes(false, nd, H, 0, false);
  const int G = team == 8 || team == 16 || team == 64 ? team : 32;
  b += (2 * (size_t)nd * ld + (size_t)(nd + 1) * (Hl + 1) + (size_t)adjoint_union(nd, H, Hl, G)) * sizeof(double2);
  b += (size_t)nd * sizeof(int);
  return (b + 15) & ~(size_t)15;
}

template <int G> static const void* gptr() { return (const void*)grad_kernel<G>; }

// Teams of 8, 16 or 32 lanes inside one warp, or of two warps (64 lanes).
static const void* pick_grad(int team) {
  switch (team) {
    case 8: return gptr<8>();
    case 16: return gptr<16>();
    case 32: return gptr<32>();
    case 64: return gptr<64>();
  }
  return nullptr;
}

template <int G> static const void* ggptr() { return (const void*)grad_grouped_kernel<G>; }

static const void* pick_grad_grouped(int team) {
  switch (team) {
    case 8: return ggptr<8>();
    case 16: return ggptr<16>();
    case 32: return ggptr<32>();
    case 64: return ggptr<64>();
  }
  return nullptr;
}

int grad_ctas_per_sm(int team, size_t smem_bytes, bool grouped) {
  const void* k = grouped ? pick_grad_grouped(team) : pick_grad(team);
  if (!k) return 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, cta_of(team), smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_grad(int team, const double2* chat, const TermParams& p, int grid, double* partials, double2* gpart,
                        cudaStream_t stream) {
  const void* k = pick_grad(team);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = (size_t)p.items_bytes + (size_t)teams_per_cta(team) * p.team_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&chat, (void*)&p, (void*)&partials, (void*)&gpart};
  return cudaLaunchKernel(k, dim3(grid), dim3(cta_of(team)), args, smem, stream);
}

cudaError_t launch_grad_grouped(int team, const double2* chat_pool, const GradSieve* sieves, int n_sieves,
                                const long long* chunk_off, long long n_chunks, int n_full, int team_bytes,
                                int items_bytes, int grid, double* partials, double2* gpart, cudaStream_t stream) {
  const void* k = pick_grad_grouped(team);
  if (!k || n_sieves <= 0 || n_full <= 0 || n_full > kMaxDim) return cudaErrorInvalidValue;
  const size_t smem = (size_t)items_bytes + (size_t)teams_per_cta(team) * team_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&chat_pool, (void*)&sieves, (void*)&n_sieves, (void*)&chunk_off, (void*)&n_chunks,
                  (void*)&n_full, (void*)&team_bytes, (void*)&items_bytes, (void*)&partials, (void*)&gpart};
  return cudaLaunchKernel(k, dim3(grid), dim3(cta_of(team)), args, smem, stream);
}

cudaError_t launch_grad_reduce(const double2* gpart, long long teams, int len, int h, double2* out,
                               cudaStream_t stream) {
  if (len <= 0) return cudaSuccess;
  grad_reduce_kernel<<<(len + 127) / 128, 128, 0, stream>>>(gpart, teams, len, h, out);
  return cudaGetLastError();
}

cudaError_t launch_batch_gather(const double2* B, long long B_stride, const double2* gamma, long long gamma_stride,
                                int M, const BatchItem* items, int n_items, double2* chat_pool, float2* chat32_pool,
                                cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
  batch_gather_kernel<<<n_items, 256, 0, stream>>>(B, B_stride, gamma, gamma_stride, M, items, chat_pool, chat32_pool);
  return cudaGetLastError();
}

template <typename R, int G, bool S> static const void* gkptr() { return (const void*)grouped_terms_kernel<R, G, S>; }

template <bool S> static const void* pick_grouped_s(bool fp32, int team) {
  if (fp32) {
    switch (team) {
      case 8: return gkptr<float, 8, S>();
      case 16: return gkptr<float, 16, S>();
      case 32: return gkptr<float, 32, S>();
      case 64: return gkptr<float, 64, S>();
      case 128: return gkptr<float, 128, S>();
    }
  } else {
    switch (team) {
      case 8: return gkptr<double, 8, S>();
      case 16: return gkptr<double, 16, S>();
      case 32: return gkptr<double, 32, S>();
      case 64: return gkptr<double, 64, S>();
      case 128: return gkptr<double, 128, S>();
    }
  }
  return nullptr;
}

static const void* pick_grouped(bool fp32, int team, bool staged) {
  return staged ? pick_grouped_s<true>(fp32, team) : pick_grouped_s<false>(fp32, team);
}

int grouped_ctas_per_sm(bool fp32, int team, size_t smem_bytes, bool staged) {
  const void* k = pick_grouped(fp32, team, staged);
  if (!k) return 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, cta_of(team), smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_grouped_terms(bool fp32, int team, const void* chat_pool, const BatchItem* jobs, int n_jobs,
                                 const long long* chunk_off, long long k_begin, long long k_end, int grid,
                                 int rounds, unsigned long long tb, unsigned long long te, int team_bytes,
                                 int items_bytes, double* partials, void* stage, double* wstage,
                                 long long stage_ld, cudaStream_t stream, int per_chunk,
                                 unsigned long long* next_chunk) {
  const bool staged = stage != nullptr;
  const void* k = pick_grouped(fp32, team, staged);
  if (!k || grid <= 0 || n_jobs <= 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)items_bytes + (size_t)teams_per_cta(team) * team_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&chat_pool, (void*)&jobs,       (void*)&n_jobs,    (void*)&chunk_off,
                  (void*)&k_begin,   (void*)&k_end,      (void*)&rounds,    (void*)&tb,
                  (void*)&te,        (void*)&team_bytes, (void*)&items_bytes, (void*)&partials,
                  (void*)&stage,     (void*)&wstage,     (void*)&stage_ld, (void*)&per_chunk,
                  (void*)&next_chunk};
  return cudaLaunchKernel(k, dim3(grid), dim3(cta_of(team)), args, smem, stream);
}

cudaError_t launch_reduce(const double* partials, long long count, int h, double* out_dd, double2* out_val,
                          cudaStream_t stream, int accumulate) {
  reduce_kernel<<<1, 256, 0, stream>>>(partials, count, h, out_dd, out_val, accumulate);
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
