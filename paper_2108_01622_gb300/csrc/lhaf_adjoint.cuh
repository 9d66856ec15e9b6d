// Adjoint of one sieve term by reverse mode through the forward steps themselves (included by
// lhaf_terms.cu after its complex helpers; teams of 8, 16, 32 or 64 lanes).
//
// The forward term (lhaf_terms.cu, sieve_terms) reduces the bordered matrix K = [[0, u], [v^T, M]]
// (M = C X_delta', u = v X_delta') to Hessenberg form H by stabilised elementary similarities
// (step k: swap of indices r_k and k+1, then K' = L A L^-1 with L = I - l e_(k+1)^T,
// l_i = A[i][k] / A[k+1][k] for i >= k+2), runs La Budde's recurrence on the trailing blocks,
//   q_j(t) = (1 - t h_jj) q_(j+1)(t) - sum_(l>j) c_jl t^(l-j+1) q_(l+1)(t),
//   c_jl = h_jl prod_(r=j+1..l) h_(r,r-1),
// truncated at degree Hl, and finishes the series of Eq. ET_poly from a = q_1 (= det(I - t M))
// and c = q_1 - q_0 (q_0 = det(I - t K)). Reverse mode runs these steps backwards:
//  1. series: f = e_h gives e_bar, z_bar, then p_bar and R_bar, then a_bar and c_bar;
//  2. La Budde: q_bar_j for j = 0, 1, ... (each complete before it is used), h_bar_jj, c_bar_jl,
//     then h_bar from the products c_jl;
//  3. elimination, k = nd-3 .. 0, with the state before each step rebuilt from the state after it
//     (A = L^-1 K' L; the multipliers and pivots were kept): with K_bar' the adjoint of K',
//       l_bar = (K'^T K_bar'[:, k+1] - K_bar' K'[k+1, :]^T) restricted to i >= k+2,
//       A_bar = L^T K_bar' L^-T, then A_bar[i][k] += l_bar_i / p, A_bar[k+1][k] -= sum l_bar_i l_i / p,
//     and both state and adjoint are swapped back;
//  4. K_bar -> weight * (dC, dv) through the pair swap and delta' scaling of X_delta'.
// About three times the forward elimination's multiply-adds per term: O(n^3), against O(h n^3)
// for a matrix polynomial.
#pragma once

// FP64 instructions issue per warp whatever the number of active lanes (an SM retires about one
// FP64 warp instruction per 16 cycles), so every phase below spreads its multiply-adds evenly over
// the team's lanes: element-wise updates as flat item lists, sums through team_dots.
//
// Team-local storage of the adjoint (shared memory, complex of type V):
//   S  nd x ld : the Hessenberg form with the multipliers (copied before La Budde), then the state
//   Kb nd x ld : the adjoint of the state
//   Qb (nd + 1) x (Hl + 1) : q_bar_j in row j; then P_j(l - 1) for the product rule (nd x Hl)
//   U  adjoint_union entries, reused by phase: the series adjoints (6 x (H + 2)); then c_bar_jl at
//      [j * Hl + l - j - 1] (nd x Hl); then the multipliers l, their adjoints l_bar (nd each) and
//      the partial sums of team_dots (dots_slots(G))
//   piv nd ints : the pivot rows r_k
__host__ __device__ constexpr int dots_np(int G) { return 2 + (kMaxDim + G - 1) / G; }
__host__ __device__ constexpr int dots_slots(int G) { return G * dots_np(G); }
__host__ __device__ constexpr int adjoint_union(int nd, int H, int Hl, int G) {
  return (nd * Hl > 6 * (H + 2) ? (nd * Hl > 2 * nd + dots_slots(G) ? nd * Hl : 2 * nd + dots_slots(G))
                                : (6 * (H + 2) > 2 * nd + dots_slots(G) ? 6 * (H + 2) : 2 * nd + dots_slots(G)));
}

// 1/k for k <= kMaxDegree + 1, rounded once at compile time (the reverse series' step divisions
// become multiplications: an FP64 division is a sequence of several FP64 instructions)
struct InvTable {
  double v[kMaxDegree + 2];
};
__host__ __device__ constexpr InvTable make_inv_table() {
  InvTable t{};
  for (int k = 1; k < kMaxDegree + 2; k++) t.v[k] = 1.0 / (double)k;
  return t;
}
__constant__ InvTable c_inv = make_inv_table();

template <typename V>
__device__ __forceinline__ V q_fwd(const V* W, int ld, int nd, int l, int m) {
  // forward q_l[m] as La Budde left it: q_l[0] = 1, q_l[m] at W[l + m - 1][l] (1 <= m <= nd - l)
  if (m == 0) return cmake<V>(1, 0);
  if (l >= nd || m > nd - l) return cmake<V>(0, 0);
  return W[(l + m - 1) * ld + l];
}

// Sums out_o = sum_(q < len) x_oq y_oq for o < no (no <= kMaxDim), with the no * len products cut
// into equal contiguous ranges, one per lane. A lane's range meets at most dots_np(G) outputs; its
// partial sums go to part[lt * dots_np(G) + u]. After a team barrier, lane per output adds the
// partials of the lanes whose ranges met it and passes the sum to done(o, sum).
// prod(o, q, x, y) loads the factors of product q of output o.
template <typename R, int G, typename Prod, typename Done>
__device__ __forceinline__ void team_dots(int no, int len, typename Cx<R>::t* part, int lt, Prod prod, Done done) {
  using V = typename Cx<R>::t;
  constexpr int NP = dots_np(G);
  const int F = no * len;
  const int c = (F + G - 1) / G;
  int f = lt * c;
  const int fe = min(f + c, F);
  if (f < fe) {
    int o = f / len, q = f - o * len, u = 0;
    V s = cmake<V>((R)0, (R)0);
    for (; f < fe; f++) {
      V x, y;
      prod(o, q, x, y);
      cmac(s, x, y);
      if (++q == len) {
        part[lt * NP + u] = s;
        u++;
        s = cmake<V>((R)0, (R)0);
        q = 0;
        o++;
      }
    }
    if (q != 0) part[lt * NP + u] = s;
  }
  team_sync<G>();
  for (int oo = lt; oo < no; oo += G) {
    V t = cmake<V>((R)0, (R)0);
    if (len > 0) {
      const int l0 = (oo * len) / c, l1 = ((oo + 1) * len - 1) / c;
      t = part[l0 * NP + (oo - (l0 * c) / len)];
      for (int l = l0 + 1; l <= l1; l++) {
        const V e = part[l * NP + (oo - (l * c) / len)];
        t.x += e.x;
        t.y += e.y;
      }
    }
    done(oo, t);
  }
}

// Steps 1 and 2: from the forward series arrays (Sa = a, Sc = c, SR, Sp, Sz, Se), the La Budde state
// in W and the Hessenberg form in S, write H_bar into Kb (zeroed here).
template <typename R, int G>
__device__ __forceinline__ void adjoint_series_labudde(const typename Cx<R>::t* W, const typename Cx<R>::t* S,
                                                       typename Cx<R>::t* Kb, typename Cx<R>::t* Qb,
                                                       typename Cx<R>::t* U, const typename Cx<R>::t* Sa,
                                                       const typename Cx<R>::t* Sc, const typename Cx<R>::t* SR,
                                                       const typename Cx<R>::t* Sp, const typename Cx<R>::t* Sz,
                                                       const typename Cx<R>::t* Se, int nd, int ld, int bord, int h,
                                                       int H, int Hl, int lt) {
  using V = typename Cx<R>::t;
  const V zero = cmake<V>((R)0, (R)0);
  const int QW = Hl + 1;
  V* eb = U;
  V* zb = U + (H + 2);
  V* pb = zb + (H + 2);
  V* Rb = pb + (H + 2);
  V* ab = Rb + (H + 2);
  V* cb = ab + (H + 2);
  (void)Sc;
  for (int x = lt; x < 6 * (H + 2); x += G) U[x] = zero;
  for (int x = lt; x < nd * ld; x += G) Kb[x] = zero;
  for (int x = lt; x < (nd + 1) * QW; x += G) Qb[x] = zero;
  team_sync<G>();
  if (lt == 0) eb[h] = cmake<V>((R)1, (R)0);
  team_sync<G>();
  // e_m = (1/m) sum_(j=1..m) z_j e_(m-j), m = h .. 1
  for (int m = h; m >= 1; m--) {
    for (int j = 1 + lt; j <= m; j += G) {  // only the lanes with work form e_bar_m / m
      const V em = eb[m];
      const R im = (R)c_inv.v[m];
      const V t = cmake<V>(em.x * im, em.y * im);
      cmac(zb[j], t, Se[m - j]);
      V e2 = eb[m - j];
      cmac(e2, t, Sz[j]);
      eb[m - j] = e2;
    }
    team_sync<G>();
  }
  // z_k = (p_k + k R_(k+1)) / 2
  for (int k = 1 + lt; k <= h; k += G) {
    const V z = zb[k];
    pb[k] = cmake<V>((R)0.5 * z.x, (R)0.5 * z.y);
    Rb[k + 1] = cmake<V>((R)0.5 * (R)k * z.x, (R)0.5 * (R)k * z.y);
  }
  team_sync<G>();
  // p_k = -k a_k - sum_(i<k) a_i p_(k-i);  R_(k+1) = c_(k+1) - sum_(i<=k) a_i R_(k+1-i); k = h .. 1
  for (int k = h; k >= 1; k--) {
    const V pk = pb[k], rk = Rb[k + 1];
    for (int i = 1 + lt; i <= k; i += G) {
      V a = ab[i];
      if (i < k) {
        cmsub(a, pk, Sp[k - i]);
        V p2 = pb[k - i];
        cmsub(p2, pk, Sa[i]);
        pb[k - i] = p2;
      } else {
        a.x = rfma(-(R)k, pk.x, a.x);
        a.y = rfma(-(R)k, pk.y, a.y);
      }
      cmsub(a, rk, SR[k + 1 - i]);
      ab[i] = a;
      V r2 = Rb[k + 1 - i];
      cmsub(r2, rk, Sa[i]);
      Rb[k + 1 - i] = r2;
    }
    if (lt == 0) {
      V c = cb[k + 1];
      c.x += rk.x;
      c.y += rk.y;
      cb[k + 1] = c;
    }
    team_sync<G>();
  }
  if (lt == 0) {  // R_1 = c_1
    V c = cb[1];
    c.x += Rb[1].x;
    c.y += Rb[1].y;
    cb[1] = c;
  }
  team_sync<G>();
  // a = q_1, c = q_1 - q_0 (bordered);  a = q_0, c = 0 (no border)
  for (int m = lt; m <= Hl; m += G) {
    const V a = (m <= H + 1) ? ab[m] : zero, c = (m <= H + 1) ? cb[m] : zero;
    if (bord) {
      if (m <= nd - 1) Qb[QW + m] = cmake<V>(a.x + c.x, a.y + c.y);
      Qb[m] = cmake<V>(-c.x, -c.y);
    } else {
      Qb[m] = a;
    }
  }
  team_sync<G>();
  // La Budde backwards, j = 0, 1, ..., nd - 1: q_bar_j is complete when j is reached (only earlier
  // steps write row j). Step j pushes it into row j + 1 through the factor (1 - t h_jj) and into
  // rows l + 1 through q_bar_(l+1)[m'] -= c_jl q_bar_j[m' + l - j + 1], l = j+1 .. j+D (D = degj - 1,
  // m' = 0 .. D - 1 - x for l = j + 1 + x). The (x, m') items are flat: rows x and D - 1 - x share
  // a block of D + 1 items.
  for (int j = 0; j < nd; j++) {
    const int degj = min(Hl, nd - j), D = degj - 1;
    const V* qbj = Qb + j * QW;
    V* qb1 = Qb + (j + 1) * QW;
    const V hjj = S[j * ld + j];
    for (int m = lt; m <= degj; m += G) {
      V t = qb1[m];
      const V g = qbj[m];
      if (m <= nd - j - 1) {
        t.x += g.x;
        t.y += g.y;
      }
      if (m + 1 <= degj) cmsub(t, hjj, qbj[m + 1]);
      qb1[m] = t;
    }
    const int nitems = ((D + 1) >> 1) * (D + 1);
    for (int w = lt; w < nitems; w += G) {
      const int b = w / (D + 1), pos = w - b * (D + 1);
      const bool first = pos < D - b;
      const int x = first ? b : D - 1 - b;
      if (!first && x == b) continue;  // odd D: the middle row belongs to its block once
      const int mp = first ? pos : pos - (D - b);
      const int l = j + 1 + x;
      V* qbl = Qb + (l + 1) * QW;
      V t = qbl[mp];
      cmsub(t, W[j * ld + l], qbj[mp + x + 2]);
      qbl[mp] = t;
    }
    team_sync<G>();
  }
  // c_bar_jl = -sum_m' q_bar_j[m' + y + 2] q_(j+y+2)[m'] (y = l - j - 1 = 0 .. D - 1) and
  // h_bar_jj = the same sum at y = -1, m' = 0 .. D - y - 1: one item per (y, j), y-major so that
  // the items of a pass have nearly equal lengths
  for (int w = lt; w < Hl * nd; w += G) {
    const int yy = w / nd, j = w - yy * nd, y = yy - 1;
    const int D = min(Hl, nd - j) - 1;
    if (y >= D) continue;
    const V* qb = Qb + j * QW + y + 2;
    const int row = j + y + 2;
    V s = zero;
    for (int mp = 0; mp < D - y; mp++) cmac(s, qb[mp], q_fwd<V>(W, ld, nd, row, mp));
    s.x = flip(s.x);
    s.y = flip(s.y);
    if (y < 0) {
      Kb[j * ld + j] = s;
    } else {
      U[j * Hl + y] = s;
    }
  }
  team_sync<G>();
  // c_jl = h_jl P_j(l), P_j(l) = prod_(r=j+1..l) h_(r,r-1). Lane per row j: h_bar_jl += c_bar_jl P_j(l);
  // then, backwards over l, T_j(l) = c_bar_jl h_jl + h_(l+1,l) T_j(l+1) and the share of row j in
  // h_bar_(l,l-1), P_j(l-1) T_j(l), in place of c_bar_jl. Lane per r then adds the shares.
  V* Pp = Qb;  // q_bar is spent
  for (int j = lt; j < nd; j += G) {
    const int nl = min(Hl - 1, nd - 1 - j);
    V P = cmake<V>((R)1, (R)0);
    for (int x = 0; x < nl; x++) {
      const int l = j + 1 + x;
      Pp[j * Hl + x] = P;
      P = cmul(P, S[l * ld + l - 1]);
      V t = Kb[j * ld + l];
      cmac(t, U[j * Hl + x], P);
      Kb[j * ld + l] = t;
    }
    V T = zero;
    for (int x = nl - 1; x >= 0; x--) {
      const int l = j + 1 + x;
      V t = cmul(U[j * Hl + x], S[j * ld + l]);
      if (x < nl - 1) cmac(t, S[(l + 1) * ld + l], T);
      T = t;
      U[j * Hl + x] = cmul(Pp[j * Hl + x], T);
    }
  }
  team_sync<G>();
  for (int r = 1 + lt; r < nd; r += G) {
    V t = Kb[r * ld + r - 1];
    for (int j = max(0, r - Hl + 1); j < r; j++) {
      const V e = U[j * Hl + r - j - 1];
      t.x += e.x;
      t.y += e.y;
    }
    Kb[r * ld + r - 1] = t;
  }
  team_sync<G>();
}

// Step 3: the elimination backwards. S holds H with the multipliers of step k in column k below
// the subdiagonal (entries below the subdiagonal are zero in the state itself), piv the pivot
// rows. On return S is the input matrix K (up to rounding) and Kb its adjoint. U holds the step's
// multipliers l (U[0 .. nd)), their adjoints l_bar (U[nd .. 2 nd), with -sum l_bar l at index
// k + 1 and 1 / p at index k) and the partial sums of team_dots.
template <typename R, int G>
__device__ __forceinline__ void adjoint_elimination(typename Cx<R>::t* S, typename Cx<R>::t* Kb,
                                                    typename Cx<R>::t* U, const int* piv, int nd, int ld, int lt) {
  using V = typename Cx<R>::t;
  constexpr int SG = G < 32 ? G : 32;
  const V zero = cmake<V>((R)0, (R)0);
  V* Lv = U;
  V* Lb = U + nd;
  V* part = U + 2 * nd;
  for (int k = nd - 3; k >= 0; k--) {
    const int k1 = k + 1, r = piv[k], m = nd - k - 2;
    const V p = S[k1 * ld + k];
    // l_bar_a = (K'^T Kb'[:, k1])_a - (Kb' K'[k1, :]^T)_a for a = k+2 .. nd-1 (row k1 of the state
    // is zero left of column k): nd + nd - k products each
    V sl = zero;  // sum_a l_bar_a l_a (this lane's outputs)
    team_dots<R, G>(
        m, 2 * nd - k, part, lt,
        [&](int o, int q, V& x, V& y) {
          const int a = k + 2 + o, j = k + q - nd;
          const bool lo = q < nd;
          x = lo ? S[q * ld + a] : Kb[a * ld + j];
          y = lo ? Kb[q * ld + k1] : S[k1 * ld + j];
          const V nx = cmake<V>(flip(x.x), flip(x.y));
          x = lo ? x : nx;
        },
        [&](int o, V s) {
          const int a = k + 2 + o;
          const V la = S[a * ld + k];
          Lv[a] = la;
          Lb[a] = s;
          cmac(sl, s, la);
        });
    // lane 0 needs the sum; with two warps and at most 32 outputs (lanes 0 .. m-1) the second
    // warp holds nothing and skips its tree (the condition is uniform over the team)
    const bool one_warp = G > 32 && m <= 32;
    if (G <= 32 || lt < 32 || !one_warp) {
#pragma unroll
      for (int off = SG / 2; off >= 1; off >>= 1) {
        sl.x += __shfl_xor_sync(0xffffffffu, sl.x, off);
        sl.y += __shfl_xor_sync(0xffffffffu, sl.y, off);
      }
    }
    if constexpr (G > 32) {  // two warps: their sums meet in the (now free) partials
      if (!one_warp) {
        team_sync<G>();
        if ((lt & 31) == 0) part[lt >> 5] = sl;
        team_sync<G>();
        sl = part[0];
        for (int w = 1; w < G / 32; w++) {
          sl.x += part[w].x;
          sl.y += part[w].y;
        }
      }
    }
    if (lt == 0) {  // -sum l_bar l and, in the free slot k, 1 / p for the multiplier adjoints
      Lb[k1] = cmake<V>(flip(sl.x), flip(sl.y));
      Lb[k] = crecip(p);
    }
    team_sync<G>();
    // A = L^-1 K' on rows a >= k+2: A[a][k] = l_a p, A[a][j] = K'[a][j] + l_a K'[k1][j] (j >= k1);
    // item (a, column), column k first
    for (int w = lt; w < m * (m + 2); w += G) {
      const int o = w / (m + 2), cc = w - o * (m + 2);
      const int a = k + 2 + o, j = k + cc;
      V t = S[a * ld + j];
      const V y = cc == 0 ? p : S[k1 * ld + j];
      t = cc == 0 ? zero : t;
      cmac(t, Lv[a], y);
      S[a * ld + j] = t;
    }
    // A_bar = L^T Kb' on row k1: Kb[k1][j] -= sum_a l_a Kb'[a][j]
    team_dots<R, G>(
        nd, m, part, lt,
        [&](int o, int q, V& x, V& y) {
          const int a = k + 2 + q;
          x = Lv[a];
          y = Kb[a * ld + o];
        },
        [&](int o, V s) {
          V t = Kb[k1 * ld + o];
          t.x -= s.x;
          t.y -= s.y;
          Kb[k1 * ld + o] = t;
        });
    team_sync<G>();
    // A_bar = (L^T Kb') L^-T on columns a >= k+2 (Kb[i][a] += Kb[i][k1] l_a), then the multiplier
    // adjoints Kb[a][k] += l_bar_a / p (a >= k+2) and Kb[k1][k] -= (sum_a l_bar_a l_a) / p: one
    // flat list of multiply-adds
    const V ip = Lb[k];
    const int n3 = nd * m;
    for (int w = lt; w < n3 + m + 1; w += G) {
      const bool cl = w < n3;
      const int i = cl ? w / m : 0;
      const int a = cl ? k + 2 + (w - i * m) : k1 + (w - n3);
      V* pt = cl ? Kb + i * ld + a : Kb + a * ld + k;
      const V x = cl ? Kb[i * ld + k1] : Lb[a];
      const V la = Lv[a];
      const V y = cl ? la : ip;
      V t = *pt;
      cmac(t, x, y);
      *pt = t;
    }
    // A = (L^-1 K') L on column k1: A[i][k1] -= sum_a A[i][a] l_a
    team_dots<R, G>(
        nd, m, part, lt,
        [&](int o, int q, V& x, V& y) {
          const int a = k + 2 + q;
          x = S[o * ld + a];
          y = Lv[a];
        },
        [&](int o, V s) {
          V t = S[o * ld + k1];
          t.x -= s.x;
          t.y -= s.y;
          S[o * ld + k1] = t;
        });
    team_sync<G>();
    // swap indices r and k1 back: rows (state: columns >= k; adjoint: every column), then columns.
    // Run by every team whatever its r (a swap of k1 with itself changes nothing): the teams of a
    // warp meet at the same barriers.
    for (int j = lt; j < nd; j += G) {
      if (j >= k) {
        const V a = S[r * ld + j], b = S[k1 * ld + j];
        S[r * ld + j] = b;
        S[k1 * ld + j] = a;
      }
      const V c = Kb[r * ld + j], d = Kb[k1 * ld + j];
      Kb[r * ld + j] = d;
      Kb[k1 * ld + j] = c;
    }
    team_sync<G>();
    for (int i = lt; i < nd; i += G) {
      const V a = S[i * ld + r], b = S[i * ld + k1];
      S[i * ld + r] = b;
      S[i * ld + k1] = a;
      const V c = Kb[i * ld + r], d = Kb[i * ld + k1];
      Kb[i * ld + r] = d;
      Kb[i * ld + k1] = c;
    }
    team_sync<G>();
  }
}

// Step 4: Ga[a][b] += weight * dC[a][b], Gv[b] += weight * dv[b] from K_bar, with K[i][bord + s] =
// chat[i][bord + (s ^ 1)] * delta'(s) for slot s and the border column unscaled. With a slot map
// (a zero-digit group's sieve), slot s of this sieve is slot smap[s] of the full problem, whose
// n_full x n_full (then n_full) sums Ga (Gv) hold.
template <typename R, int G>
__device__ __forceinline__ void adjoint_accumulate(const typename Cx<R>::t* Kb, int nd, int ld, int bord,
                                                   const int* delta, double weight, typename Cx<R>::t* Ga,
                                                   typename Cx<R>::t* Gv, const int* smap, int n_full, int lt) {
  using V = typename Cx<R>::t;
  const int n = nd - bord;
  const R wr = (R)weight;
  for (int w = lt; w < n * n; w += G) {
    const int a = w / n, b = w - (w / n) * n;
    const R s = wr * (R)delta[b >> 1];
    const V g = Kb[(bord + a) * ld + bord + (b ^ 1)];
    const int o = smap ? smap[a] * n_full + smap[b] : w;
    V t = Ga[o];
    t.x = rfma(g.x, s, t.x);
    t.y = rfma(g.y, s, t.y);
    Ga[o] = t;
  }
  if (bord) {
    for (int b = lt; b < n; b += G) {
      const V g0 = Kb[bord + (b ^ 1)], g1 = Kb[(bord + b) * ld];
      const R dl = (R)delta[b >> 1];
      const int o = smap ? smap[b] : b;
      V t = Gv[o];
      t.x = rfma(wr, rfma(g0.x, dl, g1.x), t.x);
      t.y = rfma(wr, rfma(g0.y, dl, g1.y), t.y);
      Gv[o] = t;
    }
  }
  team_sync<G>();
}
