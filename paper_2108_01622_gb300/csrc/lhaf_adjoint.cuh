// Adjoint of one sieve term by reverse mode through the forward steps themselves (included by
// lhaf_terms.cu after its complex helpers; teams of at most one warp).
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

// Team-local storage of the adjoint (all in shared memory, complex of type V):
//   S  nd x ld : the Hessenberg form with the multipliers (copied before La Budde), then the state
//   Kb nd x ld : the adjoint of the state
//   Qb (Hl + 1) x (Hl + 1) : q_bar, a window of rows j .. j + Hl (row r in slot r mod (Hl + 1));
//   Cb nd x Hl : c_bar_jl at [j][l - j - 1]
//   Sb 6 x (H + 2) : e_bar, z_bar, p_bar, R_bar, a_bar, c_bar (series)
//   Lv, Lb nd each : the step's multipliers and their adjoints
//   piv nd ints : the pivot rows r_k
template <typename V>
__device__ __forceinline__ V q_fwd(const V* W, int ld, int nd, int l, int m) {
  // forward q_l[m] as La Budde left it: q_l[0] = 1, q_l[m] at W[l + m - 1][l] (1 <= m <= nd - l)
  if (m == 0) return cmake<V>(1, 0);
  if (l >= nd || m > nd - l) return cmake<V>(0, 0);
  return W[(l + m - 1) * ld + l];
}

// Steps 1 and 2: from the forward series arrays (Sa = a, Sc = c, SR, Sp, Sz, Se), the La Budde state
// in W and the Hessenberg form in S, write H_bar into Kb (zeroed here).
template <typename R, int G>
__device__ __forceinline__ void adjoint_series_labudde(const typename Cx<R>::t* W, const typename Cx<R>::t* S,
                                                       typename Cx<R>::t* Kb, typename Cx<R>::t* Qb,
                                                       typename Cx<R>::t* Cb, typename Cx<R>::t* Sb,
                                                       const typename Cx<R>::t* Sa, const typename Cx<R>::t* Sc,
                                                       const typename Cx<R>::t* SR, const typename Cx<R>::t* Sp,
                                                       const typename Cx<R>::t* Sz, const typename Cx<R>::t* Se,
                                                       int nd, int ld, int bord, int h, int H, int Hl, int lt) {
  using V = typename Cx<R>::t;
  const V zero = cmake<V>((R)0, (R)0);
  V* eb = Sb;
  V* zb = Sb + (H + 2);
  V* pb = zb + (H + 2);
  V* Rb = pb + (H + 2);
  V* ab = Rb + (H + 2);
  V* cb = ab + (H + 2);
  for (int x = lt; x < 6 * (H + 2); x += G) Sb[x] = zero;
  for (int x = lt; x < nd * ld; x += G) Kb[x] = zero;
  for (int x = lt; x < (Hl + 1) * (Hl + 1); x += G) Qb[x] = zero;
  team_sync<G>();
  if (lt == 0) eb[h] = cmake<V>((R)1, (R)0);
  team_sync<G>();
  // e_m = (1/m) sum_(j=1..m) z_j e_(m-j), m = h .. 1
  for (int m = h; m >= 1; m--) {
    const V em = eb[m];
    const V t = cmake<V>(em.x / (R)m, em.y / (R)m);
    for (int j = 1 + lt; j <= m; j += G) {
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
      if (m <= nd - 1) Qb[1 * (Hl + 1) + m] = cmake<V>(a.x + c.x, a.y + c.y);
      Qb[m] = cmake<V>(-c.x, -c.y);
    } else {
      Qb[m] = a;
    }
  }
  team_sync<G>();
  // La Budde backwards: j = 0, 1, ..., nd - 1 (q_bar_j is complete when j is reached; step j
  // writes rows j+1 .. j+Hl of the window, and row j's slot is cleared for row j + Hl + 1)
  const int QW = Hl + 1;
  for (int j = 0; j < nd; j++) {
    const int degj = min(Hl, nd - j);
    const int nl = min(Hl - 1, nd - 1 - j);  // l = j+1 .. j+nl, d = l - j + 1 <= Hl
    V* qbj = Qb + (j % QW) * QW;
    for (int x = lt; x <= nl; x += G) {
      if (x < nl) {
        const int l = j + 1 + x, d = x + 2;
        const V c = W[j * ld + l];  // c_jl (La Budde's table over H)
        V* qbl = Qb + ((l + 1) % QW) * QW;
        const int mmax = min(Hl - d, nd - l - 1);
        V s = zero;
        for (int mp = 0; mp <= mmax; mp++) {
          const V g = qbj[mp + d];
          cmac(s, g, q_fwd(W, ld, nd, l + 1, mp));
          V t = qbl[mp];
          cmsub(t, c, g);
          qbl[mp] = t;
        }
        Cb[j * Hl + x] = cmake<V>(-s.x, -s.y);
      } else {
        const V hjj = S[j * ld + j];
        V* qb1 = Qb + ((j + 1) % QW) * QW;
        V s = zero;
        for (int m = 0; m <= degj; m++) {
          const V g = qbj[m];
          V t = qb1[m];
          if (m <= nd - j - 1) {
            t.x += g.x;
            t.y += g.y;
          }
          if (m + 1 <= degj) cmsub(t, hjj, qbj[m + 1]);
          qb1[m] = t;
          if (m >= 1) cmac(s, g, q_fwd(W, ld, nd, j + 1, m - 1));
        }
        Kb[j * ld + j] = cmake<V>(-s.x, -s.y);
      }
    }
    team_sync<G>();
    for (int m = lt; m < QW; m += G) qbj[m] = zero;  // row j is done: its slot serves row j + QW
    team_sync<G>();
  }
  // c_jl = h_jl P_j(l), P_j(l) = prod_(r=j+1..l) h_(r,r-1): h_bar_jl += c_bar_jl P_j(l) (lane per
  // row j), and h_bar_(r,r-1) += sum over j < r <= l of c_bar_jl h_jl times the product without
  // h_(r,r-1) (lane per r, so that no two lanes add into one entry)
  for (int j = lt; j < nd; j += G) {
    const int nl = min(Hl - 1, nd - 1 - j);
    V P = cmake<V>((R)1, (R)0);
    for (int x = 0; x < nl; x++) {
      const int l = j + 1 + x;
      P = cmul(P, S[l * ld + l - 1]);
      V t = Kb[j * ld + l];
      cmac(t, Cb[j * Hl + x], P);
      Kb[j * ld + l] = t;
    }
  }
  team_sync<G>();
  for (int r = 1 + lt; r < nd; r += G) {
    V acc = zero;
    V pre = cmake<V>((R)1, (R)0);
    for (int j = r - 1; j >= 0 && r - j <= Hl - 1; j--) {
      if (j < r - 1) pre = cmul(pre, S[(j + 1) * ld + j]);
      V suf = cmake<V>((R)1, (R)0);
      const int lmax = min(j + Hl - 1, nd - 1);
      for (int l = r; l <= lmax; l++) {
        if (l > r) suf = cmul(suf, S[l * ld + l - 1]);
        cmac(acc, cmul(Cb[j * Hl + (l - j - 1)], S[j * ld + l]), cmul(pre, suf));
      }
    }
    V t = Kb[r * ld + r - 1];
    t.x += acc.x;
    t.y += acc.y;
    Kb[r * ld + r - 1] = t;
  }
  team_sync<G>();
}

// Step 3: the elimination backwards. S holds H with the multipliers of step k in column k below
// the subdiagonal (entries below the subdiagonal are zero in the state itself), piv the pivot
// rows. On return S is the input matrix K (up to rounding) and Kb its adjoint.
template <typename R, int G>
__device__ __forceinline__ void adjoint_elimination(typename Cx<R>::t* S, typename Cx<R>::t* Kb,
                                                    typename Cx<R>::t* Lv, typename Cx<R>::t* Lb, const int* piv,
                                                    int nd, int ld, int lt) {
  using V = typename Cx<R>::t;
  constexpr int SG = G < 32 ? G : 32;
  const V zero = cmake<V>((R)0, (R)0);
  for (int k = nd - 3; k >= 0; k--) {
    const int k1 = k + 1, r = piv[k];
    const V p = S[k1 * ld + k];
    // multipliers of step k, and l_bar_a = (K'^T Kb'[:, k1])_a - (Kb' K'[k1, :]^T)_a for a >= k+2
    // (row k1 of the state is zero left of column k)
    V sl = zero;  // sum_a l_bar_a l_a (this lane's share)
    for (int a = k + 2 + lt; a < nd; a += G) {
      const V la = S[a * ld + k];
      V s = zero;
      for (int i = 0; i < nd; i++) cmac(s, S[i * ld + a], Kb[i * ld + k1]);
      for (int j = k; j < nd; j++) cmsub(s, Kb[a * ld + j], S[k1 * ld + j]);
      Lv[a] = la;
      Lb[a] = s;
      cmac(sl, s, la);
    }
#pragma unroll
    for (int off = SG / 2; off >= 1; off >>= 1) {
      sl.x += __shfl_xor_sync(0xffffffffu, sl.x, off);
      sl.y += __shfl_xor_sync(0xffffffffu, sl.y, off);
    }
    team_sync<G>();
    // A_bar = L^T Kb' (row k1 -= sum_a l_a Kb'[a][:]) and A = L^-1 K' (rows a >= k+2 += l_a K'[k1][:],
    // column k set to l_a p), disjoint entries
    for (int x = lt; x < 2 * nd; x += G) {
      if (x < nd) {
        const int j = x;
        V t = Kb[k1 * ld + j];
        for (int a = k + 2; a < nd; a++) cmsub(t, Lv[a], Kb[a * ld + j]);
        Kb[k1 * ld + j] = t;
      } else {
        const int a = x - nd + k + 2;
        if (a < nd) {
          const V la = Lv[a];
          S[a * ld + k] = cmul(la, p);
          for (int j = k1; j < nd; j++) {
            V t = S[a * ld + j];
            cmac(t, la, S[k1 * ld + j]);
            S[a * ld + j] = t;
          }
        }
      }
    }
    team_sync<G>();
    // A_bar = (L^T Kb') L^-T (columns a >= k+2 += A_bar[:, k1] l_a), the multiplier adjoints
    // (A_bar[a][k] += l_bar_a / p, A_bar[k1][k] -= sum l_bar l / p), and A = (L^-1 K') L
    // (column k1 -= sum_a A[:, a] l_a)
    const V ip = crecip(p);
    for (int x = lt; x < 2 * nd; x += G) {
      if (x < nd) {
        const int i = x;
        const V ck = Kb[i * ld + k1];
        for (int a = k + 2; a < nd; a++) {
          V t = Kb[i * ld + a];
          cmac(t, ck, Lv[a]);
          Kb[i * ld + a] = t;
        }
        if (i >= k + 2) {
          V t = Kb[i * ld + k];
          cmac(t, Lb[i], ip);
          Kb[i * ld + k] = t;
        } else if (i == k1) {
          V t = Kb[i * ld + k];
          cmsub(t, sl, ip);
          Kb[i * ld + k] = t;
        }
      } else {
        const int i = x - nd;
        V t = S[i * ld + k1];
        for (int a = k + 2; a < nd; a++) cmsub(t, S[i * ld + a], Lv[a]);
        S[i * ld + k1] = t;
      }
    }
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
// chat[i][bord + (s ^ 1)] * delta'(s) for slot s and the border column unscaled.
template <typename R, int G>
__device__ __forceinline__ void adjoint_accumulate(const typename Cx<R>::t* Kb, int nd, int ld, int bord,
                                                   const int* delta, double weight, typename Cx<R>::t* Ga,
                                                   typename Cx<R>::t* Gv, int lt) {
  using V = typename Cx<R>::t;
  const int n = nd - bord;
  const R wr = (R)weight;
  for (int w = lt; w < n * n; w += G) {
    const int a = w / n, b = w - (w / n) * n;
    const R s = wr * (R)delta[b >> 1];
    const V g = Kb[(bord + a) * ld + bord + (b ^ 1)];
    V t = Ga[w];
    t.x = rfma(g.x, s, t.x);
    t.y = rfma(g.y, s, t.y);
    Ga[w] = t;
  }
  if (bord) {
    for (int b = lt; b < n; b += G) {
      const V g0 = Kb[bord + (b ^ 1)], g1 = Kb[(bord + b) * ld];
      const R dl = (R)delta[b >> 1];
      V t = Gv[b];
      t.x = rfma(wr, rfma(g0.x, dl, g1.x), t.x);
      t.y = rfma(wr, rfma(g0.y, dl, g1.y), t.y);
      Gv[b] = t;
    }
  }
  team_sync<G>();
}
