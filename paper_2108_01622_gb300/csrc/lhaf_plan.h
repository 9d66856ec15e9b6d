// Host planner for the repeated-pair finite difference sieve (arXiv:2108.01622, App. B.2-B.4).
#pragma once

#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "../../include/lhaf.h"

namespace lhafgpu {

// One loop hafnian's sieve plan.
//   pairs q = 0..P-1 with repeat counts eta[q] (greedy matching of App. B.3; a leftover photon of
//   an odd pattern is paired with a pad index of loop weight 1);
//   slots 2q (left photon of pair q) and 2q+1 (right photon) carry modes slot_mode[] (-1 = pad);
//   the working dimension is nd = 2P + bord, where bord = 1 adds the loop border index 0;
//   evaluated terms are the mixed-radix numbers over radix[q] (= eta[q] + 1 except the halved
//   digit of pair hp), T = prod radix.
// A zero-digit group (split_zero_digits) is a Plan too: skip[q] = 1 removes the middle digit
// (k = eta/2) from pair q's digits, and every term's weight carries the factor wscale.
struct Plan {
  int M = 0, N = 0, h = 0, H = 0, Hl = 0, bord = 0, P = 0, nd = 0;
  int hp = 0, hp_even = 0;
  std::vector<int> slot_mode, eta, radix, skip;
  std::vector<int> src_pair;  // a zero-digit group's pairs: their index in the plan it came from
  double wscale = 1.0;
  uint64_t T = 0;
};

lhaf_status build_plan(int M, const int32_t* reps, uint32_t flags, bool loops, Plan& pl);

// Zero-digit groups of a plan. The middle digit k = eta/2 of a pair with even eta gives
// delta' = 0: both slot columns of C X_delta' (and both loop entries) vanish, and the term equals
// the one of the matrix with those two slots deleted (every power trace and loop product only sees
// the remaining slots). Each subset Z of the even pairs is one group: pairs in Z sit at their
// middle digit (deleted slots, constant weight factor C(eta, eta/2) (-1)^(eta/2)), the other even
// pairs skip it, odd pairs take every digit. Every group is closed under delta' -> -delta', so each
// halves exactly on one of its pairs. A group with no pair left contributes nothing (f = 0 for
// h >= 1) and is dropped. Returns false (subs empty) when the plan has no even pair.
bool split_zero_digits(const Plan& pl, std::vector<Plan>& subs);

// Eigenvalue-trace form of a plan (App. B.1 Eq. ET_loop with the repeated pairs of App. B.2): the
// terms are the choices of kept pairs S (|S| = k >= 1) with z_q in 1..eta_q copies of each; the
// empty choice contributes nothing (f = 0 for h >= 1). One sieve per support size k = 1..P (subs[k-1]:
// the first k pairs' slots, nd = 2k + bord, T = e_k(eta), no halving, wscale = 2^h so that the
// common 2^-h scaling of the sieve sum gives the plain inclusion/exclusion sum); table receives
// W[i][k] = e_k(eta_0..eta_{i-1}) for i, k = 0..P, row-major (P + 1) x (P + 1). False when a count
// overflows 2^62.
bool split_support_sizes(const Plan& pl, std::vector<Plan>& subs, std::vector<unsigned long long>& table);

// Bordered slot matrix (nd x nd, row-major): [0][0] = 0; [0][1+s] = [1+s][0] = v_s (gamma of the
// slot's mode, 1 for the pad); [b+s][b+t] = B[mode(s)][mode(t)] (0 when either is the pad), with B
// read from its upper triangle.
void build_chat_host(const Plan& pl, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                     std::complex<double>* chat);

// Algorithmic real flops of one term of this implementation: 8 per complex multiply-add of the
// elimination reduction, La Budde's recurrence and the series recurrences.
double lhaf_model_flops_per_term(int nd, int h, int bord);

// Modelled FP64 lane utilisation (useful lane operations / issued lane slots) for team size G.
double model_lane_efficiency(int nd, int Hl, int h, int bord, int G);

// Both parts of a complex input finite (argument validation of the host entry points).
inline bool finite_c(const lhaf_c128& z) { return std::isfinite(z.re) && std::isfinite(z.im); }

inline void dd_add_dd_host(double& hi, double& lo, double bh, double bl) {
  const double s = hi + bh;
  const double bb = s - hi;
  double err = (hi - (s - bb)) + (bh - bb);
  err += lo + bl;
  const double t = s + err;
  lo = err - (t - s);
  hi = t;
}

}  // namespace lhafgpu
