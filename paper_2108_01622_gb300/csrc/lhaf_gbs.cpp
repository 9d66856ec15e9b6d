// GBS pattern probability of a pure Gaussian state (arXiv:2108.01622, App. A, Eq. mixed_prob with
// the pure-state block form Eq. Adef): host linear algebra for the kernel matrix, then one loop
// hafnian on the GPU.
#include <cmath>
#include <complex>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_plan.h"

namespace {

using cd = std::complex<double>;
using lhafgpu::finite_c;

// In-place LU with partial pivoting of an n x n row-major matrix; returns false if singular.
// log|det| and the sign/phase of det are accumulated.
bool lu_factor(std::vector<cd>& a, int n, std::vector<int>& piv, cd& det_phase, double& log_abs_det) {
  piv.resize(n);
  det_phase = 1.0;
  log_abs_det = 0.0;
  for (int k = 0; k < n; k++) {
    int p = k;
    double best = std::abs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; i++) {
      const double v = std::abs(a[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (best == 0.0) return false;
    piv[k] = p;
    if (p != k) {
      for (int j = 0; j < n; j++) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
      det_phase = -det_phase;
    }
    const cd d = a[(size_t)k * n + k];
    log_abs_det += std::log(std::abs(d));
    det_phase *= d / std::abs(d);
    for (int i = k + 1; i < n; i++) {
      const cd l = a[(size_t)i * n + k] / d;
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; j++) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return true;
}

// Inverse from an LU factorisation (column by column).
void lu_inverse(const std::vector<cd>& lu, int n, const std::vector<int>& piv, std::vector<cd>& inv) {
  inv.assign((size_t)n * n, 0.0);
  std::vector<cd> x(n);
  for (int c = 0; c < n; c++) {
    for (int i = 0; i < n; i++) x[i] = (i == c) ? 1.0 : 0.0;
    for (int k = 0; k < n; k++)
      if (piv[k] != k) std::swap(x[k], x[piv[k]]);
    for (int i = 0; i < n; i++)
      for (int j = 0; j < i; j++) x[i] -= lu[(size_t)i * n + j] * x[j];
    for (int i = n - 1; i >= 0; i--) {
      for (int j = i + 1; j < n; j++) x[i] -= lu[(size_t)i * n + j] * x[j];
      x[i] /= lu[(size_t)i * n + i];
    }
    for (int i = 0; i < n; i++) inv[(size_t)i * n + c] = x[i];
  }
}

// Pure-state kernel (App. A, Eq. Adef) of squeezed vacuum (a -> a cosh r - a^dag sinh r), the
// interferometer a -> U a and the displacement alpha: the complex covariance sigma = S S^dag / 2,
// sigma_Q = sigma + I/2, B = first block of A = X (I - sigma_Q^-1) = -(sigma_Q^-1)[M:2M, 0:M],
// gamma = first M entries of alpha_full^dag sigma_Q^-1 and log P0 = -alpha_full^dag sigma_Q^-1
// alpha_full / 2 - log(det sigma_Q) / 2. False if sigma_Q is singular.
bool pure_state_kernel(int M, const lhaf_c128* U, const double* r, const std::vector<cd>& alpha,
                       std::vector<lhaf_c128>& B, std::vector<lhaf_c128>& gB, double& logP0) {
  const int M2 = 2 * M;
  // S = [[U, 0], [0, U*]] [[cosh r, -sinh r], [-sinh r, cosh r]]
  std::vector<cd> S((size_t)M2 * M2, 0.0);
  for (int i = 0; i < M; i++)
    for (int j = 0; j < M; j++) {
      const cd u(U[(size_t)i * M + j].re, U[(size_t)i * M + j].im);
      const double ch = std::cosh(r[j]), sh = std::sinh(r[j]);
      S[(size_t)i * M2 + j] = u * ch;
      S[(size_t)i * M2 + (M + j)] = -u * sh;
      S[(size_t)(M + i) * M2 + j] = -std::conj(u) * sh;
      S[(size_t)(M + i) * M2 + (M + j)] = std::conj(u) * ch;
    }
  std::vector<cd> sQ((size_t)M2 * M2, 0.0);
  for (int i = 0; i < M2; i++)
    for (int j = 0; j < M2; j++) {
      cd acc = 0.0;
      for (int k = 0; k < M2; k++) acc += S[(size_t)i * M2 + k] * std::conj(S[(size_t)j * M2 + k]);
      sQ[(size_t)i * M2 + j] = 0.5 * acc + (i == j ? 0.5 : 0.0);
    }
  std::vector<cd> lu = sQ, inv;
  std::vector<int> piv;
  cd phase;
  double logdet;
  if (!lu_factor(lu, M2, piv, phase, logdet)) return false;
  lu_inverse(lu, M2, piv, inv);
  B.resize((size_t)M * M);
  for (int i = 0; i < M; i++)
    for (int j = 0; j < M; j++) {
      const cd v = -inv[(size_t)(M + i) * M2 + j];
      B[(size_t)i * M + j] = {v.real(), v.imag()};
    }
  std::vector<cd> af(M2, 0.0);
  for (int i = 0; i < M; i++) {
    af[i] = alpha[i];
    af[M + i] = std::conj(alpha[i]);
  }
  gB.resize(M);
  cd quad = 0.0;
  for (int j = 0; j < M2; j++) {
    cd gj = 0.0;
    for (int i = 0; i < M2; i++) gj += std::conj(af[i]) * inv[(size_t)i * M2 + j];
    if (j < M) gB[j] = {gj.real(), gj.imag()};
    quad += gj * af[j];
  }
  logP0 = -0.5 * quad.real() - 0.5 * logdet;
  return true;
}


lhaf_status validate_pure_state(int M, const lhaf_c128* U, const double* r, const lhaf_c128* alpha) {
  for (int i = 0; i < M; i++) {
    if (!std::isfinite(r[i])) return LHAF_EINVAL;
    if (alpha && !finite_c(alpha[i])) return LHAF_EINVAL;
    for (int j = 0; j < M; j++)
      if (!finite_c(U[(size_t)i * M + j])) return LHAF_EINVAL;
  }
  return LHAF_OK;
}

}  // namespace

extern "C" lhaf_status gbs_pattern_prob(lhaf_ctx* ctx, int M, const lhaf_c128* U, const double* r,
                                        const lhaf_c128* alpha, const int32_t* n, uint32_t flags, double* prob,
                                        lhaf_c128* lhaf_B) {
  if (!ctx || M <= 0 || !U || !r || !n || !prob) return LHAF_EINVAL;
  if (flags & LHAF_DEVICE_PTRS) return LHAF_EINVAL;  // host inputs only
  for (int i = 0; i < M; i++)
    if (n[i] < 0) return LHAF_EINVAL;
  if (validate_pure_state(M, U, r, alpha) != LHAF_OK) return LHAF_EINVAL;
  std::vector<cd> a(M, 0.0);
  for (int i = 0; i < M; i++)
    if (alpha) a[i] = cd(alpha[i].re, alpha[i].im);
  std::vector<lhaf_c128> B, gB;
  double logP0 = 0.0;
  if (!pure_state_kernel(M, U, r, a, B, gB, logP0)) return LHAF_EINVAL;
  lhaf_c128 lh;
  const lhaf_status st = lhaf(ctx, M, B.data(), gB.data(), n, flags & ~LHAF_DEVICE_PTRS, &lh, nullptr);
  if (st != LHAF_OK) return st;
  double log_fact = 0.0;
  for (int i = 0; i < M; i++) log_fact += std::lgamma((double)n[i] + 1.0);
  const double mag2 = lh.re * lh.re + lh.im * lh.im;
  *prob = mag2 > 0.0 ? std::exp(logP0 - log_fact + std::log(mag2)) : 0.0;
  if (lhaf_B) *lhaf_B = lh;
  return LHAF_OK;
}

// One step of the chain-rule sampler (App. A.2): the photon number of `mode` conditioned on the
// photon numbers n of the modes sampled so far and the coherent amplitudes beta of the modes still
// in the coherent-state basis. The joint probability of (n with n_mode = k, beta) is that of the
// photon pattern n + k e_mode with zeros on the coherent modes for the state displaced by -beta
// (projecting on |beta> is counting no photons after the displacement D(-beta)), so it is
// proportional to |lhaf(B_{n + k e_mode}, gamma')|^2 / k! with gamma' the loop weights of the
// displacement alpha - beta (App. A.2); P0 and the other factorials cancel in the normalisation
// over k = 0..n_cut. The n_cut + 1 loop hafnians come from one batched-mode call (App. B.5), or
// from one batched call per outcome when its degree is above the batched mode's limit.
extern "C" lhaf_status gbs_chain_rule_step(lhaf_ctx* ctx, int M, const lhaf_c128* U, const double* r,
                                           const lhaf_c128* alpha, const lhaf_c128* beta, const int32_t* n,
                                           int mode, int n_cut, double u, uint32_t flags, double* cond,
                                           int32_t* n_drawn) {
  if (!ctx || M <= 0 || !U || !r || !n || !cond || mode < 0 || mode >= M || n_cut < 0) return LHAF_EINVAL;
  if (flags & ~(uint32_t)LHAF_PLAIN_ACCUM) return LHAF_EINVAL;
  for (int i = 0; i < M; i++)
    if (n[i] < 0 || (beta && !finite_c(beta[i]))) return LHAF_EINVAL;
  if (n[mode] != 0 || !std::isfinite(u)) return LHAF_EINVAL;
  if (validate_pure_state(M, U, r, alpha) != LHAF_OK) return LHAF_EINVAL;
  std::vector<cd> a(M, 0.0);
  for (int i = 0; i < M; i++) {
    if (alpha) a[i] = cd(alpha[i].re, alpha[i].im);
    if (beta && i != mode) a[i] -= cd(beta[i].re, beta[i].im);
  }
  std::vector<lhaf_c128> B, gB;
  double logP0 = 0.0;
  if (!pure_state_kernel(M, U, r, a, B, gB, logP0)) return LHAF_EINVAL;
  std::vector<lhaf_c128> lh(n_cut + 1);
  lhaf_status st = lhaf_batched_mode(ctx, M, B.data(), gB.data(), n, mode, n_cut, flags, lh.data(), nullptr);
  if (st == LHAF_ETOOBIG) {
    std::vector<int32_t> pats((size_t)(n_cut + 1) * M);
    std::vector<lhaf_c128> gs((size_t)(n_cut + 1) * M);
    for (int k = 0; k <= n_cut; k++)
      for (int i = 0; i < M; i++) {
        pats[(size_t)k * M + i] = i == mode ? k : n[i];
        gs[(size_t)k * M + i] = gB[i];
      }
    std::vector<lhaf_status> item(n_cut + 1, LHAF_OK);
    st = lhaf_batched(ctx, n_cut + 1, M, B.data(), gs.data(), pats.data(), flags, lh.data(), item.data(), nullptr);
    for (int k = 0; st == LHAF_OK && k <= n_cut; k++)
      if (item[k] != LHAF_OK) st = item[k];
  }
  if (st != LHAF_OK) return st;
  // weights |lhaf|^2 / k!, normalised through logarithms (the magnitudes span many decades)
  std::vector<double> lw(n_cut + 1, -INFINITY);
  double lmax = -INFINITY;
  for (int k = 0; k <= n_cut; k++) {
    const double m2 = lh[k].re * lh[k].re + lh[k].im * lh[k].im;
    if (!std::isfinite(m2)) return LHAF_EINVAL;
    if (m2 > 0.0) lw[k] = std::log(m2) - std::lgamma((double)k + 1.0);
    lmax = std::max(lmax, lw[k]);
  }
  double sum = 0.0;
  for (int k = 0; k <= n_cut; k++) {
    cond[k] = lmax > -INFINITY ? std::exp(lw[k] - lmax) : 0.0;
    sum += cond[k];
  }
  int drawn = -1;
  if (sum > 0.0) {
    for (int k = 0; k <= n_cut; k++) cond[k] /= sum;
    if (u >= 0.0 && u < 1.0) {
      double c = 0.0;
      drawn = n_cut;  // rounding of the cumulative sum: the last outcome with weight takes the rest
      while (drawn > 0 && cond[drawn] == 0.0) drawn--;
      for (int k = 0; k <= n_cut; k++) {
        c += cond[k];
        if (u < c) {
          drawn = k;
          break;
        }
      }
    }
  }
  if (n_drawn) *n_drawn = drawn;
  return LHAF_OK;
}

// GBS pattern probability of a general (mixed) Gaussian state (App. A, Eq. mixed_prob): the loop
// hafnian of the 2M x 2M matrix A = X (I - sigma_Q^-1) with index i and i + M both repeated n_i
// times (the repeated-pair sieve pairs them, App. B.2), loop weights gamma = alpha_full^dag
// sigma_Q^-1, P = Re(P0 lhaf(A_n)) / prod n_i!.
extern "C" lhaf_status gbs_pattern_prob_mixed(lhaf_ctx* ctx, int M, const lhaf_c128* sigma, const lhaf_c128* alpha,
                                              const int32_t* n, uint32_t flags, double* prob, lhaf_c128* lhaf_A) {
  if (!ctx || M <= 0 || !sigma || !n || !prob) return LHAF_EINVAL;
  if (flags & LHAF_DEVICE_PTRS) return LHAF_EINVAL;  // host inputs only
  const int M2 = 2 * M;
  for (int i = 0; i < M; i++) {
    if (n[i] < 0) return LHAF_EINVAL;
    if (alpha && !(std::isfinite(alpha[i].re) && std::isfinite(alpha[i].im))) return LHAF_EINVAL;
  }
  for (size_t e = 0; e < (size_t)M2 * M2; e++)
    if (!(std::isfinite(sigma[e].re) && std::isfinite(sigma[e].im))) return LHAF_EINVAL;
  // sigma_Q = sigma + I/2, its inverse and determinant
  std::vector<cd> lu((size_t)M2 * M2), inv;
  for (int i = 0; i < M2; i++)
    for (int j = 0; j < M2; j++) {
      const lhaf_c128 z = sigma[(size_t)i * M2 + j];
      lu[(size_t)i * M2 + j] = cd(z.re, z.im) + (i == j ? 0.5 : 0.0);
    }
  std::vector<int> piv;
  cd phase;
  double logdet;
  if (!lu_factor(lu, M2, piv, phase, logdet)) return LHAF_EINVAL;
  lu_inverse(lu, M2, piv, inv);
  // A = X (I - sigma_Q^-1): row i of A is row (i + M) mod 2M of I - sigma_Q^-1
  std::vector<lhaf_c128> A((size_t)M2 * M2);
  for (int i = 0; i < M2; i++) {
    const int r = (i + M) % M2;
    for (int j = 0; j < M2; j++) {
      const cd v = (r == j ? 1.0 : 0.0) - inv[(size_t)r * M2 + j];
      A[(size_t)i * M2 + j] = {v.real(), v.imag()};
    }
  }
  // gamma = alpha_full^dag sigma_Q^-1 and the quadratic form of P0
  std::vector<cd> af(M2, 0.0);
  for (int i = 0; i < M; i++) {
    const cd a = alpha ? cd(alpha[i].re, alpha[i].im) : cd(0.0);
    af[i] = a;
    af[M + i] = std::conj(a);
  }
  std::vector<lhaf_c128> g(M2);
  cd quad = 0.0;
  for (int j = 0; j < M2; j++) {
    cd gj = 0.0;
    for (int i = 0; i < M2; i++) gj += std::conj(af[i]) * inv[(size_t)i * M2 + j];
    g[j] = {gj.real(), gj.imag()};
    quad += gj * af[j];
  }
  // P0 = exp(-quad / 2) / sqrt(det sigma_Q), det = phase * exp(logdet)
  const cd P0 = std::exp(-0.5 * quad - 0.5 * logdet) / std::sqrt(phase);
  std::vector<int32_t> reps2(M2);
  for (int i = 0; i < M; i++) reps2[i] = reps2[M + i] = n[i];
  lhaf_c128 lh;
  const lhaf_status st = lhaf(ctx, M2, A.data(), g.data(), reps2.data(), flags & ~LHAF_DEVICE_PTRS, &lh, nullptr);
  if (st != LHAF_OK) return st;
  double log_fact = 0.0;
  for (int i = 0; i < M; i++) log_fact += std::lgamma((double)n[i] + 1.0);
  *prob = (P0 * cd(lh.re, lh.im)).real() * std::exp(-log_fact);
  if (lhaf_A) *lhaf_A = lh;
  return LHAF_OK;
}
