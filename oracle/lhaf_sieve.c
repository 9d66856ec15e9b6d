/* Test infrastructure only: a plain C restatement of the repeated-pair finite difference sieve
 * (App. B.2 and B.4, Eq. fdsieve, per-term function of Eq. ET_poly), used as the timed CPU
 * baseline and checked against the numpy oracle, brute force and closed forms. It shares nothing
 * with the GPU library. Complex FP64 (C99 double complex); sums in long double. Built with
 * LHAF_ORACLE_EXTENDED defined, the same steps run in long double complex (a 64-bit significand on
 * x86-64): an extended-precision reference of the same sum for ill-conditioned loop hafnians.
 *
 * One term, digit vector k (k_i in 0..eta_i), delta'_i = eta_i - 2 k_i, weight
 * prod_i C(eta_i, k_i) (-1)^k_i. With the reduced slot matrix C (n = 2H slots; slot i < H is the
 * left photon of pair i, slot H + i its right photon), the fixed pairing X swaps i and H + i and
 * X_delta' = X diag(delta'). Then, with M = C X_delta' and u = v X_delta',
 *   p_k = Tr(M^k)          from the characteristic polynomial of M (Householder Hessenberg form,
 *                          La Budde's recurrence, Newton's identities),
 *   s_k = u M^(k-1) v^T    by matrix-vector products,
 *   g_k = p_k / (2k) + s_k / 2,   f = [t^h] exp(sum_k g_k t^k),
 * and lhaf = 2^-h sum_k weight(k) f(k) over every digit vector (no halving).
 * Terms are numbered as itertools.product over the digit ranges (first digit slowest). */
#include <tgmath.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef LHAF_ORACLE_EXTENDED
typedef long double real_t;
typedef long double complex cplx;
#else
typedef double real_t;
typedef double complex cplx;
#endif

#define MAXN 64

/* Reduce A (n x n, row-major, overwritten) to upper Hessenberg form by Householder reflectors
 * H = I - 2 w w^H / (w^H w) applied as similarity transforms (A <- H A H). */
static void hessenberg_householder(int n, cplx* A) {
  cplx w[MAXN];
  for (int k = 0; k + 2 < n; k++) {
    real_t norm2 = 0.0;
    for (int i = k + 1; i < n; i++) norm2 += creal(A[i * n + k]) * creal(A[i * n + k]) +
                                             cimag(A[i * n + k]) * cimag(A[i * n + k]);
    if (norm2 == 0.0) continue;
    const real_t alpha = sqrt(norm2);
    const cplx x0 = A[(k + 1) * n + k];
    const real_t ax0 = cabs(x0);
    const cplx phase = ax0 > 0.0 ? x0 / ax0 : 1.0;
    for (int i = 0; i < n; i++) w[i] = 0.0;
    for (int i = k + 1; i < n; i++) w[i] = A[i * n + k];
    w[k + 1] += phase * alpha; /* w = x + e^{i arg x0} |x| e_1 */
    real_t ww = 0.0;
    for (int i = k + 1; i < n; i++) ww += creal(w[i]) * creal(w[i]) + cimag(w[i]) * cimag(w[i]);
    if (ww == 0.0) continue;
    const real_t beta = 2.0 / ww;
    /* A <- H A: rows k+1.. */
    for (int j = 0; j < n; j++) {
      cplx d = 0.0;
      for (int i = k + 1; i < n; i++) d += conj(w[i]) * A[i * n + j];
      d *= beta;
      for (int i = k + 1; i < n; i++) A[i * n + j] -= w[i] * d;
    }
    /* A <- A H: columns k+1.. */
    for (int i = 0; i < n; i++) {
      cplx d = 0.0;
      for (int j = k + 1; j < n; j++) d += A[i * n + j] * w[j];
      d *= beta;
      for (int j = k + 1; j < n; j++) A[i * n + j] -= d * conj(w[j]);
    }
  }
}

/* Characteristic polynomial det(t I - H) = t^n + c[1] t^(n-1) + ... + c[n] of an upper
 * Hessenberg H by La Budde's recurrence over the leading blocks:
 *   q_0 = 1,  q_i(t) = (t - h_ii) q_(i-1)(t) - sum_(m=1..i-1) h_(i-m,i) prod_(j=i-m+1..i) h_(j,j-1) q_(i-m-1)(t)
 * (1-based indices), with q_i stored by coefficients of t^(i-r), r = 0..i. */
static void labudde(int n, const cplx* H, cplx* c) {
  static _Thread_local cplx q[MAXN + 1][MAXN + 1];
  q[0][0] = 1.0;
  for (int i = 1; i <= n; i++) {
    for (int r = 0; r <= i; r++) q[i][r] = 0.0;
    const cplx hii = H[(i - 1) * n + (i - 1)];
    for (int r = 0; r < i; r++) {
      q[i][r] += q[i - 1][r];           /* t * q_(i-1) */
      q[i][r + 1] -= hii * q[i - 1][r]; /* -h_ii q_(i-1) */
    }
    cplx prod = 1.0;
    for (int m = 1; m <= i - 1; m++) {
      prod *= H[(i - m) * n + (i - m - 1)]; /* h_(i-m+1, i-m), 1-based */
      const cplx a = H[(i - m - 1) * n + (i - 1)] * prod;
      for (int r = 0; r <= i - m - 1; r++) q[i][r + m + 1] -= a * q[i - m - 1][r];
    }
  }
  for (int r = 0; r <= n; r++) c[r] = q[n][r];
}

/* f = [t^h] exp(sum_(k=1..h) g_k t^k): e_0 = 1, e_m = (1/m) sum_(k=1..m) k g_k e_(m-k). */
static cplx exp_coefficient(int h, const cplx* g) {
  cplx e[MAXN + 1];
  e[0] = 1.0;
  for (int m = 1; m <= h; m++) {
    cplx s = 0.0;
    for (int k = 1; k <= m; k++) s += (real_t)k * g[k] * e[m - k];
    e[m] = s / (real_t)m;
  }
  return e[h];
}

static real_t binom(int n, int k) {
  real_t c = 1.0;
  for (int i = 1; i <= k; i++) c = c * (real_t)(n - k + i) / (real_t)i;
  return c;
}

/* f of one digit vector (Eq. ET_poly with X replaced by X_delta'): n = 2H slots, C (n x n), v (n),
 * delta' per pair. hess != 0: power traces from the characteristic polynomial of the Householder
 * Hessenberg form; hess == 0: by repeated matrix products (the traces as written). */
static cplx term_f(int n, int H, const cplx* C, const cplx* v, const int* delta, int h, int hess) {
  cplx M[MAXN * MAXN], x[MAXN], y[MAXN], u[MAXN], g[MAXN + 1], p[MAXN + 1];
  for (int a = 0; a < n; a++)
    for (int j = 0; j < n; j++) {
      const int pj = j < H ? j + H : j - H, dj = delta[j < H ? j : j - H];
      M[a * n + j] = C[a * n + pj] * (real_t)dj;
    }
  for (int j = 0; j < n; j++) u[j] = v[j < H ? j + H : j - H] * (real_t)delta[j < H ? j : j - H];
  /* loop terms s_k = u M^(k-1) v^T, k = 1..h */
  cplx s[MAXN + 1];
  for (int i = 0; i < n; i++) x[i] = v[i];
  for (int k = 1; k <= h; k++) {
    cplx d = 0.0;
    for (int i = 0; i < n; i++) d += u[i] * x[i];
    s[k] = d;
    if (k < h) {
      for (int i = 0; i < n; i++) {
        cplx a = 0.0;
        for (int j = 0; j < n; j++) a += M[i * n + j] * x[j];
        y[i] = a;
      }
      for (int i = 0; i < n; i++) x[i] = y[i];
    }
  }
  /* power traces p_k = Tr(M^k), k = 1..h */
  if (hess) {
    cplx A[MAXN * MAXN], c[MAXN + 1];
    memcpy(A, M, sizeof(cplx) * n * n);
    hessenberg_householder(n, A);
    labudde(n, A, c);
    for (int k = 1; k <= h; k++) { /* Newton's identities */
      cplx acc = 0.0;
      const int jm = k - 1 < n ? k - 1 : n;
      for (int j = 1; j <= jm; j++) acc += c[j] * p[k - j];
      p[k] = -acc - (k <= n ? (real_t)k * c[k] : 0.0);
    }
  } else {
    cplx P[MAXN * MAXN], Q[MAXN * MAXN];
    memcpy(P, M, sizeof(cplx) * n * n);
    for (int k = 1; k <= h; k++) {
      cplx tr = 0.0;
      for (int i = 0; i < n; i++) tr += P[i * n + i];
      p[k] = tr;
      if (k < h) {
        for (int i = 0; i < n; i++)
          for (int j = 0; j < n; j++) {
            cplx a = 0.0;
            for (int l = 0; l < n; l++) a += P[i * n + l] * M[l * n + j];
            Q[i * n + j] = a;
          }
        memcpy(P, Q, sizeof(cplx) * n * n);
      }
    }
  }
  for (int k = 1; k <= h; k++) g[k] = p[k] / (2.0 * k) + s[k] / 2.0;
  return exp_coefficient(h, g);
}

/* Sum of weight * f over the digit vectors numbered [start, stop) (itertools.product order over
 * k_i in 0..eta_i, first digit slowest), unscaled. C: n x n complex as interleaved (re, im)
 * doubles, v: n complex, eta: H repeat counts (n = 2H). out: (re_hi, re_lo, im_hi, im_lo, sum of
 * |weight * f|), the last for the sum's condition number.
 * threads <= 0: OpenMP's default. Returns the number of threads used, or -1 on bad sizes. */
int oracle_sieve_sum(int H, const double* C_ri, const double* v_ri, const int* eta, int h, uint64_t start,
                     uint64_t stop, int hess, int threads, double* out) {
  const int n = 2 * H;
  if (H < 0 || n > MAXN || h < 0 || h > MAXN) return -1;
  cplx* C = (cplx*)malloc(sizeof(cplx) * (n * n > 0 ? n * n : 1));
  cplx* v = (cplx*)malloc(sizeof(cplx) * (n > 0 ? n : 1));
  if (!C || !v) {
    free(C);
    free(v);
    return -1;
  }
  for (int i = 0; i < n * n; i++) C[i] = C_ri[2 * i] + I * C_ri[2 * i + 1];
  for (int i = 0; i < n; i++) v[i] = v_ri[2 * i] + I * v_ri[2 * i + 1];
  long double sr = 0.0L, si = 0.0L, sa = 0.0L;
  int used = 1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel reduction(+ : sr, si, sa)
  {
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 16)
    for (long long t = (long long)start; t < (long long)stop; t++) {
      int delta[MAXN];
      real_t w = 1.0;
      unsigned long long r = (unsigned long long)t;
      for (int i = H - 1; i >= 0; i--) {
        const int k = (int)(r % (unsigned long long)(eta[i] + 1));
        r /= (unsigned long long)(eta[i] + 1);
        delta[i] = eta[i] - 2 * k;
        w *= binom(eta[i], k) * ((k & 1) ? -1.0 : 1.0);
      }
      const cplx f = (n == 0) ? 1.0 : term_f(n, H, C, v, delta, h, hess);
      sr += (long double)(w * creal(f));
      si += (long double)(w * cimag(f));
      sa += (long double)(fabs(w) * cabs(f));
    }
  }
  out[0] = (double)sr;
  out[1] = (double)(sr - (long double)out[0]);
  out[2] = (double)si;
  out[3] = (double)(si - (long double)out[2]);
  out[4] = (double)sa;
  free(C);
  free(v);
  return used;
}
