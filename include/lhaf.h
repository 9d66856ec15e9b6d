/*
 * lhaf.h -- C ABI of the GB300 loop-hafnian library (arXiv:2108.01622, "The Boundary for Quantum
 * Advantage in Gaussian Boson Sampling").
 *
 * The library evaluates the loop hafnian lhaf(B_n) of the N x N matrix B_n that is formed from a
 * complex symmetric M x M matrix B by repeating row/column i reps[i] times and putting the
 * repeated loop weights gamma on the diagonal (App. A, Eq. mixed_prob and the chain-rule variant
 * of App. A.2). It uses the finite difference sieve (App. B.4, Eq. fdsieve) over greedily matched
 * repeated pairs (App. B.2-B.3): prod_i (eta_i + 1) terms, halved by the sign symmetry of the
 * sieve. Every term runs on the GPU (FP64 by default); the signed sum is accumulated in
 * double-double.
 *
 * Conventions shared by all calls
 *   - Complex numbers are lhaf_c128 {re, im}: the layout of C99 double _Complex,
 *     std::complex<double> and torch.complex128.
 *   - B is M x M, row-major, symmetric; only entries with i <= j are read. B[m][m] is the weight of
 *     a pair of two photons in mode m; loops come from gamma.
 *   - gamma has M entries; NULL means gamma[m] = B[m][m] (the loop weights of the repeated matrix
 *     without diagonal replacement).
 *   - reps has M non-negative counts and is ALWAYS a host pointer (the host plans the pairing).
 *     reps == NULL means one photon in every mode. reps[i] = 0 drops mode i. N = sum(reps) may be 0
 *     (lhaf = 1) or odd (a pad index with loop weight 1 is added, App. B readings).
 *   - Host-pointer calls (flags without LHAF_DEVICE_PTRS) are synchronous: inputs are copied to the
 *     device, the result is copied back before the call returns.
 *   - With LHAF_DEVICE_PTRS, B, gamma and the outputs are device pointers on the context's
 *     device; the call is ordered on the context's stream and returns without synchronising.
 *   - Ownership: the caller owns every buffer; the library keeps no pointer after a call returns.
 *   - Errors are returned as lhaf_status codes; the library never exits or traps.
 */
#ifndef LHAF_GB300_H
#define LHAF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double re;
  double im;
} lhaf_c128;

typedef enum {
  LHAF_OK = 0,
  LHAF_EINVAL = 1,     /* bad argument: NULL required pointer, M <= 0, negative reps, non-finite */
  LHAF_ETOOBIG = 2,    /* working dimension above LHAF_MAX_DIM, degree above LHAF_MAX_DEGREE,
                          or more than 2^62 terms */
  LHAF_ECUDA = 3,      /* a CUDA runtime call failed (no device, launch error, ...) */
  LHAF_ETIMEOUT = 4,   /* reserved for device watchdogs */
  LHAF_ENOMEM = 5,     /* device or pinned-host allocation failed */
  LHAF_ECANCELLED = 6  /* reserved */
} lhaf_status;

/* Flags (bitwise OR). */
#define LHAF_DEVICE_PTRS 0x1u        /* B, gamma and outputs are device pointers, stream-ordered */
#define LHAF_FP32_TERMS 0x2u         /* per-term arithmetic in FP32 (accumulation stays in
                                        double-double), offered up to degree h = 18 (N <= 36
                                        photons) with a stated bound of 1e-2 relative error
                                        against FP64 (measured <= 1.2e-3 there; 2.7e-2 at
                                        N = 60): larger problems give LHAF_ETOOBIG */
#define LHAF_PLAIN_ACCUM 0x4u        /* accumulate the signed sum in plain FP64 instead of
                                        double-double (for accuracy comparisons) */
#define LHAF_NO_REPEAT_SPEEDUP 0x8u  /* pair photons one by one (all eta = 1): the sieve of the
                                        explicit duplicated-row matrix, 2^(N/2) terms */
#define LHAF_NO_LOOPS 0x10u          /* declare gamma == 0 on the occupied modes (skips the loop
                                        border); with host pointers this is detected by itself */
#define LHAF_BATCH_B_PER_ITEM 0x20u  /* lhaf_batched: B holds one M x M matrix per item */
#define LHAF_NO_ZERO_SPLIT 0x40u     /* evaluate the middle digits of even-eta pairs (delta' = 0) on
                                        the full working matrix instead of in zero-digit groups with
                                        those slots deleted (same sum; for comparisons) */
#define LHAF_ET 0x80u                /* lhaf, lhaf_range, lhaf_plan, lhaf_plan_groups,
                                        gbs_pattern_prob(_mixed): the eigenvalue-trace inclusion/
                                        exclusion sum (App. B.1 Eq. ET_loop, read with the sign
                                        (-1)^(h - |Z|); repeated pairs as in App. B.2) instead of the
                                        finite difference sieve, for accuracy comparisons (App. B.4,
                                        Fig. glynn_accuracy). Terms: every choice of kept pairs (at
                                        least one) and of z_q in 1..eta_q copies of each, prod
                                        (eta_q + 1) - 1 in all, on the shrunken matrix of the kept
                                        pairs' slots; numbered by the number of kept pairs, then
                                        by rank (lhaf_range uses this numbering; partials carry
                                        the factor 2^h, so lhaf_combine applies unchanged).
                                        Rejected (LHAF_EINVAL) by the batched calls, lhaf_grad
                                        and lhaf_noalloc. */

/* Compiled limits. */
#define LHAF_MAX_DIM 64      /* working dimension n_dim = 2 * pairs (+1 loop border) */
#define LHAF_MAX_DEGREE 256  /* h = ceil(N/2) */

typedef struct lhaf_ctx lhaf_ctx;

/* Per-call statistics (optional out-parameter). */
typedef struct {
  uint64_t terms;       /* sieve terms evaluated (after the sign-symmetry halving) */
  int32_t n_dim;        /* working matrix dimension: 2 * pairs, +1 when loops are present */
  int32_t h;            /* polynomial degree ceil(N/2) */
  int32_t pairs;        /* unique pairs after greedy matching (+1 pad pair when N is odd) */
  int32_t team;         /* GPU lanes that share one term */
  double kernel_ms;     /* device time of the term and reduction kernels (CUDA events) */
  double flops_model;   /* algorithmic real flops of this call: per term, the complex
                           multiply-adds of the elimination Hessenberg reduction, La Budde's
                           recurrence and the series, 8 flops each (lhaf_flops_per_term) */
  uint64_t h2d_bytes;   /* bytes this call copied host -> device (inputs, descriptors) */
  uint64_t d2h_bytes;   /* bytes this call copied device -> host (results) */
  int32_t launches;     /* CUDA kernels this call launched (tuning trials excluded) */
  int32_t term_launches; /* of those, launches of the sieve-term kernel (each bounded: see lhaf) */
} lhaf_stats;

/* Create a context on `device`. cuda_stream: a cudaStream_t to order work on (cudaStreamLegacy or
 * cudaStreamPerThread included), or NULL for a non-blocking stream the context creates and owns. Allocates the context's device workspace.
 * Returns LHAF_ECUDA if the device cannot be used, LHAF_ENOMEM on allocation failure. */
lhaf_status lhaf_ctx_create(lhaf_ctx** ctx, int device, void* cuda_stream);

/* Release the context and its workspace (synchronises its stream first). NULL is a no-op. */
void lhaf_ctx_destroy(lhaf_ctx* ctx);

/* Static description of a status code. */
const char* lhaf_strerror(lhaf_status status);

/* The failing CUDA call and CUDA's message of the last LHAF_ECUDA returned on this thread ("" if
 * none). Valid until the next call on this thread. */
const char* lhaf_last_error(void);

/* Plan only (host, no GPU): the greedy pairing of App. B.3 for `reps`, returning the number of
 * evaluated sieve terms after halving, the largest working dimension and the degree. `has_loops`
 * != 0 counts the loop border. Any output pointer may be NULL.
 * Evaluated terms: a pair with even eta has a middle digit (delta' = 0) whose two slot columns
 * vanish, so unless LHAF_NO_ZERO_SPLIT is given the sieve runs as zero-digit groups: for every
 * subset Z of the even pairs, Z at their middle digit with their slots deleted and the others
 * without it, each group halved by the sign symmetry on one of its own pairs. Terms are numbered
 * group after group (subsets in increasing bit order over the even pairs in pair order), which is
 * the numbering lhaf_range uses. */
lhaf_status lhaf_plan(int M, const int32_t* reps, uint32_t flags, int has_loops, uint64_t* terms,
                      int32_t* n_dim, int32_t* h, int32_t* pairs);

/* lhaf(B_n) (App. B.4 Eq. fdsieve with the repeated pairs of App. B.2-B.4).
 * out: one lhaf_c128 (host, or device with LHAF_DEVICE_PTRS). stats: host pointer or NULL.
 * Launches are bounded: every launch of the sieve-term kernel covers at most 2.5e11 model flops
 * (about a quarter second on GB300; the environment variable LHAF_LAUNCH_MFLOPS overrides, in
 * millions). Degrees up to 32 stage their term polynomials (at most 256 MB per launch) and finish
 * them one term per thread; above that the series is finished inside the team and the launch's
 * per-term partials are reduced in term order. So a long sum holds the GPU in short launches, and
 * the same range gives the same bits whichever CTA took which terms (for a given team size). */
lhaf_status lhaf(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                 const int32_t* reps, uint32_t flags, lhaf_c128* out, lhaf_stats* stats);

/* Number of zero-digit groups the sieve of `reps` runs as (0: no split, one sieve on the full
 * working matrix), with the same arguments as lhaf_plan (host only). */
lhaf_status lhaf_plan_groups(int M, const int32_t* reps, uint32_t flags, int has_loops, int32_t* groups);

/* Partial sieve sum over the evaluated-term index range [term_begin, term_end) (terms numbered
 * 0 .. terms-1 as reported by lhaf_plan). partial_dd receives 4 doubles (re_hi, re_lo, im_hi,
 * im_lo) of the UNSCALED double-double partial sum (host, or device with LHAF_DEVICE_PTRS).
 * Partials over disjoint ranges add; lhaf = 2^-h * (sum of partials over [0, terms)), see
 * lhaf_combine. This is the unit for sharding across GPUs and for checkpoint/resume. */
lhaf_status lhaf_range(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                       const int32_t* reps, uint32_t flags, uint64_t term_begin,
                       uint64_t term_end, double* partial_dd, lhaf_stats* stats);

/* Algorithmic real flops of one sieve term of this implementation for working dimension n_dim,
 * degree h and loop border flag `bordered` (8 per complex multiply-add of the elimination
 * Hessenberg reduction, La Budde's recurrence and the series recurrences). 0 for invalid sizes. */
double lhaf_flops_per_term(int n_dim, int h, int bordered);

/* Batched loop hafnians (the batch of conditional probabilities of one chain-rule step, App. A.2,
 * and the batching motivation of App. B.5): item i is lhaf(B_n) with pattern reps[i*M .. i*M+M-1].
 *   B      : one M x M matrix shared by all items, or batch x M x M with LHAF_BATCH_B_PER_ITEM.
 *   gamma  : batch x M loop weights (item i at gamma + i*M), or NULL for diag(B).
 *   reps   : HOST, batch x M.
 *   out    : batch lhaf_c128 (host, or device with LHAF_DEVICE_PTRS, like B and gamma).
 *   item_status : HOST, batch entries, or NULL: per-item LHAF_OK / LHAF_EINVAL / LHAF_ETOOBIG; a
 *            failed item's out is NaN and does not fail the call.
 *   stats  : terms = all sieve terms, n_dim / h = the largest, pairs = work units, team = lanes
 *            per term, kernel_ms = device time of the persistent launch and the reduction.
 * All items run in one persistent kernel over a queue of term ranges ordered longest first. */
lhaf_status lhaf_batched(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                         const int32_t* reps, uint32_t flags, lhaf_c128* out, lhaf_status* item_status,
                         lhaf_stats* stats);

/* Batched plan: lhaf_batched planned once for fixed patterns and replayed for new values of B and
 * gamma. Creation does the host planning of every item (greedy pairs, App. B.3), tunes the team
 * size on (B, gamma), sizes all buffers and captures the launches (slot-matrix gather, persistent
 * kernel, per-item reduction) in a CUDA graph; each exec copies the new B and gamma into the
 * plan's buffers, replays the graph on the context's stream and returns the values. The structure
 * may not depend on values: the loop border is present unless LHAF_NO_LOOPS, so items whose loop
 * weights are all zero cost what they would with loops (the result is the same).
 *   create: B, gamma, reps and flags as for lhaf_batched (B and gamma host, or device with
 *           LHAF_DEVICE_PTRS; they are only read during the call). gamma NULL fixes loops = diag(B)
 *           for every exec. The plan keeps a copy of reps. Errors: LHAF_EINVAL for bad arguments;
 *           per-item planning failures are reported by each exec's item_status, not here.
 *   exec  : B (same layout and size as at creation), gamma (NULL exactly when it was NULL at
 *           creation), out (batch lhaf_c128), item_status (HOST, batch entries, or NULL) and stats
 *           as for lhaf_batched; host or device pointers per the creation flags. Host-pointer execs
 *           are synchronous; device-pointer execs are stream-ordered. Execs of one plan must not
 *           overlap (they share its buffers); a plan is tied to its context.
 *   destroy: frees the plan (NULL is ignored); no exec of it may still be running. */
typedef struct lhaf_batch_plan lhaf_batch_plan;
lhaf_status lhaf_batched_plan_create(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                                     const int32_t* reps, uint32_t flags, lhaf_batch_plan** plan);
lhaf_status lhaf_batched_plan_exec(lhaf_batch_plan* plan, const lhaf_c128* B, const lhaf_c128* gamma,
                                   lhaf_c128* out, lhaf_status* item_status, lhaf_stats* stats);
void lhaf_batched_plan_destroy(lhaf_batch_plan* plan);

/* Batched mode of one chain-rule step (App. A.2; App. B.5): out[n] = lhaf(B_{reps + n e_mode}) for
 * n = 0..n_cut, where the batched mode has reps[mode] == 0. The fixed photons are paired greedily,
 * the batched mode's photons with themselves (floor(n/2) repeats) and an odd n's last one with the
 * fixed leftover photon or a pad index; per outcome parity one sieve runs over the fixed digits and
 * the self pair's delta' in -A..A (A = floor(n_max/2)), so each term's Hessenberg reduction and
 * characteristic polynomial serve every outcome (its series gives all degrees up to the largest).
 *   B, gamma, reps: HOST, as for lhaf() (gamma NULL: loops from diag(B)); out: HOST, n_cut + 1.
 *   The middle digits of the fixed pairs with even eta run as zero-digit groups (slots deleted,
 *   as in lhaf) unless LHAF_NO_ZERO_SPLIT is given.
 *   flags: LHAF_PLAIN_ACCUM, LHAF_NO_ZERO_SPLIT. Errors: LHAF_EINVAL for bad arguments or reps[mode] != 0;
 *   LHAF_ETOOBIG when ceil((N_fixed + n_cut)/2) exceeds 24 (the staged series limit) or the
 *   working dimension exceeds LHAF_MAX_DIM. Synchronous. */
lhaf_status lhaf_batched_mode(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                              int mode, int n_cut, uint32_t flags, lhaf_c128* out, lhaf_stats* stats);

/* Loop hafnians of one pattern for several loop-weight vectors (App. A.2 threshold sub-detectors,
 * App. B.5: only the diagonal of B_{n,beta} changes): out[g] = lhaf(B_n) with loops gamma_g. The
 * sieve's per-term Hessenberg reduction and characteristic polynomial of the couplings are shared;
 * each vector adds its loop sequence s_k = u M^(k-1) v^T from the Hessenberg form (O(h n^2)) and its
 * series.
 *   B: HOST M x M; gammas: HOST n_gamma x M (vector g at gammas + g*M); reps: HOST M;
 *   out: HOST n_gamma; stats: HOST or NULL. 1 <= n_gamma <= 256. flags: LHAF_PLAIN_ACCUM,
 *   LHAF_NO_REPEAT_SPEEDUP. Errors: LHAF_EINVAL for bad arguments (NULL, non-finite entries of the
 *   occupied modes, negative reps, other flags), LHAF_ETOOBIG when ceil(N/2) > 24 (the staged series
 *   limit) or the working dimension exceeds LHAF_MAX_DIM, LHAF_ECUDA / LHAF_ENOMEM as for lhaf(). The middle
 *   digits of even-eta pairs are evaluated on the full working matrix (no zero-digit groups); a
 *   pattern that has such digits with fewer than 16 vectors runs as lhaf_batched of the pattern
 *   repeated instead (the batch's zero-digit groups are worth more than sharing among few vectors;
 *   an item error is then returned as the call's status). Synchronous. */
lhaf_status lhaf_multi_gamma(lhaf_ctx* ctx, int M, const lhaf_c128* B, int n_gamma, const lhaf_c128* gammas,
                             const int32_t* reps, uint32_t flags, lhaf_c128* out, lhaf_stats* stats);

/* Value and gradient of lhaf(B_n) (the paper has no gradient; it follows from the definition, App.
 * B: the derivative of a matching sum with respect to one weight is the matching sum over the
 * remaining indices, e.g. d lhaf / d gamma_m = n_m lhaf(n - e_m)). Computed by a per-term adjoint
 * of the finite difference sieve on the GPU (FP64).
 *   value : HOST, lhaf(B_n).
 *   dB    : HOST M x M or NULL; dB[m][m'] = dB[m'][m] = d lhaf / d B_mm' with B symmetric (B_mm'
 *           and B_m'm one variable; the library reads i <= j only).
 *   dgamma: HOST M or NULL; d lhaf / d gamma_m. With gamma == NULL the loops are diag(B): their
 *           derivative is added to dB[m][m] and dgamma is not written.
 * The adjoint runs in reverse through the term's own steps (series, La Budde's recurrence, the
 * elimination). As in lhaf, the middle digits of even-eta pairs run as zero-digit groups on their
 * smaller matrices (at most 4096 groups; LHAF_NO_ZERO_SPLIT: every term on the full matrix).
 * flags: LHAF_PLAIN_ACCUM, LHAF_NO_ZERO_SPLIT, LHAF_NO_REPEAT_SPEEDUP. The environment variable
 * LHAF_GRAD_TEAM = 8, 16, 32 or 64 forces the lanes per term (default: the most resident warps).
 * Host pointers only (LHAF_DEVICE_PTRS, LHAF_FP32_TERMS and LHAF_ET give LHAF_EINVAL). */
lhaf_status lhaf_grad(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                      uint32_t flags, lhaf_c128* value, lhaf_c128* dB, lhaf_c128* dgamma);

/* lhaf_grad for a batch of outcomes of one state (the log-probability batches of a GBS training
 * step): item i uses reps[i * M ..] and gammas[i * M ..] (gammas NULL: loops from diag(B)) with the
 * shared M x M matrix B. All items' slot matrices go up in one copy, their adjoint launches and
 * reductions run back to back on the context's stream, and one synchronisation ends the call.
 *   values      : HOST, batch values.
 *   dB          : HOST batch x M x M or NULL (as lhaf_grad, item after item).
 *   dgamma      : HOST batch x M or NULL (written only when gammas is given).
 *   item_status : HOST batch statuses or NULL. With it the call returns LHAF_OK once the batch ran
 *                 and a failed item (bad counts or values, too large) has its status there and
 *                 zeros in its outputs; without it the first item error is returned.
 * Host pointers only (LHAF_DEVICE_PTRS and LHAF_FP32_TERMS give LHAF_EINVAL). */
lhaf_status lhaf_grad_batched(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B, const lhaf_c128* gammas,
                              const int32_t* reps, uint32_t flags, lhaf_c128* values, lhaf_c128* dB,
                              lhaf_c128* dgamma, lhaf_status* item_status);

/* GBS pattern probability of a pure Gaussian state (App. A, Eq. mixed_prob with the pure-state
 * block form Eq. Adef): squeezed vacuum in every mode (a -> a cosh r - a^dag sinh r), then the
 * interferometer a -> U a, then the displacement alpha. On the host: the complex covariance
 * sigma = S S^dag / 2, sigma_Q = sigma + I/2, B = first block of A = X (I - sigma_Q^-1),
 * gamma = first M entries of alpha_full^dag sigma_Q^-1, P0 = exp(-alpha_full^dag sigma_Q^-1
 * alpha_full / 2) / sqrt(det sigma_Q); on the GPU: lhaf(B_n). Result P = P0 |lhaf|^2 / prod n_i!.
 *   U: HOST M x M row-major; r: HOST M squeezing parameters; alpha: HOST M (NULL = no displacement);
 *   n: HOST M photon counts; prob: HOST double; lhaf_B: HOST, optional (the loop hafnian).
 * flags: LHAF_FP32_TERMS / LHAF_PLAIN_ACCUM / LHAF_NO_REPEAT_SPEEDUP as for lhaf(). */
lhaf_status gbs_pattern_prob(lhaf_ctx* ctx, int M, const lhaf_c128* U, const double* r, const lhaf_c128* alpha,
                             const int32_t* n, uint32_t flags, double* prob, lhaf_c128* lhaf_B);

/* GBS pattern probability of a general (mixed) Gaussian state (App. A, Eq. mixed_prob): with the
 * complex covariance sigma (2M x 2M in the basis (a_1..a_M, a_1^dag..a_M^dag), App. A) and the mean
 * alpha, sigma_Q = sigma + I/2, A = X (I - sigma_Q^-1) (2M x 2M), gamma = alpha_full^dag
 * sigma_Q^-1, P0 = exp(-alpha_full^dag sigma_Q^-1 alpha_full / 2) / sqrt(det sigma_Q), and
 * P = Re(P0 lhaf(A_n)) / prod n_i!, where A_n repeats index i and i + M n_i times each (the
 * repeated-pair sieve of App. B.2 over pairs of equal counts: prod (n_i + 1) terms, halved). This
 * covers lossy states exactly, without a pure-state decomposition.
 *   sigma: HOST 2M x 2M row-major; alpha: HOST M or NULL; n: HOST M; prob: HOST;
 *   lhaf_A: HOST, optional (the loop hafnian of A_n). flags as for lhaf() (host pointers; with
 *   LHAF_ET the paper's lhafmix inclusion/exclusion form). Errors: LHAF_EINVAL for NULL, negative
 *   counts, non-finite entries or a singular sigma_Q; otherwise those of lhaf(). */
lhaf_status gbs_pattern_prob_mixed(lhaf_ctx* ctx, int M, const lhaf_c128* sigma, const lhaf_c128* alpha,
                                   const int32_t* n, uint32_t flags, double* prob, lhaf_c128* lhaf_A);

/* One step of the chain-rule sampler (App. A.2) for the pure state of gbs_pattern_prob: the
 * distribution of the photon number of `mode` given the photon numbers n of the modes sampled so
 * far and the coherent amplitudes beta of the modes still in the coherent-state basis, under the
 * cutoff n_cut: cond[k] = P(n + k e_mode, beta) / sum_j P(n + j e_mode, beta), k = 0..n_cut, where
 * P(n + k e_mode, beta) is proportional to |lhaf(B_{n + k e_mode})|^2 / k! with the loop weights
 * gamma' of the displacement alpha - beta (App. A.2). The loop hafnians come from one
 * lhaf_batched_mode call (App. B.5), or one lhaf_batched call over the n_cut + 1 patterns when
 * ceil((N + n_cut)/2) is above its limit.
 *   U, r, alpha: HOST, as for gbs_pattern_prob (alpha NULL = no displacement);
 *   beta: HOST M or NULL (no coherent modes); beta[i] must be 0 for the modes already sampled in
 *     photon number (beta[mode] is ignored: this step replaces it);
 *   n: HOST M photon numbers (0 on coherent modes), n[mode] == 0;
 *   u: a uniform number in [0, 1) to draw the outcome with (its inverse cumulative distribution),
 *     or any value outside [0, 1) to draw nothing;
 *   cond: HOST n_cut + 1; n_drawn: HOST or NULL, the drawn photon number (-1 if none was drawn or
 *     every weight is 0, in which case cond is all zeros).
 * flags: LHAF_PLAIN_ACCUM only. Errors: LHAF_EINVAL for bad arguments; the errors of the
 * loop-hafnian calls. Synchronous. */
lhaf_status gbs_chain_rule_step(lhaf_ctx* ctx, int M, const lhaf_c128* U, const double* r, const lhaf_c128* alpha,
                                const lhaf_c128* beta, const int32_t* n, int mode, int n_cut, double u,
                                uint32_t flags, double* cond, int32_t* n_drawn);

/* Host-side double-double sum of `count` partials (4 doubles each, as from lhaf_range) scaled
 * by 2^-h (exact). */
lhaf_status lhaf_combine(int count, const double* partials_dd, int32_t h, lhaf_c128* out);

/* Allocation-free lhaf (no counterpart in the paper). For callers that cannot call cudaMalloc or
 * cudaFree: code where another allocator (a framework's caching allocator, a pre-reserved memory
 * pool) owns the device memory, or loops that must not take the implicit device synchronisation of
 * an allocation. Same result as lhaf() with LHAF_DEVICE_PTRS, without a context.
 *   device      : the GPU to run on (made current for the call, the previous device is restored).
 *   cuda_stream : cudaStream_t the work is ordered on (NULL = legacy default stream); the call
 *                 returns without synchronising.
 *   B, gamma    : DEVICE pointers as for lhaf() (gamma may be NULL); reps: HOST pointer.
 *   out         : DEVICE pointer to one lhaf_c128.
 *   flags       : LHAF_FP32_TERMS, LHAF_PLAIN_ACCUM, LHAF_NO_REPEAT_SPEEDUP, LHAF_NO_LOOPS.
 * Scratch: a fixed 224 KiB device array inside the library (slot matrix for working dimension
 * <= LHAF_MAX_DIM plus partial sums of at most 4096 GPU teams), held by every GPU that loads the
 * library until the process exits. Larger problems are rejected with LHAF_ETOOBIG; the number of
 * terms is not limited (teams loop over more terms). Every call made outside stream capture looks
 * up the array's device address (cudaGetSymbolAddress, so the address is found again after
 * cudaDeviceReset) and caches it per device; a call made while its stream is capturing uses the
 * cached address, so make the first call on each device before any stream capture. All calls share the one array and it keeps the last call's contents (nothing in
 * it needs to start at zero): calls that overlap on the GPU, e.g. on two streams, race and give
 * wrong results; order them on one stream or synchronise between them. */
lhaf_status lhaf_noalloc(int device, void* cuda_stream, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                         const int32_t* reps, uint32_t flags, lhaf_c128* out);

/* Measurement utility (no counterpart in the paper): FP64 fused multiply-add throughput of
 * `device` in GFLOP/s (2 flops per FMA), from independent FMA chains over every SM for a few tens
 * of milliseconds. The sieve kernels are bound by this rate; it is the roofline denominator. */
lhaf_status lhaf_fp64_probe(int device, double* gflops);

#ifdef __cplusplus
}
#endif

#endif /* LHAF_GB300_H */
