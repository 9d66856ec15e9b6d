// Internal declarations shared by the host planner/API and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lhafgpu {

constexpr int kMaxDim = 64;      // working dimension limit (slots + loop border)
constexpr int kMaxPairs = 32;    // pairs limit (kMaxDim / 2)
constexpr int kMaxDegree = 256;  // h limit

// Per-launch description of one loop hafnian's sieve (App. B.2-B.4), passed by value.
struct TermParams {
  int nd;        // working dimension (2 * P slots, + bord)
  int ld;        // leading dimension of the shared working matrix (odd, >= nd)
  int bord;      // 1 when the loop border (index 0) is present
  int h;         // degree of the coefficient taken: ceil(N/2)
  int H;         // series length: h + bord
  int Hl;        // La Budde truncation: min(H, nd)
  int P;         // pairs
  int hp;        // index of the pair whose digit is halved
  int hp_even;   // 1 when eta[hp] is even (its middle digit is counted once)
  int plain;     // 1: plain FP64 accumulation instead of double-double
  unsigned skip_mask;  // bit q: pair q's digits skip the middle one (k = eta/2) of a zero-digit group
  double wscale;       // constant weight factor of every term (1, or a zero-digit group's factor)
  int n_items;   // push-item table entries: Hl (Hl - 1) / 2
  int team_bytes;   // shared bytes per team
  int items_bytes;  // shared bytes for the item table + 1/k table
  int eta[kMaxPairs];
  int radix[kMaxPairs];
  unsigned long long t_begin, t_end;  // evaluated-term index range
  unsigned long long rounds;          // terms per team (uniform, last round may be idle)
  unsigned long long total_teams;
  unsigned long long t_lo;            // terms below t_lo are outside the range (weight 0)
  int stage_pad;                      // 1: stage out-of-range terms too, with weight 0
  int bq;                             // batched-mode self pair (its digit k gives delta' = bA - k), or -1
  int bA;                             // largest self-pair repeat of the batched mode
  // Eigenvalue-trace variant (App. B.1, B.2): et_P > 0 makes every term one choice of P = this
  // sieve's pair count kept pairs out of the et_P pairs of the full slot matrix (et_ndf x et_ndf,
  // at element offset et_off from this sieve's own), ranked through et_table (et_P + 1 squared
  // entries, W[i][k] = e_k(eta_0..eta_{i-1}) over the full pairs, whose counts are in eta[]).
  int et_P;
  int et_ndf;
  int pad3_;
  long long et_off;
  const unsigned long long* et_table;
  // Several loop-weight vectors on one sieve (App. B.5, staged, no loop border): ng > 0 stages,
  // besides d_M, the loop sequences s_k (k <= min(h, nd)) of each of the ng slot loop-weight
  // vectors at gv (ng x nd, double2 on the slots), in rows h + g h + k - 1.
  int ng;
  int pad4_;
  const void* gv;
};

static_assert(sizeof(TermParams) % 8 == 0, "TermParams is copied as 8-byte words");

// One sieve of a grouped launch: a loop hafnian's whole sieve or one of its zero-digit groups.
struct BatchItem {
  TermParams p;         // the sieve (t_end = its term count; the kernel sets the chunk range)
  long long chat_off;   // element offset of the item's slot matrix in the pool
  unsigned long long base;  // first term number of this sieve in its loop hafnian's numbering
  int src;              // index of the loop hafnian (its B and gamma) this sieve belongs to
  int pad;
  int slot_mode[kMaxDim];
};

// Launch the FP64 (fp32 = false) or FP32 term kernel. chat is the bordered slot matrix (nd x nd,
// row-major) in double2 (fp32 = false) or float2. Without `stage` every team finishes its terms
// and writes 4 doubles (its double-double partial) to partials. With `stage`, each term's
// characteristic-polynomial coefficients go to stage (coefficient-major, stage_ld terms per row,
// term index t - t_begin) and its weight to wstage; series_kernel finishes them.
cudaError_t launch_terms(bool fp32, int team, const void* chat, const TermParams& p, int grid,
                         double* partials, cudaStream_t stream, void* stage = nullptr,
                         double* wstage = nullptr, long long stage_ld = 0);

// One loop hafnian over several sieves (its zero-digit groups, `jobs`, slot matrices in chat_pool
// at jobs[j].chat_off): the terms are cut into chunks of teams_per_cta(team) terms that never
// straddle two sieves (job j owns chunks chunk_off[j] .. chunk_off[j+1]-1; its last chunk is
// padded). CTA c takes chunks k_begin + c + r * grid (r < rounds, below k_end), so the teams of a
// CTA always share one sieve. Terms outside [tb, te) of the loop hafnian's numbering (jobs[j].base
// + local index) and padding carry weight 0. With `stage`, chunk k's terms go to columns
// (k - k_begin) * teams_per_cta + team; without, each team writes its double-double partial:
// one per team over all its chunks, or (per_chunk) one per chunk and team at that column.
// With next_chunk (a zeroed device counter) CTAs take chunks k_begin + atomicAdd(next_chunk, 1)
// until k_end instead of the fixed grid-strided rounds.
cudaError_t launch_grouped_terms(bool fp32, int team, const void* chat_pool, const BatchItem* jobs, int n_jobs,
                                 const long long* chunk_off, long long k_begin, long long k_end, int grid,
                                 int rounds, unsigned long long tb, unsigned long long te, int team_bytes,
                                 int items_bytes, double* partials, void* stage, double* wstage,
                                 long long stage_ld, cudaStream_t stream, int per_chunk = 0,
                                 unsigned long long* next_chunk = nullptr);
int grouped_ctas_per_sm(bool fp32, int team, size_t smem_bytes, bool staged);
// Staged series of a grouped launch with each column's own degree and border (from its sieve):
// weighted values (re, 0, im, 0) per column into values. h_max bounds the degrees.
cudaError_t launch_series_values(bool fp32, const void* stage, const double* wstage, long long count,
                                 long long stage_ld, const BatchItem* jobs, int n_jobs, const long long* chunk_off,
                                 long long k_begin, int tpc, int h_max, double* values, cudaStream_t stream);
// Batched mode (App. B.5): series of count staged terms to degree h_max, then per outcome t the
// weight coef[t * (2A + 1) + delta_self + A] (delta_self staged in wstage[stage_ld + term]) times
// e_{h_out[t]}, summed per 64-term block into partials[4 * (t * blocks + block)].
cudaError_t launch_series_modes(bool fp32, const void* stage, const double* wstage, long long count,
                                long long stage_ld, int h_max, int bord, int n_out, const int* h_out,
                                const double* coef, int A, double* partials, cudaStream_t stream);
// Several loop-weight vectors on shared terms (TermParams::ng): series of count staged terms for
// each of ng vectors (grid y), partials[4 (g blocks + block)] with blocks = series_blocks(count).
cudaError_t launch_series_multi(const void* stage, const double* wstage, long long count, long long stage_ld, int h,
                                int kr, int ng, int plain, double* partials, cudaStream_t stream);
// Shared bytes per team of the staged FP64 term kernel with the loop-vector buffers of ng > 0.
size_t multi_team_bytes(int nd, int H);
// acc[4 * seg_item[s]] += double-double sum of entries seg_begin[s] .. seg_begin[s+1]-1.
cudaError_t launch_segment_reduce(const double* entries, const long long* seg_begin, const int* seg_item, int n_seg,
                                  int plain, double* acc, cudaStream_t stream);
// out[i] = 2^-item_h[i] * acc[i] (item_h < 0: 1; item_h == INT_MAX: NaN).
cudaError_t launch_item_finalize(const double* acc, const int* item_h, int n_items, double2* out,
                                 cudaStream_t stream);

// Shared bytes one CTA needs, and CTA size, for a team size.
int cta_threads(int team);
int teams_per_cta(int team);
size_t team_shared_bytes(bool fp32, int nd, int H, int P, bool staged = false);
size_t cta_shared_bytes(bool fp32, int team, int nd, int H, int Hl, int P, bool staged = false);
int max_ctas_per_sm(bool fp32, int team, size_t smem_bytes, bool staged = false);

// Staged series: count terms (one per thread), partials: 4 doubles per block.
constexpr int kStageMaxDegree = 24;
// One loop hafnian (lhaf, lhaf_range) stages its term polynomials up to this degree: the series
// then runs one term per thread instead of on a warp with shuffle reductions (series_kernel keeps
// (4h + 5) x 64 complex values in shared memory: 136 KB at h = 32).
constexpr int kStageMaxDegreeSingle = 32;
// FP32 per-term arithmetic is offered up to this degree (N <= 36 photons), where its stated error
// bound (1e-2 relative against FP64) holds with margin: measured on GB300 at most 1.2e-3 on
// GBS-shaped and block-diagonal instances up to N = 36, but up to 7.6e-2 at N = 42 and 2.7e-2 at
// N = 60. Larger problems with LHAF_FP32_TERMS are refused with LHAF_ETOOBIG.
constexpr int kFp32MaxDegree = 18;
size_t series_shared_bytes(bool fp32, int h);
long long series_blocks(long long count);
cudaError_t launch_series(bool fp32, const void* stage, const double* wstage, long long count,
                          long long stage_ld, int h, int bord, int plain, double* partials,
                          cudaStream_t stream);

// Double-double reduction of `count` partials (4 doubles each): out_dd (4 doubles, unscaled; with
// accumulate != 0 added to its previous content) and out_val (complex, scaled by 2^-h). Either
// output may be NULL.
cudaError_t launch_reduce(const double* partials, long long count, int h, double* out_dd,
                          double2* out_val, cudaStream_t stream, int accumulate = 0);

// Batched persistent kernel and its helpers.
size_t cta_table_bytes(bool fp32, int Hl, int H);
cudaError_t launch_batch_gather(const double2* B, long long B_stride, const double2* gamma,
                                long long gamma_stride, int M, const BatchItem* items, int n_items,
                                double2* chat_pool, float2* chat32_pool, cudaStream_t stream);

// Adjoint: shared bytes per team, occupancy, the value+gradient kernel and the cross-team sum.
size_t grad_team_bytes(int nd, int H, int h, int bord, int team);  // team: 8, 16, 32 or 64 lanes
int grad_ctas_per_sm(int team, size_t smem_bytes, bool grouped = false);
cudaError_t launch_grad(int team, const double2* chat, const TermParams& p, int grid, double* partials,
                        double2* gpart, cudaStream_t stream);

// One sieve of the adjoint over zero-digit groups: its term parameters (t_end = its term count),
// its slot matrix at chat_off in the pool, and the full problem's slot of each of its slots.
struct GradSieve {
  TermParams p;
  long long chat_off;
  int smap[kMaxDim];
};
static_assert(sizeof(GradSieve) % 8 == 0, "GradSieve is copied as 8-byte words");

// The adjoint over several sieves in one launch: chunks of teams_per_cta(team) terms of one sieve
// (sieve j owns chunks chunk_off[j] .. chunk_off[j+1]-1), CTA c taking chunks c, c + grid, ...;
// each team keeps its gradient sums in the full problem's n_full slots (gpart slice
// n_full^2 + n_full per team) and its dd value partial (4 doubles per team in partials).
cudaError_t launch_grad_grouped(int team, const double2* chat_pool, const GradSieve* sieves, int n_sieves,
                                const long long* chunk_off, long long n_chunks, int n_full, int team_bytes,
                                int items_bytes, int grid, double* partials, double2* gpart, cudaStream_t stream);
cudaError_t launch_grad_reduce(const double2* gpart, long long teams, int len, int h, double2* out,
                               cudaStream_t stream);

// Gather the bordered slot matrix from device B (M x M, upper triangle read) and gamma.
// slot_mode: modes of the 2P slots (-1 = pad). gamma may be NULL (diag(B) is used).
cudaError_t launch_gather(const double2* B, const double2* gamma, int M, const int* slot_mode_host,
                          int P, int bord, double2* chat, float2* chat32, cudaStream_t stream);

// Failed CUDA call: remember "what: CUDA message" for lhaf_last_error() and return LHAF_ECUDA (3).
int record_cuda(cudaError_t e, const char* what);
void record_message(const char* msg);

}  // namespace lhafgpu
