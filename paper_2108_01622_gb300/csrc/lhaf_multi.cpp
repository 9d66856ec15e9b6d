// Loop hafnians of one pattern for several loop-weight vectors (arXiv:2108.01622, App. A.2 and App.
// B.5): the threshold sub-detectors of one mode change only the diagonal of B_{n,beta}, so the
// sieve's per-term Hessenberg reduction and characteristic polynomial of M = C X_delta' (the
// couplings, without loops) serve every vector. Per vector g and term the loop sequence
// s_k = u M^(k-1) v^T (v the vector's slot loop weights, u = v X_delta') follows from the Hessenberg
// form in O(h n^2) (the reduction's swaps and multipliers carry u and v into its basis), and its
// series gives f_g; the terms' weights are shared. Staged series only (h <= 24).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_ctx.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"

using namespace lhafgpu;

namespace {

constexpr int kMaxGammaVectors = 256;
// Below this many vectors a pattern with zero-digit groups runs as one batch of single loop
// hafnians instead: the batch deletes the delta' = 0 slots group by group, which the shared
// reduction here cannot, and on GB300 that is worth more than sharing the reduction among few
// vectors (the 40-photon collision pattern: the shared reduction ran 4 vectors at 0.94x the batch;
// from 16 vectors on it wins, 1.03x to 1.12x). The dispatch itself does no more host work than a
// plan: the batch checks the values.
constexpr int kMultiMinVectorsWithGroups = 16;

}  // namespace

extern "C" lhaf_status lhaf_multi_gamma(lhaf_ctx* ctx, int M, const lhaf_c128* B, int n_gamma,
                                        const lhaf_c128* gammas, const int32_t* reps, uint32_t flags, lhaf_c128* out,
                                        lhaf_stats* stats) {
  if (!ctx || M <= 0 || !B || !gammas || !reps || !out || n_gamma < 1 || n_gamma > kMaxGammaVectors)
    return LHAF_EINVAL;
  if (flags & ~(uint32_t)(LHAF_PLAIN_ACCUM | LHAF_NO_REPEAT_SPEEDUP)) return LHAF_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  for (int a = 0; a < M; a++)
    if (reps[a] < 0) return LHAF_EINVAL;
  Plan pl;
  lhaf_status st = build_plan(M, reps, flags, true, pl);
  if (st != LHAF_OK) return st;
  if ((pl.N + 1) / 2 > kStageMaxDegree) return LHAF_ETOOBIG;  // the staged series limit (either path)
  if (pl.N > 0 && n_gamma < kMultiMinVectorsWithGroups) {
    int even = 0;  // zero-digit groups exist: split_zero_digits' condition, without building them
    for (int q = 0; q < pl.P; q++) even += (pl.eta[q] >= 2 && pl.eta[q] % 2 == 0) ? 1 : 0;
    if (even >= 1 && even <= 20) {  // few vectors on a pattern with zero-digit groups: batch them (it checks the values)
      std::vector<int32_t> rr((size_t)n_gamma * M);
      for (int g = 0; g < n_gamma; g++) std::memcpy(rr.data() + (size_t)g * M, reps, sizeof(int32_t) * M);
      std::vector<lhaf_status> ist(n_gamma);
      st = lhaf_batched(ctx, n_gamma, M, B, gammas, rr.data(), flags, out, ist.data(), stats);
      if (st != LHAF_OK) return st;
      for (lhaf_status x : ist)
        if (x != LHAF_OK) return x;
      return LHAF_OK;
    }
  }
  for (int a = 0; a < M; a++) {
    if (reps[a] == 0) continue;
    for (int g = 0; g < n_gamma; g++)
      if (!finite_c(gammas[(size_t)g * M + a])) return LHAF_EINVAL;
    for (int b = 0; b < M; b++)
      if (reps[b] > 0 && !finite_c(B[(size_t)std::min(a, b) * M + std::max(a, b)])) return LHAF_EINVAL;
  }
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e = cudaSetDevice(ctx->device); e != cudaSuccess)
    return (lhaf_status)record_cuda(e, "cudaSetDevice");
  if (pl.N == 0) {  // empty pattern: lhaf = 1 for every vector
    for (int g = 0; g < n_gamma; g++) out[g] = {1.0, 0.0};
    return LHAF_OK;
  }
  // the couplings alone: no loop border (the loops enter through each vector's sequence)
  Plan pm = pl;
  pm.bord = 0;
  pm.nd = 2 * pm.P;
  pm.H = pm.h;
  pm.Hl = std::min(pm.H, pm.nd);
  if (pm.h > kStageMaxDegree) return LHAF_ETOOBIG;
  const int nd = pm.nd, h = pm.h, ng = n_gamma;
  const int rows = h * (1 + ng);

  BatchWork& w = ctx->bw;
  cudaStream_t s = ctx->stream;
  if (w.uploaded) {
    if (const cudaError_t e = cudaEventSynchronize(w.uploaded); e != cudaSuccess)
      return (lhaf_status)record_cuda(e, "cudaEventSynchronize");
  } else if (cudaEventCreateWithFlags(&w.uploaded, cudaEventDisableTiming) != cudaSuccess) {
    w.uploaded = nullptr;
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventCreate");
  }
  const size_t gv_bytes = sizeof(double2) * (size_t)ng * nd;
  if (!w.in_gamma.reserve(gv_bytes) || !w.h_in.reserve(gv_bytes) || !w.acc.reserve(sizeof(double) * 4 * ng) ||
      !w.out.reserve(sizeof(double2) * ng) || !w.h_out.reserve(sizeof(double2) * ng) ||
      !w.item_h.reserve(sizeof(int) * ng) || !w.h_item_h.reserve(sizeof(int) * ng))
    return LHAF_ENOMEM;
  // slot loop weights of every vector (the pad slot of an odd pattern has loop weight 1)
  double2* hv = static_cast<double2*>(w.h_in.p);
  for (int g = 0; g < ng; g++)
    for (int q = 0; q < nd; q++) {
      const int m = pm.slot_mode[q];
      const lhaf_c128 z = m >= 0 ? gammas[(size_t)g * M + m] : lhaf_c128{1.0, 0.0};
      hv[(size_t)g * nd + q] = make_double2(z.re, z.im);
    }
  int* hh = static_cast<int*>(w.h_item_h.p);
  for (int g = 0; g < ng; g++) hh[g] = h;
  build_chat_host(pm, M, B, nullptr, (std::complex<double>*)ctx->h_chat);
  uint64_t h2d = gv_bytes + sizeof(int) * (uint64_t)ng + sizeof(double2) * (uint64_t)nd * nd;
  if (cudaMemcpyAsync(w.in_gamma.p, hv, gv_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(w.item_h.p, hh, sizeof(int) * ng, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(ctx->d_chat, ctx->h_chat, sizeof(double2) * nd * nd, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(w.acc.p, 0, sizeof(double) * 4 * ng, s) != cudaSuccess ||
      cudaEventRecord(w.uploaded, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "multi-vector setup");
  // staging: d_M rows and every vector's loop sequence per term
  uint64_t cap = ((size_t)256 << 20) / ((size_t)rows * sizeof(double2));
  cap = std::min<uint64_t>(cap, (uint64_t)ctx->partial_cap * 64 / (uint64_t)ng);
  cap = std::min<uint64_t>(cap, std::max<uint64_t>(pl.T, 64));
  cap = std::max<uint64_t>(cap, 64);
  if (!ensure_stage(ctx, (size_t)rows * sizeof(double2) * cap, cap)) return LHAF_ENOMEM;
  if (!w.entries.reserve(4 * sizeof(double) * (size_t)ng * (size_t)series_blocks((long long)cap)))
    return LHAF_ENOMEM;
  // team: 8 lanes up to working dimension 32, else 16 (the loop sequences reduce across one
  // warp's lanes, so teams stay within a warp); a larger team if the CTA does not fit
  const size_t tb = multi_team_bytes(nd, pm.H);
  int team = 0, occ = 0;
  for (int g : {8, 16, 32}) {
    if (g == 8 && nd > 32) continue;
    TermParams q;
    fill_params(pm, false, true, g, flags, q);
    const size_t smem = (size_t)q.items_bytes + (size_t)teams_per_cta(g) * tb;
    if (smem > 227 * 1024) continue;
    const int o = max_ctas_per_sm(false, g, smem, true);
    if (o <= 0) continue;
    team = g;
    occ = o;
    break;
  }
  if (team == 0) return LHAF_ETOOBIG;
  occ = ctas_per_sm_override(occ);
  TermParams p;
  fill_params(pm, false, true, team, flags, p);
  p.team_bytes = (int)tb;
  p.ng = ng;
  p.gv = w.in_gamma.p;
  const int tpc = teams_per_cta(team);
  const uint64_t max_ctas = (uint64_t)ctx->sms * (uint64_t)std::max(occ, 1);
  const uint64_t T = pl.T;
  const int kr = std::min(h, nd);
  // per launch: ng segments of `blocks` partials each, one per vector
  if (!w.h_seg_begin.reserve(sizeof(long long) * (ng + 1)) || !w.seg_begin.reserve(sizeof(long long) * (ng + 1)) ||
      !w.h_seg_item.reserve(sizeof(int) * ng) || !w.seg_item.reserve(sizeof(int) * ng))
    return LHAF_ENOMEM;
  if (stats) cudaEventRecord(ctx->ev0, s);
  int launches = 0;
  long long last_blocks = -1;
  for (uint64_t t0 = 0; t0 < T; t0 += cap) {
    const uint64_t t1 = std::min<uint64_t>(T, t0 + cap), nn = t1 - t0;
    const long long blocks = series_blocks((long long)nn);
    if (blocks != last_blocks) {  // segment table for this launch size (at most two distinct sizes)
      if (cudaEventSynchronize(w.uploaded) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "multi-vector segment wait");
      long long* sb = static_cast<long long*>(w.h_seg_begin.p);
      int* si = static_cast<int*>(w.h_seg_item.p);
      for (int g = 0; g <= ng; g++) sb[g] = (long long)g * blocks;
      for (int g = 0; g < ng; g++) si[g] = g;
      if (cudaMemcpyAsync(w.seg_begin.p, sb, sizeof(long long) * (ng + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(w.seg_item.p, si, sizeof(int) * ng, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaEventRecord(w.uploaded, s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "multi-vector segments");
      h2d += sizeof(long long) * (ng + 1) + sizeof(int) * ng;
      last_blocks = blocks;
    }
    unsigned long long rounds = 1;
    const uint64_t grid = balanced_grid(nn, tpc, max_ctas, &rounds);
    p.total_teams = grid * (uint64_t)tpc;
    p.rounds = rounds;
    p.t_begin = t0;
    p.t_end = t1;
    p.t_lo = 0;
    p.stage_pad = 0;  // only the chunk's own terms are staged (columns < nn <= cap)
    cudaError_t e = launch_terms(false, team, ctx->d_chat, p, (int)grid, ctx->d_partials, s, ctx->d_stage,
                                 ctx->d_wstage, (long long)cap);
    if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "multi-vector terms kernel");
    e = launch_series_multi(ctx->d_stage, ctx->d_wstage, (long long)nn, (long long)cap, h, kr, ng,
                            (flags & LHAF_PLAIN_ACCUM) ? 1 : 0, (double*)w.entries.p, s);
    if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "multi-vector series kernel");
    e = launch_segment_reduce((const double*)w.entries.p, (const long long*)w.seg_begin.p,
                              (const int*)w.seg_item.p, ng, (flags & LHAF_PLAIN_ACCUM) ? 1 : 0, (double*)w.acc.p, s);
    if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "multi-vector reduction");
    launches += 3;
  }
  if (launch_item_finalize((const double*)w.acc.p, (const int*)w.item_h.p, ng, (double2*)w.out.p, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "multi-vector scaling");
  launches++;
  if (stats) cudaEventRecord(ctx->ev1, s);
  if (cudaEventRecord(w.uploaded, s) != cudaSuccess ||
      cudaMemcpyAsync(w.h_out.p, w.out.p, sizeof(double2) * ng, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "multi-vector result copy");
  if (const cudaError_t e = cudaStreamSynchronize(s); e != cudaSuccess)
    return (lhaf_status)record_cuda(e, "cudaStreamSynchronize");
  std::memcpy(out, w.h_out.p, sizeof(double2) * ng);
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->kernel_ms = ms;
    stats->terms = T;
    stats->n_dim = nd;
    stats->h = h;
    stats->pairs = pm.P;
    stats->team = team;
    // the reduction and characteristic polynomial once, and per vector the transformed vectors,
    // min(h, n) - 1 Hessenberg products and the series (8 flops per complex multiply-add)
    const double per_vec = 8.0 * ((double)nd * nd + (double)(kr - 1) * nd * (nd + 3) / 2.0 + (double)kr * nd) +
                           8.0 * (double)h * h;
    stats->flops_model = (double)T * (lhaf_model_flops_per_term(nd, h, 0) + (double)ng * per_vec);
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = sizeof(double2) * (uint64_t)ng;
    stats->launches = launches;
  }
  return LHAF_OK;
}
