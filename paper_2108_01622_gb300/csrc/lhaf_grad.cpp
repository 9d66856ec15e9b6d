// Value and gradient of lhaf(B_n) with respect to B (as a symmetric variable) and gamma, from the
// per-term adjoint of the finite difference sieve (App. B.4). Not part of the paper.
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

extern "C" lhaf_status lhaf_grad(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                                 uint32_t flags, lhaf_c128* value, lhaf_c128* dB, lhaf_c128* dgamma) {
  if (!ctx || M <= 0 || !B || !value) return LHAF_EINVAL;
  if (flags & (LHAF_DEVICE_PTRS | LHAF_FP32_TERMS | LHAF_ET)) return LHAF_EINVAL;  // host inputs, FP64, sieve
  for (int i = 0; i < M; i++) {
    const int r = reps ? reps[i] : 1;
    if (r < 0) return LHAF_EINVAL;
    if (gamma && !(std::isfinite(gamma[i].re) && std::isfinite(gamma[i].im))) return LHAF_EINVAL;
    for (int j = i; j < M; j++) {
      const lhaf_c128 z = B[(size_t)i * M + j];
      if (!(std::isfinite(z.re) && std::isfinite(z.im))) return LHAF_EINVAL;
    }
  }
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaSetDevice");
  Plan pl;
  lhaf_status st = build_plan(M, reps, flags, true, pl);
  if (st != LHAF_OK) return st;
  bool any_loop = pl.N > 0 && (pl.N % 2 == 1);
  for (int s = 0; s < 2 * pl.P && !any_loop; s++) {
    const int m = pl.slot_mode[s];
    const lhaf_c128 g = gamma ? gamma[m] : B[(size_t)m * M + m];
    any_loop = (g.re != 0.0 || g.im != 0.0);
  }
  if (!any_loop && pl.N > 0) {
    // gamma = 0 on the occupied modes and N even: every loop derivative vanishes (a matching of
    // an odd number of photons needs a loop); the border is dropped
    st = build_plan(M, reps, flags, false, pl);
    if (st != LHAF_OK) return st;
  }
  if (dB) std::memset(dB, 0, sizeof(lhaf_c128) * (size_t)M * M);
  if (dgamma) std::memset(dgamma, 0, sizeof(lhaf_c128) * M);
  if (pl.N == 0) {
    *value = {1.0, 0.0};
    return LHAF_OK;
  }
  const int nd = pl.nd, n = nd - pl.bord;
  // slot matrix
  build_chat_host(pl, M, B, gamma, (std::complex<double>*)ctx->h_chat);
  if (cudaMemcpyAsync(ctx->d_chat, ctx->h_chat, sizeof(double2) * nd * nd, cudaMemcpyHostToDevice, ctx->stream) !=
      cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "slot matrix upload");
  // team size: largest number of resident warps, preferring 16 or 32 lanes per term
  const size_t tb = grad_team_bytes(nd, pl.H, pl.h, pl.bord);
  const size_t ib = cta_table_bytes(false, pl.Hl, pl.H);
  int team = 0, occ = 0;
  double best = -1.0;
  for (int g : {16, 32, 64, 8, 128}) {
    const size_t smem = ib + (size_t)teams_per_cta(g) * tb;
    if (smem > 227 * 1024) continue;
    const int o = grad_ctas_per_sm(g, smem);
    if (o <= 0) continue;
    const double warps = (double)o * cta_threads(g) / 32.0;
    const double score = std::min(warps, 8.0) + (g == 16 || g == 32 ? 0.5 : 0.0);
    if (score > best) {
      best = score;
      team = g;
      occ = o;
    }
  }
  if (team == 0) return LHAF_ETOOBIG;
  TermParams p;
  fill_params(pl, false, false, team, flags & LHAF_PLAIN_ACCUM, p);
  p.team_bytes = (int)tb;
  p.items_bytes = (int)ib;
  const int tpc = teams_per_cta(team);
  uint64_t grid = (pl.T + tpc - 1) / tpc;
  grid = std::min<uint64_t>(grid, (uint64_t)ctx->sms * (uint64_t)occ);
  if (grid < 1) grid = 1;
  p.total_teams = grid * (uint64_t)tpc;
  if (p.total_teams > ctx->partial_cap) return LHAF_ETOOBIG;
  p.rounds = (pl.T + p.total_teams - 1) / p.total_teams;
  p.t_begin = 0;
  p.t_end = pl.T;
  const int len = n * n + n;
  if (!ctx->b_gpart.reserve(sizeof(double2) * (size_t)len * p.total_teams) ||
      !ctx->b_gout.reserve(sizeof(double2) * (size_t)len) || !ctx->hb_gout.reserve(sizeof(double2) * (size_t)len))
    return LHAF_ENOMEM;
  if (launch_grad(team, ctx->d_chat, p, (int)grid, ctx->d_partials, (double2*)ctx->b_gpart.p, ctx->stream) !=
      cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "adjoint kernel");
  if (launch_reduce(ctx->d_partials, (long long)p.total_teams, pl.h, ctx->d_out, (double2*)(ctx->d_out + 4),
                    ctx->stream) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "value reduction");
  if (launch_grad_reduce((const double2*)ctx->b_gpart.p, (long long)p.total_teams, len, pl.h, (double2*)ctx->b_gout.p,
                         ctx->stream) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "gradient reduction");
  if (cudaMemcpyAsync(ctx->h_out, ctx->d_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
      cudaMemcpyAsync(ctx->hb_gout.p, ctx->b_gout.p, sizeof(double2) * len, cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "result copy");
  if (const cudaError_t e_ = (cudaStreamSynchronize(ctx->stream)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaStreamSynchronize");
  *value = {ctx->h_out[4], ctx->h_out[5]};
  const std::complex<double>* g = static_cast<const std::complex<double>*>(ctx->hb_gout.p);
  // slot derivatives -> modes: B[m][m'] (m <= m') collects dC over slot pairs with those modes
  std::vector<std::complex<double>> dsym((size_t)M * M, 0.0), dgam(M, 0.0);
  for (int a = 0; a < n; a++) {
    const int ma = pl.slot_mode[a];
    if (ma < 0) continue;
    for (int b = 0; b < n; b++) {
      const int mb = pl.slot_mode[b];
      if (mb < 0) continue;
      const int lo = std::min(ma, mb), hi = std::max(ma, mb);
      dsym[(size_t)lo * M + hi] += g[(size_t)a * n + b];
    }
    if (pl.bord) dgam[ma] += g[(size_t)n * n + a];
  }
  if (!gamma)  // loops taken from diag(B): the loop derivative belongs to B[m][m]
    for (int m = 0; m < M; m++) dsym[(size_t)m * M + m] += dgam[m];
  if (dB)
    for (int i = 0; i < M; i++)
      for (int j = i; j < M; j++) {
        const std::complex<double> v = dsym[(size_t)i * M + j];
        dB[(size_t)i * M + j] = {v.real(), v.imag()};
        dB[(size_t)j * M + i] = {v.real(), v.imag()};
      }
  if (dgamma && gamma)
    for (int m = 0; m < M; m++) dgamma[m] = {dgam[m].real(), dgam[m].imag()};
  return LHAF_OK;
}
