// Value and gradient of lhaf(B_n) with respect to B (as a symmetric variable) and gamma, from the
// per-term adjoint of the finite difference sieve (App. B.4). Not part of the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_ctx.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"

using namespace lhafgpu;

namespace {

// One loop hafnian's adjoint launch: its plan, team, term parameters and gradient length.
struct GradJob {
  Plan pl;
  int team = 0;
  uint64_t grid = 0;
  int len = 0;  // n * n slot-matrix entries, then n loop entries
  TermParams p;
};

lhaf_status grad_validate(int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps) {
  for (int i = 0; i < M; i++) {
    const int r = reps ? reps[i] : 1;
    if (r < 0) return LHAF_EINVAL;
    if (gamma && !(std::isfinite(gamma[i].re) && std::isfinite(gamma[i].im))) return LHAF_EINVAL;
    for (int j = i; j < M; j++) {
      const lhaf_c128 z = B[(size_t)i * M + j];
      if (!(std::isfinite(z.re) && std::isfinite(z.im))) return LHAF_EINVAL;
    }
  }
  return LHAF_OK;
}

// Plan, loop border, team size and term parameters of one item (host only).
lhaf_status grad_plan(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                      uint32_t flags, GradJob& J) {
  Plan& pl = J.pl;
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
  if (pl.N == 0) return LHAF_OK;
  const int nd = pl.nd, n = nd - pl.bord;
  // team size: largest number of resident warps, preferring 16 or 32 lanes per term
  const size_t ib = cta_table_bytes(false, pl.Hl, pl.H);
  size_t tb = 0;
  int occ = 0;
  double best = -1.0;
  J.team = 0;
  const char* env = std::getenv("LHAF_GRAD_TEAM");  // forces 8, 16, 32 or 64 lanes per term
  const int forced = env ? std::atoi(env) : 0;
  for (int g : {16, 32, 8, 64}) {
    if (forced && g != forced) continue;
    const size_t tg = grad_team_bytes(nd, pl.H, pl.h, pl.bord, g);
    const size_t smem = ib + (size_t)teams_per_cta(g) * tg;
    if (smem > 227 * 1024) continue;
    const int o = grad_ctas_per_sm(g, smem);
    if (o <= 0) continue;
    const double warps = (double)o * cta_threads(g) / 32.0;
    const double score = std::min(warps, 8.0) + (g == 16 || g == 32 ? 0.5 : 0.0);
    if (score > best) {
      best = score;
      J.team = g;
      occ = o;
      tb = tg;
    }
  }
  if (J.team == 0) return LHAF_ETOOBIG;
  TermParams& p = J.p;
  fill_params(pl, false, false, J.team, flags & LHAF_PLAIN_ACCUM, p);
  p.team_bytes = (int)tb;
  p.items_bytes = (int)ib;
  const int tpc = teams_per_cta(J.team);
  uint64_t grid = (pl.T + tpc - 1) / tpc;
  grid = std::min<uint64_t>(grid, (uint64_t)ctx->sms * (uint64_t)occ);
  if (grid < 1) grid = 1;
  J.grid = grid;
  p.total_teams = grid * (uint64_t)tpc;
  if (p.total_teams > ctx->partial_cap) return LHAF_ETOOBIG;
  p.rounds = (pl.T + p.total_teams - 1) / p.total_teams;
  p.t_begin = 0;
  p.t_end = pl.T;
  J.len = n * n + n;
  return LHAF_OK;
}

// Adjoint launch, value reduction and gradient reduction of one item, ordered on the context's
// stream: the slot matrix at chat, 6 doubles (dd value, value) at out6, the len gradient sums at
// gout. The per-team gradient partials use ctx->b_gpart (reserved by the caller).
lhaf_status grad_enqueue(lhaf_ctx* ctx, const GradJob& J, const double2* chat, double* out6, double2* gout) {
  if (launch_grad(J.team, chat, J.p, (int)J.grid, ctx->d_partials, (double2*)ctx->b_gpart.p, ctx->stream) !=
      cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "adjoint kernel");
  if (launch_reduce(ctx->d_partials, (long long)J.p.total_teams, J.pl.h, out6, (double2*)(out6 + 4), ctx->stream) !=
      cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "value reduction");
  if (launch_grad_reduce((const double2*)ctx->b_gpart.p, (long long)J.p.total_teams, J.len, J.pl.h, gout,
                         ctx->stream) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "gradient reduction");
  return LHAF_OK;
}

// Slot derivatives -> modes: B[m][m'] (m <= m') collects dC over the slot pairs with those modes;
// dB symmetric, dgamma only when gamma was given (else the loop part goes to dB's diagonal).
void grad_scatter(const Plan& pl, int M, const std::complex<double>* g, bool has_gamma, lhaf_c128* dB,
                  lhaf_c128* dgamma) {
  const int n = pl.nd - pl.bord;
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
  if (!has_gamma)
    for (int m = 0; m < M; m++) dsym[(size_t)m * M + m] += dgam[m];
  if (dB)
    for (int i = 0; i < M; i++)
      for (int j = i; j < M; j++) {
        const std::complex<double> v = dsym[(size_t)i * M + j];
        dB[(size_t)i * M + j] = {v.real(), v.imag()};
        dB[(size_t)j * M + i] = {v.real(), v.imag()};
      }
  if (dgamma && has_gamma)
    for (int m = 0; m < M; m++) dgamma[m] = {dgam[m].real(), dgam[m].imag()};
}

}  // namespace

extern "C" lhaf_status lhaf_grad(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                                 uint32_t flags, lhaf_c128* value, lhaf_c128* dB, lhaf_c128* dgamma) {
  if (!ctx || M <= 0 || !B || !value) return LHAF_EINVAL;
  if (flags & (LHAF_DEVICE_PTRS | LHAF_FP32_TERMS | LHAF_ET)) return LHAF_EINVAL;  // host inputs, FP64, sieve
  lhaf_status st = grad_validate(M, B, gamma, reps);
  if (st != LHAF_OK) return st;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaSetDevice");
  GradJob J;
  st = grad_plan(ctx, M, B, gamma, reps, flags, J);
  if (st != LHAF_OK) return st;
  if (dB) std::memset(dB, 0, sizeof(lhaf_c128) * (size_t)M * M);
  if (dgamma) std::memset(dgamma, 0, sizeof(lhaf_c128) * M);
  if (J.pl.N == 0) {
    *value = {1.0, 0.0};
    return LHAF_OK;
  }
  const int nd = J.pl.nd;
  build_chat_host(J.pl, M, B, gamma, (std::complex<double>*)ctx->h_chat);
  if (cudaMemcpyAsync(ctx->d_chat, ctx->h_chat, sizeof(double2) * nd * nd, cudaMemcpyHostToDevice, ctx->stream) !=
      cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "slot matrix upload");
  if (!ctx->b_gpart.reserve(sizeof(double2) * (size_t)J.len * J.p.total_teams) ||
      !ctx->b_gout.reserve(sizeof(double2) * (size_t)J.len) || !ctx->hb_gout.reserve(sizeof(double2) * (size_t)J.len))
    return LHAF_ENOMEM;
  st = grad_enqueue(ctx, J, ctx->d_chat, ctx->d_out, (double2*)ctx->b_gout.p);
  if (st != LHAF_OK) return st;
  if (cudaMemcpyAsync(ctx->h_out, ctx->d_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
      cudaMemcpyAsync(ctx->hb_gout.p, ctx->b_gout.p, sizeof(double2) * J.len, cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "result copy");
  if (const cudaError_t e_ = (cudaStreamSynchronize(ctx->stream)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaStreamSynchronize");
  *value = {ctx->h_out[4], ctx->h_out[5]};
  grad_scatter(J.pl, M, static_cast<const std::complex<double>*>(ctx->hb_gout.p), gamma != nullptr, dB, dgamma);
  return LHAF_OK;
}

extern "C" lhaf_status lhaf_grad_batched(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B, const lhaf_c128* gammas,
                                         const int32_t* reps, uint32_t flags, lhaf_c128* values, lhaf_c128* dB,
                                         lhaf_c128* dgamma, lhaf_status* item_status) {
  if (!ctx || batch < 0 || M <= 0 || !B || !reps || !values) return LHAF_EINVAL;
  if (flags & (LHAF_DEVICE_PTRS | LHAF_FP32_TERMS | LHAF_ET)) return LHAF_EINVAL;  // host inputs, FP64, sieve
  if (batch == 0) return LHAF_OK;
  lhaf_status st = LHAF_OK;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaSetDevice");
  std::vector<GradJob> jobs(batch);
  std::vector<lhaf_status> ist(batch, LHAF_OK);
  std::vector<size_t> chat_off(batch, 0), gout_off(batch, 0);
  size_t pool = 0, gtot = 0, gpart = 1;
  for (int i = 0; i < batch; i++) {
    const lhaf_c128* gi = gammas ? gammas + (size_t)i * M : nullptr;
    const int32_t* ri = reps + (size_t)i * M;
    ist[i] = grad_validate(M, B, gi, ri);
    if (ist[i] == LHAF_OK) ist[i] = grad_plan(ctx, M, B, gi, ri, flags, jobs[i]);
    if (ist[i] != LHAF_OK || jobs[i].pl.N == 0) continue;
    chat_off[i] = pool;
    pool += (size_t)jobs[i].pl.nd * jobs[i].pl.nd;
    gout_off[i] = gtot;
    gtot += (size_t)jobs[i].len;
    gpart = std::max(gpart, (size_t)jobs[i].len * (size_t)jobs[i].p.total_teams);
  }
  BatchWork& w = ctx->bw;
  if (!w.h_chat.reserve(sizeof(double2) * std::max<size_t>(pool, 1)) ||
      !w.chat.reserve(sizeof(double2) * std::max<size_t>(pool, 1)) ||
      !w.out.reserve(sizeof(double) * 6 * (size_t)batch) || !w.h_out.reserve(sizeof(double) * 6 * (size_t)batch) ||
      !ctx->b_gpart.reserve(sizeof(double2) * gpart) ||
      !ctx->b_gout.reserve(sizeof(double2) * std::max<size_t>(gtot, 1)) ||
      !ctx->hb_gout.reserve(sizeof(double2) * std::max<size_t>(gtot, 1)))
    return LHAF_ENOMEM;
  if (w.uploaded) cudaEventSynchronize(w.uploaded);  // an earlier upload still reads the pinned buffer
  std::complex<double>* hc = static_cast<std::complex<double>*>(w.h_chat.p);
  for (int i = 0; i < batch; i++)
    if (ist[i] == LHAF_OK && jobs[i].pl.N > 0)
      build_chat_host(jobs[i].pl, M, B, gammas ? gammas + (size_t)i * M : nullptr, hc + chat_off[i]);
  if (pool && cudaMemcpyAsync(w.chat.p, hc, sizeof(double2) * pool, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "slot matrix upload");
  double* out = static_cast<double*>(w.out.p);
  double2* gout = static_cast<double2*>(ctx->b_gout.p);
  for (int i = 0; i < batch; i++) {
    if (ist[i] != LHAF_OK || jobs[i].pl.N == 0) continue;
    st = grad_enqueue(ctx, jobs[i], static_cast<const double2*>(w.chat.p) + chat_off[i], out + 6 * (size_t)i,
                      gout + gout_off[i]);
    if (st != LHAF_OK) return st;
  }
  if (cudaMemcpyAsync(w.h_out.p, w.out.p, sizeof(double) * 6 * (size_t)batch, cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess ||
      (gtot && cudaMemcpyAsync(ctx->hb_gout.p, ctx->b_gout.p, sizeof(double2) * gtot, cudaMemcpyDeviceToHost,
                               ctx->stream) != cudaSuccess))
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "result copy");
  if (const cudaError_t e_ = (cudaStreamSynchronize(ctx->stream)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaStreamSynchronize");
  const double* ho = static_cast<const double*>(w.h_out.p);
  const std::complex<double>* hg = static_cast<const std::complex<double>*>(ctx->hb_gout.p);
  lhaf_status first = LHAF_OK;
  for (int i = 0; i < batch; i++) {
    lhaf_c128* dBi = dB ? dB + (size_t)i * M * M : nullptr;
    lhaf_c128* dgi = dgamma ? dgamma + (size_t)i * M : nullptr;
    if (dBi) std::memset(dBi, 0, sizeof(lhaf_c128) * (size_t)M * M);
    if (dgi) std::memset(dgi, 0, sizeof(lhaf_c128) * M);
    values[i] = {0.0, 0.0};
    if (item_status) item_status[i] = ist[i];
    if (ist[i] != LHAF_OK) {
      if (first == LHAF_OK) first = ist[i];
      continue;
    }
    if (jobs[i].pl.N == 0) {
      values[i] = {1.0, 0.0};
      continue;
    }
    values[i] = {ho[6 * (size_t)i + 4], ho[6 * (size_t)i + 5]};
    grad_scatter(jobs[i].pl, M, hg + gout_off[i], gammas != nullptr, dBi, dgi);
  }
  return item_status ? LHAF_OK : first;
}
