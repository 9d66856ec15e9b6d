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
  // zero-digit groups (empty: one sieve on the full matrix): their plans, descriptors (slot
  // matrices at chat_off in a pool of `pool` entries) and chunk offsets
  std::vector<Plan> subs;
  std::vector<GradSieve> sv;
  std::vector<long long> chunk_off;
  size_t pool = 0;
};

// At most this many zero-digit groups per loop hafnian run as one grouped adjoint launch (more,
// and the full matrix is used: the descriptors would outweigh the saved work).
constexpr size_t kGradMaxSieves = 4096;

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
  // zero-digit groups (App. B.4's middle digits of even pairs give delta' = 0, deleting two slots):
  // the adjoint runs every group on its own smaller matrix unless LHAF_NO_ZERO_SPLIT is given
  std::vector<Plan> subs;
  const bool grouped = !(flags & LHAF_NO_ZERO_SPLIT) && split_zero_digits(pl, subs) && subs.size() >= 2 &&
                       subs.size() <= kGradMaxSieves;
  // team size: largest number of resident warps, preferring 16 or 32 lanes per term (the full plan
  // has the largest matrix and tables of all its groups)
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
    const int o = grad_ctas_per_sm(g, smem, grouped);
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
  uint64_t chunks = (pl.T + tpc - 1) / tpc;
  if (grouped) {
    J.chunk_off.assign(1, 0);
    for (const Plan& sub : subs) {
      GradSieve g;
      std::memset(&g, 0, sizeof(g));
      fill_params(sub, false, false, J.team, flags & LHAF_PLAIN_ACCUM, g.p);
      g.p.team_bytes = (int)tb;
      g.p.items_bytes = (int)ib;
      g.p.t_end = sub.T;
      g.chat_off = (long long)J.pool;
      J.pool += (size_t)sub.nd * sub.nd;
      for (int q = 0; q < sub.P; q++) {  // pair q of the group is pair src_pair[q] of the full plan
        g.smap[2 * q] = 2 * sub.src_pair[q];
        g.smap[2 * q + 1] = 2 * sub.src_pair[q] + 1;
      }
      J.sv.push_back(g);
      J.chunk_off.push_back(J.chunk_off.back() + (long long)((sub.T + tpc - 1) / tpc));
    }
    J.subs = std::move(subs);
    chunks = (uint64_t)J.chunk_off.back();
  }
  uint64_t grid = std::min<uint64_t>(chunks, (uint64_t)ctx->sms * (uint64_t)occ);
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

// Slot matrices of a job's sieves (its zero-digit groups, or the full plan) into chat (host).
void grad_build_chats(const GradJob& J, int M, const lhaf_c128* B, const lhaf_c128* gamma, std::complex<double>* chat) {
  if (J.sv.empty()) {
    build_chat_host(J.pl, M, B, gamma, chat);
    return;
  }
  for (size_t g = 0; g < J.subs.size(); g++) build_chat_host(J.subs[g], M, B, gamma, chat + J.sv[g].chat_off);
}

size_t grad_chat_entries(const GradJob& J) { return J.sv.empty() ? (size_t)J.pl.nd * J.pl.nd : J.pool; }

// Adjoint launch, value reduction and gradient reduction of one item, ordered on the context's
// stream: the slot matrix at chat, 6 doubles (dd value, value) at out6, the len gradient sums at
// gout. The per-team gradient partials use ctx->b_gpart (reserved by the caller).
lhaf_status grad_enqueue(lhaf_ctx* ctx, const GradJob& J, const double2* chat, double* out6, double2* gout,
                         const GradSieve* sv = nullptr, const long long* chunk_off = nullptr) {
  if (J.sv.empty()) {
    if (launch_grad(J.team, chat, J.p, (int)J.grid, ctx->d_partials, (double2*)ctx->b_gpart.p, ctx->stream) !=
        cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "adjoint kernel");
  } else {
    if (launch_grad_grouped(J.team, chat, sv, (int)J.sv.size(), chunk_off, J.chunk_off.back(), J.pl.nd - J.pl.bord,
                            J.p.team_bytes, J.p.items_bytes, (int)J.grid, ctx->d_partials,
                            (double2*)ctx->b_gpart.p, ctx->stream) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "grouped adjoint kernel");
  }
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
  const double2* chat = ctx->d_chat;
  const GradSieve* dsv = nullptr;
  const long long* dco = nullptr;
  if (J.sv.empty()) {
    build_chat_host(J.pl, M, B, gamma, (std::complex<double>*)ctx->h_chat);
    if (cudaMemcpyAsync(ctx->d_chat, ctx->h_chat, sizeof(double2) * nd * nd, cudaMemcpyHostToDevice, ctx->stream) !=
        cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "slot matrix upload");
  } else {
    // the zero-digit groups' slot matrices, descriptors and chunk offsets in the context's group buffers
    BatchWork& w = ctx->gw;
    const size_t ns = J.sv.size();
    if (w.uploaded) {
      if (const cudaError_t e = cudaEventSynchronize(w.uploaded); e != cudaSuccess)
        return (lhaf_status)record_cuda(e, "cudaEventSynchronize");
    } else if (cudaEventCreateWithFlags(&w.uploaded, cudaEventDisableTiming) != cudaSuccess) {
      w.uploaded = nullptr;
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventCreate");
    }
    if (!w.h_chat.reserve(sizeof(double2) * J.pool) || !w.chat.reserve(sizeof(double2) * J.pool) ||
        !w.h_items.reserve(sizeof(GradSieve) * ns) || !w.items.reserve(sizeof(GradSieve) * ns) ||
        !w.h_chunks.reserve(sizeof(long long) * (ns + 1)) || !w.chunks.reserve(sizeof(long long) * (ns + 1)))
      return LHAF_ENOMEM;
    grad_build_chats(J, M, B, gamma, static_cast<std::complex<double>*>(w.h_chat.p));
    std::memcpy(w.h_items.p, J.sv.data(), sizeof(GradSieve) * ns);
    std::memcpy(w.h_chunks.p, J.chunk_off.data(), sizeof(long long) * (ns + 1));
    if (cudaMemcpyAsync(w.chat.p, w.h_chat.p, sizeof(double2) * J.pool, cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(w.items.p, w.h_items.p, sizeof(GradSieve) * ns, cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(w.chunks.p, w.h_chunks.p, sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess ||
        cudaEventRecord(w.uploaded, ctx->stream) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "group upload");
    chat = static_cast<const double2*>(w.chat.p);
    dsv = static_cast<const GradSieve*>(w.items.p);
    dco = static_cast<const long long*>(w.chunks.p);
  }
  if (!ctx->b_gpart.reserve(sizeof(double2) * (size_t)J.len * J.p.total_teams) ||
      !ctx->b_gout.reserve(sizeof(double2) * (size_t)J.len) || !ctx->hb_gout.reserve(sizeof(double2) * (size_t)J.len))
    return LHAF_ENOMEM;
  st = grad_enqueue(ctx, J, chat, ctx->d_out, (double2*)ctx->b_gout.p, dsv, dco);
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
  std::vector<size_t> chat_off(batch, 0), gout_off(batch, 0), sv_off(batch, 0), co_off(batch, 0);
  size_t pool = 0, gtot = 0, gpart = 1, nsv = 0, nco = 0;
  for (int i = 0; i < batch; i++) {
    const lhaf_c128* gi = gammas ? gammas + (size_t)i * M : nullptr;
    const int32_t* ri = reps + (size_t)i * M;
    ist[i] = grad_validate(M, B, gi, ri);
    if (ist[i] == LHAF_OK) ist[i] = grad_plan(ctx, M, B, gi, ri, flags, jobs[i]);
    if (ist[i] != LHAF_OK || jobs[i].pl.N == 0) continue;
    chat_off[i] = pool;
    pool += grad_chat_entries(jobs[i]);
    sv_off[i] = nsv;
    nsv += jobs[i].sv.size();
    co_off[i] = nco;
    nco += jobs[i].chunk_off.size();
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
  // the items' zero-digit group descriptors and chunk offsets (ctx->gw)
  BatchWork& gw = ctx->gw;
  if (nsv) {
    if (gw.uploaded) {
      if (const cudaError_t e = cudaEventSynchronize(gw.uploaded); e != cudaSuccess)
        return (lhaf_status)record_cuda(e, "cudaEventSynchronize");
    }
    if (!gw.h_items.reserve(sizeof(GradSieve) * nsv) || !gw.items.reserve(sizeof(GradSieve) * nsv) ||
        !gw.h_chunks.reserve(sizeof(long long) * nco) || !gw.chunks.reserve(sizeof(long long) * nco))
      return LHAF_ENOMEM;
  }
  if (w.uploaded) cudaEventSynchronize(w.uploaded);  // an earlier upload still reads the pinned buffer
  std::complex<double>* hc = static_cast<std::complex<double>*>(w.h_chat.p);
  for (int i = 0; i < batch; i++)
    if (ist[i] == LHAF_OK && jobs[i].pl.N > 0) {
      grad_build_chats(jobs[i], M, B, gammas ? gammas + (size_t)i * M : nullptr, hc + chat_off[i]);
      if (!jobs[i].sv.empty()) {
        std::memcpy(static_cast<GradSieve*>(gw.h_items.p) + sv_off[i], jobs[i].sv.data(),
                    sizeof(GradSieve) * jobs[i].sv.size());
        std::memcpy(static_cast<long long*>(gw.h_chunks.p) + co_off[i], jobs[i].chunk_off.data(),
                    sizeof(long long) * jobs[i].chunk_off.size());
      }
    }
  if (pool && cudaMemcpyAsync(w.chat.p, hc, sizeof(double2) * pool, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "slot matrix upload");
  if (nsv && (cudaMemcpyAsync(gw.items.p, gw.h_items.p, sizeof(GradSieve) * nsv, cudaMemcpyHostToDevice,
                              ctx->stream) != cudaSuccess ||
              cudaMemcpyAsync(gw.chunks.p, gw.h_chunks.p, sizeof(long long) * nco, cudaMemcpyHostToDevice,
                              ctx->stream) != cudaSuccess))
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "group upload");
  double* out = static_cast<double*>(w.out.p);
  double2* gout = static_cast<double2*>(ctx->b_gout.p);
  for (int i = 0; i < batch; i++) {
    if (ist[i] != LHAF_OK || jobs[i].pl.N == 0) continue;
    st = grad_enqueue(ctx, jobs[i], static_cast<const double2*>(w.chat.p) + chat_off[i], out + 6 * (size_t)i,
                      gout + gout_off[i], static_cast<const GradSieve*>(gw.items.p) + sv_off[i],
                      static_cast<const long long*>(gw.chunks.p) + co_off[i]);
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
