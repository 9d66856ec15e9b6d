// Batched loop hafnians (the chain-rule sampler's conditional probabilities, App. A.2 and
// App. B.5): many lhaf(B_n) of uneven size in one persistent launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_ctx.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"

using namespace lhafgpu;

namespace {

bool finite_c(const lhaf_c128& z) { return std::isfinite(z.re) && std::isfinite(z.im); }

}  // namespace

extern "C" lhaf_status lhaf_batched(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                                    const int32_t* reps, uint32_t flags, lhaf_c128* out, lhaf_status* item_status,
                                    lhaf_stats* stats) {
  if (!ctx || batch < 0 || M <= 0 || !B || !reps || (batch > 0 && !out)) return LHAF_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (batch == 0) return LHAF_OK;
  const bool dev = (flags & LHAF_DEVICE_PTRS) != 0;
  const bool per_item_B = (flags & LHAF_BATCH_B_PER_ITEM) != 0;
  const bool fp32 = (flags & LHAF_FP32_TERMS) != 0;
  const long long B_stride = per_item_B ? (long long)M * M : 0;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaSetDevice");

  // ---- plans ----
  std::vector<Plan> plans(batch);
  std::vector<lhaf_status> st(batch, LHAF_OK);
  std::vector<int> item_h(batch, 0);
  for (int i = 0; i < batch; i++) {
    const int32_t* r = reps + (size_t)i * M;
    const lhaf_c128* Bi = B + (size_t)i * B_stride;
    const lhaf_c128* gi = gamma ? gamma + (size_t)i * M : nullptr;
    bool loops = !(flags & LHAF_NO_LOOPS);
    if (!dev) {
      // validate the entries this item reads
      for (int a = 0; a < M && st[i] == LHAF_OK; a++) {
        if (r[a] < 0) st[i] = LHAF_EINVAL;
        if (r[a] <= 0) continue;
        if (gi && !finite_c(gi[a])) st[i] = LHAF_EINVAL;
        for (int b = a; b < M; b++)
          if (r[b] > 0 && !finite_c(Bi[(size_t)a * M + b])) st[i] = LHAF_EINVAL;
      }
    }
    if (st[i] == LHAF_OK) st[i] = build_plan(M, r, flags, loops, plans[i]);
    if (st[i] == LHAF_OK && !dev && loops && plans[i].N > 0) {
      bool any = false;
      for (int s = 0; s < 2 * plans[i].P && !any; s++) {
        const int m = plans[i].slot_mode[s];
        if (m < 0) {
          any = true;
          break;
        }
        const lhaf_c128 g = gi ? gi[m] : Bi[(size_t)m * M + m];
        any = (g.re != 0.0 || g.im != 0.0);
      }
      if (!any) st[i] = build_plan(M, r, flags, false, plans[i]);
    }
    if (st[i] != LHAF_OK) {
      item_h[i] = INT_MAX;
    } else if (plans[i].N == 0) {
      item_h[i] = -1;
    } else {
      item_h[i] = plans[i].h;
    }
  }
  if (item_status)
    for (int i = 0; i < batch; i++) item_status[i] = st[i];
  // items with sieve terms to evaluate (valid plan, N > 0)
  std::vector<char> runnable(batch, 0);
  for (int i = 0; i < batch; i++) runnable[i] = (st[i] == LHAF_OK && plans[i].N > 0) ? 1 : 0;

  // ---- per-item descriptors, slot-matrix pool, costs ----
  std::vector<int> work;  // items with terms
  for (int i = 0; i < batch; i++)
    if (runnable[i]) work.push_back(i);
  if (!ctx->hb_items.reserve(sizeof(BatchItem) * batch) || !ctx->b_items.reserve(sizeof(BatchItem) * batch) ||
      !ctx->hb_item_h.reserve(sizeof(int) * batch) || !ctx->b_item_h.reserve(sizeof(int) * batch) ||
      !ctx->hb_unit_begin.reserve(sizeof(int) * (batch + 1)) || !ctx->b_unit_begin.reserve(sizeof(int) * (batch + 1)) ||
      !ctx->b_out.reserve(sizeof(double2) * batch) || !ctx->hb_out.reserve(sizeof(double2) * batch))
    return LHAF_ENOMEM;
  BatchItem* hitems = static_cast<BatchItem*>(ctx->hb_items.p);
  long long pool = 0;
  int nd_max = 0, H_max = 0, Hl_max = 0, rep = -1;
  double cost_max = -1.0, cost_total = 0.0;
  std::vector<double> fpt(batch, 0.0);
  for (int i = 0; i < batch; i++) {
    std::memset(&hitems[i], 0, sizeof(BatchItem));
    if (!runnable[i]) continue;
    const Plan& pl = plans[i];
    fill_params(pl, fp32, false, 32, flags, hitems[i].p);
    hitems[i].chat_off = pool;
    for (int s = 0; s < kMaxDim; s++) hitems[i].slot_mode[s] = s < 2 * pl.P ? pl.slot_mode[s] : -1;
    pool += (long long)pl.nd * pl.nd;
    nd_max = std::max(nd_max, pl.nd);
    H_max = std::max(H_max, pl.H);
    Hl_max = std::max(Hl_max, pl.Hl);
    fpt[i] = lhaf_model_flops_per_term(pl.nd, pl.h, pl.bord);
    const double c = fpt[i] * (double)pl.T;
    cost_total += c;
    if (c > cost_max) {
      cost_max = c;
      rep = i;
    }
  }
  std::memcpy(ctx->hb_item_h.p, item_h.data(), sizeof(int) * batch);

  cudaStream_t s = ctx->stream;
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  if (!ctx->b_chat.reserve(sizeof(double2) * std::max<long long>(pool, 1)) ||
      (fp32 && !ctx->b_chat32.reserve(sizeof(float2) * std::max<long long>(pool, 1))))
    return LHAF_ENOMEM;
  (void)cs;
  // descriptors first (the device gather reads them)
  if (cudaMemcpyAsync(ctx->b_items.p, hitems, sizeof(BatchItem) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:131");
  if (dev) {
    if (launch_batch_gather((const double2*)B, B_stride, (const double2*)gamma, M, M, (const BatchItem*)ctx->b_items.p,
                            batch, (double2*)ctx->b_chat.p, fp32 ? (float2*)ctx->b_chat32.p : nullptr, s) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:135");
  } else {
    if (!ctx->hb_chat.reserve(sizeof(double2) * std::max<long long>(pool, 1))) return LHAF_ENOMEM;
    std::complex<double>* hc = static_cast<std::complex<double>*>(ctx->hb_chat.p);
    for (int i : work)
      build_chat_host(plans[i], M, B + (size_t)i * B_stride, gamma ? gamma + (size_t)i * M : nullptr,
                      hc + hitems[i].chat_off);
    if (fp32) {
      if (!ctx->hb_chat32.reserve(sizeof(float2) * std::max<long long>(pool, 1))) return LHAF_ENOMEM;
      float2* h32 = static_cast<float2*>(ctx->hb_chat32.p);
      for (long long e = 0; e < pool; e++) h32[e] = make_float2((float)hc[e].real(), (float)hc[e].imag());
      if (cudaMemcpyAsync(ctx->b_chat32.p, h32, sizeof(float2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:147");
    } else if (pool > 0) {
      if (cudaMemcpyAsync(ctx->b_chat.p, hc, sizeof(double2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:150");
    }
  }

  // Items of degree <= kStageMaxDegree stage their term polynomials and finish them one term per
  // thread (series_units_kernel); larger degrees finish each term in the team (inline).
  const char* env_stage = std::getenv("LHAF_STAGE");
  const bool stage_ok = !(env_stage && env_stage[0] == '0');
  bool any_inline = false;
  int h_max_staged = 0;
  for (int i : work) {
    if (stage_ok && plans[i].h <= kStageMaxDegree) {
      h_max_staged = std::max(h_max_staged, plans[i].h);
    } else {
      any_inline = true;
    }
  }

  // ---- team size: tuned on the costliest item, shared-memory layout for the largest ----
  int team = 16, occ = 0;
  const void* chat_pool = fp32 ? ctx->b_chat32.p : ctx->b_chat.p;
  size_t team_bytes = 0, items_bytes = 0;
  if (rep >= 0) {
    const char* chatp = static_cast<const char*>(chat_pool) + (size_t)hitems[rep].chat_off * (fp32 ? 8 : 16);
    int occ_rep = 0;
    // tuned with the single-lhaf kernel on the costliest item's slot matrix (in the pool)
    team = pick_team(ctx, fp32, plans[rep], false, 1, chatp, &occ_rep);
    (void)occ_rep;
    if (team == 0) team = 32;
    team_bytes = team_shared_bytes(fp32, nd_max, H_max, 0, any_inline ? false : true);
    items_bytes = cta_table_bytes(fp32, Hl_max, H_max);
    // the fused series reuses the team area: (4h + 5) entries per CTA thread
    const size_t series_bytes = (size_t)(4 * h_max_staged + 5) * cta_threads(team) * (fp32 ? 8 : 16);
    if (h_max_staged > 0 && (size_t)teams_per_cta(team) * team_bytes < series_bytes)
      team_bytes = ((series_bytes + teams_per_cta(team) - 1) / teams_per_cta(team) + 15) & ~(size_t)15;
    while (items_bytes + (size_t)teams_per_cta(team) * team_bytes > 227 * 1024 && team < 128) {
      team *= 2;
      const size_t sb = (size_t)(4 * h_max_staged + 5) * cta_threads(team) * (fp32 ? 8 : 16);
      team_bytes = team_shared_bytes(fp32, nd_max, H_max, 0, any_inline ? false : true);
      if (h_max_staged > 0 && (size_t)teams_per_cta(team) * team_bytes < sb)
        team_bytes = ((sb + teams_per_cta(team) - 1) / teams_per_cta(team) + 15) & ~(size_t)15;
    }
    occ = batched_ctas_per_sm(fp32, team, items_bytes + (size_t)teams_per_cta(team) * team_bytes);
    if (occ <= 0) return LHAF_ETOOBIG;
  }
  const int TEAMS = teams_per_cta(team);

  // ---- work units: term ranges of similar cost, queue ordered longest first ----
  std::vector<BatchUnit> units;
  std::vector<double> ucost;
  std::vector<int> unit_begin(batch + 1, 0);
  const long long n_ctas = (long long)ctx->sms * std::max(occ, 1);
  const double target = cost_total / (double)(n_ctas * 8);
  for (int i = 0; i < batch; i++) {
    unit_begin[i] = (int)units.size();
    if (!runnable[i]) continue;
    const uint64_t T = plans[i].T;
    uint64_t ut = (uint64_t)std::ceil(target / std::max(fpt[i], 1.0));
    ut = std::min<uint64_t>(ut, 4096);  // bounds the per-CTA staging region
    ut = std::max<uint64_t>(ut, (uint64_t)TEAMS);
    ut = ((ut + TEAMS - 1) / TEAMS) * TEAMS;
    for (uint64_t t0 = 0; t0 < T; t0 += ut) {
      BatchUnit u;
      u.item = i;
      u.pad = 0;
      u.t0 = t0;
      u.t1 = std::min<uint64_t>(T, t0 + ut);
      u.stage_off = -1;
      u.w_off = 0;
      units.push_back(u);
      ucost.push_back(fpt[i] * (double)(u.t1 - u.t0));
    }
  }
  unit_begin[batch] = (int)units.size();
  const int n_units = (int)units.size();
  std::vector<int> queue(n_units);
  std::iota(queue.begin(), queue.end(), 0);
  std::stable_sort(queue.begin(), queue.end(), [&](int a, int b) { return ucost[a] > ucost[b]; });

  // Staged units: each CTA stages the polynomials of the unit it runs in a private region of
  // region_elems entries (the largest staged unit) and finishes them itself.
  const size_t cs_b = fp32 ? sizeof(float2) : sizeof(double2);
  const long long grid_b = std::min<long long>(n_ctas, std::max(n_units, 1));
  long long region_elems = 0, w_region = 0;
  for (const BatchUnit& u : units) {
    const Plan& pl = plans[u.item];
    if (!(stage_ok && pl.h <= kStageMaxDegree)) continue;
    const long long rows = pl.bord ? 2 * (long long)pl.h + 1 : (long long)pl.h;
    region_elems = std::max(region_elems, rows * (long long)(u.t1 - u.t0));
    w_region = std::max(w_region, (long long)(u.t1 - u.t0));
  }
  for (BatchUnit& u : units) {
    const Plan& pl = plans[u.item];
    const bool staged_u = stage_ok && pl.h <= kStageMaxDegree;
    u.stage_off = staged_u ? region_elems : -1;
    u.w_off = staged_u ? w_region : 0;
  }
  if (region_elems > 0 && (!ctx->b_stage.reserve((size_t)region_elems * grid_b * cs_b) ||
                           !ctx->b_wstage.reserve((size_t)w_region * grid_b * sizeof(double))))
    return LHAF_ENOMEM;

  if (!ctx->hb_units.reserve(sizeof(BatchUnit) * std::max(n_units, 1)) ||
      !ctx->b_units.reserve(sizeof(BatchUnit) * std::max(n_units, 1)) ||
      !ctx->hb_queue.reserve(sizeof(int) * std::max(n_units, 1)) ||
      !ctx->b_queue.reserve(sizeof(int) * std::max(n_units, 1)) || !ctx->b_next.reserve(sizeof(int)) ||
      !ctx->b_partials.reserve(sizeof(double) * 4 * (size_t)std::max(n_units, 1) * TEAMS))
    return LHAF_ENOMEM;
  std::memcpy(ctx->hb_units.p, units.data(), sizeof(BatchUnit) * n_units);
  std::memcpy(ctx->hb_queue.p, queue.data(), sizeof(int) * n_units);
  std::memcpy(ctx->hb_unit_begin.p, unit_begin.data(), sizeof(int) * (batch + 1));

  if (stats) {
    uint64_t terms = 0;
    double flops = 0.0;
    for (int i : work) {
      terms += plans[i].T;
      flops += fpt[i] * (double)plans[i].T;
    }
    stats->terms = terms;
    stats->n_dim = nd_max;
    stats->h = 0;
    for (int i : work) stats->h = std::max(stats->h, plans[i].h);
    stats->pairs = n_units;
    stats->team = team;
    stats->flops_model = flops;
  }

  // ---- launches ----
  bool ok = cudaMemcpyAsync(ctx->b_units.p, ctx->hb_units.p, sizeof(BatchUnit) * n_units, cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync(ctx->b_queue.p, ctx->hb_queue.p, sizeof(int) * n_units, cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync(ctx->b_unit_begin.p, ctx->hb_unit_begin.p, sizeof(int) * (batch + 1),
                            cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(ctx->b_item_h.p, ctx->hb_item_h.p, sizeof(int) * batch, cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemsetAsync(ctx->b_next.p, 0, sizeof(int), s) == cudaSuccess;
  if (!ok) return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:287");
  if (stats) cudaEventRecord(ctx->ev0, s);
  if (n_units > 0) {
    if (launch_batched(fp32, team, chat_pool, (const BatchItem*)ctx->b_items.p, (const BatchUnit*)ctx->b_units.p,
                       (const int*)ctx->b_queue.p, n_units, (int*)ctx->b_next.p, (double*)ctx->b_partials.p,
                       (int)team_bytes, (int)items_bytes, (int)grid_b, s, region_elems ? ctx->b_stage.p : nullptr,
                       region_elems ? (double*)ctx->b_wstage.p : nullptr) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:294");
  }
  double2* dout = dev ? (double2*)out : (double2*)ctx->b_out.p;
  if (launch_batch_reduce((const double*)ctx->b_partials.p, (const int*)ctx->b_unit_begin.p, (const int*)ctx->b_item_h.p,
                          TEAMS, batch, dout, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:299");
  if (stats) cudaEventRecord(ctx->ev1, s);
  if (!dev) {
    if (cudaMemcpyAsync(ctx->hb_out.p, ctx->b_out.p, sizeof(double2) * batch, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "lhaf_batched.cpp:303");
  }
  if (!dev || stats) {
    if (const cudaError_t e_ = (cudaStreamSynchronize(s)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaStreamSynchronize");
  }
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->kernel_ms = ms;
  }
  if (!dev) std::memcpy(out, ctx->hb_out.p, sizeof(double2) * batch);
  return LHAF_OK;
}
