// Batched loop hafnians (the chain-rule sampler's conditional probabilities, App. A.2 and
// App. B.5): many lhaf(B_n) of uneven size in one persistent launch, either planned per call
// (lhaf_batched) or planned once and replayed from a captured CUDA graph (lhaf_batched_plan_*).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_ctx.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"

using namespace lhafgpu;

namespace {

bool finite_c(const lhaf_c128& z) { return std::isfinite(z.re) && std::isfinite(z.im); }

// Everything the launches of one planned batch need.
struct BatchLaunch {
  int batch = 0, M = 0;
  bool fp32 = false;
  int team = 0, teams = 1, team_bytes = 0, items_bytes = 0, grid = 0, n_units = 0;
  long long region_elems = 0;
  long long B_stride = 0;
  int n_desc = 0;  // sieve descriptors (items, or their zero-digit groups)
  uint64_t h2d = 0;  // bytes planning copied host -> device
  int prep_launches = 0;  // kernels planning launched (the slot-matrix gather)
  uint64_t terms = 0;
  double flops = 0.0;
  int nd_max = 0, h_max = 0;
};

// Validity of the host entries item i reads (its occupied rows and columns of B, its gamma).
lhaf_status validate_item(int M, const int32_t* r, const lhaf_c128* Bi, const lhaf_c128* gi) {
  for (int a = 0; a < M; a++) {
    if (r[a] < 0) return LHAF_EINVAL;
    if (r[a] == 0) continue;
    if (gi && !finite_c(gi[a])) return LHAF_EINVAL;
    for (int b = a; b < M; b++)
      if (r[b] > 0 && !finite_c(Bi[(size_t)a * M + b])) return LHAF_EINVAL;
  }
  return LHAF_OK;
}

// Host planning of a batch into the buffers w: per-item plans and status, descriptors, the
// slot-matrix pool (built on the host from host inputs, or gathered on the device from device
// inputs), the team size (tuned on the costliest item), the work units and their queue. All
// uploads are ordered on the context's stream. B and gamma are host pointers unless dev_inputs.
lhaf_status prepare_batch(lhaf_ctx* ctx, BatchWork& w, int batch, int M, const lhaf_c128* B,
                          const lhaf_c128* gamma, const int32_t* reps, uint32_t flags, bool dev_inputs,
                          std::vector<lhaf_status>& st, BatchLaunch& L, uint64_t range_tb = 0,
                          uint64_t range_te = UINT64_MAX) {
  const bool per_item_B = (flags & LHAF_BATCH_B_PER_ITEM) != 0;
  const bool fp32 = (flags & LHAF_FP32_TERMS) != 0;
  // the previous planning's uploads read the pinned buffers rewritten below: let them finish
  if (w.uploaded) {
    if (const cudaError_t e_ = cudaEventSynchronize(w.uploaded); e_ != cudaSuccess)
      return (lhaf_status)record_cuda(e_, "cudaEventSynchronize");
  } else if (cudaEventCreateWithFlags(&w.uploaded, cudaEventDisableTiming) != cudaSuccess) {
    w.uploaded = nullptr;
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventCreate");
  }
  L = BatchLaunch();
  L.batch = batch;
  L.M = M;
  L.fp32 = fp32;
  L.B_stride = per_item_B ? (long long)M * M : 0;
  cudaStream_t s = ctx->stream;

  // ---- plans ----
  std::vector<Plan> plans(batch);
  st.assign(batch, LHAF_OK);
  std::vector<int> item_h(batch, 0);
  for (int i = 0; i < batch; i++) {
    const int32_t* r = reps + (size_t)i * M;
    const lhaf_c128* Bi = B + (size_t)i * L.B_stride;
    const lhaf_c128* gi = gamma ? gamma + (size_t)i * M : nullptr;
    const bool loops = !(flags & LHAF_NO_LOOPS);
    if (!dev_inputs) {
      st[i] = validate_item(M, r, Bi, gi);
    } else {
      for (int a = 0; a < M && st[i] == LHAF_OK; a++)
        if (r[a] < 0) st[i] = LHAF_EINVAL;
    }
    if (st[i] == LHAF_OK) st[i] = build_plan(M, r, flags, loops, plans[i]);
    if (st[i] == LHAF_OK && !dev_inputs && loops && plans[i].N > 0) {
      // host inputs: the loop border is dropped when no loop weight of the item is nonzero
      bool any = false;
      for (int q = 0; q < 2 * plans[i].P && !any; q++) {
        const int m = plans[i].slot_mode[q];
        if (m < 0) {
          any = true;
          break;
        }
        const lhaf_c128 g = gi ? gi[m] : Bi[(size_t)m * M + m];
        any = (g.re != 0.0 || g.im != 0.0);
      }
      if (!any) st[i] = build_plan(M, r, flags, false, plans[i]);
    }
    item_h[i] = st[i] != LHAF_OK ? INT_MAX : (plans[i].N == 0 ? -1 : plans[i].h);
  }
  // ---- sieves: one per item, or its zero-digit groups (numbered in order) ----
  struct Job {
    int item;
    Plan pl;
    uint64_t base;  // first term number of the job in its item's numbering
  };
  std::vector<Job> jobs;
  std::vector<int> job_begin(batch + 1, 0);
  for (int i = 0; i < batch; i++) {
    job_begin[i] = (int)jobs.size();
    if (!(st[i] == LHAF_OK && plans[i].N > 0)) continue;
    std::vector<Plan> subs;
    if (!(flags & LHAF_NO_ZERO_SPLIT) && split_zero_digits(plans[i], subs)) {
      uint64_t base = 0;
      for (Plan& sp : subs) {
        const uint64_t T = sp.T;
        jobs.push_back({i, std::move(sp), base});
        base += T;
      }
    } else {
      jobs.push_back({i, plans[i], 0});
    }
  }
  job_begin[batch] = (int)jobs.size();
  const int n_jobs = (int)jobs.size();

  // ---- per-sieve descriptors, slot-matrix pool, costs ----
  const int n_desc = std::max(n_jobs, 1);
  if (!w.h_items.reserve(sizeof(BatchItem) * n_desc) || !w.items.reserve(sizeof(BatchItem) * n_desc) ||
      !w.h_item_h.reserve(sizeof(int) * batch) || !w.item_h.reserve(sizeof(int) * batch) ||
      !w.h_unit_begin.reserve(sizeof(int) * (batch + 1)) || !w.unit_begin.reserve(sizeof(int) * (batch + 1)) ||
      !w.out.reserve(sizeof(double2) * batch) || !w.h_out.reserve(sizeof(double2) * batch))
    return LHAF_ENOMEM;
  BatchItem* hitems = static_cast<BatchItem*>(w.h_items.p);
  std::memset(hitems, 0, sizeof(BatchItem) * n_desc);
  long long pool = 0;
  int nd_max = 0, H_max = 0, Hl_max = 0, rep = -1;
  double cost_max = -1.0, cost_total = 0.0;
  std::vector<double> fpt(n_desc, 0.0);
  for (int j = 0; j < n_jobs; j++) {
    const Plan& pl = jobs[j].pl;
    fill_params(pl, fp32, false, 32, flags, hitems[j].p);
    hitems[j].chat_off = pool;
    hitems[j].src = jobs[j].item;
    for (int q = 0; q < kMaxDim; q++) hitems[j].slot_mode[q] = q < 2 * pl.P ? pl.slot_mode[q] : -1;
    pool += (long long)pl.nd * pl.nd;
    nd_max = std::max(nd_max, pl.nd);
    H_max = std::max(H_max, pl.H);
    Hl_max = std::max(Hl_max, pl.Hl);
    fpt[j] = lhaf_model_flops_per_term(pl.nd, pl.h, pl.bord);
    const double c = fpt[j] * (double)pl.T;
    cost_total += c;
    if (c > cost_max) {
      cost_max = c;
      rep = j;
    }
  }
  std::memcpy(w.h_item_h.p, item_h.data(), sizeof(int) * batch);
  if (!w.chat.reserve(sizeof(double2) * std::max<long long>(pool, 1)) ||
      (fp32 && !w.chat32.reserve(sizeof(float2) * std::max<long long>(pool, 1))))
    return LHAF_ENOMEM;
  L.n_desc = n_jobs;
  // descriptors first (the device gather reads them)
  if (n_jobs > 0 &&
      cudaMemcpyAsync(w.items.p, hitems, sizeof(BatchItem) * n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched descriptors");
  L.h2d += sizeof(BatchItem) * (uint64_t)n_jobs;
  if (dev_inputs) {
    if (launch_batch_gather((const double2*)B, L.B_stride, (const double2*)gamma, M, M, (const BatchItem*)w.items.p,
                            n_jobs, (double2*)w.chat.p, fp32 ? (float2*)w.chat32.p : nullptr, s) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batch gather");
    if (n_jobs > 0) L.prep_launches++;
  } else {
    L.h2d += (uint64_t)pool * (fp32 ? sizeof(float2) : sizeof(double2));
    if (!w.h_chat.reserve(sizeof(double2) * std::max<long long>(pool, 1))) return LHAF_ENOMEM;
    std::complex<double>* hc = static_cast<std::complex<double>*>(w.h_chat.p);
    for (int j = 0; j < n_jobs; j++) {
      const int i = jobs[j].item;
      build_chat_host(jobs[j].pl, M, B + (size_t)i * L.B_stride, gamma ? gamma + (size_t)i * M : nullptr,
                      hc + hitems[j].chat_off);
    }
    if (fp32) {
      if (!w.h_chat32.reserve(sizeof(float2) * std::max<long long>(pool, 1))) return LHAF_ENOMEM;
      float2* h32 = static_cast<float2*>(w.h_chat32.p);
      for (long long e = 0; e < pool; e++) h32[e] = make_float2((float)hc[e].real(), (float)hc[e].imag());
      if (cudaMemcpyAsync(w.chat32.p, h32, sizeof(float2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched slot matrices");
    } else if (pool > 0) {
      if (cudaMemcpyAsync(w.chat.p, hc, sizeof(double2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched slot matrices");
    }
  }

  // Items of degree <= kStageMaxDegree stage their term polynomials and finish them one term per
  // thread inside the CTA; larger degrees finish each term in the team (inline).
  const char* env_stage = std::getenv("LHAF_STAGE");
  const bool stage_ok = !(env_stage && env_stage[0] == '0');
  bool any_inline = false;
  int h_max_staged = 0;
  for (const Job& jb : jobs) {
    if (stage_ok && jb.pl.h <= kStageMaxDegree) {
      h_max_staged = std::max(h_max_staged, jb.pl.h);
    } else {
      any_inline = true;
    }
  }

  // ---- team size: tuned on the costliest item, shared-memory layout for the largest ----
  int team = 16, occ = 0;
  const void* chat_pool = fp32 ? w.chat32.p : w.chat.p;
  size_t team_bytes = 0, items_bytes = 0;
  if (rep >= 0) {
    const char* chatp = static_cast<const char*>(chat_pool) + (size_t)hitems[rep].chat_off * (fp32 ? 8 : 16);
    int occ_rep = 0;
    // tuned with the single-lhaf kernel on the costliest item's slot matrix (in the pool)
    team = pick_team(ctx, fp32, jobs[rep].pl, false, 1, chatp, &occ_rep);
    if (team == 0) team = 32;
    auto layout = [&](int g) {
      team_bytes = team_shared_bytes(fp32, nd_max, H_max, 0, !any_inline);
      items_bytes = cta_table_bytes(fp32, Hl_max, H_max);
      // the fused series reuses the team area: (4h + 5) entries per CTA thread
      const size_t series_bytes = (size_t)(4 * h_max_staged + 5) * cta_threads(g) * (fp32 ? 8 : 16);
      if (h_max_staged > 0 && (size_t)teams_per_cta(g) * team_bytes < series_bytes)
        team_bytes = ((series_bytes + teams_per_cta(g) - 1) / teams_per_cta(g) + 15) & ~(size_t)15;
    };
    layout(team);
    while (items_bytes + (size_t)teams_per_cta(team) * team_bytes > 227 * 1024 && team < 128) {
      team *= 2;
      layout(team);
    }
    occ = batched_ctas_per_sm(fp32, team, items_bytes + (size_t)teams_per_cta(team) * team_bytes);
    if (occ <= 0) return LHAF_ETOOBIG;
    occ = ctas_per_sm_override(occ);
  }
  const int TEAMS = teams_per_cta(team);

  // ---- work units: term ranges of similar cost, queue ordered longest first ----
  std::vector<BatchUnit> units;
  std::vector<double> ucost;
  std::vector<int> unit_begin(batch + 1, 0);
  const long long n_ctas = (long long)ctx->sms * std::max(occ, 1);
  const double target = cost_total / (double)(n_ctas * 8);
  uint64_t terms_run = 0;
  double flops_run = 0.0;
  for (int i = 0; i < batch; i++) {
    unit_begin[i] = (int)units.size();
    for (int j = job_begin[i]; j < job_begin[i + 1]; j++) {
      // this job's part of the item's term range [range_tb, range_te) (whole range for batches)
      const uint64_t base = jobs[j].base, T = jobs[j].pl.T;
      const uint64_t lo = range_tb > base ? std::min<uint64_t>(range_tb - base, T) : 0;
      const uint64_t hi = range_te > base ? std::min<uint64_t>(range_te - base, T) : 0;
      if (hi <= lo) continue;
      terms_run += hi - lo;
      flops_run += fpt[j] * (double)(hi - lo);
      uint64_t ut = (uint64_t)std::ceil(target / std::max(fpt[j], 1.0));
      ut = std::min<uint64_t>(ut, 4096);  // bounds the per-CTA staging region
      ut = std::max<uint64_t>(ut, (uint64_t)TEAMS);
      ut = ((ut + TEAMS - 1) / TEAMS) * TEAMS;
      for (uint64_t t0 = lo; t0 < hi; t0 += ut) {
        BatchUnit u;
        u.item = j;
        u.pad = 0;
        u.t0 = t0;
        u.t1 = std::min<uint64_t>(hi, t0 + ut);
        u.stage_off = -1;
        u.w_off = 0;
        units.push_back(u);
        ucost.push_back(fpt[j] * (double)(u.t1 - u.t0));
      }
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
    const Plan& pl = jobs[u.item].pl;
    if (!(stage_ok && pl.h <= kStageMaxDegree)) continue;
    const long long rows = pl.bord ? 2 * (long long)pl.h + 1 : (long long)pl.h;
    region_elems = std::max(region_elems, rows * (long long)(u.t1 - u.t0));
    w_region = std::max(w_region, (long long)(u.t1 - u.t0));
  }
  for (BatchUnit& u : units) {
    const Plan& pl = jobs[u.item].pl;
    const bool staged_u = stage_ok && pl.h <= kStageMaxDegree;
    u.stage_off = staged_u ? region_elems : -1;
    u.w_off = staged_u ? w_region : 0;
  }
  if (region_elems > 0 && (!w.stage.reserve((size_t)region_elems * grid_b * cs_b) ||
                           !w.wstage.reserve((size_t)w_region * grid_b * sizeof(double))))
    return LHAF_ENOMEM;

  if (!w.h_units.reserve(sizeof(BatchUnit) * std::max(n_units, 1)) ||
      !w.units.reserve(sizeof(BatchUnit) * std::max(n_units, 1)) ||
      !w.h_queue.reserve(sizeof(int) * std::max(n_units, 1)) || !w.queue.reserve(sizeof(int) * std::max(n_units, 1)) ||
      !w.next.reserve(sizeof(int)) || !w.partials.reserve(sizeof(double) * 4 * (size_t)std::max(n_units, 1) * TEAMS))
    return LHAF_ENOMEM;
  std::memcpy(w.h_units.p, units.data(), sizeof(BatchUnit) * n_units);
  std::memcpy(w.h_queue.p, queue.data(), sizeof(int) * n_units);
  std::memcpy(w.h_unit_begin.p, unit_begin.data(), sizeof(int) * (batch + 1));
  const bool ok =
      (n_units == 0 ||
       (cudaMemcpyAsync(w.units.p, w.h_units.p, sizeof(BatchUnit) * n_units, cudaMemcpyHostToDevice, s) ==
            cudaSuccess &&
        cudaMemcpyAsync(w.queue.p, w.h_queue.p, sizeof(int) * n_units, cudaMemcpyHostToDevice, s) == cudaSuccess)) &&
      cudaMemcpyAsync(w.unit_begin.p, w.h_unit_begin.p, sizeof(int) * (batch + 1), cudaMemcpyHostToDevice, s) ==
          cudaSuccess &&
      cudaMemcpyAsync(w.item_h.p, w.h_item_h.p, sizeof(int) * batch, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (!ok) return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched work units");
  L.h2d += (sizeof(BatchUnit) + sizeof(int)) * (uint64_t)n_units + sizeof(int) * (uint64_t)(2 * batch + 1);
  if (cudaEventRecord(w.uploaded, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventRecord");

  L.team = team;
  L.teams = TEAMS;
  L.team_bytes = (int)team_bytes;
  L.items_bytes = (int)items_bytes;
  L.grid = (int)grid_b;
  L.n_units = n_units;
  L.region_elems = region_elems;
  L.terms = terms_run;
  L.flops = flops_run;
  for (const Job& jb : jobs) L.h_max = std::max(L.h_max, jb.pl.h);
  L.nd_max = nd_max;
  return LHAF_OK;
}

// The launches of a prepared batch on stream s: queue reset, persistent kernel, per-item
// reduction into out (device, batch complex values).
lhaf_status enqueue_batch(BatchWork& w, const BatchLaunch& L, double2* out, cudaStream_t s,
                          double* out_dd = nullptr) {
  if (cudaMemsetAsync(w.next.p, 0, sizeof(int), s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched queue reset");
  if (L.n_units > 0) {
    const void* chat_pool = L.fp32 ? w.chat32.p : w.chat.p;
    if (launch_batched(L.fp32, L.team, chat_pool, (const BatchItem*)w.items.p, (const BatchUnit*)w.units.p,
                       (const int*)w.queue.p, L.n_units, (int*)w.next.p, (double*)w.partials.p, L.team_bytes,
                       L.items_bytes, L.grid, s, L.region_elems ? w.stage.p : nullptr,
                       L.region_elems ? (double*)w.wstage.p : nullptr) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched kernel");
  }
  if (launch_batch_reduce((const double*)w.partials.p, (const int*)w.unit_begin.p, (const int*)w.item_h.p, L.teams,
                          L.batch, out, s, out_dd) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched reduction");
  return LHAF_OK;
}

// Kernels of one enqueue_batch: the persistent kernel (when there is work) and the reduction.
int enqueue_launches(const BatchLaunch& L) { return (L.n_units > 0 ? 1 : 0) + 1; }

void fill_stats(const BatchLaunch& L, lhaf_stats* stats) {
  stats->h2d_bytes = L.h2d;
  stats->launches = L.prep_launches + enqueue_launches(L);
  stats->terms = L.terms;
  stats->n_dim = L.nd_max;
  stats->h = L.h_max;
  stats->pairs = L.n_units;
  stats->team = L.team;
  stats->flops_model = L.flops;
}

}  // namespace

extern "C" lhaf_status lhaf_batched(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                                    const int32_t* reps, uint32_t flags, lhaf_c128* out, lhaf_status* item_status,
                                    lhaf_stats* stats) {
  if (!ctx || batch < 0 || M <= 0 || !B || !reps || (batch > 0 && !out)) return LHAF_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (batch == 0) return LHAF_OK;
  const bool dev = (flags & LHAF_DEVICE_PTRS) != 0;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess)
    return (lhaf_status)record_cuda(e_, "cudaSetDevice");
  std::vector<lhaf_status> st;
  BatchLaunch L;
  BatchWork& w = ctx->bw;
  lhaf_status rc = prepare_batch(ctx, w, batch, M, B, gamma, reps, flags, dev, st, L);
  if (item_status && (int)st.size() == batch)
    for (int i = 0; i < batch; i++) item_status[i] = st[i];
  if (rc != LHAF_OK) return rc;
  cudaStream_t s = ctx->stream;
  if (stats) cudaEventRecord(ctx->ev0, s);
  rc = enqueue_batch(w, L, dev ? (double2*)out : (double2*)w.out.p, s);
  if (rc != LHAF_OK) return rc;
  if (stats) cudaEventRecord(ctx->ev1, s);
  if (!dev &&
      cudaMemcpyAsync(w.h_out.p, w.out.p, sizeof(double2) * batch, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched result copy");
  if (!dev || stats) {
    if (const cudaError_t e_ = (cudaStreamSynchronize(s)); e_ != cudaSuccess)
      return (lhaf_status)record_cuda(e_, "cudaStreamSynchronize");
  }
  if (stats) {
    fill_stats(L, stats);
    stats->d2h_bytes = dev ? 0 : sizeof(double2) * (uint64_t)batch;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->kernel_ms = ms;
  }
  if (!dev) std::memcpy(out, w.h_out.p, sizeof(double2) * batch);
  return LHAF_OK;
}

namespace lhafgpu {

lhaf_status run_split_single(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                             uint32_t flags, bool dev_inputs, uint64_t tb, uint64_t te, double* dd_dst,
                             double2* val_dst, lhaf_stats* stats) {
  std::vector<lhaf_status> st;
  BatchLaunch L;
  BatchWork& w = ctx->bw;
  lhaf_status rc = prepare_batch(ctx, w, 1, M, B, gamma, reps, flags & ~LHAF_BATCH_B_PER_ITEM, dev_inputs, st, L, tb,
                                 te);
  if (rc != LHAF_OK) return rc;
  if (st[0] != LHAF_OK) return st[0];
  if (stats) cudaEventRecord(ctx->ev0, ctx->stream);
  rc = enqueue_batch(w, L, val_dst, ctx->stream, dd_dst);
  if (rc != LHAF_OK) return rc;
  if (stats) {
    cudaEventRecord(ctx->ev1, ctx->stream);
    fill_stats(L, stats);
    stats->kernel_ms = 0.0;
  }
  return LHAF_OK;
}

}  // namespace lhafgpu

// ---------------------------------------------------------------------------------------------
// Batched plan: planning, tuning and buffers once; the launches captured in a CUDA graph.
// ---------------------------------------------------------------------------------------------

struct lhaf_batch_plan {
  lhaf_ctx* ctx = nullptr;
  BatchWork w;
  BatchLaunch L;
  std::vector<lhaf_status> st;
  std::vector<int32_t> reps;  // batch x M, for the checks of host inputs
  uint32_t flags = 0;
  bool with_gamma = false;
  long long B_elems = 0, g_elems = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~lhaf_batch_plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    w.release();
  }
};

namespace {

// Copies B and gamma (host or device per the plan's flags) into the plan's input buffers. Host
// inputs go through pinned staging, which is free: every host-input call synchronises before it
// returns.
lhaf_status load_inputs(lhaf_batch_plan* pl, const lhaf_c128* B, const lhaf_c128* gamma) {
  lhaf_ctx* ctx = pl->ctx;
  const bool dev = (pl->flags & LHAF_DEVICE_PTRS) != 0;
  const size_t bB = sizeof(lhaf_c128) * (size_t)pl->B_elems, bg = sizeof(lhaf_c128) * (size_t)pl->g_elems;
  const void* srcB = B;
  const void* srcg = gamma;
  cudaMemcpyKind kind = cudaMemcpyDeviceToDevice;
  if (!dev) {
    if (!pl->w.h_in.reserve(bB + bg)) return LHAF_ENOMEM;
    char* h = static_cast<char*>(pl->w.h_in.p);
    std::memcpy(h, B, bB);
    if (pl->with_gamma) std::memcpy(h + bB, gamma, bg);
    srcB = h;
    srcg = h + bB;
    kind = cudaMemcpyHostToDevice;
  }
  if (cudaMemcpyAsync(pl->w.in_B.p, srcB, bB, kind, ctx->stream) != cudaSuccess ||
      (pl->with_gamma && cudaMemcpyAsync(pl->w.in_gamma.p, srcg, bg, kind, ctx->stream) != cudaSuccess))
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched plan input copy");
  return LHAF_OK;
}

}  // namespace

extern "C" lhaf_status lhaf_batched_plan_create(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B,
                                                const lhaf_c128* gamma, const int32_t* reps, uint32_t flags,
                                                lhaf_batch_plan** plan) {
  if (!plan) return LHAF_EINVAL;
  *plan = nullptr;
  if (!ctx || batch <= 0 || M <= 0 || !B || !reps) return LHAF_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess)
    return (lhaf_status)record_cuda(e_, "cudaSetDevice");
  lhaf_batch_plan* pl = new (std::nothrow) lhaf_batch_plan();
  if (!pl) return LHAF_ENOMEM;
  pl->ctx = ctx;
  pl->flags = flags;
  pl->with_gamma = gamma != nullptr;
  pl->B_elems = (flags & LHAF_BATCH_B_PER_ITEM) ? (long long)batch * M * M : (long long)M * M;
  pl->g_elems = (long long)batch * M;
  pl->reps.assign(reps, reps + (size_t)batch * M);
  auto fail = [&](lhaf_status rc) {
    cudaStreamSynchronize(ctx->stream);  // no copy into the plan's buffers is left in flight
    delete pl;
    return rc;
  };
  if (!pl->w.in_B.reserve(sizeof(lhaf_c128) * (size_t)pl->B_elems) ||
      (pl->with_gamma && !pl->w.in_gamma.reserve(sizeof(lhaf_c128) * (size_t)pl->g_elems)))
    return fail(LHAF_ENOMEM);
  lhaf_status rc = load_inputs(pl, B, gamma);
  if (rc != LHAF_OK) return fail(rc);
  // The structure may not depend on the values: the loop border is present unless LHAF_NO_LOOPS,
  // and the slot matrices are gathered on the device from the plan's input buffers.
  rc = prepare_batch(ctx, pl->w, batch, M, (const lhaf_c128*)pl->w.in_B.p,
                     pl->with_gamma ? (const lhaf_c128*)pl->w.in_gamma.p : nullptr, reps, flags | LHAF_DEVICE_PTRS,
                     true, pl->st, pl->L);
  if (rc != LHAF_OK) return fail(rc);
  if (const cudaError_t e_ = cudaStreamSynchronize(ctx->stream); e_ != cudaSuccess)
    return fail((lhaf_status)record_cuda(e_, "cudaStreamSynchronize"));
  // capture: gather -> queue reset -> persistent kernel -> reduction
  if (cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) != cudaSuccess)
    return fail((lhaf_status)record_cuda(cudaPeekAtLastError(), "capture stream"));
  if (cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail((lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaStreamBeginCapture"));
  bool cap_ok = launch_batch_gather((const double2*)pl->w.in_B.p, pl->L.B_stride,
                                    pl->with_gamma ? (const double2*)pl->w.in_gamma.p : nullptr, M, M,
                                    (const BatchItem*)pl->w.items.p, pl->L.n_desc, (double2*)pl->w.chat.p,
                                    pl->L.fp32 ? (float2*)pl->w.chat32.p : nullptr, pl->cap) == cudaSuccess;
  if (cap_ok) cap_ok = enqueue_batch(pl->w, pl->L, (double2*)pl->w.out.p, pl->cap) == LHAF_OK;
  const cudaError_t ec = cudaStreamEndCapture(pl->cap, &pl->graph);
  if (!cap_ok || ec != cudaSuccess)
    return fail((lhaf_status)record_cuda(ec != cudaSuccess ? ec : cudaErrorUnknown, "batched graph capture"));
  if (const cudaError_t e_ = cudaGraphInstantiate(&pl->exec, pl->graph, 0); e_ != cudaSuccess)
    return fail((lhaf_status)record_cuda(e_, "cudaGraphInstantiate"));
  *plan = pl;
  return LHAF_OK;
}

extern "C" lhaf_status lhaf_batched_plan_exec(lhaf_batch_plan* pl, const lhaf_c128* B, const lhaf_c128* gamma,
                                              lhaf_c128* out, lhaf_status* item_status, lhaf_stats* stats) {
  if (!pl || !B || !out) return LHAF_EINVAL;
  if ((gamma != nullptr) != pl->with_gamma) return LHAF_EINVAL;
  lhaf_ctx* ctx = pl->ctx;
  const int batch = pl->L.batch, M = pl->L.M;
  const bool dev = (pl->flags & LHAF_DEVICE_PTRS) != 0;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess)
    return (lhaf_status)record_cuda(e_, "cudaSetDevice");
  // host inputs: an item reading a non-finite entry gets LHAF_EINVAL and NaN
  std::vector<lhaf_status> st = pl->st;
  if (!dev)
    for (int i = 0; i < batch; i++)
      if (st[i] == LHAF_OK)
        st[i] = validate_item(M, pl->reps.data() + (size_t)i * M, B + (size_t)i * pl->L.B_stride,
                              gamma ? gamma + (size_t)i * M : nullptr);
  lhaf_status rc = load_inputs(pl, B, gamma);
  if (rc != LHAF_OK) return rc;
  cudaStream_t s = ctx->stream;
  if (stats) cudaEventRecord(ctx->ev0, s);
  if (const cudaError_t e_ = cudaGraphLaunch(pl->exec, s); e_ != cudaSuccess)
    return (lhaf_status)record_cuda(e_, "cudaGraphLaunch");
  if (stats) cudaEventRecord(ctx->ev1, s);
  const size_t ob = sizeof(double2) * batch;
  const bool copy_ok =
      dev ? cudaMemcpyAsync(out, pl->w.out.p, ob, cudaMemcpyDeviceToDevice, s) == cudaSuccess
          : cudaMemcpyAsync(pl->w.h_out.p, pl->w.out.p, ob, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (!copy_ok) return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched plan result copy");
  if (!dev || stats) {
    if (const cudaError_t e_ = (cudaStreamSynchronize(s)); e_ != cudaSuccess)
      return (lhaf_status)record_cuda(e_, "cudaStreamSynchronize");
  }
  if (!dev) {
    std::memcpy(out, pl->w.h_out.p, ob);
    for (int i = 0; i < batch; i++)
      if (st[i] != LHAF_OK) out[i] = {NAN, NAN};
  }
  if (item_status)
    for (int i = 0; i < batch; i++) item_status[i] = st[i];
  if (stats) {
    fill_stats(pl->L, stats);
    // a replay copies only the inputs and results; its graph holds the gather and enqueue_batch
    stats->h2d_bytes = dev ? 0 : sizeof(lhaf_c128) * (uint64_t)(pl->B_elems + (pl->with_gamma ? pl->g_elems : 0));
    stats->d2h_bytes = dev ? 0 : ob;
    stats->launches = 1 + enqueue_launches(pl->L);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->kernel_ms = ms;
  }
  return LHAF_OK;
}

extern "C" void lhaf_batched_plan_destroy(lhaf_batch_plan* pl) {
  if (!pl) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(pl->ctx->device);
  delete pl;
  cudaSetDevice(prev);
}
