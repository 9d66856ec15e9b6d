// Batched loop hafnians (the chain-rule sampler's conditional probabilities, App. A.2, and the
// batching motivation of App. B.5): many lhaf(B_n) of uneven size, planned per call
// (lhaf_batched) or planned once and replayed from a captured CUDA graph (lhaf_batched_plan_*).
//
// Every item becomes one sieve, or its zero-digit groups (several smaller sieves). Sieves are
// sorted into classes by series mode (staged for degrees up to kStageMaxDegree, inline above) and
// working dimension, so each class gets its own team size, shared-memory layout and occupancy.
// A class runs as grouped terms launches (grid-strided chunks that never straddle two sieves) over
// chunk ranges sized to a staging budget; each launch ends in per-column values (the staged series,
// one term per thread, or the teams' per-chunk partials) that a segmented reduction adds to each
// item's double-double accumulator. A last kernel scales by 2^-h per item.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_ctx.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"

using namespace lhafgpu;

namespace {

// Per-launch budget of staged coefficient rows (staged classes) or per-chunk partials (inline).
constexpr size_t kLaunchBytes = (size_t)192 << 20;

// Working-dimension class bounds: a class holds the sieves with nd in (previous bound, bound].
constexpr int kClassBounds[] = {8, 10, 12, 14, 16, 18, 20, 22, 24, 26, 28, 30, 32, 36, 40, 44, 48, 56, 64};
constexpr int kNumBounds = (int)(sizeof(kClassBounds) / sizeof(kClassBounds[0]));

struct GLaunch {
  long long c0 = 0, c1 = 0;  // chunk range of the class
  int grid = 0, rounds = 0;
  long long sb_off = 0;      // first of its n_seg + 1 segment boundaries
  long long si_off = 0;      // first of its n_seg segment items
  int n_seg = 0;
};

struct GClass {
  bool staged = false;
  int team = 0, tpc = 1;
  int team_bytes = 0, items_bytes = 0;
  int h_max = 0, rows_max = 0;
  long long desc_off = 0;   // first descriptor of the class
  long long chunk_off = 0;  // first of its n_jobs + 1 chunk offsets
  int n_jobs = 0;
  long long cols_cap = 0;   // columns one launch stages (row stride of the staging buffer)
  std::vector<GLaunch> launches;
};

// Everything the launches of one planned batch need.
struct BatchLaunch {
  int batch = 0, M = 0;
  bool fp32 = false;
  long long B_stride = 0;
  int n_desc = 0;
  int plain = 0;
  std::vector<GClass> classes;
  uint64_t h2d = 0;       // bytes planning copied host -> device
  int prep_launches = 0;  // kernels planning launched (the slot-matrix gather)
  uint64_t terms = 0;
  double flops = 0.0;
  int nd_max = 0, h_max = 0, team = 0;
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

// Host planning of a batch into the buffers w: per-item plans and status, the sieves (zero-digit
// groups unless LHAF_NO_ZERO_SPLIT), their descriptors and slot matrices (built on the host from
// host inputs, or gathered on the device from device inputs), the classes with their tuned team
// sizes, and every launch's chunk range and item segments. All uploads are ordered on the
// context's stream. B and gamma are host pointers unless dev_inputs.
lhaf_status prepare_batch(lhaf_ctx* ctx, BatchWork& w, int batch, int M, const lhaf_c128* B,
                          const lhaf_c128* gamma, const int32_t* reps, uint32_t flags, bool dev_inputs,
                          std::vector<lhaf_status>& st, BatchLaunch& L) {
  const bool per_item_B = (flags & LHAF_BATCH_B_PER_ITEM) != 0;
  const bool fp32 = (flags & LHAF_FP32_TERMS) != 0;
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  // the previous planning's uploads read the pinned buffers rewritten below: let them finish
  if (w.uploaded) {
    if (const cudaError_t e = cudaEventSynchronize(w.uploaded); e != cudaSuccess)
      return (lhaf_status)record_cuda(e, "cudaEventSynchronize");
  } else if (cudaEventCreateWithFlags(&w.uploaded, cudaEventDisableTiming) != cudaSuccess) {
    w.uploaded = nullptr;
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventCreate");
  }
  L = BatchLaunch();
  L.batch = batch;
  L.M = M;
  L.fp32 = fp32;
  L.plain = (flags & LHAF_PLAIN_ACCUM) ? 1 : 0;
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
    if (st[i] == LHAF_OK && fp32 && plans[i].h > kFp32MaxDegree) st[i] = LHAF_ETOOBIG;  // FP32 beyond its bound
    item_h[i] = st[i] != LHAF_OK ? INT_MAX : (plans[i].N == 0 ? -1 : plans[i].h);
  }

  // ---- sieves, sorted into classes (series mode, working dimension), items in order ----
  const char* env_stage = std::getenv("LHAF_STAGE");
  const bool stage_ok = !(env_stage && env_stage[0] == '0');
  struct Job {
    int item;
    Plan pl;
  };
  std::vector<Job> jobs;
  for (int i = 0; i < batch; i++) {
    if (!(st[i] == LHAF_OK && plans[i].N > 0)) continue;
    std::vector<Plan> subs;
    if (!(flags & LHAF_NO_ZERO_SPLIT) && split_zero_digits(plans[i], subs)) {
      for (Plan& sp : subs) jobs.push_back({i, std::move(sp)});
    } else {
      jobs.push_back({i, plans[i]});
    }
  }
  const int n_jobs = (int)jobs.size();
  std::vector<std::vector<int>> members(2 * kNumBounds);
  for (int j = 0; j < n_jobs; j++) {
    const Plan& pl = jobs[j].pl;
    int b = 0;
    while (b + 1 < kNumBounds && pl.nd > kClassBounds[b]) b++;
    const bool staged = stage_ok && pl.h <= kStageMaxDegree;
    members[(staged ? 0 : kNumBounds) + b].push_back(j);
  }

  // ---- descriptors and slot-matrix pool, class after class ----
  const int n_desc = std::max(n_jobs, 1);
  if (!w.counter.reserve(sizeof(unsigned long long)) || !w.h_items.reserve(sizeof(BatchItem) * n_desc) ||
      !w.items.reserve(sizeof(BatchItem) * n_desc) ||
      !w.h_item_h.reserve(sizeof(int) * batch) || !w.item_h.reserve(sizeof(int) * batch) ||
      !w.acc.reserve(sizeof(double) * 4 * batch) || !w.out.reserve(sizeof(double2) * batch) ||
      !w.h_out.reserve(sizeof(double2) * batch))
    return LHAF_ENOMEM;
  BatchItem* desc = static_cast<BatchItem*>(w.h_items.p);
  std::memset(desc, 0, sizeof(BatchItem) * n_desc);
  std::vector<int> order;  // descriptor index -> job
  long long pool = 0;
  for (int c = 0; c < 2 * kNumBounds; c++) {
    if (members[c].empty()) continue;
    GClass cl;
    cl.staged = c < kNumBounds;
    cl.desc_off = (long long)order.size();
    cl.n_jobs = (int)members[c].size();
    for (int j : members[c]) {
      const Plan& pl = jobs[j].pl;
      BatchItem& d = desc[order.size()];
      fill_params(pl, fp32, cl.staged, 32, flags, d.p);
      d.p.t_end = pl.T;  // the sieve's term count (the kernel sets the per-chunk range)
      d.chat_off = pool;
      d.base = 0;
      d.src = jobs[j].item;
      for (int q = 0; q < kMaxDim; q++) d.slot_mode[q] = q < 2 * pl.P ? pl.slot_mode[q] : -1;
      pool += (long long)pl.nd * pl.nd;
      order.push_back(j);
    }
    L.classes.push_back(std::move(cl));
  }
  std::memcpy(w.h_item_h.p, item_h.data(), sizeof(int) * batch);
  if (!w.chat.reserve(sizeof(double2) * std::max<long long>(pool, 1)) ||
      (fp32 && !w.chat32.reserve(sizeof(float2) * std::max<long long>(pool, 1))))
    return LHAF_ENOMEM;
  L.n_desc = n_jobs;
  if (n_jobs > 0 &&
      cudaMemcpyAsync(w.items.p, desc, sizeof(BatchItem) * n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched descriptors");
  L.h2d += sizeof(BatchItem) * (uint64_t)n_jobs;
  if (dev_inputs) {
    if (launch_batch_gather((const double2*)B, L.B_stride, (const double2*)gamma, M, M, (const BatchItem*)w.items.p,
                            n_jobs, (double2*)w.chat.p, fp32 ? (float2*)w.chat32.p : nullptr, s) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batch gather");
    if (n_jobs > 0) L.prep_launches++;
  } else if (pool > 0) {
    if (!w.h_chat.reserve(sizeof(double2) * pool)) return LHAF_ENOMEM;
    std::complex<double>* hc = static_cast<std::complex<double>*>(w.h_chat.p);
    for (int d = 0; d < n_jobs; d++) {
      const int i = jobs[order[d]].item;
      build_chat_host(jobs[order[d]].pl, M, B + (size_t)i * L.B_stride, gamma ? gamma + (size_t)i * M : nullptr,
                      hc + desc[d].chat_off);
    }
    if (fp32) {
      if (!w.h_chat32.reserve(sizeof(float2) * pool)) return LHAF_ENOMEM;
      float2* h32 = static_cast<float2*>(w.h_chat32.p);
      for (long long e = 0; e < pool; e++) h32[e] = make_float2((float)hc[e].real(), (float)hc[e].imag());
      if (cudaMemcpyAsync(w.chat32.p, h32, sizeof(float2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched slot matrices");
    } else if (cudaMemcpyAsync(w.chat.p, hc, sizeof(double2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched slot matrices");
    }
    L.h2d += (uint64_t)pool * cs;
  }

  // ---- per class: team size, layout, occupancy, chunks, launches and segments ----
  std::vector<long long> chunk_off_all, seg_begin_all;
  std::vector<int> seg_item_all;
  size_t stage_bytes_max = 0, wstage_max = 0, entries_max = 0;
  const void* pool_ptr = fp32 ? w.chat32.p : w.chat.p;
  for (GClass& cl : L.classes) {
    int nd_max = 0, P_max = 0, Hl_max = 0, H_max = 0;
    long long rep = cl.desc_off;
    double cost_max = -1.0;
    for (long long d = cl.desc_off; d < cl.desc_off + cl.n_jobs; d++) {
      const Plan& pl = jobs[order[d]].pl;
      nd_max = std::max(nd_max, pl.nd);
      P_max = std::max(P_max, pl.P);
      Hl_max = std::max(Hl_max, pl.Hl);
      H_max = std::max(H_max, pl.H);
      cl.h_max = std::max(cl.h_max, pl.h);
      cl.rows_max = std::max(cl.rows_max, pl.bord ? 2 * pl.h + 1 : pl.h);
      const double fpt = lhaf_model_flops_per_term(pl.nd, pl.h, pl.bord);
      L.terms += pl.T;
      L.flops += fpt * (double)pl.T;
      L.h_max = std::max(L.h_max, pl.h);
      L.nd_max = std::max(L.nd_max, pl.nd);
      if (fpt * (double)pl.T > cost_max) {
        cost_max = fpt * (double)pl.T;
        rep = d;
      }
    }
    // team tuned on the class's costliest sieve (its slot matrix is in the pool already); a
    // staged trial stages into the context's buffer, grown here for it when that is possible
    const Plan& rp = jobs[order[rep]].pl;
    if (cl.staged) {
      const int rows = rp.bord ? 2 * rp.h + 1 : rp.h;
      const uint64_t trial = std::min<uint64_t>(rp.T, (uint64_t)ctx->partial_cap);
      ensure_stage(ctx, (size_t)rows * cs * trial, trial);  // on failure the tuner skips staged trials
    }
    int occ = 0;
    const char* chatp = static_cast<const char*>(pool_ptr) + (size_t)desc[rep].chat_off * cs;
    int team = pick_team(ctx, fp32, rp, cl.staged, 3, chatp, &occ);
    if (team == 0) team = 32;
    auto layout = [&](int g) {
      cl.team_bytes = (int)team_shared_bytes(fp32, nd_max, H_max, P_max, cl.staged);
      cl.items_bytes = (int)cta_table_bytes(fp32, Hl_max, H_max);
      return (size_t)cl.items_bytes + (size_t)teams_per_cta(g) * (size_t)cl.team_bytes;
    };
    while (layout(team) > 227 * 1024 && team < 128) team *= 2;
    const size_t smem = layout(team);
    if (smem > 227 * 1024) return LHAF_ETOOBIG;
    const int occ_g = grouped_ctas_per_sm(fp32, team, smem, cl.staged);
    if (occ_g <= 0) return LHAF_ETOOBIG;
    occ = ctas_per_sm_override(std::min(occ > 0 ? occ : occ_g, occ_g));
    cl.team = team;
    cl.tpc = teams_per_cta(team);
    L.team = std::max(L.team, team);
    // chunks of tpc terms per sieve; this class's offsets follow the previous classes'
    cl.chunk_off = (long long)chunk_off_all.size();
    std::vector<long long> coff(cl.n_jobs + 1, 0);
    for (int q = 0; q < cl.n_jobs; q++) {
      const uint64_t T = jobs[order[cl.desc_off + q]].pl.T;
      coff[q + 1] = coff[q] + (long long)((T + cl.tpc - 1) / cl.tpc);
    }
    chunk_off_all.insert(chunk_off_all.end(), coff.begin(), coff.end());
    // columns per launch: staged rows and weights plus the value entries, within the budget
    const size_t col_bytes =
        (cl.staged ? (size_t)cl.rows_max * cs + sizeof(double) : (size_t)0) + 4 * sizeof(double);
    long long cols = (long long)(kLaunchBytes / col_bytes);
    cols = std::max<long long>(cols / cl.tpc, 1) * cl.tpc;
    cl.cols_cap = cols;
    const long long chunks_per_launch = cols / cl.tpc;
    const long long n_chunks = coff[cl.n_jobs];
    const uint64_t max_ctas = (uint64_t)ctx->sms * (uint64_t)occ;
    for (long long c0 = 0; c0 < n_chunks; c0 += chunks_per_launch) {
      GLaunch lg;
      lg.c0 = c0;
      lg.c1 = std::min(n_chunks, c0 + chunks_per_launch);
      unsigned long long rounds = 1;
      lg.grid = (int)balanced_grid((uint64_t)(lg.c1 - lg.c0), 1, max_ctas, &rounds);
      lg.rounds = (int)rounds;
      // item segments over the launch's columns: adjacent ranges, consecutive sieves of one item
      // merged; boundaries b_0 = 0 < b_1 < ... < b_n_seg = columns
      lg.sb_off = (long long)seg_begin_all.size();
      lg.si_off = (long long)seg_item_all.size();
      seg_begin_all.push_back(0);
      int cur = -1;
      for (int q = 0; q < cl.n_jobs; q++) {
        const long long a = std::max(coff[q], lg.c0), b = std::min(coff[q + 1], lg.c1);
        if (b <= a) continue;
        const int item = jobs[order[cl.desc_off + q]].item;
        const long long eb = (b - lg.c0) * cl.tpc;
        if (item == cur) {
          seg_begin_all.back() = eb;
        } else {
          seg_begin_all.push_back(eb);
          seg_item_all.push_back(item);
          lg.n_seg++;
          cur = item;
        }
      }
      cl.launches.push_back(lg);
      if (cl.staged) {
        stage_bytes_max = std::max(stage_bytes_max, (size_t)cl.rows_max * cs * (size_t)cols);
        wstage_max = std::max(wstage_max, (size_t)cols);
      }
      entries_max = std::max(entries_max, (size_t)((lg.c1 - lg.c0) * cl.tpc));
    }
  }
  if (!w.h_chunks.reserve(sizeof(long long) * std::max<size_t>(chunk_off_all.size(), 1)) ||
      !w.chunks.reserve(sizeof(long long) * std::max<size_t>(chunk_off_all.size(), 1)) ||
      !w.h_seg_begin.reserve(sizeof(long long) * std::max<size_t>(seg_begin_all.size(), 1)) ||
      !w.seg_begin.reserve(sizeof(long long) * std::max<size_t>(seg_begin_all.size(), 1)) ||
      !w.h_seg_item.reserve(sizeof(int) * std::max<size_t>(seg_item_all.size(), 1)) ||
      !w.seg_item.reserve(sizeof(int) * std::max<size_t>(seg_item_all.size(), 1)) ||
      !w.entries.reserve(4 * sizeof(double) * std::max<size_t>(entries_max, 1)) ||
      (stage_bytes_max > 0 && (!w.stage.reserve(stage_bytes_max) || !w.wstage.reserve(sizeof(double) * wstage_max))))
    return LHAF_ENOMEM;
  std::memcpy(w.h_chunks.p, chunk_off_all.data(), sizeof(long long) * chunk_off_all.size());
  std::memcpy(w.h_seg_begin.p, seg_begin_all.data(), sizeof(long long) * seg_begin_all.size());
  std::memcpy(w.h_seg_item.p, seg_item_all.data(), sizeof(int) * seg_item_all.size());
  const bool ok =
      (chunk_off_all.empty() || cudaMemcpyAsync(w.chunks.p, w.h_chunks.p, sizeof(long long) * chunk_off_all.size(),
                                                cudaMemcpyHostToDevice, s) == cudaSuccess) &&
      (seg_begin_all.empty() || cudaMemcpyAsync(w.seg_begin.p, w.h_seg_begin.p,
                                                sizeof(long long) * seg_begin_all.size(), cudaMemcpyHostToDevice,
                                                s) == cudaSuccess) &&
      (seg_item_all.empty() || cudaMemcpyAsync(w.seg_item.p, w.h_seg_item.p, sizeof(int) * seg_item_all.size(),
                                               cudaMemcpyHostToDevice, s) == cudaSuccess) &&
      cudaMemcpyAsync(w.item_h.p, w.h_item_h.p, sizeof(int) * batch, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (!ok) return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched launch tables");
  L.h2d += sizeof(long long) * (chunk_off_all.size() + seg_begin_all.size()) + sizeof(int) * seg_item_all.size() +
           sizeof(int) * (size_t)batch;
  if (cudaEventRecord(w.uploaded, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventRecord");
  return LHAF_OK;
}

// The launches of a prepared batch on stream s: accumulator reset; per class and chunk range the
// grouped terms kernel, the series (staged classes) and the segmented reduction; then the per-item
// scaling into out (device, batch complex values).
lhaf_status enqueue_batch(BatchWork& w, const BatchLaunch& L, double2* out, cudaStream_t s) {
  if (cudaMemsetAsync(w.acc.p, 0, sizeof(double) * 4 * L.batch, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched accumulator reset");
  const void* pool_ptr = L.fp32 ? w.chat32.p : w.chat.p;
  const BatchItem* items = (const BatchItem*)w.items.p;
  const long long* chunks = (const long long*)w.chunks.p;
  const long long* segb = (const long long*)w.seg_begin.p;
  const int* segi = (const int*)w.seg_item.p;
  for (const GClass& cl : L.classes) {
    const BatchItem* cj = items + cl.desc_off;
    const long long* cc = chunks + cl.chunk_off;
    for (const GLaunch& lg : cl.launches) {
      if (cudaMemsetAsync(w.counter.p, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "chunk queue reset");
      cudaError_t e = launch_grouped_terms(
          L.fp32, cl.team, pool_ptr, cj, cl.n_jobs, cc, lg.c0, lg.c1, lg.grid, lg.rounds, 0ull, ~0ull,
          cl.team_bytes, cl.items_bytes, cl.staged ? nullptr : (double*)w.entries.p,
          cl.staged ? w.stage.p : nullptr, cl.staged ? (double*)w.wstage.p : nullptr,
          cl.staged ? cl.cols_cap : 0, s, cl.staged ? 0 : 1, (unsigned long long*)w.counter.p);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "grouped terms kernel");
      if (cl.staged) {
        e = launch_series_values(L.fp32, w.stage.p, (const double*)w.wstage.p, (lg.c1 - lg.c0) * cl.tpc, cl.cols_cap,
                                 cj, cl.n_jobs, cc, lg.c0, cl.tpc, cl.h_max, (double*)w.entries.p, s);
        if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "series kernel");
      }
      e = launch_segment_reduce((const double*)w.entries.p, segb + lg.sb_off, segi + lg.si_off, lg.n_seg, L.plain,
                                (double*)w.acc.p, s);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "segmented reduction");
    }
  }
  if (launch_item_finalize((const double*)w.acc.p, (const int*)w.item_h.p, L.batch, out, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched scaling");
  return LHAF_OK;
}

// Kernels of one enqueue_batch.
int enqueue_launches(const BatchLaunch& L) {
  int n = 1;
  for (const GClass& cl : L.classes)
    for (const GLaunch& lg : cl.launches) n += (cl.staged ? 2 : 1) + (lg.n_seg > 0 ? 1 : 0);
  return n;
}

void fill_stats(const BatchLaunch& L, lhaf_stats* stats) {
  stats->h2d_bytes = L.h2d;
  stats->launches = L.prep_launches + enqueue_launches(L);
  stats->terms = L.terms;
  stats->n_dim = L.nd_max;
  stats->h = L.h_max;
  stats->pairs = (int32_t)L.classes.size();
  stats->team = L.team;
  stats->flops_model = L.flops;
}

}  // namespace

extern "C" lhaf_status lhaf_batched(lhaf_ctx* ctx, int batch, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                                    const int32_t* reps, uint32_t flags, lhaf_c128* out, lhaf_status* item_status,
                                    lhaf_stats* stats) {
  if (!ctx || batch < 0 || M <= 0 || !B || !reps || (batch > 0 && !out)) return LHAF_EINVAL;
  if (flags & LHAF_ET) return LHAF_EINVAL;  // the eigenvalue-trace variant runs through lhaf / lhaf_range
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
  if (flags & LHAF_ET) return LHAF_EINVAL;
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
  // capture: gather -> accumulator reset -> grouped launches -> scaling
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
    // a replay copies only the inputs and results; its graph holds the gather and the launches
    stats->h2d_bytes = dev ? 0 : sizeof(lhaf_c128) * (uint64_t)(pl->B_elems + (pl->with_gamma ? pl->g_elems : 0));
    stats->d2h_bytes = dev ? 0 : ob;
    stats->launches = (pl->L.n_desc > 0 ? 1 : 0) + enqueue_launches(pl->L);
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
