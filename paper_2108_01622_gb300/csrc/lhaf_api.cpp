// Host side of the loop-hafnian library: pairing planner (App. B.3), slot matrix, term-space
// partition, team-size choice, workspace and the C ABI of include/lhaf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"
#include "lhaf_ctx.h"

using namespace lhafgpu;

namespace lhafgpu {
static thread_local char g_last_error[512] = "";
int record_cuda(cudaError_t e, const char* what) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();  // clear a non-sticky error so it is not reported twice
  return LHAF_ECUDA;
}
void record_message(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace lhafgpu

extern "C" const char* lhaf_last_error(void) { return lhafgpu::g_last_error; }

extern "C" const char* lhaf_strerror(lhaf_status s) {
  switch (s) {
    case LHAF_OK: return "ok";
    case LHAF_EINVAL: return "invalid argument";
    case LHAF_ETOOBIG: return "problem exceeds compiled limits (dimension, degree or term count)";
    case LHAF_ECUDA: return "CUDA runtime error";
    case LHAF_ETIMEOUT: return "device watchdog expired";
    case LHAF_ENOMEM: return "out of memory";
    case LHAF_ECANCELLED: return "cancelled";
  }
  return "unknown status";
}

extern "C" void lhaf_ctx_destroy(lhaf_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->d_chat);
  cudaFree(ctx->d_chat32);
  cudaFree(ctx->d_partials);
  cudaFree(ctx->d_out);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_wstage);
  cudaFreeHost(ctx->h_chat);
  cudaFreeHost(ctx->h_chat32);
  cudaFreeHost(ctx->h_out);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->tev0) cudaEventDestroy(ctx->tev0);
  if (ctx->tev1) cudaEventDestroy(ctx->tev1);
  ctx->bw.release();
  ctx->gw.release();
  ctx->b_gpart.release();
  ctx->b_gout.release();
  ctx->hb_gout.release();
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaSetDevice(prev);
  delete ctx;
}

extern "C" lhaf_status lhaf_ctx_create(lhaf_ctx** out, int device, void* cuda_stream) {
  if (!out) return LHAF_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LHAF_ECUDA;
  lhaf_ctx* c = new (std::nothrow) lhaf_ctx();
  if (!c) return LHAF_ENOMEM;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaSetDevice");
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaStreamCreate");
    }
    c->own_stream = true;
  }
  c->partial_cap = (size_t)c->sms * 32 * 16;  // max CTAs/SM x max teams/CTA
  const size_t nchat = (size_t)kMaxDim * kMaxDim;
  bool ok = cudaMalloc(&c->d_chat, nchat * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&c->d_chat32, nchat * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&c->d_partials, c->partial_cap * 4 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->d_out, 8 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&c->h_chat, nchat * sizeof(double2)) == cudaSuccess &&
            cudaMallocHost(&c->h_chat32, nchat * sizeof(float2)) == cudaSuccess &&
            cudaMallocHost(&c->h_out, 8 * sizeof(double)) == cudaSuccess &&
            cudaEventCreate(&c->ev0) == cudaSuccess && cudaEventCreate(&c->ev1) == cudaSuccess &&
            cudaEventCreate(&c->tev0) == cudaSuccess && cudaEventCreate(&c->tev1) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lhaf_ctx_destroy(c);
    return LHAF_ENOMEM;
  }
  *out = c;
  return LHAF_OK;
}

// Terms the sieve evaluates: the plan's, or the sum over its zero-digit groups, or over the
// support sizes of the eigenvalue-trace form (0 when its counts overflow).
static uint64_t evaluated_terms(const Plan& pl, uint32_t flags) {
  std::vector<Plan> subs;
  if (flags & LHAF_ET) {
    std::vector<unsigned long long> tab;
    if (pl.N == 0) return pl.T;
    if (!split_support_sizes(pl, subs, tab)) return 0;
    uint64_t T = 0;
    for (const Plan& s : subs) T += s.T;
    return T;
  }
  if (pl.N == 0 || (flags & LHAF_NO_ZERO_SPLIT) || !split_zero_digits(pl, subs)) return pl.T;
  uint64_t T = 0;
  for (const Plan& s : subs) T += s.T;
  return T;
}

extern "C" lhaf_status lhaf_plan(int M, const int32_t* reps, uint32_t flags, int has_loops, uint64_t* terms,
                                 int32_t* n_dim, int32_t* h, int32_t* pairs) {
  Plan pl;
  lhaf_status st = build_plan(M, reps, flags, has_loops != 0, pl);
  if (st != LHAF_OK) return st;
  const uint64_t T = evaluated_terms(pl, flags);
  if (T == 0) return LHAF_ETOOBIG;  // eigenvalue-trace counts above 2^62
  if (terms) *terms = T;
  if (n_dim) *n_dim = pl.nd;
  if (h) *h = pl.h;
  if (pairs) *pairs = pl.P;
  return LHAF_OK;
}

extern "C" lhaf_status lhaf_plan_groups(int M, const int32_t* reps, uint32_t flags, int has_loops, int32_t* groups) {
  if (!groups) return LHAF_EINVAL;
  Plan pl;
  lhaf_status st = build_plan(M, reps, flags, has_loops != 0, pl);
  if (st != LHAF_OK) return st;
  std::vector<Plan> subs;
  if (flags & LHAF_ET) {
    std::vector<unsigned long long> tab;
    *groups = (pl.N > 0 && split_support_sizes(pl, subs, tab)) ? (int32_t)subs.size() : 0;
    return LHAF_OK;
  }
  *groups = (pl.N > 0 && !(flags & LHAF_NO_ZERO_SPLIT) && split_zero_digits(pl, subs)) ? (int32_t)subs.size() : 0;
  return LHAF_OK;
}

extern "C" lhaf_status lhaf_combine(int count, const double* p, int32_t h, lhaf_c128* out) {
  if (count < 0 || (count > 0 && !p) || !out || h < 0) return LHAF_EINVAL;
  double rh = 0, rl = 0, ih = 0, il = 0;
  for (int i = 0; i < count; i++) {
    dd_add_dd_host(rh, rl, p[4 * i + 0], p[4 * i + 1]);
    dd_add_dd_host(ih, il, p[4 * i + 2], p[4 * i + 3]);
  }
  out->re = std::ldexp(rh + rl, -h);
  out->im = std::ldexp(ih + il, -h);
  return LHAF_OK;
}


namespace lhafgpu {

void fill_params(const Plan& pl, bool fp32, bool staged, int team, uint32_t flags, TermParams& p) {
  std::memset(&p, 0, sizeof(p));
  p.nd = pl.nd;
  p.ld = pl.nd | 1;
  p.bord = pl.bord;
  p.h = pl.h;
  p.H = pl.H;
  p.Hl = pl.Hl;
  p.P = pl.P;
  p.hp = pl.hp;
  p.hp_even = pl.hp_even;
  p.plain = (flags & LHAF_PLAIN_ACCUM) ? 1 : 0;
  p.skip_mask = 0u;
  for (int q = 0; q < pl.P && q < (int)pl.skip.size(); q++)
    if (pl.skip[q]) p.skip_mask |= 1u << q;
  p.wscale = pl.wscale;
  p.bq = -1;  // no batched-mode self pair
  p.bA = 0;
  p.n_items = pl.Hl * (pl.Hl - 1) / 2;
  p.team_bytes = (int)team_shared_bytes(fp32, pl.nd, pl.H, pl.P, staged);
  p.items_bytes = (int)(cta_shared_bytes(fp32, team, pl.nd, pl.H, pl.Hl, pl.P, staged) -
                        (size_t)teams_per_cta(team) * p.team_bytes);
  for (int q = 0; q < pl.P; q++) {
    p.eta[q] = pl.eta[q];
    p.radix[q] = pl.radix[q];
  }
}

// Resident CTAs per SM used for a launch: the occupancy limit, or fewer if LHAF_CTAS_PER_SM asks.
int ctas_per_sm_override(int occ) {
  const char* env = std::getenv("LHAF_CTAS_PER_SM");
  const int c = env ? std::atoi(env) : 0;
  return (c > 0 && c < occ) ? c : occ;
}

// Grid for n terms at tpc teams per CTA and at most max_ctas resident CTAs: the fewest rounds,
// then the fewest CTAs that finish n terms in that many rounds (so that at most tpc - 1 teams of
// the last round evaluate a padding term instead of a whole round's worth).
uint64_t balanced_grid(uint64_t n, int tpc, uint64_t max_ctas, unsigned long long* rounds) {
  if (max_ctas < 1) max_ctas = 1;
  uint64_t grid = (n + tpc - 1) / tpc;
  if (grid > max_ctas) grid = max_ctas;
  if (grid < 1) grid = 1;
  uint64_t r = (n + grid * tpc - 1) / (grid * tpc);
  if (r < 1) r = 1;
  const uint64_t teams = (n + r - 1) / r;
  grid = (teams + tpc - 1) / tpc;
  if (grid < 1) grid = 1;
  *rounds = (n + grid * tpc - 1) / (grid * tpc);
  if (*rounds < 1) *rounds = 1;
  return grid;
}

// Team size (lanes per term) and resident CTAs per SM. LHAF_TEAM forces the team size. Otherwise
// each candidate that fits in shared memory runs a short slice of real terms (two rounds of the
// resident grid), timed with CUDA events, at its occupancy limit and at the largest smaller CTA
// count that gives every SM sub-partition the same number of warps (the sub-partitions share the
// SM's FP64 unit, and one with an extra warp finishes last); the fastest per term is cached for
// the problem shape. Problems too small to time meaningfully use a model of FP64 lane utilisation
// times sub-partition coverage instead.
int pick_team(lhaf_ctx* ctx, bool fp32, const Plan& pl, bool staged, int family, const void* chat,
              int* ctas_per_sm) {
  const char* env = std::getenv("LHAF_TEAM");
  const int forced = env ? std::atoi(env) : 0;
  const int cands[5] = {8, 16, 32, 64, 128};
  int occs[5] = {0, 0, 0, 0, 0};
  double model_best = -1.0;
  int model_g = 0;
  for (int c = 0; c < 5; c++) {
    const int g = cands[c];
    if (forced && g != forced) continue;
    const size_t smem = cta_shared_bytes(fp32, g, pl.nd, pl.H, pl.Hl, pl.P, staged);
    if (smem > 227 * 1024) continue;
    occs[c] = max_ctas_per_sm(fp32, g, smem, staged);
    if (occs[c] <= 0) continue;
    const double warps = (double)occs[c] * cta_threads(g) / 32.0;
    const double score = model_lane_efficiency(pl.nd, pl.Hl, pl.h, pl.bord, g) * std::min(1.0, warps / 4.0) *
                         (warps >= 8.0 ? 1.0 : 0.9);
    if (score > model_best) {
      model_best = score;
      model_g = g;
    }
  }
  if (model_g == 0) return 0;
  auto occ_of = [&](int g) {
    for (int c = 0; c < 5; c++)
      if (cands[c] == g) return occs[c];
    return 0;
  };
  if (forced) {
    *ctas_per_sm = occ_of(forced);
    return forced;
  }
  const TuneKey key{fp32 ? 1 : 0, staged ? 1 : 0, pl.nd, pl.Hl, pl.h, pl.bord, family};
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end()) {
    *ctas_per_sm = it->second >> 16;
    return it->second & 0xffff;
  }
  const char* env_tune = std::getenv("LHAF_AUTOTUNE");
  const bool tune = !(env_tune && env_tune[0] == '0');
  int best_g = model_g, best_occ = occ_of(model_g);
  if (tune && chat) {
    double best_per_term = 1e300;
    bool too_small = false;
    for (int c = 0; c < 5 && !too_small; c++) {
      const int g = cands[c];
      if (occs[c] <= 0) continue;
      const int wpc = cta_threads(g) / 32;
      int occ_bal = occs[c];
      while (occ_bal > 0 && (occ_bal * wpc) % 4 != 0) occ_bal--;
      const int trials[2] = {occs[c], (occ_bal > 0 && occ_bal != occs[c] && occ_bal * wpc >= 4) ? occ_bal : 0};
      for (int o : trials) {
        if (o <= 0) continue;
        TermParams p;
        fill_params(pl, fp32, staged, g, 0, p);
        const uint64_t grid = (uint64_t)ctx->sms * (uint64_t)o;
        p.total_teams = grid * (uint64_t)teams_per_cta(g);
        if (p.total_teams > ctx->partial_cap) continue;
        const uint64_t S = std::min<uint64_t>(pl.T, 2 * p.total_teams);
        if (S < p.total_teams) {  // fewer terms than teams: too small to tell apart, use the model
          best_g = model_g;
          best_occ = occ_of(model_g);
          too_small = true;
          break;
        }
        p.rounds = (S + p.total_teams - 1) / p.total_teams;
        p.t_begin = 0;
        p.t_end = S;
        // the trial stages its own S terms at stride S (rows x S entries, within the buffer the
        // caller sized for rows x chunk with S <= chunk)
        void* stage = staged ? ctx->d_stage : nullptr;
        const long long stage_ld = staged ? (long long)S : 0;
        if (staged) {
          const size_t rows = pl.bord ? 2 * (size_t)pl.h + 1 : (size_t)pl.h;
          if (rows * S * (fp32 ? sizeof(float2) : sizeof(double2)) > ctx->stage_bytes || S > ctx->wstage_terms)
            continue;
        }
        float ms = 0.f;
        // one warm-up launch, then the fastest of three timed ones
        float best_ms = 1e30f;
        for (int rep = 0; rep < 4; rep++) {
          cudaEventRecord(ctx->tev0, ctx->stream);
          if (launch_terms(fp32, g, chat, p, (int)grid, ctx->d_partials, ctx->stream, stage, ctx->d_wstage,
                           stage_ld) != cudaSuccess) {
            cudaGetLastError();
            best_ms = -1.f;
            break;
          }
          cudaEventRecord(ctx->tev1, ctx->stream);
          cudaEventSynchronize(ctx->tev1);
          cudaEventElapsedTime(&ms, ctx->tev0, ctx->tev1);
          if (rep > 0 && ms < best_ms) best_ms = ms;
        }
        ms = best_ms;
        if (ms <= 0.f) continue;
        const double per_term = ms / (double)S;
        if (per_term < best_per_term) {
          best_per_term = per_term;
          best_g = g;
          best_occ = o;
        }
      }
    }
  }
  ctx->tuned[key] = best_g | (best_occ << 16);
  *ctas_per_sm = best_occ;
  return best_g;
}

}  // namespace lhafgpu

namespace {

bool has_loops_host(const Plan& pl, int M, const lhaf_c128* B, const lhaf_c128* gamma) {
  for (int s = 0; s < 2 * pl.P; s++) {
    const int m = pl.slot_mode[s];
    if (m < 0) return true;
    const lhaf_c128 g = gamma ? gamma[m] : B[(size_t)m * M + m];
    if (g.re != 0.0 || g.im != 0.0) return true;
  }
  return false;
}

lhaf_status validate_host_inputs(int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps) {
  for (int i = 0; i < M; i++) {
    const int r = reps ? reps[i] : 1;
    if (r < 0) return LHAF_EINVAL;
    if (r == 0) continue;
    for (int j = 0; j < M; j++) {
      const int r2 = reps ? reps[j] : 1;
      if (r2 == 0) continue;
      const int lo = std::min(i, j), hi = std::max(i, j);
      if (!finite_c(B[(size_t)lo * M + hi])) return LHAF_EINVAL;
    }
    if (gamma && !finite_c(gamma[i])) return LHAF_EINVAL;
  }
  return LHAF_OK;
}

// Staging buffer for the series kernel: grown on demand (terms x coefficient rows).
constexpr size_t kStageBytesMax = (size_t)256 << 20;

// Every launch of the sieve-term kernel covers at most kLaunchModelFlops of model work (about 0.25 s
// at GB300's FP64 rate; LHAF_LAUNCH_MFLOPS overrides, in millions). Unstaged launches (series
// finished inside the team, h > kStageMaxDegreeSingle) also hold at most kMaxChunkParts term
// slots, whose per-chunk partials are reduced in chunk order, so that a launch's sum does not
// depend on which CTA took which chunk (staged launches write their terms by column already).
constexpr double kLaunchModelFlops = 2.5e11;
constexpr uint64_t kMaxChunkParts = (uint64_t)1 << 21;

double launch_flops_budget() {
  const char* env = std::getenv("LHAF_LAUNCH_MFLOPS");
  const double v = env ? std::atof(env) * 1e6 : 0.0;
  return v > 0.0 ? v : kLaunchModelFlops;
}

}  // namespace

bool lhafgpu::ensure_stage(lhaf_ctx* ctx, size_t bytes, size_t terms) {
  if (ctx->stage_bytes >= bytes && ctx->wstage_terms >= terms) return true;
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_wstage);
  ctx->d_stage = nullptr;
  ctx->d_wstage = nullptr;
  ctx->stage_bytes = ctx->wstage_terms = 0;
  if (cudaMalloc(&ctx->d_stage, bytes) != cudaSuccess || cudaMalloc(&ctx->d_wstage, terms * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->d_stage);
    ctx->d_stage = nullptr;
    return false;
  }
  ctx->stage_bytes = bytes;
  ctx->wstage_terms = terms;
  return true;
}

namespace {

// One loop hafnian over its zero-digit groups `subs` (numbered group after group), restricted to
// [tb, te): grid-strided chunks that never straddle two groups (grouped_terms_kernel), then, for
// degrees up to kStageMaxDegreeSingle, the staged series one term per thread; both in launches sized to
// the staging buffer. Writes the unscaled dd partial to dd_dst and/or the value to val_dst.
lhaf_status run_grouped(lhaf_ctx* ctx, const Plan& pl, const std::vector<Plan>& subs, int M, const lhaf_c128* B,
                        const lhaf_c128* gamma, uint32_t flags, bool dev, uint64_t tb, uint64_t te, double* dd_dst,
                        double2* val_dst, lhaf_stats* stats, bool timed,
                        const std::vector<unsigned long long>* et_tab = nullptr) {
  const bool fp32 = (flags & LHAF_FP32_TERMS) != 0;
  const char* env_stage = std::getenv("LHAF_STAGE");
  bool staged = pl.h <= kStageMaxDegreeSingle && !(env_stage && env_stage[0] == '0');
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  const int rows = pl.bord ? 2 * pl.h + 1 : pl.h;
  BatchWork& w = ctx->gw;
  cudaStream_t s = ctx->stream;
  // the previous call's uploads read the pinned buffers rewritten below
  if (w.uploaded) {
    if (const cudaError_t e = cudaEventSynchronize(w.uploaded); e != cudaSuccess)
      return (lhaf_status)record_cuda(e, "cudaEventSynchronize");
  } else if (cudaEventCreateWithFlags(&w.uploaded, cudaEventDisableTiming) != cudaSuccess) {
    w.uploaded = nullptr;
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventCreate");
  }
  const int nj = (int)subs.size();
  const size_t et_bytes = et_tab ? sizeof(unsigned long long) * et_tab->size() : 0;
  if (et_tab && (!w.et_table.reserve(et_bytes) || !w.h_et_table.reserve(et_bytes))) return LHAF_ENOMEM;
  if (!w.counter.reserve(sizeof(unsigned long long)) || !w.h_items.reserve(sizeof(BatchItem) * nj) ||
      !w.items.reserve(sizeof(BatchItem) * nj) ||
      !w.h_chunks.reserve(sizeof(long long) * (nj + 1)) || !w.chunks.reserve(sizeof(long long) * (nj + 1)))
    return LHAF_ENOMEM;
  BatchItem* jobs = static_cast<BatchItem*>(w.h_items.p);
  std::memset(jobs, 0, sizeof(BatchItem) * nj);
  // Term numbering follows subs. A whole loop hafnian's sieves run in classes of equal working
  // dimension (largest first), each launch with the shared memory and occupancy of its class, when
  // the sieve is large enough that a launch per class costs less than the smaller classes gain
  // from their higher occupancy (measured on GB300: 12 % slower at 34,560 terms, 4 % faster at
  // 622,080); below 2048 terms per SM one launch runs every sieve.
  std::vector<uint64_t> orig_base(nj);
  uint64_t T_all = 0;
  for (int j = 0; j < nj; j++) {
    orig_base[j] = T_all;
    T_all += subs[j].T;
  }
  const char* env_cls = std::getenv("LHAF_ND_CLASSES");
  // A whole sieve always runs largest working dimension first, so that the chunks left for the
  // last wave of the queue are the cheapest ones.
  const bool big = T_all >= 2048ull * (uint64_t)std::max(ctx->sms, 1);
  const bool whole = nj > 1 && tb == 0 && te == T_all;
  const bool by_class = whole && (env_cls ? env_cls[0] == '1' : big);  // LHAF_ND_CLASSES=0/1 forces it
  std::vector<int> order(nj);
  for (int j = 0; j < nj; j++) order[j] = j;
  if (whole)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return subs[a].nd > subs[b].nd; });
  long long pool = 0;
  int nd_max = 0, P_max = 0, Hl_max = 0, rep = 0;
  double cost_max = -1.0;
  std::vector<uint64_t> bases(nj);
  for (int j = 0; j < nj; j++) {
    const Plan& sp = subs[order[j]];
    const uint64_t base = orig_base[order[j]];
    fill_params(sp, fp32, staged, 32, flags, jobs[j].p);
    jobs[j].p.t_end = sp.T;  // the sieve's term count (the kernel sets the per-chunk range)
    jobs[j].chat_off = pool;
    jobs[j].base = base;
    jobs[j].src = 0;
    for (int q = 0; q < kMaxDim; q++) jobs[j].slot_mode[q] = q < 2 * sp.P ? sp.slot_mode[q] : -1;
    if (et_tab) {
      // eigenvalue-trace support size sp.P: terms read the full slot matrix, which is the last
      // sieve's (all pairs kept), with the full pairs' counts
      jobs[j].p.et_P = pl.P;
      jobs[j].p.et_ndf = pl.nd;
      jobs[j].p.et_table = static_cast<const unsigned long long*>(w.et_table.p);
      for (int q = 0; q < pl.P; q++) jobs[j].p.eta[q] = pl.eta[q];
    }
    bases[j] = base;
    pool += (long long)sp.nd * sp.nd;
    nd_max = std::max(nd_max, sp.nd);
    P_max = std::max(P_max, sp.P);
    Hl_max = std::max(Hl_max, sp.Hl);
    const double c = lhaf_model_flops_per_term(sp.nd, sp.h, sp.bord) * (double)sp.T;
    if (c > cost_max) {
      cost_max = c;
      rep = j;
    }
  }
  if (!w.chat.reserve(sizeof(double2) * std::max<long long>(pool, 1)) ||
      (fp32 && !w.chat32.reserve(sizeof(float2) * std::max<long long>(pool, 1))))
    return LHAF_ENOMEM;
  if (et_tab) {
    int full = -1;  // the sieve that keeps every pair: its slot matrix is the full one
    for (int j = 0; j < nj; j++)
      if (subs[order[j]].P == pl.P) full = j;
    if (full < 0) return LHAF_EINVAL;
    for (int j = 0; j < nj; j++) jobs[j].p.et_off = jobs[full].chat_off - jobs[j].chat_off;
    std::memcpy(w.h_et_table.p, et_tab->data(), et_bytes);
    if (cudaMemcpyAsync(w.et_table.p, w.h_et_table.p, et_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "eigenvalue-trace rank table");
  }
  uint64_t h2d = sizeof(BatchItem) * (uint64_t)nj + et_bytes;
  int launches = 0, term_launches = 0;
  if (cudaMemcpyAsync(w.items.p, jobs, sizeof(BatchItem) * nj, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "group descriptors");
  if (dev) {
    if (launch_batch_gather((const double2*)B, 0, (const double2*)gamma, 0, M, (const BatchItem*)w.items.p, nj,
                            (double2*)w.chat.p, fp32 ? (float2*)w.chat32.p : nullptr, s) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "group slot-matrix gather");
    launches++;
  } else {
    if (!w.h_chat.reserve(sizeof(double2) * std::max<long long>(pool, 1))) return LHAF_ENOMEM;
    std::complex<double>* hc = static_cast<std::complex<double>*>(w.h_chat.p);
    for (int j = 0; j < nj; j++) build_chat_host(subs[order[j]], M, B, gamma, hc + jobs[j].chat_off);
    if (fp32) {
      if (!w.h_chat32.reserve(sizeof(float2) * std::max<long long>(pool, 1))) return LHAF_ENOMEM;
      float2* h32 = static_cast<float2*>(w.h_chat32.p);
      for (long long e = 0; e < pool; e++) h32[e] = make_float2((float)hc[e].real(), (float)hc[e].imag());
      if (cudaMemcpyAsync(w.chat32.p, h32, sizeof(float2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "group slot matrices");
    } else if (cudaMemcpyAsync(w.chat.p, hc, sizeof(double2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "group slot matrices");
    }
    h2d += (uint64_t)pool * cs;
  }
  // staging buffer first: the tuner's staged trial writes into it
  uint64_t cap_cols = 0;
  if (staged) {
    cap_cols = kStageBytesMax / ((size_t)rows * cs);
    cap_cols = std::min<uint64_t>(cap_cols, (uint64_t)ctx->partial_cap * 64);  // series blocks of 64 terms
    cap_cols = std::min<uint64_t>(cap_cols, T_all + 128 * (uint64_t)nj);     // at most every term plus padding
    if (!ensure_stage(ctx, (size_t)rows * cs * cap_cols, cap_cols)) staged = false;
  }
  const void* pool_ptr = fp32 ? w.chat32.p : w.chat.p;
  // launch classes: runs of sieves with one working dimension (one class when not by_class), each
  // with the team size tuned on its costliest sieve, its shared memory and its occupancy
  struct LaunchClass {
    int j0, j1, team, tpc, occ;
    long long c0, c1;
    size_t team_bytes, items_bytes;
  };
  std::vector<LaunchClass> classes;
  int team_rep = 0;  // the team of the class holding the costliest sieve (reported in stats)
  std::vector<long long> chunk_off(nj + 1, 0);
  for (int j0 = 0; j0 < nj;) {
    int j1 = j0 + 1;
    if (by_class)
      while (j1 < nj && subs[order[j1]].nd == subs[order[j0]].nd) j1++;
    else
      j1 = nj;
    int ndc = 0, Pc = 0, Hlc = 0, repc = j0;
    double costc = -1.0;
    for (int j = j0; j < j1; j++) {
      const Plan& sj = subs[order[j]];
      ndc = std::max(ndc, sj.nd);
      Pc = std::max(Pc, sj.P);
      Hlc = std::max(Hlc, sj.Hl);
      const double c = lhaf_model_flops_per_term(sj.nd, sj.h, sj.bord) * (double)sj.T;
      if (c > costc) {
        costc = c;
        repc = j;
      }
    }
    LaunchClass lc;
    lc.j0 = j0;
    lc.j1 = j1;
    int occ_t = 0;
    const char* chatp = static_cast<const char*>(pool_ptr) + (size_t)jobs[repc].chat_off * cs;
    lc.team = pick_team(ctx, fp32, subs[order[repc]], staged, 2, chatp, &occ_t);
    if (lc.team == 0) return LHAF_ETOOBIG;
    lc.tpc = teams_per_cta(lc.team);
    if (staged && cap_cols < (uint64_t)lc.tpc) return LHAF_ETOOBIG;  // a launch stages whole chunks
    lc.team_bytes = team_shared_bytes(fp32, ndc, pl.H, Pc, staged);
    lc.items_bytes = cta_table_bytes(fp32, Hlc, pl.H);
    const size_t smem_c = lc.items_bytes + (size_t)lc.tpc * lc.team_bytes;
    if (smem_c > 227 * 1024) return LHAF_ETOOBIG;
    const int occ_g = grouped_ctas_per_sm(fp32, lc.team, smem_c, staged);
    if (occ_g <= 0) return LHAF_ETOOBIG;
    lc.occ = ctas_per_sm_override(std::min(occ_t > 0 ? occ_t : occ_g, occ_g));
    if (rep >= j0 && rep < j1) team_rep = lc.team;
    // chunks of the class's tpc terms per sieve
    for (int j = j0; j < j1; j++)
      chunk_off[j + 1] = chunk_off[j] + (long long)((subs[order[j]].T + lc.tpc - 1) / lc.tpc);
    classes.push_back(lc);
    j0 = j1;
  }
  // the chunk range covering [tb, te) (one class when the range is partial)
  auto chunk_of = [&](uint64_t t) -> long long {  // chunk holding term t (t < T_all)
    int j = 0;
    while (j + 1 < nj && bases[j + 1] <= t) j++;
    return chunk_off[j] + (long long)((t - bases[j]) / classes[0].tpc);
  };
  long long kb = 0, ke = 0;
  if (whole) {
    ke = chunk_off[nj];  // the whole sieve (its sieves reordered by working dimension)
  } else if (te > tb) {
    kb = chunk_of(tb);
    ke = chunk_of(te - 1) + 1;
  }
  for (LaunchClass& lc : classes) {
    lc.c0 = std::max<long long>(chunk_off[lc.j0], kb);
    lc.c1 = std::min<long long>(chunk_off[lc.j1], ke);
  }
  long long* hco = static_cast<long long*>(w.h_chunks.p);
  std::memcpy(hco, chunk_off.data(), sizeof(long long) * (nj + 1));
  if (cudaMemcpyAsync(w.chunks.p, hco, sizeof(long long) * (nj + 1), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "group chunk offsets");
  h2d += sizeof(long long) * (uint64_t)(nj + 1);
  if (cudaEventRecord(w.uploaded, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventRecord");

  double* acc_dd = dd_dst ? dd_dst : ctx->d_out;
  if (timed) cudaEventRecord(ctx->ev0, s);
  int ci = 0;
  bool first = true;
  for (size_t cl = 0; cl < classes.size(); cl++) {
    const LaunchClass& lc = classes[cl];
    const bool last_class = cl + 1 == classes.size();
    if (lc.c1 <= lc.c0 && !(first && last_class)) continue;  // nothing of the range in this class
    first = false;
    // bounded launches: the class's costliest sieve sets the terms per launch (flop budget), and
    // the staging buffer (staged) or the per-chunk partial slots (inline series) cap it
    double fpt = 1.0;
    for (int j = lc.j0; j < lc.j1; j++) {
      const Plan& sj = subs[order[j]];
      fpt = std::max(fpt, lhaf_model_flops_per_term(sj.nd, sj.h, sj.bord));
    }
    const double budget_chunks = std::max(1.0, launch_flops_budget() / fpt / lc.tpc);
    long long span = 1;
    if (staged) {
      span = std::max<long long>(1, (long long)std::min<double>((double)(cap_cols / lc.tpc), budget_chunks));
    } else {
      span = std::max<long long>(1, (long long)std::min<double>(budget_chunks, (double)(kMaxChunkParts / lc.tpc)));
      span = std::min<long long>(span, std::max<long long>(1, lc.c1 - lc.c0));
      if (!w.parts.reserve(sizeof(double) * 4 * (size_t)span * (size_t)lc.tpc)) return LHAF_ENOMEM;
    }
    const uint64_t max_ctas = (uint64_t)ctx->sms * (uint64_t)lc.occ;
    long long c0 = lc.c0;
    do {
      const long long c1 = std::max(c0, std::min<long long>(lc.c1, c0 + std::max<long long>(span, 1)));
      const long long n = c1 - c0;  // chunks in this launch
      long long nparts = 0;
      if (n > 0) {
        unsigned long long rounds = 1;
        const uint64_t grid = balanced_grid((uint64_t)n, 1, max_ctas, &rounds);
        if (cudaMemsetAsync(w.counter.p, 0, sizeof(unsigned long long), s) != cudaSuccess)
          return (lhaf_status)record_cuda(cudaPeekAtLastError(), "chunk queue reset");
        cudaError_t e = launch_grouped_terms(fp32, lc.team, pool_ptr, (const BatchItem*)w.items.p, nj,
                                             (const long long*)w.chunks.p, c0, c1, (int)grid, (int)rounds, tb, te,
                                             (int)lc.team_bytes, (int)lc.items_bytes,
                                             staged ? ctx->d_partials : static_cast<double*>(w.parts.p),
                                             staged ? ctx->d_stage : nullptr, staged ? ctx->d_wstage : nullptr,
                                             staged ? (long long)cap_cols : 0, s, staged ? 0 : 1,
                                             (unsigned long long*)w.counter.p);
        if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "grouped terms kernel");
        launches++;
        term_launches++;
        if (staged) {
          e = launch_series(fp32, ctx->d_stage, ctx->d_wstage, n * lc.tpc, (long long)cap_cols, pl.h, pl.bord,
                            (flags & LHAF_PLAIN_ACCUM) ? 1 : 0, ctx->d_partials, s);
          if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "series kernel");
          launches++;
          nparts = series_blocks(n * lc.tpc);
        } else {
          nparts = n * lc.tpc;  // one partial per chunk term slot, in chunk order
        }
      }
      bool last = last_class && c1 >= lc.c1;
      if (!last && c1 >= lc.c1) {  // the last class with chunks in the range ends the sum
        last = true;
        for (size_t k2 = cl + 1; k2 < classes.size(); k2++)
          if (classes[k2].c1 > classes[k2].c0) last = false;
      }
      cudaError_t e = launch_reduce(staged ? ctx->d_partials : static_cast<double*>(w.parts.p), nparts, pl.h, acc_dd,
                                    last ? val_dst : nullptr, s, ci > 0 ? 1 : 0);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "reduction kernel");
      launches++;
      c0 = c1;
      ci++;
      if (last) break;
    } while (c0 < lc.c1);
  }
  if (timed) cudaEventRecord(ctx->ev1, s);
  if (stats) {
    double flops = 0.0;
    for (int j = 0; j < nj; j++) {
      const Plan& sj = subs[order[j]];
      const uint64_t lo = std::max<uint64_t>(tb, bases[j]), hi = std::min<uint64_t>(te, bases[j] + sj.T);
      if (hi > lo) flops += (double)(hi - lo) * lhaf_model_flops_per_term(sj.nd, sj.h, sj.bord);
    }
    stats->terms = te - tb;
    stats->n_dim = nd_max;
    stats->h = pl.h;
    stats->pairs = pl.P;
    stats->team = team_rep;
    stats->flops_model = flops;
    stats->kernel_ms = 0.0;
    stats->launches = launches;
    stats->term_launches = term_launches;
    stats->h2d_bytes = h2d;
  }
  return LHAF_OK;
}

lhaf_status lhaf_common(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                        uint32_t flags, bool ranged, uint64_t tb, uint64_t te, lhaf_c128* out, double* partial_dd,
                        lhaf_stats* stats) {
  if (!ctx || M <= 0 || !B) return LHAF_EINVAL;
  if (!ranged && !out) return LHAF_EINVAL;
  if (ranged && !partial_dd) return LHAF_EINVAL;
  const bool dev = (flags & LHAF_DEVICE_PTRS) != 0;
  if (!dev) {
    lhaf_status v = validate_host_inputs(M, B, gamma, reps);
    if (v != LHAF_OK) return v;
  } else if (reps) {
    for (int i = 0; i < M; i++)
      if (reps[i] < 0) return LHAF_EINVAL;
  }
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e_ = (cudaSetDevice(ctx->device)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaSetDevice");
  Plan pl;
  // Loop border: with host inputs, detected from gamma; with device inputs, present unless the
  // caller declares LHAF_NO_LOOPS.
  bool loops = !(flags & LHAF_NO_LOOPS);
  lhaf_status st = build_plan(M, reps, flags, loops, pl);
  if (st != LHAF_OK) return st;
  if ((flags & LHAF_FP32_TERMS) && pl.h > kFp32MaxDegree) return LHAF_ETOOBIG;  // beyond its stated bound
  if (!dev && loops && pl.N > 0 && !has_loops_host(pl, M, B, gamma)) {
    st = build_plan(M, reps, flags, false, pl);
    if (st != LHAF_OK) return st;
  }
  if (stats) std::memset(stats, 0, sizeof(*stats));
  std::vector<Plan> subs;
  std::vector<unsigned long long> et_tab;
  const bool et = (flags & LHAF_ET) != 0;
  if (et && pl.N > 0 && !split_support_sizes(pl, subs, et_tab)) return LHAF_ETOOBIG;
  const bool split = et ? pl.N > 0 : (pl.N > 0 && !(flags & LHAF_NO_ZERO_SPLIT) && split_zero_digits(pl, subs));
  uint64_t T_eval = pl.T;
  if (split) {
    T_eval = 0;
    for (const Plan& sp : subs) T_eval += sp.T;
  }
  if (ranged) {
    if (tb > te || te > T_eval) return LHAF_EINVAL;
  } else {
    tb = 0;
    te = T_eval;
  }
  if (pl.N == 0) {  // empty pattern: lhaf = 1 (one empty matching)
    if (ranged) {
      const double v[4] = {tb < te ? 1.0 : 0.0, 0.0, 0.0, 0.0};
      if (dev) return cudaMemcpyAsync(partial_dd, v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess
                          ? LHAF_OK
                          : LHAF_ECUDA;
      std::memcpy(partial_dd, v, sizeof(v));
      return LHAF_OK;
    }
    lhaf_c128 one = {1.0, 0.0};
    if (dev) {
      return cudaMemcpyAsync(out, &one, sizeof(one), cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess ? LHAF_OK
                                                                                                         : LHAF_ECUDA;
    }
    *out = one;
    return LHAF_OK;
  }
  const bool fp32 = (flags & LHAF_FP32_TERMS) != 0;
  const bool timed = stats != nullptr;
  double* dd_dst = ranged ? (dev ? partial_dd : ctx->d_out) : nullptr;
  double2* val_dst = ranged ? nullptr : (dev ? (double2*)out : (double2*)(ctx->d_out + 4));
  (void)fp32;
  if (!split) subs.assign(1, pl);  // one sieve on the full working matrix
  st = run_grouped(ctx, pl, subs, M, B, gamma, flags, dev, tb, te, dd_dst, val_dst, stats, timed,
                   et ? &et_tab : nullptr);
  if (st != LHAF_OK) return st;
  if (stats) stats->d2h_bytes = dev ? 0 : 6 * sizeof(double);
  if (!dev) {
    cudaError_t e = cudaMemcpyAsync(ctx->h_out, ctx->d_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "result copy");
  }
  if (!dev || timed) {
    if (const cudaError_t e_ = (cudaStreamSynchronize(ctx->stream)); e_ != cudaSuccess) return (lhaf_status)record_cuda(e_, "cudaStreamSynchronize");
  }
  if (timed) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->kernel_ms = ms;
  }
  if (!dev) {
    if (ranged) {
      std::memcpy(partial_dd, ctx->h_out, 4 * sizeof(double));
    } else {
      out->re = ctx->h_out[4];
      out->im = ctx->h_out[5];
    }
  }
  return LHAF_OK;
}

}  // namespace

extern "C" lhaf_status lhaf(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma, const int32_t* reps,
                            uint32_t flags, lhaf_c128* out, lhaf_stats* stats) {
  return lhaf_common(ctx, M, B, gamma, reps, flags, false, 0, 0, out, nullptr, stats);
}

extern "C" lhaf_status lhaf_range(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                                  const int32_t* reps, uint32_t flags, uint64_t term_begin, uint64_t term_end,
                                  double* partial_dd, lhaf_stats* stats) {
  return lhaf_common(ctx, M, B, gamma, reps, flags, true, term_begin, term_end, nullptr, partial_dd, stats);
}

extern "C" double lhaf_flops_per_term(int n_dim, int h, int bordered) {
  if (n_dim < 2 || n_dim > kMaxDim || h < 1) return 0.0;
  return lhaf_model_flops_per_term(n_dim, h, bordered ? 1 : 0);
}
