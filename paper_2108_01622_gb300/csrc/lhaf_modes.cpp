// Batched mode of one chain-rule step (arXiv:2108.01622, App. A.2 and App. B.5): the loop
// hafnians of n_fixed + n e_mode for every n = 0..n_cut with one sieve per outcome parity.
//
// The fixed photons are paired greedily (App. B.3); the batched mode's 2a photons (a = floor(n/2))
// form a self pair repeated a times, and an odd n's last photon pairs with the fixed pattern's
// leftover photon, or with a pad index of loop weight 1. For a parity class the self pair's
// delta' = a - 2k runs over -A..A (A = the class's largest a), and every term (fixed digits and the
// self delta') needs one Hessenberg reduction and characteristic polynomial; its series to the
// class's largest degree gives e_h for every outcome's degree h_n, and outcome n weighs the term
// by C(a, (a - delta')/2) (-1)^((a - delta')/2) where that digit exists.
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

double binom_host(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double c = 1.0;
  for (int i = 1; i <= k; i++) c = c * (double)(n - k + i) / (double)i;
  return std::round(c);
}

}  // namespace

extern "C" lhaf_status lhaf_batched_mode(lhaf_ctx* ctx, int M, const lhaf_c128* B, const lhaf_c128* gamma,
                                         const int32_t* reps, int mode, int n_cut, uint32_t flags, lhaf_c128* out,
                                         lhaf_stats* stats) {
  if (!ctx || M <= 0 || !B || !reps || !out || mode < 0 || mode >= M || n_cut < 0) return LHAF_EINVAL;
  if (flags & (LHAF_DEVICE_PTRS | LHAF_FP32_TERMS | LHAF_NO_REPEAT_SPEEDUP | LHAF_ET)) return LHAF_EINVAL;
  if (reps[mode] != 0) return LHAF_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  // the entries every outcome reads must be finite (the batched mode's row and loop included)
  for (int a = 0; a < M; a++) {
    if (reps[a] < 0) return LHAF_EINVAL;
    if (reps[a] == 0 && a != mode) continue;
    if (gamma && !finite_c(gamma[a])) return LHAF_EINVAL;
    for (int b = 0; b < M; b++) {
      if (reps[b] == 0 && b != mode) continue;
      if (!finite_c(B[(size_t)std::min(a, b) * M + std::max(a, b)])) return LHAF_EINVAL;
    }
  }
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (const cudaError_t e = cudaSetDevice(ctx->device); e != cudaSuccess)
    return (lhaf_status)record_cuda(e, "cudaSetDevice");
  Plan pf;
  lhaf_status st = build_plan(M, reps, flags, true, pf);
  if (st != LHAF_OK) return st;
  const int N_fixed = pf.N;
  struct PairDef {
    int a, b, eta;
  };
  std::vector<PairDef> fixed;
  int pad_q = -1;
  for (int q = 0; q < pf.P; q++) {
    fixed.push_back({pf.slot_mode[2 * q], pf.slot_mode[2 * q + 1], pf.eta[q]});
    if (pf.slot_mode[2 * q + 1] < 0) pad_q = q;
  }
  const int n_out_all = n_cut + 1;
  std::vector<int> item_h(n_out_all);
  for (int n = 0; n <= n_cut; n++) item_h[n] = (N_fixed + n == 0) ? -1 : (N_fixed + n + 1) / 2;

  BatchWork& w = ctx->bw;
  cudaStream_t s = ctx->stream;
  if (w.uploaded) {
    if (const cudaError_t e = cudaEventSynchronize(w.uploaded); e != cudaSuccess)
      return (lhaf_status)record_cuda(e, "cudaEventSynchronize");
  } else if (cudaEventCreateWithFlags(&w.uploaded, cudaEventDisableTiming) != cudaSuccess) {
    w.uploaded = nullptr;
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "cudaEventCreate");
  }
  if (!w.acc.reserve(sizeof(double) * 4 * n_out_all) || !w.out.reserve(sizeof(double2) * n_out_all) ||
      !w.h_out.reserve(sizeof(double2) * n_out_all) || !w.item_h.reserve(sizeof(int) * n_out_all) ||
      !w.h_item_h.reserve(sizeof(int) * n_out_all))
    return LHAF_ENOMEM;
  uint64_t terms_all = 0, h2d = sizeof(int) * (uint64_t)n_out_all;
  double flops_all = 0.0;
  int launches = 0, team_used = 0, nd_max = 0;

  // host staging of the per-class tables: [coefficients | outcome degrees | segments] per class
  struct ClassRun {
    Plan pl;
    int A = 0, bq = -1;
    std::vector<int> outs;  // outcome indices n of the class
  };
  std::vector<ClassRun> runs;
  for (int c = 0; c < 2; c++) {
    ClassRun cr;
    for (int n = c; n <= n_cut; n += 2)
      if (N_fixed + n > 0) cr.outs.push_back(n);
    if (cr.outs.empty()) continue;
    const int n_max = cr.outs.back();
    cr.A = n_max / 2;
    std::vector<PairDef> pairs = fixed;
    if (c == 1) {
      if (pad_q >= 0) {
        pairs[pad_q].b = mode;  // the fixed leftover photon pairs with the batched mode's last one
      } else {
        pairs.push_back({mode, -1, 1});  // the batched mode's last photon pairs with a pad index
      }
    }
    if (cr.A >= 1) {
      cr.bq = (int)pairs.size();
      pairs.push_back({mode, mode, cr.A});
    }
    Plan& p = cr.pl;
    p.M = M;
    p.N = N_fixed + n_max;
    p.h = (p.N + 1) / 2;
    if (p.h > kStageMaxDegree) return LHAF_ETOOBIG;  // the outcome series run staged
    p.P = (int)pairs.size();
    bool loops = false;
    for (const PairDef& d : pairs) {
      for (int m : {d.a, d.b}) {
        if (m < 0) {
          loops = true;
          continue;
        }
        const lhaf_c128 g = gamma ? gamma[m] : B[(size_t)m * M + m];
        if (g.re != 0.0 || g.im != 0.0) loops = true;
      }
    }
    p.bord = loops ? 1 : 0;
    p.nd = 2 * p.P + p.bord;
    if (p.P > kMaxPairs || p.nd > kMaxDim) return LHAF_ETOOBIG;
    p.H = p.h + p.bord;
    p.Hl = std::min(p.H, p.nd);
    p.slot_mode.resize(2 * p.P);
    p.eta.resize(p.P);
    p.radix.resize(p.P);
    p.skip.assign(p.P, 0);
    for (int q = 0; q < p.P; q++) {
      p.slot_mode[2 * q] = pairs[q].a;
      p.slot_mode[2 * q + 1] = pairs[q].b;
      p.eta[q] = pairs[q].eta;
    }
    // sign symmetry: an odd pair's digit halves exactly; else the self pair's delta' >= 0 (x2 for
    // delta' > 0)
    int hp = -1;
    for (int q = 0; q < p.P; q++)
      if (q != cr.bq && p.eta[q] % 2 == 1) {
        hp = q;
        break;
      }
    int hp_even = 0;
    if (hp < 0) hp = cr.bq;
    if (hp < 0) {
      // only even fixed pairs: the largest one's digit halves with its middle digit counted once
      hp = 0;
      for (int q = 1; q < p.P; q++)
        if (p.eta[q] > p.eta[hp]) hp = q;
      hp_even = 1;
    }
    p.hp = hp;
    p.hp_even = hp_even;
    uint64_t T = 1;
    for (int q = 0; q < p.P; q++) {
      int r;
      if (q == cr.bq) {
        r = (q == hp) ? cr.A + 1 : 2 * cr.A + 1;
      } else if (q == hp) {
        r = hp_even ? p.eta[q] / 2 + 1 : (p.eta[q] + 1) / 2;
      } else {
        r = p.eta[q] + 1;
      }
      p.radix[q] = r;
      T *= (uint64_t)r;
      if (T > ((uint64_t)1 << 62)) return LHAF_ETOOBIG;
    }
    p.T = T;
    runs.push_back(std::move(cr));
  }

  // Zero-digit groups of the fixed pairs (as for one loop hafnian): the middle digit of a fixed pair
  // with even eta gives delta' = 0, whose two slots vanish from the term. For every subset Z of
  // those pairs one sieve keeps Z at the middle digit with the slots deleted (constant weight
  // factor C(eta, eta/2) (-1)^(eta/2)) and lets the other even fixed pairs skip it; each such
  // group is closed under delta' -> -delta' and halves exactly on an odd fixed pair, else on an
  // even one without its middle digit, else on the self pair. Each group is its own launches and
  // uploads, so classes below 256 terms per SM (where that overhead outweighs the smaller
  // matrices: a 20-photon step ran 3.1 ms unsplit, 4.8 ms split) stay whole; LHAF_MODE_SPLIT=1 / 0
  // forces the split on or off.
  if (!(flags & LHAF_NO_ZERO_SPLIT)) {
    const char* env_split = std::getenv("LHAF_MODE_SPLIT");
    const uint64_t min_T = 256ull * (uint64_t)std::max(ctx->sms, 1);
    std::vector<ClassRun> split;
    for (const ClassRun& cr : runs) {
      const Plan& p = cr.pl;
      std::vector<int> even;
      for (int q = 0; q < p.P; q++)
        if (q != cr.bq && p.eta[q] >= 2 && p.eta[q] % 2 == 0) even.push_back(q);
      const bool want = env_split ? env_split[0] == '1' : p.T >= min_T;
      if (even.empty() || even.size() > 12 || !want) {
        split.push_back(cr);
        continue;
      }
      const int ne = (int)even.size();
      for (uint32_t zmask = 0; zmask < (1u << ne); zmask++) {
        std::vector<char> inZ(p.P, 0);
        double ws = 1.0;
        for (int b = 0; b < ne; b++)
          if (zmask >> b & 1) {
            const int q = even[b], e = p.eta[q];
            inZ[q] = 1;
            ws *= ((e / 2) % 2 ? -1.0 : 1.0) * binom_host(e, e / 2);
          }
        ClassRun sc;
        sc.A = cr.A;
        sc.outs = cr.outs;
        Plan& g = sc.pl;
        g.M = p.M;
        g.N = p.N;
        g.h = p.h;
        g.H = p.H;
        g.bord = p.bord;
        g.wscale = ws;
        for (int q = 0; q < p.P; q++) {
          if (inZ[q]) continue;
          if (q == cr.bq) sc.bq = (int)g.eta.size();
          g.slot_mode.push_back(p.slot_mode[2 * q]);
          g.slot_mode.push_back(p.slot_mode[2 * q + 1]);
          g.eta.push_back(p.eta[q]);
          g.skip.push_back((q != cr.bq && p.eta[q] % 2 == 0) ? 1 : 0);
        }
        g.P = (int)g.eta.size();
        if (g.P == 0) continue;  // every remaining delta' is 0: f = 0 (h >= 1 here)
        g.nd = 2 * g.P + g.bord;
        g.Hl = std::min(g.H, g.nd);
        int hp = -1;
        for (int q = 0; q < g.P && hp < 0; q++)
          if (q != sc.bq && g.eta[q] % 2 == 1) hp = q;
        for (int q = 0; q < g.P && hp < 0; q++)
          if (q != sc.bq && g.skip[q]) hp = q;
        if (hp < 0) hp = sc.bq;
        if (hp < 0) continue;  // unreachable: a remaining pair is odd, skips its middle or is the self pair
        g.hp = hp;
        g.hp_even = 0;
        g.radix.resize(g.P);
        uint64_t T = 1;
        for (int q = 0; q < g.P; q++) {
          int r;
          if (q == sc.bq) {
            r = (q == hp) ? sc.A + 1 : 2 * sc.A + 1;
          } else if (q == hp) {
            r = (g.eta[q] % 2) ? (g.eta[q] + 1) / 2 : g.eta[q] / 2;
            g.skip[q] = 0;  // its digits k < eta/2 never reach the middle
          } else {
            r = g.eta[q] + 1 - g.skip[q];
          }
          g.radix[q] = r;
          T *= (uint64_t)r;
        }
        g.T = T;
        split.push_back(std::move(sc));
      }
    }
    runs.swap(split);
  }

  std::memcpy(w.h_item_h.p, item_h.data(), sizeof(int) * n_out_all);
  if (cudaMemsetAsync(w.acc.p, 0, sizeof(double) * 4 * n_out_all, s) != cudaSuccess ||
      cudaMemcpyAsync(w.item_h.p, w.h_item_h.p, sizeof(int) * n_out_all, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode setup");
  if (stats) cudaEventRecord(ctx->ev0, s);
  for (const ClassRun& cr : runs) {
    const Plan& pl = cr.pl;
    const int A = cr.A;
    const int n_out = (int)cr.outs.size();
    // the previous uploads read the pinned buffers (slot matrix, tables) rewritten below
    if (cudaEventRecord(w.uploaded, s) != cudaSuccess || cudaEventSynchronize(w.uploaded) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode upload wait");
    // slot matrix
    build_chat_host(pl, M, B, gamma, (std::complex<double>*)ctx->h_chat);
    if (cudaMemcpyAsync(ctx->d_chat, ctx->h_chat, sizeof(double2) * pl.nd * pl.nd, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode slot matrix");
    h2d += sizeof(double2) * (uint64_t)pl.nd * pl.nd;
    // staging: rows of every term, its weight and its self delta' (second weight row)
    const int rows = pl.bord ? 2 * pl.h + 1 : pl.h;
    uint64_t cap = ((size_t)256 << 20) / ((size_t)rows * sizeof(double2));
    cap = std::min<uint64_t>(cap, (uint64_t)ctx->partial_cap * 64);
    cap = std::min<uint64_t>(cap, std::max<uint64_t>(pl.T, 64));
    if (!ensure_stage(ctx, (size_t)rows * sizeof(double2) * cap, 2 * cap)) return LHAF_ENOMEM;
    int occ = 0;
    const int team = pick_team(ctx, false, pl, true, 4, ctx->d_chat, &occ);
    if (team == 0) return LHAF_ETOOBIG;
    occ = ctas_per_sm_override(occ);
    team_used = std::max(team_used, team);
    nd_max = std::max(nd_max, pl.nd);
    TermParams p;
    fill_params(pl, false, true, team, flags, p);
    p.bq = cr.bq;
    p.bA = A;
    // outcome tables: degrees and coefficients (delta' = -A..A)
    std::vector<int> h_out(n_out);
    std::vector<double> coef((size_t)n_out * (2 * A + 1), 0.0);
    for (int t = 0; t < n_out; t++) {
      const int n = cr.outs[t], a = n / 2;
      h_out[t] = (N_fixed + n + 1) / 2;
      for (int dl = -A; dl <= A; dl++) {
        if (std::abs(dl) > a || ((a - dl) & 1)) continue;
        const int k = (a - dl) / 2;
        coef[(size_t)t * (2 * A + 1) + (dl + A)] = ((k & 1) ? -1.0 : 1.0) * binom_host(a, k);
      }
    }
    // chunks and their segments (one per outcome: its blocks' partials)
    const uint64_t T = pl.T;
    const uint64_t n_chunks = (T + cap - 1) / cap;
    std::vector<long long> segb;
    std::vector<int> segi;
    std::vector<long long> sb_off(n_chunks), si_off(n_chunks);
    for (uint64_t ck = 0; ck < n_chunks; ck++) {
      const uint64_t nn = std::min<uint64_t>(T, (ck + 1) * cap) - ck * cap;
      const long long blocks = series_blocks((long long)nn);
      sb_off[ck] = (long long)segb.size();
      si_off[ck] = (long long)segi.size();
      for (int t = 0; t <= n_out; t++) segb.push_back((long long)t * blocks);
      for (int t = 0; t < n_out; t++) segi.push_back(cr.outs[t]);
    }
    const size_t tab_bytes = sizeof(int) * h_out.size() + sizeof(double) * coef.size();
    if (!w.h_chunks.reserve(tab_bytes + 16) || !w.chunks.reserve(tab_bytes + 16) ||
        !w.h_seg_begin.reserve(sizeof(long long) * segb.size()) || !w.seg_begin.reserve(sizeof(long long) * segb.size()) ||
        !w.h_seg_item.reserve(sizeof(int) * segi.size()) || !w.seg_item.reserve(sizeof(int) * segi.size()) ||
        !w.entries.reserve(4 * sizeof(double) * (size_t)n_out * (size_t)series_blocks((long long)cap)))
      return LHAF_ENOMEM;
    // coefficient table first (8-byte aligned), then the outcome degrees
    char* ht = static_cast<char*>(w.h_chunks.p);
    std::memcpy(ht, coef.data(), sizeof(double) * coef.size());
    std::memcpy(ht + sizeof(double) * coef.size(), h_out.data(), sizeof(int) * h_out.size());
    std::memcpy(w.h_seg_begin.p, segb.data(), sizeof(long long) * segb.size());
    std::memcpy(w.h_seg_item.p, segi.data(), sizeof(int) * segi.size());
    if (cudaMemcpyAsync(w.chunks.p, w.h_chunks.p, tab_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.seg_begin.p, w.h_seg_begin.p, sizeof(long long) * segb.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(w.seg_item.p, w.h_seg_item.p, sizeof(int) * segi.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode tables");
    h2d += tab_bytes + sizeof(long long) * segb.size() + sizeof(int) * segi.size();
    const double* d_coef = static_cast<const double*>(w.chunks.p);
    const int* d_hout = reinterpret_cast<const int*>(static_cast<const char*>(w.chunks.p) + sizeof(double) * coef.size());
    const int tpc = teams_per_cta(team);
    const uint64_t max_ctas = (uint64_t)ctx->sms * (uint64_t)std::max(occ, 1);
    for (uint64_t ck = 0; ck < n_chunks; ck++) {
      const uint64_t t0 = ck * cap, t1 = std::min<uint64_t>(T, t0 + cap), nn = t1 - t0;
      unsigned long long rounds = 1;
      const uint64_t grid = balanced_grid(nn, tpc, max_ctas, &rounds);
      p.total_teams = grid * (uint64_t)tpc;
      p.rounds = rounds;
      p.t_begin = t0;
      p.t_end = t1;
      cudaError_t e = launch_terms(false, team, ctx->d_chat, p, (int)grid, ctx->d_partials, s, ctx->d_stage,
                                   ctx->d_wstage, (long long)cap);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "batched-mode terms kernel");
      e = launch_series_modes(false, ctx->d_stage, ctx->d_wstage, (long long)nn, (long long)cap, pl.h, pl.bord, n_out,
                              d_hout, d_coef, A, (double*)w.entries.p, s);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "batched-mode series kernel");
      e = launch_segment_reduce((const double*)w.entries.p, (const long long*)w.seg_begin.p + sb_off[ck],
                                (const int*)w.seg_item.p + si_off[ck], n_out, (flags & LHAF_PLAIN_ACCUM) ? 1 : 0,
                                (double*)w.acc.p, s);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "batched-mode reduction");
      launches += 3;
    }
    terms_all += T;
    flops_all += (double)T * lhaf_model_flops_per_term(pl.nd, pl.h, pl.bord);
  }
  if (launch_item_finalize((const double*)w.acc.p, (const int*)w.item_h.p, n_out_all, (double2*)w.out.p, s) !=
      cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode scaling");
  launches++;
  if (stats) cudaEventRecord(ctx->ev1, s);
  if (cudaEventRecord(w.uploaded, s) != cudaSuccess ||
      cudaMemcpyAsync(w.h_out.p, w.out.p, sizeof(double2) * n_out_all, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode result copy");
  if (const cudaError_t e = cudaStreamSynchronize(s); e != cudaSuccess)
    return (lhaf_status)record_cuda(e, "cudaStreamSynchronize");
  std::memcpy(out, w.h_out.p, sizeof(double2) * n_out_all);
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats->kernel_ms = ms;
    stats->terms = terms_all;
    stats->n_dim = nd_max;
    stats->h = (N_fixed + n_cut + 1) / 2;
    stats->pairs = (int32_t)runs.size();
    stats->team = team_used;
    stats->flops_model = flops_all;
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = sizeof(double2) * (uint64_t)n_out_all;
    stats->launches = launches;
  }
  return LHAF_OK;
}
