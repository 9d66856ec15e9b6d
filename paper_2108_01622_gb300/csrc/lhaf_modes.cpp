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
  int launches = 0, team_used = 0, nd_max_all = 0;

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
  // One parity class at a time: the slot matrices of all its sieves (zero-digit groups) in one
  // pool, one chunk queue over all of them (grouped launches, largest working dimension first,
  // chunks never straddle two sieves), the series of every staged column, one segment per outcome.
  for (int cls = 0; cls < 2; cls++) {
    std::vector<int> members;
    for (int ri = 0; ri < (int)runs.size(); ri++)
      if ((runs[ri].outs[0] & 1) == cls) members.push_back(ri);
    if (members.empty()) continue;
    std::stable_sort(members.begin(), members.end(),
                     [&](int a, int b) { return runs[a].pl.nd > runs[b].pl.nd; });
    const ClassRun& c0 = runs[members[0]];
    const int A = c0.A, n_out = (int)c0.outs.size();
    const int h = c0.pl.h, bord = c0.pl.bord, H = c0.pl.H;
    const int nj = (int)members.size();
    // the previous class's uploads read the pinned buffers rewritten below
    if (cudaEventRecord(w.uploaded, s) != cudaSuccess || cudaEventSynchronize(w.uploaded) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode upload wait");
    long long pool = 0;
    for (int ri : members) pool += (long long)runs[ri].pl.nd * runs[ri].pl.nd;
    if (!w.h_items.reserve(sizeof(BatchItem) * nj) || !w.items.reserve(sizeof(BatchItem) * nj) ||
        !w.h_chat.reserve(sizeof(double2) * pool) || !w.chat.reserve(sizeof(double2) * pool) ||
        !w.counter.reserve(sizeof(unsigned long long)))
      return LHAF_ENOMEM;
    BatchItem* jobs = static_cast<BatchItem*>(w.h_items.p);
    std::memset(jobs, 0, sizeof(BatchItem) * nj);
    std::complex<double>* hc = static_cast<std::complex<double>*>(w.h_chat.p);
    int nd_max = 0, P_max = 0, Hl_max = 0, rep = 0;
    double cost_max = -1.0;
    long long off = 0;
    for (int j = 0; j < nj; j++) {
      const ClassRun& cr = runs[members[j]];
      const Plan& g = cr.pl;
      fill_params(g, false, true, 32, flags, jobs[j].p);
      jobs[j].p.bq = cr.bq;
      jobs[j].p.bA = A;
      jobs[j].p.t_end = g.T;  // the sieve's term count (the kernel sets the per-chunk range)
      jobs[j].chat_off = off;
      for (int q = 0; q < kMaxDim; q++) jobs[j].slot_mode[q] = q < 2 * g.P ? g.slot_mode[q] : -1;
      build_chat_host(g, M, B, gamma, hc + off);
      off += (long long)g.nd * g.nd;
      nd_max = std::max(nd_max, g.nd);
      P_max = std::max(P_max, g.P);
      Hl_max = std::max(Hl_max, g.Hl);
      const double c = lhaf_model_flops_per_term(g.nd, g.h, g.bord) * (double)g.T;
      if (c > cost_max) {
        cost_max = c;
        rep = j;
      }
    }
    if (cudaMemcpyAsync(w.items.p, jobs, sizeof(BatchItem) * nj, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.chat.p, hc, sizeof(double2) * pool, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode sieves");
    h2d += sizeof(BatchItem) * (uint64_t)nj + sizeof(double2) * (uint64_t)pool;
    // staging first (the tuner's staged trial writes into it): coefficient rows of every term, its
    // weight and its self delta' (second weight row), at most 256 MB of rows per launch
    const int rows = bord ? 2 * h + 1 : h;
    uint64_t T_class = 0;
    for (int ri : members) T_class += runs[ri].pl.T;
    uint64_t cap = ((size_t)256 << 20) / ((size_t)rows * sizeof(double2));
    cap = std::min<uint64_t>(cap, (uint64_t)ctx->partial_cap * 64);
    cap = std::min<uint64_t>(cap, T_class + 32ull * (uint64_t)nj);  // every term plus chunk padding
    cap = std::max<uint64_t>(cap, 32);
    if (!ensure_stage(ctx, (size_t)rows * sizeof(double2) * cap, 2 * cap)) return LHAF_ENOMEM;
    // team size on the costliest sieve, the class's shared memory and occupancy
    int occ = 0;
    const double2* rep_chat = static_cast<const double2*>(w.chat.p) + jobs[rep].chat_off;
    const int team = pick_team(ctx, false, runs[members[rep]].pl, true, 4, rep_chat, &occ);
    if (team == 0) return LHAF_ETOOBIG;
    const int tpc = teams_per_cta(team);
    const size_t team_bytes = team_shared_bytes(false, nd_max, H, P_max, true);
    const size_t items_bytes = cta_table_bytes(false, Hl_max, H);
    const size_t smem = items_bytes + (size_t)tpc * team_bytes;
    if (smem > 227 * 1024) return LHAF_ETOOBIG;
    const int occ_g = grouped_ctas_per_sm(false, team, smem, true);
    if (occ_g <= 0) return LHAF_ETOOBIG;
    occ = ctas_per_sm_override(std::min(occ > 0 ? occ : occ_g, occ_g));
    team_used = std::max(team_used, team);
    nd_max_all = std::max(nd_max_all, nd_max);
    // chunks of tpc terms per sieve
    std::vector<long long> chunk_off(nj + 1, 0);
    for (int j = 0; j < nj; j++)
      chunk_off[j + 1] = chunk_off[j] + (long long)((runs[members[j]].pl.T + tpc - 1) / tpc);
    const long long n_chunks = chunk_off[nj];
    const long long span = std::max<long long>(1, (long long)(cap / tpc));  // chunks per launch
    // outcome tables: coefficients (delta' = -A..A) and degrees, after the chunk offsets
    std::vector<int> h_out(n_out);
    std::vector<double> coef((size_t)n_out * (2 * A + 1), 0.0);
    for (int t = 0; t < n_out; t++) {
      const int n = c0.outs[t], a = n / 2;
      h_out[t] = (N_fixed + n + 1) / 2;
      for (int dl = -A; dl <= A; dl++) {
        if (std::abs(dl) > a || ((a - dl) & 1)) continue;
        const int k = (a - dl) / 2;
        coef[(size_t)t * (2 * A + 1) + (dl + A)] = ((k & 1) ? -1.0 : 1.0) * binom_host(a, k);
      }
    }
    // per launch: the segments of its blocks (one per outcome)
    std::vector<long long> segb;
    std::vector<int> segi;
    std::vector<long long> sb_off, si_off;
    for (long long k0 = 0; k0 < n_chunks; k0 += span) {
      const long long nn = (std::min(n_chunks, k0 + span) - k0) * tpc;
      const long long blocks = series_blocks(nn);
      sb_off.push_back((long long)segb.size());
      si_off.push_back((long long)segi.size());
      for (int t = 0; t <= n_out; t++) segb.push_back((long long)t * blocks);
      for (int t = 0; t < n_out; t++) segi.push_back(c0.outs[t]);
    }
    const size_t tab_bytes =
        sizeof(long long) * (nj + 1) + sizeof(double) * coef.size() + sizeof(int) * h_out.size();
    if (!w.h_chunks.reserve(tab_bytes + 16) || !w.chunks.reserve(tab_bytes + 16) ||
        !w.h_seg_begin.reserve(sizeof(long long) * segb.size()) ||
        !w.seg_begin.reserve(sizeof(long long) * segb.size()) || !w.h_seg_item.reserve(sizeof(int) * segi.size()) ||
        !w.seg_item.reserve(sizeof(int) * segi.size()) ||
        !w.entries.reserve(4 * sizeof(double) * (size_t)n_out * (size_t)series_blocks((long long)(span * tpc))))
      return LHAF_ENOMEM;
    char* ht = static_cast<char*>(w.h_chunks.p);
    std::memcpy(ht, chunk_off.data(), sizeof(long long) * (nj + 1));
    std::memcpy(ht + sizeof(long long) * (nj + 1), coef.data(), sizeof(double) * coef.size());
    std::memcpy(ht + sizeof(long long) * (nj + 1) + sizeof(double) * coef.size(), h_out.data(),
                sizeof(int) * h_out.size());
    std::memcpy(w.h_seg_begin.p, segb.data(), sizeof(long long) * segb.size());
    std::memcpy(w.h_seg_item.p, segi.data(), sizeof(int) * segi.size());
    if (cudaMemcpyAsync(w.chunks.p, w.h_chunks.p, tab_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.seg_begin.p, w.h_seg_begin.p, sizeof(long long) * segb.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(w.seg_item.p, w.h_seg_item.p, sizeof(int) * segi.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      return (lhaf_status)record_cuda(cudaPeekAtLastError(), "batched-mode tables");
    h2d += tab_bytes + sizeof(long long) * segb.size() + sizeof(int) * segi.size();
    const long long* d_chunks = static_cast<const long long*>(w.chunks.p);
    const double* d_coef = reinterpret_cast<const double*>(static_cast<const char*>(w.chunks.p) +
                                                           sizeof(long long) * (nj + 1));
    const int* d_hout = reinterpret_cast<const int*>(static_cast<const char*>(w.chunks.p) +
                                                     sizeof(long long) * (nj + 1) + sizeof(double) * coef.size());
    const uint64_t max_ctas = (uint64_t)ctx->sms * (uint64_t)std::max(occ, 1);
    int li = 0;
    for (long long k0 = 0; k0 < n_chunks; k0 += span, li++) {
      const long long k1 = std::min(n_chunks, k0 + span);
      const long long nn = (k1 - k0) * tpc;  // staged columns of this launch (padding included)
      unsigned long long rounds = 1;
      const uint64_t grid = balanced_grid((uint64_t)(k1 - k0), 1, max_ctas, &rounds);
      if (cudaMemsetAsync(w.counter.p, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return (lhaf_status)record_cuda(cudaPeekAtLastError(), "chunk queue reset");
      cudaError_t e = launch_grouped_terms(false, team, w.chat.p, (const BatchItem*)w.items.p, nj, d_chunks, k0, k1,
                                           (int)grid, (int)rounds, 0ull, ~0ull, (int)team_bytes, (int)items_bytes,
                                           ctx->d_partials, ctx->d_stage, ctx->d_wstage, (long long)cap, s, 0,
                                           (unsigned long long*)w.counter.p);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "batched-mode terms kernel");
      e = launch_series_modes(false, ctx->d_stage, ctx->d_wstage, nn, (long long)cap, h, bord, n_out, d_hout, d_coef,
                              A, (double*)w.entries.p, s);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "batched-mode series kernel");
      e = launch_segment_reduce((const double*)w.entries.p, (const long long*)w.seg_begin.p + sb_off[li],
                                (const int*)w.seg_item.p + si_off[li], n_out, (flags & LHAF_PLAIN_ACCUM) ? 1 : 0,
                                (double*)w.acc.p, s);
      if (e != cudaSuccess) return (lhaf_status)record_cuda(e, "batched-mode reduction");
      launches += 3;
    }
    for (int ri : members) {
      terms_all += runs[ri].pl.T;
      flops_all += (double)runs[ri].pl.T * lhaf_model_flops_per_term(runs[ri].pl.nd, runs[ri].pl.h, runs[ri].pl.bord);
    }
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
    stats->n_dim = nd_max_all;
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
