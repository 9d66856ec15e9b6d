// Greedy pair matching (App. B.3), sieve term space (App. B.4) and cost models.
#include "lhaf_plan.h"

#include <algorithm>
#include <cmath>
#include <utility>

#include "lhaf_internal.h"

namespace lhafgpu {

lhaf_status build_plan(int M, const int32_t* reps, uint32_t flags, bool loops, Plan& pl) {
  pl = Plan();
  if (M <= 0) return LHAF_EINVAL;
  pl.M = M;
  long long N = 0;
  std::vector<std::pair<int, int>> cnt;  // (count, mode)
  for (int m = 0; m < M; m++) {
    const int r = reps ? reps[m] : 1;
    if (r < 0) return LHAF_EINVAL;
    if (r > 0) cnt.push_back({r, m});
    N += r;
  }
  if (N > 2LL * kMaxDegree) return LHAF_ETOOBIG;
  pl.N = (int)N;
  if (N == 0) {
    pl.T = 1;
    return LHAF_OK;
  }
  struct Pair {
    int a, b, eta;
  };
  std::vector<Pair> pairs;
  int leftover = -1;
  if (flags & LHAF_NO_REPEAT_SPEEDUP) {
    // every photon paired singly: the sieve of the explicit duplicated-row matrix
    std::vector<int> photons;
    for (auto& cm : cnt)
      for (int k = 0; k < cm.first; k++) photons.push_back(cm.second);
    size_t i = 0;
    for (; i + 1 < photons.size(); i += 2) pairs.push_back({photons[i], photons[i + 1], 1});
    if (i < photons.size()) leftover = photons[i];
  } else {
    // App. B.3: sort counts descending (ties: ascending mode); if n1 >= 2 n2 make floor(n1/2)
    // copies of (m1, m1), else n2 copies of (m1, m2); drop zeros; repeat while > 1 photon remains.
    long long rem = N;
    while (rem > 1) {
      std::stable_sort(cnt.begin(), cnt.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        if (x.first != y.first) return x.first > y.first;
        return x.second < y.second;
      });
      const int n1 = cnt[0].first, m1 = cnt[0].second;
      const int n2 = cnt.size() > 1 ? cnt[1].first : 0;
      if (n1 >= 2 * n2) {
        const int eta = n1 / 2;
        pairs.push_back({m1, m1, eta});
        cnt[0].first -= 2 * eta;
        rem -= 2 * eta;
      } else {
        pairs.push_back({m1, cnt[1].second, n2});
        cnt[0].first -= n2;
        cnt[1].first = 0;
        rem -= 2 * n2;
      }
      cnt.erase(std::remove_if(cnt.begin(), cnt.end(), [](const std::pair<int, int>& x) { return x.first == 0; }),
                cnt.end());
    }
    if (rem == 1) leftover = cnt[0].second;
  }
  if (leftover >= 0) pairs.push_back({leftover, -1, 1});  // pad index: loop weight 1, no couplings
  pl.P = (int)pairs.size();
  pl.bord = (loops || leftover >= 0) ? 1 : 0;
  pl.nd = 2 * pl.P + pl.bord;
  if (pl.P > kMaxPairs || pl.nd > kMaxDim) return LHAF_ETOOBIG;
  pl.h = (int)((N + 1) / 2);
  if (pl.h > kMaxDegree) return LHAF_ETOOBIG;
  pl.H = pl.h + pl.bord;
  pl.Hl = std::min(pl.H, pl.nd);
  pl.slot_mode.resize(2 * pl.P);
  pl.eta.resize(pl.P);
  pl.radix.resize(pl.P);
  pl.skip.assign(pl.P, 0);
  for (int q = 0; q < pl.P; q++) {
    pl.slot_mode[2 * q] = pairs[q].a;
    pl.slot_mode[2 * q + 1] = pairs[q].b;
    pl.eta[q] = pairs[q].eta;
  }
  // Sign symmetry (App. B.4): delta' -> -delta' leaves weight * f unchanged, so one digit is
  // halved. Prefer a pair with odd eta (exact half); otherwise the pair with the largest eta,
  // whose middle digit (delta' = 0) is counted once.
  int hp = -1;
  for (int q = 0; q < pl.P; q++)
    if (pl.eta[q] % 2 == 1) {
      hp = q;
      break;
    }
  if (hp < 0) {
    hp = 0;
    for (int q = 1; q < pl.P; q++)
      if (pl.eta[q] > pl.eta[hp]) hp = q;
  }
  pl.hp = hp;
  pl.hp_even = (pl.eta[hp] % 2 == 0) ? 1 : 0;
  long double T = 1.0L;
  uint64_t Ti = 1;
  for (int q = 0; q < pl.P; q++) {
    int r = pl.eta[q] + 1;
    if (q == hp) r = pl.hp_even ? pl.eta[q] / 2 + 1 : (pl.eta[q] + 1) / 2;
    pl.radix[q] = r;
    T *= (long double)r;
    if (T > 4.6e18L) return LHAF_ETOOBIG;  // 2^62
    Ti *= (uint64_t)r;
  }
  pl.T = Ti;
  return LHAF_OK;
}

bool split_support_sizes(const Plan& pl, std::vector<Plan>& subs, std::vector<unsigned long long>& table) {
  subs.clear();
  const int P = pl.P;
  const unsigned long long lim = 1ull << 62;
  table.assign((size_t)(P + 1) * (P + 1), 0ull);
  table[0] = 1ull;  // W[0][0]: the empty choice
  for (int i = 1; i <= P; i++) {
    const unsigned long long e = (unsigned long long)pl.eta[i - 1];
    for (int k = 0; k <= i; k++) {
      const unsigned long long out = table[(size_t)(i - 1) * (P + 1) + k];
      const unsigned long long in = k ? table[(size_t)(i - 1) * (P + 1) + k - 1] : 0ull;
      if (in > lim / e || out > lim - in * e) return false;
      table[(size_t)i * (P + 1) + k] = out + in * e;
    }
  }
  if (pl.h > 1000) return false;  // 2^h must stay a finite double
  for (int k = 1; k <= P; k++) {
    Plan s;
    s.M = pl.M;
    s.N = pl.N;
    s.h = pl.h;
    s.H = pl.H;
    s.bord = pl.bord;
    s.P = k;
    s.nd = 2 * k + pl.bord;
    s.Hl = std::min(s.H, s.nd);
    s.hp = -1;  // no sign symmetry: every term is evaluated
    s.hp_even = 0;
    s.wscale = std::ldexp(1.0, pl.h);
    for (int q = 0; q < k; q++) {
      s.slot_mode.push_back(pl.slot_mode[2 * q]);
      s.slot_mode.push_back(pl.slot_mode[2 * q + 1]);
      s.eta.push_back(pl.eta[q]);
      s.radix.push_back(pl.eta[q] + 1);
      s.skip.push_back(0);
    }
    s.T = table[(size_t)P * (P + 1) + k];
    if (s.T == 0) continue;
    subs.push_back(std::move(s));
  }
  return true;
}

bool split_zero_digits(const Plan& pl, std::vector<Plan>& subs) {
  subs.clear();
  std::vector<int> even;
  for (int q = 0; q < pl.P; q++)
    if (pl.eta[q] >= 2 && pl.eta[q] % 2 == 0) even.push_back(q);
  if (even.empty() || even.size() > 20) return false;
  const int ne = (int)even.size();
  for (uint32_t zmask = 0; zmask < (1u << ne); zmask++) {
    std::vector<char> inZ(pl.P, 0);
    double ws = 1.0;
    for (int b = 0; b < ne; b++)
      if (zmask >> b & 1) {
        const int q = even[b], e = pl.eta[q];
        inZ[q] = 1;
        // C(e, e/2) (-1)^(e/2), exact in double for the counts allowed here
        double c = 1.0;
        for (int i = 1; i <= e / 2; i++) c = c * (double)(e / 2 + i) / (double)i;
        ws *= ((e / 2) % 2) ? -c : c;
      }
    Plan s;
    s.M = pl.M;
    s.N = pl.N;
    s.h = pl.h;
    s.H = pl.H;
    s.bord = pl.bord;
    s.wscale = ws;
    for (int q = 0; q < pl.P; q++) {
      if (inZ[q]) continue;
      s.src_pair.push_back(q);
      s.slot_mode.push_back(pl.slot_mode[2 * q]);
      s.slot_mode.push_back(pl.slot_mode[2 * q + 1]);
      s.eta.push_back(pl.eta[q]);
      s.skip.push_back(pl.eta[q] % 2 == 0 ? 1 : 0);
    }
    s.P = (int)s.eta.size();
    if (s.P == 0) continue;  // every delta' = 0: f = 0
    s.nd = 2 * s.P + s.bord;
    s.Hl = std::min(s.H, s.nd);
    // halving: the first odd pair (digits k < (eta+1)/2), else the first pair, whose digits
    // without the middle split into k < eta/2 and their mirror images
    int hp = -1;
    for (int q = 0; q < s.P; q++)
      if (s.eta[q] % 2 == 1) {
        hp = q;
        break;
      }
    if (hp < 0) hp = 0;
    s.hp = hp;
    s.hp_even = 0;
    s.radix.resize(s.P);
    uint64_t T = 1;
    for (int q = 0; q < s.P; q++) {
      int r = s.eta[q] + 1 - s.skip[q];
      if (q == hp) {
        r = (s.eta[q] % 2) ? (s.eta[q] + 1) / 2 : s.eta[q] / 2;
        s.skip[q] = 0;  // its digits k < eta/2 never reach the middle
      }
      s.radix[q] = r;
      T *= (uint64_t)r;
    }
    s.T = T;
    subs.push_back(std::move(s));
  }
  return true;
}

void build_chat_host(const Plan& pl, int M, const lhaf_c128* B, const lhaf_c128* gamma, std::complex<double>* chat) {
  const int nd = pl.nd, b = pl.bord, n = 2 * pl.P;
  auto Bat = [&](int i, int j) {
    const int lo = std::min(i, j), hi = std::max(i, j);
    const lhaf_c128 z = B[(size_t)lo * M + hi];
    return std::complex<double>(z.re, z.im);
  };
  for (int i = 0; i < nd * nd; i++) chat[i] = 0.0;
  if (b) {
    for (int s = 0; s < n; s++) {
      const int m = pl.slot_mode[s];
      std::complex<double> v = 1.0;
      if (m >= 0) v = gamma ? std::complex<double>(gamma[m].re, gamma[m].im) : Bat(m, m);
      chat[0 * nd + (b + s)] = v;
      chat[(b + s) * nd + 0] = v;
    }
  }
  for (int s = 0; s < n; s++)
    for (int t = 0; t < n; t++) {
      const int ms = pl.slot_mode[s], mt = pl.slot_mode[t];
      if (ms >= 0 && mt >= 0) chat[(b + s) * nd + (b + t)] = Bat(ms, mt);
    }
}

static long long push_items_valid(int nd, int Hl, int l) {
  const int deg = nd - l - 1;
  long long c = 0;
  for (int d = 2; d <= Hl; d++) {
    if (l - d + 1 < 0) break;
    const int emax = std::min(Hl - d, deg);
    if (emax >= 0) c += emax + 1;
  }
  return c;
}

double lhaf_model_flops_per_term(int nd, int h, int bord) {
  const int H = h + bord, Hl = std::min(H, nd);
  double macs = 0.0;
  for (int k = 0; k + 2 < nd; k++) {
    const double m = nd - k - 1;
    macs += (m - 1) + (m - 1) * m + nd * (m - 1);
  }
  for (int j = 0; j < nd - 1; j++) macs += 2.0 * std::min(Hl - 1, nd - 1 - j);
  for (int l = nd - 1; l >= 0; l--) macs += (double)push_items_valid(nd, Hl, l) + std::min(Hl, nd - l);
  for (int k = 1; k <= h; k++) macs += 3.0 * k - 1.0;
  return 8.0 * macs;
}

static double rnd(double items, int G) { return items > 0 ? std::ceil(items / G) * G : 0.0; }

double model_lane_efficiency(int nd, int Hl, int h, int bord, int G) {
  (void)bord;
  double useful = 0.0, slots = 0.0;
  for (int k = 0; k + 2 < nd; k++) {
    const double m = nd - k - 1;
    useful += (m - 1) + (m - 1) * m + nd * (m - 1);
    slots += rnd(m - 1, G) + rnd((m - 1) * m, G) + rnd(nd, G) * (m - 1) + 3.0 * G;
  }
  for (int j0 = 0; j0 < nd - 1; j0 += G) {
    int dm = 0;
    for (int j = j0; j < std::min(nd - 1, j0 + G); j++) {
      dm = std::max(dm, std::min(Hl - 1, nd - 1 - j));
      useful += 2.0 * std::min(Hl - 1, nd - 1 - j);
    }
    slots += 2.0 * dm * G;
  }
  for (int l = nd - 1; l >= 0; l--) {
    const int deg = nd - l - 1;
    const int E = std::min(deg, Hl - 2);
    const double npe = E >= 0 ? (E + 1.0) * (Hl - 1) - E * (E + 1.0) / 2 : 0.0;
    const int dmx = std::min(Hl, l + 1);
    const double npd = dmx >= 2 ? (dmx - 1.0) * (2.0 * Hl - dmx) / 2 : 0.0;
    const double nq = std::min(Hl, nd - l);
    useful += (double)push_items_valid(nd, Hl, l) + nq;
    slots += rnd(std::min(npe, npd) + nq, 2 * G);
  }
  const int SG = std::min(G, 32);
  const double lg = std::log2((double)SG);
  for (int k = 1; k <= h; k++) {
    useful += 3.0 * k - 1.0;
    slots += (2.0 * std::ceil((double)k / SG) + std::ceil((double)k / SG)) * G + 3.0 * lg * 0.5 * G;
  }
  return slots > 0 ? useful / slots : 0.0;
}

}  // namespace lhafgpu
