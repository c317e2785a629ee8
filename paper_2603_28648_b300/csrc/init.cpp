// Sector rule of the initial MPS (bond dimensions per quantum-number sector).
//
// At a bond with b sites on the labelled side:
//   cap(q) = min(exact number of block states with label q,
//                number of states of the other L-b sites that complete q to
//                the target, product dimension reachable from bond b-1)
//   w(q)   = cap(q) exp(-(n - N b/L)^2 / 18) exp(-(s/2)^2 / 4.5)
// min(D, sum cap) is split in proportion to w by water filling with caps, then
// floors plus largest remainders (ties: smaller label first); a final
// right-to-left pass caps each sector by the states it can continue into.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "core.hpp"

namespace qd {

// Exact number of block states (U(1)) or multiplets (SU(2)) per label. In
// SU(2) the four label shifts are the coupling channels of a site multiplet,
// and a doublet coupled to a singlet gives spin 1/2 only (no negative 2S).
static std::map<QN, double> counts(int nsites, bool su2) {
  std::map<QN, double> cur{{QN{0, 0}, 1.0}};
  for (int k = 0; k < nsites; ++k) {
    std::map<QN, double> nxt;
    for (auto& kv : cur)
      for (int s = 0; s < NSITE; ++s) {
        const QN q = kv.first + SITE_QN[s];
        if (su2 && q.s < 0) continue;
        nxt[q] += kv.second;
      }
    cur.swap(nxt);
  }
  return cur;
}

static std::map<QN, int> allocate(int D, const std::map<QN, long long>& caps,
                                  const std::map<QN, double>& w) {
  long long total = 0;
  for (auto& kv : caps) total += kv.second;
  long long Dt = std::min<long long>(D, total);
  std::map<QN, double> alloc;
  std::vector<QN> freeq;
  for (auto& kv : caps) {
    alloc[kv.first] = 0.0;
    if (kv.second > 0 && w.at(kv.first) > 0) freeq.push_back(kv.first);
  }
  double remaining = (double)Dt;
  while (!freeq.empty() && remaining > 1e-12) {
    double wsum = 0;
    for (auto& q : freeq) wsum += w.at(q);
    std::vector<QN> over;
    for (auto& q : freeq)
      if (alloc[q] + remaining * w.at(q) / wsum >= (double)caps.at(q)) over.push_back(q);
    if (over.empty()) {
      for (auto& q : freeq) alloc[q] += remaining * w.at(q) / wsum;
      remaining = 0;
      break;
    }
    for (auto& q : over) {
      remaining -= (double)caps.at(q) - alloc[q];
      alloc[q] = (double)caps.at(q);
      freeq.erase(std::find(freeq.begin(), freeq.end(), q));
    }
  }
  std::map<QN, long long> ints;
  long long used = 0;
  for (auto& kv : alloc) {
    ints[kv.first] = (long long)std::floor(kv.second + 1e-9);
    used += ints[kv.first];
  }
  long long left = Dt - used;
  std::vector<QN> order;
  for (auto& kv : alloc) order.push_back(kv.first);
  std::stable_sort(order.begin(), order.end(), [&](const QN& a, const QN& b) {
    double fa = alloc[a] - ints[a], fb = alloc[b] - ints[b];
    if (fa != fb) return fa > fb;
    return a < b;
  });
  for (auto& q : order) {
    if (left <= 0) break;
    if (ints[q] < caps.at(q)) {
      ints[q]++;
      left--;
    }
  }
  std::map<QN, int> out;
  for (auto& kv : ints)
    if (kv.second > 0) out[kv.first] = (int)kv.second;
  return out;
}

std::vector<std::map<QN, int>> mps_structure(int L, int N, int two_s, int D, bool su2) {
  std::vector<std::map<QN, int>> bonds(L + 1);
  bonds[0][QN{0, 0}] = 1;
  bonds[L][QN{N, two_s}] = 1;
  std::vector<std::map<QN, double>> cnt(L + 1);
  for (int b = 0; b <= L; ++b) cnt[b] = counts(b, su2);
  const QN target{N, two_s};
  for (int b = 1; b < L; ++b) {
    std::map<QN, long long> prod;
    for (auto& kv : bonds[b - 1])
      for (int s = 0; s < NSITE; ++s) {
        const QN q = kv.first + SITE_QN[s];
        if (su2 && q.s < 0) continue;
        prod[q] += kv.second;
      }
    std::map<QN, long long> caps;
    std::map<QN, double> w;
    for (auto& kv : cnt[b]) {
      const QN q = kv.first;
      double comp = 0.0;
      if (su2) {
        // multiplets of the other L-b sites that couple with q to the target spin
        for (auto& r : cnt[L - b])
          if (r.first.n == N - q.n && std::abs(q.s - r.first.s) <= two_s && q.s + r.first.s >= two_s)
            comp += r.second;
      } else {
        auto it = cnt[L - b].find(target - q);
        comp = it == cnt[L - b].end() ? 0.0 : it->second;
      }
      double c = std::min(kv.second, comp);
      auto pit = prod.find(q);
      double pc = pit == prod.end() ? 0.0 : (double)pit->second;
      c = std::min(c, pc);
      if (c <= 0) continue;
      long long cap = (long long)std::min(c, 1e15);
      caps[q] = cap;
      double dn = q.n - (double)N * b / L;
      w[q] = (double)cap * std::exp(-dn * dn / 18.0) * std::exp(-(q.s / 2.0) * (q.s / 2.0) / (2 * 1.5 * 1.5));
    }
    bonds[b] = allocate(D, caps, w);
  }
  for (int b = L - 1; b >= 1; --b) {
    for (auto it = bonds[b].begin(); it != bonds[b].end();) {
      long long cont = 0;
      for (int s = 0; s < NSITE; ++s) {
        auto jt = bonds[b + 1].find(it->first + SITE_QN[s]);
        if (jt != bonds[b + 1].end()) cont += jt->second;
      }
      it->second = (int)std::min<long long>(it->second, cont);
      if (it->second <= 0) it = bonds[b].erase(it);
      else ++it;
    }
  }
  return bonds;
}

}  // namespace qd
