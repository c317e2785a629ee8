// Configuration-space warm start (host code, no device). The paper converges
// its large runs with an SU(2)-aware dynamically extended active space
// procedure (DEAS, Legeza et al. 2003; Numerical benchmark section), whose
// warm-up sweep takes the environment of each step from a small configuration
// space instead of states of a previous sweep. Here a set of configurations
// (determinants, or SU(2) configuration state functions) becomes an exact MPS
// whose left bond bases are the configurations' prefixes; with the centre at
// the right end, a right-to-left half sweep then optimises against a left
// environment spanned by those prefixes.
//
// Selection energies are quadratic forms of the occupations:
//   U(1), x = spin-orbital occupations (0/1):
//     E(x) = sum_k h_kk x_k + 1/2 sum_{k != l} g_kl x_k x_l,
//     g_kl = (pp|qq) - [same spin] (pq|qp)   (k on orbital p, l on q),
//   which is <D|H|D> (Slater-Condon);
//   SU(2), n = spatial occupations (0/1/2): the average of <D|H|D> over the
//   determinants of n,
//     E(n) = sum_p h_pp n_p + sum_p n_p (n_p - 1)/2 (pp|pp)
//            + sum_{p<q} n_p n_q ((pp|qq) - 1/2 (pq|qp)).
// Both are E(x) = c.x + 1/2 x^T B x with a symmetric B (U(1): B_kk = 0; SU(2):
// c_p = h_pp - 1/2 (pp|pp), B_pp = (pp|pp), B_pq = (pp|qq) - 1/2 (pq|qp)), so
// an excitation x = x_ref + delta costs
//   E = E_ref + delta.(c + B x_ref) + 1/2 delta^T B delta,
// a few terms for the at most four nonzero entries of delta.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <stdexcept>
#include <string>

#include "configs.hpp"
#include "core.hpp"

namespace qd {

void configs_to_mps(int L, bool su2, int N, int two_s, int n, const uint8_t* steps, const double* coef,
                    ImportArrays& out) {
  if (L < 2 || n < 1 || !steps || !coef) throw std::invalid_argument("L >= 2 and one configuration at least");
  const QN target{N, two_s};
  double nrm = 0.0;
  for (int k = 0; k < n; ++k) {
    if (!std::isfinite(coef[k])) throw std::invalid_argument("non-finite coefficient");
    nrm += coef[k] * coef[k];
    QN acc{0, 0};
    for (int p = 0; p < L; ++p) {
      const uint8_t st = steps[(size_t)k * L + p];
      if (st >= NSITE) throw std::invalid_argument("step outside 0..3");
      acc = acc + SITE_QN[st];
      if (su2 && acc.s < 0) throw std::invalid_argument("spin coupling below zero");
    }
    if (acc != target) throw std::invalid_argument("configuration outside the target sector");
  }
  if (!(nrm > 0)) throw std::invalid_argument("all coefficients are zero");
  const int c = L - 2;
  auto label = [&](int k, int len) {
    QN q{0, 0};
    for (int p = 0; p < len; ++p) q = q + SITE_QN[steps[(size_t)k * L + p]];
    return q;
  };
  auto prefix = [&](int k, int len) { return std::string((const char*)steps + (size_t)k * L, (size_t)len); };
  // distinct prefixes of each bond, by label, in lexicographic order
  std::vector<std::map<QN, std::map<std::string, int>>> pre(c + 1);
  for (int b = 0; b <= c; ++b)
    for (int k = 0; k < n; ++k) pre[b][label(k, b)].emplace(prefix(k, b), 0);
  std::vector<Basis> bonds(L + 1);
  for (auto& B : bonds) B.su2 = su2;
  for (int b = 0; b <= c; ++b)
    for (auto& kv : pre[b]) {
      int i = 0;
      for (auto& s : kv.second) s.second = i++;
      bonds[b].add(kv.first, (int)kv.second.size());
    }
  bonds[L].add(QN{0, 0}, 1);
  out = ImportArrays{};
  out.L = L;
  out.center = c;
  for (int b = 0; b <= L; ++b) {
    out.nsec.push_back(b == c + 1 ? 0 : bonds[b].nsec());
    if (b == c + 1) continue;
    for (int s = 0; s < bonds[b].nsec(); ++s) {
      out.sec.push_back(bonds[b].q[s].n);
      out.sec.push_back(bonds[b].q[s].s);
      out.sec.push_back(bonds[b].dim[s]);
    }
  }
  // left sites: selectors U_q[(x, i) row, x' column] = 1 for x' = x followed by i
  for (int p = 0; p < c; ++p) {
    const ProdBasis pb = make_prod(bonds[p], true);
    for (int q = 0; q < pb.prod.nsec(); ++q) {
      const int t = bonds[p + 1].find(pb.prod.q[q]);
      if (t < 0) continue;
      const int rows = pb.prod.dim[q], cols = bonds[p + 1].dim[t];
      std::vector<double> M((size_t)rows * cols, 0.0);
      for (auto& kv : pre[p + 1].at(pb.prod.q[q])) {
        const std::string par = kv.first.substr(0, p);
        QN ql{0, 0};
        for (char ch : par) ql = ql + SITE_QN[(uint8_t)ch];
        const int x = bonds[p].find(ql);
        const int sub = pb.find(x, (uint8_t)kv.first[p]);
        if (x < 0 || sub < 0 || pb.subs[sub].prod != q) throw std::logic_error("prefix outside the product basis");
        M[(size_t)(pb.subs[sub].off + pre[p].at(ql).at(par)) * cols + kv.second] = 1.0;
      }
      out.data.insert(out.data.end(), M.begin(), M.end());
    }
  }
  // the two-site wavefunction at (L-2, L-1); the right block is the vacuum
  const ProdBasis Lp = make_prod(bonds[c], true), Rp = make_prod(bonds[L], false);
  const PsiLayout lay = make_psi_layout(Lp, Rp, target);
  std::vector<double> psi((size_t)lay.size, 0.0);
  for (int k = 0; k < n; ++k) {
    const QN ql = label(k, c);
    const int x = bonds[c].find(ql);
    const int r = pre[c].at(ql).at(prefix(k, c));
    const int i = steps[(size_t)k * L + c];
    int j = steps[(size_t)k * L + c + 1];
    if (su2 && j == 2) j = 1;   // the last doublet couples to the vacuum as spin 1/2
    const int blk = lay.find(Lp.find(x, i), Rp.find(0, j));
    if (blk < 0) throw std::invalid_argument("configuration outside the target sector");
    psi[(size_t)lay.blks[blk].off + r] += coef[k];
  }
  out.data.insert(out.data.end(), psi.begin(), psi.end());
}

namespace {

struct Cand {
  double e;
  int level;
  std::vector<uint8_t> steps;
};

bool before(const Cand& a, const Cand& b) {
  if (a.e != b.e) return a.e < b.e;
  if (a.level != b.level) return a.level < b.level;
  return a.steps < b.steps;
}

// the nmax smallest candidates by before(), in a max-heap
struct Best {
  size_t nmax;
  std::vector<Cand> heap;
  static bool cmp(const Cand& a, const Cand& b) { return before(a, b); }
  bool admits(double e) const {
    return heap.size() < nmax || e <= heap.front().e;
  }
  void offer(Cand&& c) {
    if (heap.size() < nmax) {
      heap.push_back(std::move(c));
      std::push_heap(heap.begin(), heap.end(), cmp);
    } else if (before(c, heap.front())) {
      std::pop_heap(heap.begin(), heap.end(), cmp);
      heap.back() = std::move(c);
      std::push_heap(heap.begin(), heap.end(), cmp);
    }
  }
};

// orbitals by increasing h_pp, ties by index
std::vector<int> aufbau_order(int L, const double* h) {
  std::vector<int> o(L);
  std::iota(o.begin(), o.end(), 0);
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return h[a * L + a] < h[b * L + b]; });
  return o;
}

double Vx(const double* V, int L, int p, int q, int r, int s) {
  return V[(((size_t)p * L + q) * L + r) * L + s];
}

int select_u1(int L, int N, int two_s, const double* h, const double* V, Best& best) {
  const int na = (N + two_s) / 2, nb = (N - two_s) / 2;
  const int M = 2 * L;   // spin-orbital k = 2p + sigma
  std::vector<double> cvec(M), B((size_t)M * M, 0.0);
  for (int k = 0; k < M; ++k) cvec[k] = h[(k / 2) * L + k / 2];
  for (int k = 0; k < M; ++k)
    for (int l = 0; l < M; ++l) {
      if (k == l) continue;
      const int p = k / 2, q = l / 2;
      double g = Vx(V, L, p, p, q, q);
      if ((k & 1) == (l & 1)) g -= Vx(V, L, p, q, q, p);
      B[(size_t)k * M + l] = g;
    }
  const std::vector<int> ord = aufbau_order(L, h);
  std::vector<int> x(M, 0);
  for (int i = 0; i < na; ++i) x[2 * ord[i]] = 1;
  for (int i = 0; i < nb; ++i) x[2 * ord[i] + 1] = 1;
  double eref = 0.0;
  std::vector<double> G(M);
  for (int k = 0; k < M; ++k) {
    double bx = 0.0;
    for (int l = 0; l < M; ++l) bx += B[(size_t)k * M + l] * x[l];
    G[k] = cvec[k] + bx;
    eref += x[k] * (cvec[k] + 0.5 * bx);
  }
  std::vector<int> occ[2], vir[2];
  for (int k = 0; k < M; ++k) (x[k] ? occ : vir)[k & 1].push_back(k);
  std::vector<uint8_t> st(L);
  int count = 0;   // determinants visited
  auto emit = [&](const int* rem, const int* add, int m) {
    // delta = -1 on rem, +1 on add
    double e = eref;
    int dk[4];
    double dv[4];
    for (int i = 0; i < m; ++i) {
      dk[i] = rem[i];
      dv[i] = -1.0;
      dk[m + i] = add[i];
      dv[m + i] = 1.0;
    }
    for (int i = 0; i < 2 * m; ++i) {
      e += dv[i] * G[dk[i]];
      for (int j = 0; j < 2 * m; ++j) e += 0.5 * dv[i] * dv[j] * B[(size_t)dk[i] * M + dk[j]];
    }
    ++count;
    if (!best.admits(e)) return;
    for (int k = 0; k < m; ++k) x[rem[k]] = 0, x[add[k]] = 1;
    for (int p = 0; p < L; ++p) st[p] = (uint8_t)(x[2 * p] + 2 * x[2 * p + 1]);
    for (int k = 0; k < m; ++k) x[rem[k]] = 1, x[add[k]] = 0;
    best.offer(Cand{e, m, st});
  };
  emit(nullptr, nullptr, 0);
  for (int s = 0; s < 2; ++s)
    for (int i : occ[s])
      for (int a : vir[s]) {
        const int r[1] = {i}, d[1] = {a};
        emit(r, d, 1);
      }
  for (int s = 0; s < 2; ++s)   // both electrons of one spin
    for (size_t i = 0; i < occ[s].size(); ++i)
      for (size_t j = i + 1; j < occ[s].size(); ++j)
        for (size_t a = 0; a < vir[s].size(); ++a)
          for (size_t b = a + 1; b < vir[s].size(); ++b) {
            const int r[2] = {occ[s][i], occ[s][j]}, d[2] = {vir[s][a], vir[s][b]};
            emit(r, d, 2);
          }
  for (int i : occ[0])   // one electron of each spin
    for (int a : vir[0])
      for (int j : occ[1])
        for (int b : vir[1]) {
          const int r[2] = {i, j}, d[2] = {a, b};
          emit(r, d, 2);
        }
  return count;
}

int select_su2(int L, int N, int two_s, const double* h, const double* V, Best& best) {
  const int nd = (N - two_s) / 2;
  std::vector<double> cvec(L), B((size_t)L * L);
  for (int p = 0; p < L; ++p) {
    cvec[p] = h[p * L + p] - 0.5 * Vx(V, L, p, p, p, p);
    for (int q = 0; q < L; ++q)
      B[(size_t)p * L + q] = p == q ? Vx(V, L, p, p, p, p) : Vx(V, L, p, p, q, q) - 0.5 * Vx(V, L, p, q, q, p);
  }
  const std::vector<int> ord = aufbau_order(L, h);
  std::vector<int> nref(L, 0);
  for (int i = 0; i < nd; ++i) nref[ord[i]] = 2;
  for (int i = nd; i < nd + two_s; ++i) nref[ord[i]] = 1;
  double eref = 0.0;
  std::vector<double> G(L);
  for (int p = 0; p < L; ++p) {
    double bn = 0.0;
    for (int q = 0; q < L; ++q) bn += B[(size_t)p * L + q] * nref[q];
    G[p] = cvec[p] + bn;
    eref += nref[p] * (cvec[p] + 0.5 * bn);
  }
  std::vector<int> n = nref;
  std::vector<uint8_t> st(L);
  int count = 0;   // couplings offered
  // every genealogical coupling of the open shells of n with final spin two_s
  auto couplings = [&](double e, int level) {
    std::vector<int> open;
    for (int p = 0; p < L; ++p)
      if (n[p] == 1) open.push_back(p);
    const int k = (int)open.size();
    if (k < two_s || (k - two_s) % 2) return;
    for (int p = 0; p < L; ++p) st[p] = n[p] == 2 ? 3 : 0;
    // up steps u and down steps k - u with u - (k - u) = two_s; running spin >= 0
    std::vector<int> path(k, 1);
    auto rec = [&](auto&& self, int i, int s) -> void {
      if (i == k) {
        if (s != two_s) return;
        for (int t = 0; t < k; ++t) st[open[t]] = (uint8_t)path[t];
        ++count;
        best.offer(Cand{e, level, st});
        return;
      }
      if (s - (k - i) > two_s) return;           // cannot come down to two_s any more
      if (s + (k - i) < two_s) return;           // cannot reach two_s any more
      path[i] = 1;
      self(self, i + 1, s + 1);
      if (s > 0) {
        path[i] = 2;
        self(self, i + 1, s - 1);
      }
    };
    rec(rec, 0, 0);
  };
  auto visit = [&](const int* rem, const int* add, int m) {
    // rem / add: orbitals losing / gaining one electron each (an orbital may
    // appear twice); no orbital both loses and gains
    double e = eref;
    for (int i = 0; i < m; ++i) {
      e -= G[rem[i]];
      e += G[add[i]];
    }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        e += 0.5 * (B[(size_t)rem[i] * L + rem[j]] + B[(size_t)add[i] * L + add[j]]) -
             B[(size_t)rem[i] * L + add[j]];
    if (!best.admits(e)) return;
    for (int i = 0; i < m; ++i) --n[rem[i]], ++n[add[i]];
    couplings(e, m);
    for (int i = 0; i < m; ++i) ++n[rem[i]], --n[add[i]];
  };
  visit(nullptr, nullptr, 0);
  std::vector<int> src, dst;   // orbitals that can lose / gain an electron
  for (int p = 0; p < L; ++p) {
    if (nref[p] > 0) src.push_back(p);
    if (nref[p] < 2) dst.push_back(p);
  }
  for (int r : src)
    for (int a : dst) {
      if (r == a) continue;
      const int rr[1] = {r}, aa[1] = {a};
      visit(rr, aa, 1);
    }
  // two electrons: removal pairs r1 <= r2 (equal only from a doubly occupied
  // orbital), addition pairs a1 <= a2 (equal only into an empty one)
  for (size_t i = 0; i < src.size(); ++i)
    for (size_t j = i; j < src.size(); ++j) {
      const int r1 = src[i], r2 = src[j];
      if (r1 == r2 && nref[r1] < 2) continue;
      for (size_t a = 0; a < dst.size(); ++a)
        for (size_t b = a; b < dst.size(); ++b) {
          const int a1 = dst[a], a2 = dst[b];
          if (a1 == a2 && nref[a1] > 0) continue;
          if (a1 == r1 || a1 == r2 || a2 == r1 || a2 == r2) continue;
          const int rr[2] = {r1, r2}, aa[2] = {a1, a2};
          visit(rr, aa, 2);
        }
    }
  return count;
}

}  // namespace

int select_configs(int L, bool su2, int N, int two_s, const double* h, const double* V, int nmax,
                   std::vector<uint8_t>& steps, std::vector<double>& energy) {
  if (L < 2 || nmax < 1 || !h || !V) throw std::invalid_argument("L >= 2, nmax >= 1");
  if (N < 0 || N > 2 * L || ((N + two_s) & 1)) throw std::invalid_argument("target outside the Fock space");
  if (su2) {
    if (two_s < 0 || (N - two_s) / 2 + two_s > L || two_s > N) throw std::invalid_argument("target outside the Fock space");
  } else if ((N + two_s) / 2 < 0 || (N + two_s) / 2 > L || (N - two_s) / 2 < 0 || (N - two_s) / 2 > L) {
    throw std::invalid_argument("target outside the Fock space");
  }
  Best best{(size_t)nmax, {}};
  if (su2) select_su2(L, N, two_s, h, V, best);
  else select_u1(L, N, two_s, h, V, best);
  std::sort(best.heap.begin(), best.heap.end(), before);
  steps.clear();
  energy.clear();
  for (auto& c : best.heap) {
    steps.insert(steps.end(), c.steps.begin(), c.steps.end());
    energy.push_back(c.e);
  }
  return (int)best.heap.size();
}

}  // namespace qd
