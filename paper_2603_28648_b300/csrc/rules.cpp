// Complementary-operator rules: how the operators of an enlarged block
// (block (x) site) are written in terms of the block's renormalized operators
// and exact single-site matrices.
//
// Spin-orbital form of the active-space Hamiltonian (k = 2p + sigma):
//   H = sum t_kl a+_k a_l + 1/2 sum w_ijkl a+_i a+_j a_k a_l,
//   t_kl = h_{p_k p_l} d(s_k, s_l),  w_ijkl = (p_i p_l | p_j p_k) d(s_i, s_l) d(s_j, s_k).
// Operators kept by a block at cut c (left = sites [0,c), right = [c,L)):
//   every block: I, C_k = a+_k (k in block), S_m (m outside), H
//   normal pairs:        A_kl = a+_k a+_l (k<l), B_kl = a+_k a_l   (k, l in block)
//   complementary pairs: P_ij = 1/2 sum_{kl in block} w_ijkl a_k a_l   (i<j outside)
//                        Q_il = sum_{jk in block} (w_ijkl - w_ijlk) a+_j a_k   (i,l outside)
//   S^B_m = 1/2 sum_{j in B} t_mj a_j + sum_{jkl in B} w_mjkl a+_j a_k a_l.
// Left blocks hold normal pairs up to a switch cut and complementary pairs
// beyond it, right blocks the reverse, so that normal pairs sit on the side
// with fewer modes when the switch is at the middle of the chain (the N/2
// rule); with the switch at L every left block is normal. Decomposition at a
// cut L|R with normal pairs on the left:
//   H = H_L + H_R + sum_{i in L} (a+_i S^R_i - a_i (S^R_i)^+)
//     + sum_{m in R} (-S^L_m a+_m + (S^L_m)^+ a_m)
//     + 2 sum_{i<j in L} (A_ij P_ij + A_ij^+ P_ij^+) + sum_{il in L} B_il Q_il;
// with normal pairs on the right the last line reads
//     + 2 sum_{i<j in R} (P_ij A_ij + P_ij^+ A_ij^+) + sum_{jk in R} Q_jk B_jk.
// The switch itself is the enlargement of a normal block into a
// complementary one: the block-block part of P'_ij and Q'_il is a sum over
// the block's A_kl and B_jk weighted by w.
// A product O_X O_s on X (x) site acts as (O_X P_X^{p(O_s)}) (x) O_s; a
// product O_s O_Y on site (x) Y as (O_s P_s^{p(O_Y)}) (x) O_Y.
#include <algorithm>
#include <atomic>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>
#include <climits>
#include <cmath>
#include <cstdint>
#include <set>
#include <tuple>
#include <map>
#include <unordered_map>
#include <stdexcept>
#include <vector>

#include "core.hpp"

namespace qd {

std::vector<Key> block_keys(bool left, bool normal, int c, int L) {
  // own modes [m0, m1), outside modes [o0, o1) (the left block's or the right's complement)
  const int m0 = left ? 0 : 2 * c, m1 = left ? 2 * c : 2 * L;
  const int o0 = left ? 2 * c : 0, o1 = left ? 2 * L : 2 * c;
  std::vector<Key> k;
  k.push_back(Key(F_I));
  for (int a = m0; a < m1; ++a) k.push_back(Key(F_C, a));
  const int p0 = normal ? m0 : o0, p1 = normal ? m1 : o1;
  for (int a = p0; a < p1; ++a)
    for (int b = a + 1; b < p1; ++b) k.push_back(Key(normal ? F_A : F_P, a, b));
  for (int a = p0; a < p1; ++a)
    for (int b = p0; b < p1; ++b) k.push_back(Key(normal ? F_B : F_Q, a, b));
  for (int m = o0; m < o1; ++m) k.push_back(Key(F_S, m));
  k.push_back(Key(F_H));
  return k;
}

namespace {

// Site-operator monomials: normal-ordered products of a+_up, a+_dn, a_up,
// a_dn on one site. The 16 of them are a basis of the 4x4 matrices; every
// site factor of a contribution is split on this basis so that the block
// parts multiplying the same monomial can be summed once.
struct Monos {
  Mat4 m[16];
  double inv[16][16];
  Monos() {
    const Mat4 I4 = Mat4::id();
    Mat4 c0 = cre(0), c1 = cre(1), a0 = ann(0), a1 = ann(1);
    Mat4 list[16] = {I4, c0, c1, a0, a1, c0 * c1, c0 * a0, c0 * a1, c1 * a0, c1 * a1, a0 * a1,
                     c0 * c1 * a0, c0 * c1 * a1, c0 * a0 * a1, c1 * a0 * a1, c0 * c1 * a0 * a1};
    double M[16][32];
    for (int k = 0; k < 16; ++k) {
      m[k] = list[k];
      for (int e = 0; e < 16; ++e) M[e][k] = list[k].v[e];
    }
    for (int r = 0; r < 16; ++r)
      for (int c = 0; c < 16; ++c) M[r][16 + c] = (r == c);
    for (int c = 0; c < 16; ++c) {  // Gauss-Jordan with partial pivoting
      int piv = c;
      for (int r = c + 1; r < 16; ++r)
        if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
      for (int k = 0; k < 32; ++k) std::swap(M[c][k], M[piv][k]);
      double d = M[c][c];
      for (int k = 0; k < 32; ++k) M[c][k] /= d;
      for (int r = 0; r < 16; ++r)
        if (r != c && M[r][c] != 0.0) {
          double f = M[r][c];
          for (int k = 0; k < 32; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < 16; ++r)
      for (int c = 0; c < 16; ++c) inv[r][c] = M[r][16 + c];
  }
  // coefficients x_k with o = sum_k x_k m[k]
  void split(const Mat4& o, double x[16]) const {
    for (int k = 0; k < 16; ++k) {
      double s = 0;
      for (int e = 0; e < 16; ++e) s += inv[k][e] * o.v[e];
      x[k] = std::fabs(s) < 1e-15 ? 0.0 : s;
    }
  }
};
const Monos& monos() {
  static Monos M;
  return M;
}

// f(0..n-1) on up to 16 host threads (items are independent and write only
// their own results); the first exception of any item is rethrown
void parallel_for(size_t n, const std::function<void(size_t)>& f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const unsigned nt = (unsigned)std::min<size_t>(std::min(hw, 16u), n / 32);
  if (nt <= 1) {
    for (size_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<size_t> next{0};
  std::exception_ptr err;
  std::mutex mu;
  std::vector<std::thread> ts;
  for (unsigned t = 0; t < nt; ++t)
    ts.emplace_back([&]() {
      try {
        for (size_t i; (i = next.fetch_add(1)) < n;) f(i);
      } catch (...) {
        std::lock_guard<std::mutex> g(mu);
        if (!err) err = std::current_exception();
        next = n;
      }
    });
  for (auto& t : ts) t.join();
  if (err) std::rethrow_exception(err);
}

struct Ctx {
  const EnvBlock& B;
  const Integrals& I;
  Enlarged& E;
  const ProdBasis& pb;
  struct Pending {
    Key key;
    bool odd;
    std::vector<Contrib> cs;
  };
  std::vector<Pending> pending;
  Ctx(const EnvBlock& b, const Integrals& i, Enlarged& e, bool for_enlarge = true) : B(b), I(i), E(e), pb(e.pb) {
    if (for_enlarge) pending.reserve(16 + 8 * (size_t)i.L * i.L);  // complementary operators of one block
  }

  const OpView* get(Key k) const {
    auto it = B.ops.find(k);
    if (it == B.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  }

  // expand coef * (src (x) o) into references on the enlarged basis
  void expand(const std::vector<BRef>& src, const Mat4& o, double coef, bool par,
              std::vector<BRef>& out) const {
    if (coef == 0.0 || o.zero()) return;
    for (const BRef& b : src) {
      for (int i = 0; i < NSITE; ++i)
        for (int i2 = 0; i2 < NSITE; ++i2) {
          double v = o(i, i2);
          if (v == 0.0) continue;
          BRef r = b;
          double sgn = 1.0;
          r.r = pb.find(b.r, i);
          r.c = pb.find(b.c, i2);
          if (par) {
            if (E.left) { if (B.basis.q[b.c].n & 1) sgn = -1.0; }
            else if (SITE_QN[i2].n & 1) sgn = -1.0;
          }
          r.sc = b.sc * coef * v * sgn;
          out.push_back(r);
        }
    }
  }
  std::vector<BRef> src_blocks(const OpView* src, bool T) const {
    if (src) return T ? transpose(*src).blocks : src->blocks;
    std::vector<BRef> v;
    for (int x = 0; x < B.basis.nsec(); ++x) {
      BRef b;
      b.r = b.c = x;
      b.ptr = 0;
      b.rows = b.cols = b.ld = B.basis.dim[x];
      v.push_back(b);
    }
    return v;
  }

  void view(Key k, const std::vector<Contrib>& cs, bool odd) {
    OpView v;
    v.odd = odd;
    for (auto& c : cs) expand(src_blocks(c.src, c.srcT), c.o, c.coef, c.par, v.blocks);
    if (!v.blocks.empty()) E.ops[k] = v;
  }

  void materialize(Key k, std::vector<Contrib>&& cs, bool odd) {
    pending.push_back({k, odd, std::move(cs)});
  }

  // Group every pending operator's contributions by (site monomial, parity
  // flag). A group with one block operator stays a reference; a group with
  // several is summed once into new storage on the block basis.
  struct Item { const OpView* src; bool T; double coef; };
  struct Group { Mat4 o; bool par; std::vector<Item> items; };
  struct Plan { std::vector<Group> groups; };

  // Groups with at least WIDE items whose sources are stored, untransposed,
  // dense blocks with one quantum-number change are batched by (orientation,
  // change). In a batch with groups t and sources s (ordered by address),
  // every block position (r, c) of the sources is one problem
  //   Z[t, :] = sum_s W[t, s] src_s(r, c)[:]    (Z: groups x block elements)
  // whose K dimension runs over the sources: a run of sources whose blocks at
  // (r, c) lie at equal distances is one segment (A = columns of W, B = the
  // blocks as rows of a strided matrix), any other source a segment of K = 1.
  // A group of transposed sources sums the untransposed blocks and takes the
  // transpose of the result. The refs of each group go to `summed`.
  static constexpr size_t WIDE = 8;
  void batch_sums(const std::vector<Plan>& plans, Launch& lb, std::set<std::pair<size_t, size_t>>& in_batch,
                  std::map<std::pair<size_t, size_t>, std::vector<BRef>>& summed, Executor& ex) {
    struct SrcInfo { bool ok; QN dq; };
    std::unordered_map<const OpView*, SrcInfo> info;
    auto inspect = [&](const OpView* src) -> const SrcInfo& {
      auto it = info.find(src);
      if (it != info.end()) return it->second;
      SrcInfo si{src != nullptr && !src->blocks.empty(), QN{}};
      if (si.ok) {
        std::set<std::pair<int, int>> seen;
        si.dq = B.basis.q[src->blocks[0].c] - B.basis.q[src->blocks[0].r];
        for (const BRef& b : src->blocks)
          if (b.ident() || b.tr || b.ld != b.cols || b.rows != B.basis.dim[b.r] || b.cols != B.basis.dim[b.c] ||
              B.basis.q[b.c] - B.basis.q[b.r] != si.dq || !seen.insert({b.r, b.c}).second) {
            si.ok = false;
            break;
          }
      }
      return info.emplace(src, si).first->second;
    };
    std::map<std::tuple<bool, int, int>, std::vector<std::pair<size_t, size_t>>> batches;
    for (size_t n = 0; n < plans.size(); ++n)
      for (size_t g = 0; g < plans[n].groups.size(); ++g) {
        const Group& grp = plans[n].groups[g];
        if (grp.items.size() < WIDE) continue;
        const bool T = grp.items[0].T;
        const SrcInfo& s0 = inspect(grp.items[0].src);
        bool ok = s0.ok;
        for (const Item& itm : grp.items) {
          if (!ok) break;
          const SrcInfo& si = inspect(itm.src);
          ok = itm.T == T && si.ok && si.dq == s0.dq;
        }
        if (ok) batches[std::make_tuple(T, s0.dq.n, s0.dq.s)].push_back({n, g});
      }
    for (auto& kv : batches) {
      const bool T = std::get<0>(kv.first);
      const auto& tg = kv.second;
      std::vector<const OpView*> src;
      std::unordered_map<const OpView*, int> col;
      for (auto& ng : tg)
        for (const Item& itm : plans[ng.first].groups[ng.second].items)
          if (col.emplace(itm.src, 0).second) src.push_back(itm.src);
      std::sort(src.begin(), src.end(),
                [](const OpView* a, const OpView* b) { return a->blocks[0].ptr < b->blocks[0].ptr; });
      for (size_t k = 0; k < src.size(); ++k) col[src[k]] = (int)k;
      const int nt = (int)tg.size(), K = (int)src.size();
      std::vector<double> W((size_t)nt * K, 0.0);
      for (int t = 0; t < nt; ++t)
        for (const Item& itm : plans[tg[t].first].groups[tg[t].second].items) W[(size_t)t * K + col[itm.src]] += itm.coef;
      std::map<std::pair<int, int>, std::vector<const BRef*>> at;  // position -> block of each source
      for (int k = 0; k < K; ++k)
        for (const BRef& b : src[k]->blocks) {
          auto& v = at[{b.r, b.c}];
          if (v.empty()) v.assign(K, nullptr);
          v[k] = &b;
        }
      int64_t total = 0;
      for (auto& pv : at) total += (int64_t)nt * B.basis.dim[pv.first.first] * B.basis.dim[pv.first.second];
      const uint64_t wdev = ex.alloc((int64_t)W.size());
      E.owned.push_back(wdev);
      ex.upload(wdev, W.data(), (int64_t)W.size());
      const uint64_t store = ex.alloc(total);
      E.owned.push_back(store);
      std::vector<std::vector<BRef>> refs(nt);
      int64_t off = 0;
      for (auto& pv : at) {
        const int rows = B.basis.dim[pv.first.first], cols = B.basis.dim[pv.first.second];
        const int e = rows * cols;
        const auto& v = pv.second;
        Prob p;
        p.c = store + 8ull * off; p.cbuf = B_ABS;
        p.m = nt; p.n = e; p.ldc = e; p.beta = 0;
        p.seg0 = (int)lb.segs.size();
        for (int k = 0; k < K;) {
          if (!v[k]) { ++k; continue; }
          int k1 = k + 1;
          int64_t stride = 0;
          for (; k1 < K && v[k1] && v[k1]->sc == v[k]->sc; ++k1) {
            const int64_t d = (int64_t)v[k1]->ptr - (int64_t)v[k1 - 1]->ptr;
            if (k1 == k + 1) {
              if (d <= 0 || d % 8 || d / 8 < e || d / 8 > INT32_MAX) break;
              stride = d;
            } else if (d != stride) {
              break;
            }
          }
          Seg sg;
          sg.a = wdev + 8ull * k; sg.abuf = B_ABS; sg.lda = K; sg.ta = 0;
          sg.b = v[k]->ptr; sg.bbuf = B_ABS; sg.ldb = k1 - k > 1 ? (int)(stride / 8) : e; sg.tb = 0;
          sg.k = k1 - k;
          sg.sc = v[k]->sc;
          lb.segs.push_back(sg);
          lb.flops += 2.0 * nt * e * sg.k;
          k = k1;
        }
        p.nseg = (int)lb.segs.size() - p.seg0;
        lb.probs.push_back(p);
        for (int t = 0; t < nt; ++t) {
          BRef r;
          r.r = pv.first.first; r.c = pv.first.second;
          r.ptr = p.c + 8ull * t * e;
          r.rows = rows; r.cols = cols; r.ld = cols; r.tr = false; r.sc = 1.0;
          refs[t].push_back(r);
        }
        off += (int64_t)nt * e;
      }
      for (int t = 0; t < nt; ++t) {
        OpView z;
        z.blocks = std::move(refs[t]);
        summed[tg[t]] = T ? transpose(z).blocks : std::move(z.blocks);
        in_batch.insert(tg[t]);
      }
    }
  }

  void finish(Executor& ex) {
    const Monos& M = monos();
    std::vector<Plan> plans(pending.size());
    // every pending operator is planned on its own (independent, any thread)
    parallel_for(pending.size(), [&](size_t n) {
      int gi[16][2];                             // (monomial, par) -> group
      for (auto& row : gi) row[0] = row[1] = -1;
      std::vector<std::unordered_map<uintptr_t, int>> where;  // per group: (source, transposed) -> item
      auto& G = plans[n].groups;
      for (const Contrib& c : pending[n].cs) {
        if (c.coef == 0.0 || c.o.zero()) continue;
        double x[16];
        M.split(c.o, x);
        const uintptr_t id = reinterpret_cast<uintptr_t>(c.src) * 2 + (c.srcT ? 1 : 0);
        for (int k = 0; k < 16; ++k) {
          if (x[k] == 0.0) continue;
          int& g = gi[k][c.par ? 1 : 0];
          if (g < 0) {
            g = (int)G.size();
            G.push_back({M.m[k], c.par, {}});
            where.emplace_back();
          }
          auto ins = where[g].emplace(id, (int)G[g].items.size());
          if (ins.second) G[g].items.push_back({c.src, c.srcT, c.coef * x[k]});
          else G[g].items[ins.first->second].coef += c.coef * x[k];
        }
      }
    });
    // block lists of the sources (transposes built once)
    std::unordered_map<uintptr_t, std::vector<BRef>> blocks_of;
    auto blocks = [&](const OpView* src, bool T) -> const std::vector<BRef>& {
      const uintptr_t id = reinterpret_cast<uintptr_t>(src) * 2 + (T ? 1 : 0);
      auto it = blocks_of.find(id);
      if (it != blocks_of.end()) return it->second;
      return blocks_of.emplace(id, src_blocks(src, T)).first->second;
    };
    std::map<std::pair<size_t, size_t>, std::vector<BRef>> summed;
    // wide sums as GEMMs: summed groups of many stored operators, all with the
    // same orientation and quantum-number change, are evaluated together
    Launch lb;
    std::set<std::pair<size_t, size_t>> in_batch;
    if (E.batched) batch_sums(plans, lb, in_batch, summed, ex);
    // block lists of every source that is summed or referenced below
    // (transposes built once), filled here so that the parallel parts only
    // read the cache
    for (size_t n = 0; n < plans.size(); ++n)
      for (size_t g = 0; g < plans[n].groups.size(); ++g)
        if (!in_batch.count({n, g}))
          for (auto& itm : plans[n].groups[g].items) blocks(itm.src, itm.T);
    auto blocks_ro = [&](const OpView* src, bool T) -> const std::vector<BRef>& {
      return blocks_of.at(reinterpret_cast<uintptr_t>(src) * 2 + (T ? 1 : 0));
    };
    // summed groups: each group's destination blocks (offsets in order of first
    // appearance, problems in block-key order), then the groups' storage,
    // problems and segments laid out one group after the other
    struct Mat {
      size_t n, g;
      std::map<std::pair<int, int>, std::pair<int64_t, std::pair<int, int>>> blk;  // key -> local offset, shape
      int64_t size = 0, off = 0;
      size_t nseg = 0, seg0 = 0, prob0 = 0;
    };
    std::vector<Mat> mats;
    for (size_t n = 0; n < plans.size(); ++n)
      for (size_t g = 0; g < plans[n].groups.size(); ++g)
        if (plans[n].groups[g].items.size() >= 2 && !in_batch.count({n, g})) {
          mats.emplace_back();
          mats.back().n = n;
          mats.back().g = g;
        }
    parallel_for(mats.size(), [&](size_t mi) {
      Mat& mt = mats[mi];
      for (auto& itm : plans[mt.n].groups[mt.g].items)
        for (const BRef& b : blocks_ro(itm.src, itm.T)) {
          auto ins = mt.blk.emplace(std::make_pair(b.r, b.c), std::make_pair(mt.size, std::make_pair(b.rows, b.cols)));
          if (ins.second) mt.size += (int64_t)b.rows * b.cols;
          ++mt.nseg;
        }
    });
    int64_t total = 0;
    size_t nseg = 0, nprob = 0;
    for (auto& mt : mats) {
      mt.off = total;
      mt.seg0 = nseg;
      mt.prob0 = nprob;
      total += mt.size;
      nseg += mt.nseg;
      nprob += mt.blk.size();
    }
    if (nseg + lb.segs.size() > (size_t)INT32_MAX) throw std::runtime_error("enlarge: summation task list too long");
    uint64_t store = total ? ex.alloc(total) : 0;
    if (store) E.owned.push_back(store);
    Launch l;
    l.segs.resize(nseg);
    l.probs.resize(nprob);
    // each group's problems and segments (grouped by destination block in key
    // order, item order within a block) and block references, in place
    std::vector<std::vector<BRef>> refs(mats.size());
    parallel_for(mats.size(), [&](size_t mi) {
      const Mat& mt = mats[mi];
      const auto& grp = plans[mt.n].groups[mt.g];
      std::map<std::pair<int, int>, int> kidx;
      for (auto& kv : mt.blk) kidx.emplace(kv.first, (int)kidx.size());
      std::vector<int> key_of;
      key_of.reserve(mt.nseg);
      std::vector<size_t> start(kidx.size() + 1, 0);
      for (auto& itm : grp.items)
        for (const BRef& b : blocks_ro(itm.src, itm.T)) {
          key_of.push_back(kidx.at({b.r, b.c}));
          start[key_of.back() + 1]++;
        }
      for (size_t i = 0; i < kidx.size(); ++i) start[i + 1] += start[i];
      std::vector<size_t> pos(start.begin(), start.end() - 1);
      size_t e = 0;
      for (auto& itm : grp.items)
        for (const BRef& b : blocks_ro(itm.src, itm.T)) {
          Seg sg;
          sg.a = 0; sg.abuf = B_ABS; sg.k = b.rows; sg.sc = itm.coef * b.sc;
          if (b.ident()) { sg.b = 0; sg.bbuf = B_ABS; }
          else { sg.b = b.ptr; sg.bbuf = B_ABS; sg.ldb = b.ld; sg.tb = b.tr ? 1 : 0; }
          l.segs[mt.seg0 + pos[key_of[e++]]++] = sg;
        }
      int q = 0;
      refs[mi].reserve(mt.blk.size());
      for (auto& kv : mt.blk) {
        Prob pr;
        pr.c = store + 8ull * (mt.off + kv.second.first); pr.cbuf = B_ABS;
        pr.m = kv.second.second.first; pr.n = kv.second.second.second; pr.ldc = pr.n; pr.beta = 0;
        pr.seg0 = (int)(mt.seg0 + start[q]);
        pr.nseg = (int)(start[q + 1] - start[q]);
        l.probs[mt.prob0 + q] = pr;
        ++q;
        BRef r;
        r.r = kv.first.first; r.c = kv.first.second; r.ptr = pr.c;
        r.rows = pr.m; r.cols = pr.n; r.ld = pr.n; r.tr = false; r.sc = 1.0;
        refs[mi].push_back(r);
      }
    });
    for (size_t mi = 0; mi < mats.size(); ++mi) summed[{mats[mi].n, mats[mi].g}] = std::move(refs[mi]);
    if (!lb.empty()) {  // the GEMM-batched sums join the same launch
      const int base = (int)l.segs.size();
      for (Prob pr : lb.probs) {
        pr.seg0 += base;
        l.probs.push_back(pr);
      }
      l.segs.insert(l.segs.end(), lb.segs.begin(), lb.segs.end());
      l.flops += lb.flops;
    }
    if (!l.empty()) ex.run(l, 0, 0);
    // the operators' views, independently; then stored in key order
    std::vector<OpView> views(plans.size());
    parallel_for(plans.size(), [&](size_t n) {
      OpView& v = views[n];
      v.odd = pending[n].odd;
      for (size_t g = 0; g < plans[n].groups.size(); ++g) {
        auto& grp = plans[n].groups[g];
        if (grp.items.size() >= 2) {
          expand(summed.at({n, g}), grp.o, 1.0, grp.par, v.blocks);
        } else if (grp.items.size() == 1) {
          auto& itm = grp.items[0];
          expand(blocks_ro(itm.src, itm.T), grp.o, itm.coef, grp.par, v.blocks);
        }
      }
    });
    for (size_t n = 0; n < plans.size(); ++n)
      if (!views[n].blocks.empty()) E.ops[pending[n].key] = std::move(views[n]);
  }
};

Mat4 site_three(const Integrals& I, int m, const int sm[2]) {
  Mat4 r;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        double w = I.w(m, sm[a], sm[b], sm[c]);
        if (w != 0.0) r = r + cre(a) * ann(b) * ann(c) * w;
      }
  return r;
}

// S^s_m of a single site for m outside the site
Mat4 site_S(const Integrals& I, int m, const int sm[2]) {
  Mat4 r = site_three(I, m, sm);
  for (int j = 0; j < 2; ++j) r = r + ann(j) * (0.5 * I.t(m, sm[j]));
  return r;
}

Mat4 site_H(const Integrals& I, const int sm[2]) {
  Mat4 r;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      r = r + cre(a) * ann(b) * I.t(sm[a], sm[b]);
      for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2; ++d) {
          double w = I.w(sm[a], sm[b], sm[c], sm[d]);
          if (w != 0.0) r = r + cre(a) * cre(b) * ann(c) * ann(d) * (0.5 * w);
        }
    }
  return r;
}

Contrib C_(const OpView* src, bool T, const Mat4& o, double coef, bool par) {
  Contrib c;
  c.src = src;
  c.srcT = T;
  c.o = o;
  c.coef = coef;
  c.par = par;
  return c;
}

}  // namespace

OpView product_view(const EnvBlock& B, const Integrals& I, Enlarged& E, const std::vector<Contrib>& cs, bool odd) {
  Ctx x(B, I, E, false);
  OpView v;
  v.odd = odd;
  for (const Contrib& c : cs) x.expand(x.src_blocks(c.src, c.srcT), c.o, c.coef, c.par, v.blocks);
  return v;
}

void enlarge(const EnvBlock& B, const Integrals& I, Executor& ex, Enlarged& E, double* flops, bool normal) {
  if (normal && !B.normal) throw std::logic_error("enlarge: complementary pair operators cannot become normal");
  const int L = I.L;
  E.left = B.left;
  E.normal = normal;
  E.ops.clear();
  E.pb = make_prod(B.basis, B.left);
  Ctx x(B, I, E);
  const Mat4 I4 = Mat4::id();
  const bool src_normal = B.normal;
  // site parts of the complementary operators (both modes on the site)
  auto site_P = [&](int i, int j, const int sm[2]) {
    Mat4 P;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) P = P + ann(a) * ann(b) * (0.5 * I.w(i, j, sm[a], sm[b]));
    return P;
  };
  auto site_Q = [&](int i, int l, const int sm[2]) {
    Mat4 Q;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) Q = Q + cre(a) * ann(b) * I.q(i, sm[a], sm[b], l);
    return Q;
  };
  // block-block part of P_ij and Q_il (i, j, l outside the block) from the
  // block's normal pairs: 1/2 sum_{k,l} w_ijkl a_k a_l = -sum_{k<l} 1/2 (w_ijkl - w_ijlk) A_kl^T,
  // sum_{j,k} (w_ijkl - w_ijlk) a+_j a_k = sum_{j,k} q_ijkl B_jk; `m0`, `m1` bound the block's modes
  auto pairs_P_from_A = [&](int i, int j, int m0, int m1, std::vector<Contrib>& cs) {
    for (int k = m0; k < m1; ++k)
      for (int l = k + 1; l < m1; ++l) {
        auto A = x.get(Key(F_A, k, l));
        if (!A) continue;
        const double w = -0.5 * (I.w(i, j, k, l) - I.w(i, j, l, k));
        if (w != 0.0) cs.push_back(C_(A, true, I4, w, false));
      }
  };
  auto pairs_Q_from_B = [&](int i, int l, int m0, int m1, std::vector<Contrib>& cs) {
    for (int j = m0; j < m1; ++j)
      for (int k = m0; k < m1; ++k) {
        auto Bjk = x.get(Key(F_B, j, k));
        if (!Bjk) continue;
        const double q = I.q(i, j, k, l);
        if (q != 0.0) cs.push_back(C_(Bjk, false, I4, q, false));
      }
  };
  if (B.left) {
    const int c = B.cut;          // X = [0, c), site p = c
    E.cut = c + 1;
    const int sm[2] = {2 * c, 2 * c + 1};
    const int nx = 2 * c;
    const int y0 = 2 * (c + 1);   // first mode outside the enlarged block
    x.view(Key(F_I), {C_(nullptr, false, I4, 1.0, false)}, false);
    for (int k = 0; k < nx; ++k)
      if (auto C = x.get(Key(F_C, k))) x.view(Key(F_C, k), {C_(C, false, I4, 1.0, false)}, true);
    for (int s = 0; s < 2; ++s) x.view(Key(F_C, sm[s]), {C_(nullptr, false, cre(s), 1.0, true)}, true);
    if (normal) {
      // A'_kl, k < l
      for (int k = 0; k < nx; ++k)
        for (int l = k + 1; l < nx; ++l)
          if (auto A = x.get(Key(F_A, k, l))) x.view(Key(F_A, k, l), {C_(A, false, I4, 1.0, false)}, false);
      for (int k = 0; k < nx; ++k)
        for (int s = 0; s < 2; ++s)
          if (auto C = x.get(Key(F_C, k))) x.view(Key(F_A, k, sm[s]), {C_(C, false, cre(s), 1.0, true)}, false);
      x.view(Key(F_A, sm[0], sm[1]), {C_(nullptr, false, cre(0) * cre(1), 1.0, false)}, false);
      // B'_kl
      for (int k = 0; k < nx; ++k)
        for (int l = 0; l < nx; ++l)
          if (auto Bk = x.get(Key(F_B, k, l))) x.view(Key(F_B, k, l), {C_(Bk, false, I4, 1.0, false)}, false);
      for (int k = 0; k < nx; ++k)
        for (int s = 0; s < 2; ++s)
          if (auto C = x.get(Key(F_C, k))) {
            x.view(Key(F_B, k, sm[s]), {C_(C, false, ann(s), 1.0, true)}, false);       // a+_k(X) a_l(s)
            x.view(Key(F_B, sm[s], k), {C_(C, true, cre(s), -1.0, true)}, false);       // a+_k(s) a_l(X) = -a_l a+_k
          }
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          x.view(Key(F_B, sm[a], sm[b]), {C_(nullptr, false, cre(a) * ann(b), 1.0, false)}, false);
    } else {
      // P'_ij = 1/2 sum_{kl in X+s} w_ijkl a_k a_l, i < j outside
      for (int i = y0; i < 2 * L; ++i)
        for (int j = i + 1; j < 2 * L; ++j) {
          std::vector<Contrib> cs;
          if (src_normal) pairs_P_from_A(i, j, 0, nx, cs);
          else if (auto P = x.get(Key(F_P, i, j))) cs.push_back(C_(P, false, I4, 1.0, false));
          // (X,s) and (s,X): (a_l)_X (a_s)_s with 1/2 (w_ijls - w_ijsl)
          for (int l = 0; l < nx; ++l) {
            auto C = x.get(Key(F_C, l));
            if (!C) continue;
            for (int s = 0; s < 2; ++s) {
              const double w = 0.5 * (I.w(i, j, l, sm[s]) - I.w(i, j, sm[s], l));
              if (w != 0.0) cs.push_back(C_(C, true, ann(s), w, true));
            }
          }
          cs.push_back(C_(nullptr, false, site_P(i, j, sm), 1.0, false));
          x.materialize(Key(F_P, i, j), std::move(cs), false);
        }
      // Q'_il = sum_{jk in X+s} q_ijkl a+_j a_k, i, l outside
      for (int i = y0; i < 2 * L; ++i)
        for (int l = y0; l < 2 * L; ++l) {
          std::vector<Contrib> cs;
          if (src_normal) pairs_Q_from_B(i, l, 0, nx, cs);
          else if (auto Q = x.get(Key(F_Q, i, l))) cs.push_back(C_(Q, false, I4, 1.0, false));
          for (int j = 0; j < nx; ++j) {
            auto C = x.get(Key(F_C, j));
            if (!C) continue;
            for (int s = 0; s < 2; ++s) {
              const double q1 = I.q(i, j, sm[s], l);    // (X,s): (a+_j)_X (a_s)_s
              if (q1 != 0.0) cs.push_back(C_(C, false, ann(s), q1, true));
              const double q2 = -I.q(i, sm[s], j, l);   // (s,X): (a+_s)_s (a_j)_X = -(a_j)_X (a+_s)_s
              if (q2 != 0.0) cs.push_back(C_(C, true, cre(s), q2, true));
            }
          }
          cs.push_back(C_(nullptr, false, site_Q(i, l, sm), 1.0, false));
          x.materialize(Key(F_Q, i, l), std::move(cs), false);
        }
    }
    // S'_m, m outside the enlarged block
    for (int m = y0; m < 2 * L; ++m) {
      std::vector<Contrib> cs;
      if (auto S = x.get(Key(F_S, m))) cs.push_back(C_(S, false, I4, 1.0, false));
      for (int j = 0; j < 2; ++j) cs.push_back(C_(nullptr, false, ann(j), 0.5 * I.t(m, sm[j]), true));
      for (int s = 0; s < 2; ++s) {
        const int l = sm[s];
        if (src_normal) {
          for (int j = 0; j < nx; ++j)
            for (int k = 0; k < nx; ++k) {
              auto Bjk = x.get(Key(F_B, j, k));
              if (!Bjk) continue;
              double w1 = I.w(m, j, k, l);       // (X,X,s): (a+_j a_k)_X (a_l)_s
              double w2 = -I.w(m, j, l, k);      // (X,s,X): -(a+_j a_k)_X (a_l)_s, roles k<->l
              if (w1 + w2 != 0.0) cs.push_back(C_(Bjk, false, ann(s), w1 + w2, true));
            }
          // (s,X,X): (a_k a_l)_X (a+_j)_s with j = site mode; (a_k a_l) = -A_kl^T (k<l)
          const int j = sm[s];
          for (int k = 0; k < nx; ++k)
            for (int l2 = k + 1; l2 < nx; ++l2) {
              auto A = x.get(Key(F_A, k, l2));
              if (!A) continue;
              double w = -I.w(m, j, k, l2) + I.w(m, j, l2, k);
              if (w != 0.0) cs.push_back(C_(A, true, cre(s), w, true));
            }
        } else {
          // (X,X,s) + (X,s,X) = Q^X_{m,l} (a_l)_s; (s,X,X) = 2 (a+_l)_s P^X_{m,l} = -2 P^X_{l,m} (a+_l)_s
          if (auto Q = x.get(Key(F_Q, m, l))) cs.push_back(C_(Q, false, ann(s), 1.0, true));
          if (auto P = x.get(Key(F_P, l, m))) cs.push_back(C_(P, false, cre(s), -2.0, true));
        }
      }
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          for (int j = 0; j < nx; ++j) {
            auto C = x.get(Key(F_C, j));
            if (!C) continue;
            double w = I.w(m, j, sm[a], sm[b]);                 // (X,s,s): a+_j (a_a a_b)_s
            if (w != 0.0) cs.push_back(C_(C, false, ann(a) * ann(b), w, false));
            double w2 = -I.w(m, sm[a], j, sm[b]) + I.w(m, sm[a], sm[b], j);  // (s,X,s) + (s,s,X)
            if (w2 != 0.0) cs.push_back(C_(C, true, cre(a) * ann(b), w2, false));
          }
        }
      cs.push_back(C_(nullptr, false, site_three(I, m, sm), 1.0, true));
      x.materialize(Key(F_S, m), std::move(cs), true);
    }
    // H'
    {
      std::vector<Contrib> cs;
      if (auto H = x.get(Key(F_H))) cs.push_back(C_(H, false, I4, 1.0, false));
      cs.push_back(C_(nullptr, false, site_H(I, sm), 1.0, false));
      for (int i = 0; i < nx; ++i)
        if (auto C = x.get(Key(F_C, i))) {
          Mat4 Ss = site_S(I, i, sm);
          cs.push_back(C_(C, false, Ss, 1.0, true));
          cs.push_back(C_(C, true, Ss.T(), -1.0, true));
        }
      for (int s = 0; s < 2; ++s)
        if (auto S = x.get(Key(F_S, sm[s]))) {
          cs.push_back(C_(S, false, cre(s), -1.0, true));
          cs.push_back(C_(S, true, ann(s), 1.0, true));
        }
      if (src_normal) {
        // normal pairs of X with the site's complementary P, Q
        for (int i = 0; i < nx; ++i)
          for (int j = i + 1; j < nx; ++j)
            if (auto A = x.get(Key(F_A, i, j))) {
              Mat4 P = site_P(i, j, sm);
              cs.push_back(C_(A, false, P, 2.0, false));
              cs.push_back(C_(A, true, P.T(), 2.0, false));
            }
        for (int i = 0; i < nx; ++i)
          for (int l = 0; l < nx; ++l)
            if (auto Bil = x.get(Key(F_B, i, l))) cs.push_back(C_(Bil, false, site_Q(i, l, sm), 1.0, false));
      } else {
        // complementary pairs of X with the site's normal A, B:
        // 2 (P^X_{s0 s1} A^s + P^X+ A^s+) + sum_ab Q^X_{ab} B^s_ab
        if (auto P = x.get(Key(F_P, sm[0], sm[1]))) {
          const Mat4 A = cre(0) * cre(1);
          cs.push_back(C_(P, false, A, 2.0, false));
          cs.push_back(C_(P, true, A.T(), 2.0, false));
        }
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            if (auto Q = x.get(Key(F_Q, sm[a], sm[b]))) cs.push_back(C_(Q, false, cre(a) * ann(b), 1.0, false));
      }
      x.materialize(Key(F_H), std::move(cs), false);
    }
  } else {
    const int c = B.cut - 1;      // site p = c, Y = [c+1, L)
    E.cut = c;
    const int mc = 2 * c;                     // modes outside the enlarged block: < 2c
    const int sm[2] = {2 * c, 2 * c + 1};
    const int y0 = 2 * (c + 1);
    x.view(Key(F_I), {C_(nullptr, false, I4, 1.0, false)}, false);
    if (E.local) {
      // matrix units |a><b| of every orbital of s + Y: the site's own (site part
      // first, no string), the block's carried over with the site's parity when
      // the unit changes the particle number by one
      static const int NOCC[4] = {0, 1, 1, 2};
      for (int u = 0; u < 16; ++u) {
        const bool odd = (NOCC[u / 4] + NOCC[u % 4]) & 1;
        Mat4 m;
        m(u / 4, u % 4) = 1.0;
        x.view(Key(F_L, c, u), {C_(nullptr, false, m, 1.0, false)}, odd);
        for (int j = c + 1; j < L; ++j)
          if (auto U = x.get(Key(F_L, j, u))) x.view(Key(F_L, j, u), {C_(U, false, I4, 1.0, odd)}, odd);
      }
    }
    for (int s = 0; s < 2; ++s) x.view(Key(F_C, sm[s]), {C_(nullptr, false, cre(s), 1.0, false)}, true);
    for (int k = y0; k < 2 * L; ++k)
      if (auto C = x.get(Key(F_C, k))) x.view(Key(F_C, k), {C_(C, false, I4, 1.0, true)}, true);
    if (normal) {
      // A'_kl, k < l in s+Y (site modes come first)
      for (int k = y0; k < 2 * L; ++k)
        for (int l = k + 1; l < 2 * L; ++l)
          if (auto A = x.get(Key(F_A, k, l))) x.view(Key(F_A, k, l), {C_(A, false, I4, 1.0, false)}, false);
      for (int s = 0; s < 2; ++s)
        for (int l = y0; l < 2 * L; ++l)
          if (auto C = x.get(Key(F_C, l))) x.view(Key(F_A, sm[s], l), {C_(C, false, cre(s), 1.0, true)}, false);
      x.view(Key(F_A, sm[0], sm[1]), {C_(nullptr, false, cre(0) * cre(1), 1.0, false)}, false);
      // B'_kl
      for (int k = y0; k < 2 * L; ++k)
        for (int l = y0; l < 2 * L; ++l)
          if (auto Bk = x.get(Key(F_B, k, l))) x.view(Key(F_B, k, l), {C_(Bk, false, I4, 1.0, false)}, false);
      for (int s = 0; s < 2; ++s)
        for (int k = y0; k < 2 * L; ++k)
          if (auto C = x.get(Key(F_C, k))) {
            x.view(Key(F_B, sm[s], k), {C_(C, true, cre(s), 1.0, true)}, false);    // (a+_s)_s (a_k)_Y
            x.view(Key(F_B, k, sm[s]), {C_(C, false, ann(s), -1.0, true)}, false);  // a+_k(Y) a_s(s) = -(a_s)_s (a+_k)_Y
          }
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          x.view(Key(F_B, sm[a], sm[b]), {C_(nullptr, false, cre(a) * ann(b), 1.0, false)}, false);
    } else {
      // P'_ij, i < j < 2c
      for (int i = 0; i < mc; ++i)
        for (int j = i + 1; j < mc; ++j) {
          std::vector<Contrib> cs;
          if (src_normal) pairs_P_from_A(i, j, y0, 2 * L, cs);
          else if (auto P = x.get(Key(F_P, i, j))) cs.push_back(C_(P, false, I4, 1.0, false));
          for (int s = 0; s < 2; ++s)
            for (int l = y0; l < 2 * L; ++l) {
              auto C = x.get(Key(F_C, l));
              if (!C) continue;
              double w = 0.5 * (I.w(i, j, sm[s], l) - I.w(i, j, l, sm[s]));
              if (w != 0.0) cs.push_back(C_(C, true, ann(s), w, true));
            }
          cs.push_back(C_(nullptr, false, site_P(i, j, sm), 1.0, false));
          x.materialize(Key(F_P, i, j), std::move(cs), false);
        }
      // Q'_il, i, l < 2c
      for (int i = 0; i < mc; ++i)
        for (int l = 0; l < mc; ++l) {
          std::vector<Contrib> cs;
          if (src_normal) pairs_Q_from_B(i, l, y0, 2 * L, cs);
          else if (auto Q = x.get(Key(F_Q, i, l))) cs.push_back(C_(Q, false, I4, 1.0, false));
          for (int s = 0; s < 2; ++s)
            for (int k = y0; k < 2 * L; ++k) {
              auto C = x.get(Key(F_C, k));
              if (!C) continue;
              double q1 = I.q(i, sm[s], k, l);    // (s,Y): a+_j(s) a_k(Y)
              if (q1 != 0.0) cs.push_back(C_(C, true, cre(s), q1, true));
              double q2 = -I.q(i, k, sm[s], l);   // (Y,s): a+_j(Y) a_k(s) = -a_k a+_j
              if (q2 != 0.0) cs.push_back(C_(C, false, ann(s), q2, true));
            }
          cs.push_back(C_(nullptr, false, site_Q(i, l, sm), 1.0, false));
          x.materialize(Key(F_Q, i, l), std::move(cs), false);
        }
    }
    // S'_m, m < 2c
    for (int m = 0; m < mc; ++m) {
      std::vector<Contrib> cs;
      if (auto S = x.get(Key(F_S, m))) cs.push_back(C_(S, false, I4, 1.0, true));
      Mat4 t1;
      for (int j = 0; j < 2; ++j) t1 = t1 + ann(j) * (0.5 * I.t(m, sm[j]));
      cs.push_back(C_(nullptr, false, t1, 1.0, false));
      for (int s = 0; s < 2; ++s) {
        if (src_normal) {
          // (s,Y,Y): (a+_s)_s sum_{kl} w_mskl a_k a_l = -(a+_s)_s sum_{k<l} (w_mskl - w_mslk) A_kl^T
          for (int k = y0; k < 2 * L; ++k)
            for (int l = k + 1; l < 2 * L; ++l) {
              auto A = x.get(Key(F_A, k, l));
              if (!A) continue;
              const double w = -(I.w(m, sm[s], k, l) - I.w(m, sm[s], l, k));
              if (w != 0.0) cs.push_back(C_(A, true, cre(s), w, false));
            }
          // (Y,Y,s) + (Y,s,Y): (a_s)_s sum_{jk} (w_mjks - w_mjsk) B_jk
          for (int j = y0; j < 2 * L; ++j)
            for (int k = y0; k < 2 * L; ++k) {
              auto Bjk = x.get(Key(F_B, j, k));
              if (!Bjk) continue;
              const double w = I.w(m, j, k, sm[s]) - I.w(m, j, sm[s], k);
              if (w != 0.0) cs.push_back(C_(Bjk, false, ann(s), w, false));
            }
        } else {
          if (auto P = x.get(Key(F_P, m, sm[s]))) cs.push_back(C_(P, false, cre(s), 2.0, false));
          if (auto Q = x.get(Key(F_Q, m, sm[s]))) cs.push_back(C_(Q, false, ann(s), 1.0, false));
        }
      }
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int k = y0; k < 2 * L; ++k) {
            auto C = x.get(Key(F_C, k));
            if (!C) continue;
            // (s,s,Y): (a+_a a_b)_s (a_k)_Y ; (s,Y,s): -(a+_a a_b)_s (a_k)_Y
            double w1 = I.w(m, sm[a], sm[b], k) - I.w(m, sm[a], k, sm[b]);
            if (w1 != 0.0) cs.push_back(C_(C, true, cre(a) * ann(b), w1, true));
            // (Y,s,s): (a_a a_b)_s (a+_k)_Y
            double w2 = I.w(m, k, sm[a], sm[b]);
            if (w2 != 0.0) cs.push_back(C_(C, false, ann(a) * ann(b), w2, true));
          }
      cs.push_back(C_(nullptr, false, site_three(I, m, sm), 1.0, false));
      x.materialize(Key(F_S, m), std::move(cs), true);
    }
    // H'
    {
      std::vector<Contrib> cs;
      cs.push_back(C_(nullptr, false, site_H(I, sm), 1.0, false));
      if (auto H = x.get(Key(F_H))) cs.push_back(C_(H, false, I4, 1.0, false));
      for (int s = 0; s < 2; ++s)
        if (auto S = x.get(Key(F_S, sm[s]))) {
          cs.push_back(C_(S, false, cre(s), 1.0, true));
          cs.push_back(C_(S, true, ann(s), -1.0, true));
        }
      for (int m = y0; m < 2 * L; ++m)
        if (auto C = x.get(Key(F_C, m))) {
          Mat4 Ss = site_S(I, m, sm);
          cs.push_back(C_(C, false, Ss, -1.0, true));
          cs.push_back(C_(C, true, Ss.T(), 1.0, true));
        }
      if (src_normal) {
        // the site's complementary P, Q with the normal pairs of Y:
        // 2 sum_{i<j in Y} (P^s_ij A_ij + P^s_ij+ A_ij+) + sum_{jk in Y} Q^s_jk B_jk
        for (int i = y0; i < 2 * L; ++i)
          for (int j = i + 1; j < 2 * L; ++j)
            if (auto A = x.get(Key(F_A, i, j))) {
              Mat4 P = site_P(i, j, sm);
              cs.push_back(C_(A, false, P, 2.0, false));
              cs.push_back(C_(A, true, P.T(), 2.0, false));
            }
        for (int j = y0; j < 2 * L; ++j)
          for (int k = y0; k < 2 * L; ++k)
            if (auto Bjk = x.get(Key(F_B, j, k))) cs.push_back(C_(Bjk, false, site_Q(j, k, sm), 1.0, false));
      } else {
        if (auto P = x.get(Key(F_P, sm[0], sm[1]))) {
          Mat4 A = cre(0) * cre(1);
          cs.push_back(C_(P, false, A, 2.0, false));
          cs.push_back(C_(P, true, A.T(), 2.0, false));
        }
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            if (auto Q = x.get(Key(F_Q, sm[a], sm[b]))) cs.push_back(C_(Q, false, cre(a) * ann(b), 1.0, false));
      }
      x.materialize(Key(F_H), std::move(cs), false);
    }
  }
  x.finish(ex);
  (void)flops;
}

}  // namespace qd
