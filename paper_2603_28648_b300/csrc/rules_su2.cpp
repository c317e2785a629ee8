// Spin-adapted (SU(2)) complementary-operator rules: the reduced operators of
// an enlarged block (block (x) one site) from the block's renormalized reduced
// operators and exact single-site reduced matrices, and the operator-product
// terms of H at the centre. Bond dimensions count SU(2) multiplets (the
// paper's Numerical procedure section); every operator is stored as reduced
// matrix elements between multiplets, so its blocks are those of the
// multiplet basis, not of its M components.
//
// Tensor operators (spatial orbitals; rank in brackets; doubled ranks in code):
//   c_p = a+_p (1/2), c_{p,+1/2} = a+_{p up}, c_{p,-1/2} = a+_{p dn}
//   d_p = adjoint tensor of c_p (1/2): d_{p,+1/2} = a_{p dn}, d_{p,-1/2} = -a_{p up}
//   A^k_pq = [c_p x c_q]^k, B^k_pq = [c_p x d_q]^k, k = 0, 1, stored for p <= q
//   (A^k_qp = (-1)^k A^k_pq; B^k_qp = (-1)^k adjoint(B^k_pq));
//   [d_p x d_q]^k = -adjoint(A^k_pq);
//   T_m = 1/2 sum_q h_mq d_q + sum_{q,r,s} (ms|qr) E_qr d_s  (1/2), E_qr = -sqrt(2) B^0_qr,
//   P^k_pr = sum_{s,q} (pq|rs) [d_s x d_q]^k and
//   Q^0_ij = sum_{k,l} (2 (ij|kl) - (il|kj)) B^0_kl, Q^1_ij = sqrt(3) sum_{k,l} (il|kj) B^1_kl
//   (sums over the block's orbitals; P^k_rp = (-1)^k P^k_pr, Q^k_ji = (-1)^k adjoint(Q^k_ij),
//   stored for p <= r, i <= j).
// Every block keeps c of its orbitals, T of the orbitals outside it and H;
// the pair operators are A, B of its own orbitals (normal) or P, Q of the
// orbitals outside it (complementary). Left blocks at cuts up to the switch
// and right blocks beyond it hold normal pairs, so that at every cut exactly
// one side does; without a switch the normal pairs are on the left everywhere,
// with the switch at L/2 they are on the side with fewer orbitals (the N/2
// rule). At a cut L|R with normal pairs on the left the Hamiltonian is the sum
// of scalar couplings (each "+ h.c." adds the Hermitian conjugate,
// [X x Y]^0 -> e [X~ x Y~]^0 with e = -1 for two odd operators):
//   H = H_L + H_R - sqrt(2) sum_{p in L} [c_p x T_p]^0 - sqrt(2) sum_{m in R} [T_m x c_m]^0 + h.c.
//     + sum_{p<=r in L} f_pr (-1)^(1+k) sqrt(2k+1) [A^k_pr x P^k_pr]^0 + h.c.   (f = 1, or 1/2 at p = r)
//     + sum_{i<j in L} [B^k_ij x Q^k_ij]^0 + h.c. + sum_i [B^k_ii x Q^k_ii]^0;
// with normal pairs on the right the pair sums run over R with the same
// coefficients, [P^k_pr x A^k_pr]^0 and [Q^k_ij x B^k_ij]^0.
// The reduced element of a product O_1 O_2 of operators on the two parts of a
// coupled basis (part 1 first in the fermion order) is the 9j factor of
// su2::coupled times (-1)^(parity of O_2 x particle number of the part-1 ket).
// The three-operator terms of T on an enlarged block are reordered so that
// the operators of one part come first and recoupled with 6j symbols
// (su2::swap23, su2::assoc); the derivation of each coefficient is written
// next to it.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <exception>
#include <functional>
#include <map>
#include <mutex>
#include <stdexcept>
#include <thread>
#include <unordered_map>
#include <vector>

#include "core.hpp"
#include "su2.hpp"

namespace qd {

namespace {

const double SQ2 = std::sqrt(2.0);
const double SQ3 = std::sqrt(3.0);

// site multiplets 0: |0> (n 0, S 0), 1: the doublet (n 1, S 1/2), 2: |updn> (n 2, S 0)
const int MULT_S[3] = {0, 1, 0};
const int MULT_N[3] = {0, 1, 2};
inline int mult_of(int ch) { return ch == 0 ? 0 : (ch == 3 ? 2 : 1); }

// reduced 3x3 matrix of a site tensor operator
struct S3 {
  double v[3][3];
  S3() {
    for (auto& r : v)
      for (double& x : r) x = 0.0;
  }
  S3 operator+(const S3& o) const {
    S3 r;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) r.v[a][b] = v[a][b] + o.v[a][b];
    return r;
  }
  S3 operator*(double s) const {
    S3 r;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) r.v[a][b] = v[a][b] * s;
    return r;
  }
  bool zero() const {
    for (auto& r : v)
      for (double x : r)
        if (x != 0.0) return false;
    return true;
  }
};

S3 s_ident() {
  S3 r;
  for (int a = 0; a < 3; ++a) r.v[a][a] = 1.0;
  return r;
}
// <1/2||c||0> = 1, <2||c||1/2> = -sqrt(2) (a+_dn a+_up|0> = -|updn>, CG <1/2 -1/2; 1/2 1/2|0 0> = -1/sqrt(2))
S3 s_c() {
  S3 r;
  r.v[1][0] = 1.0;
  r.v[2][1] = -SQ2;
  return r;
}
S3 s_adj(const S3& m, int k) {
  S3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (m.v[a][b] != 0.0) r.v[b][a] = m.v[a][b] * su2::adjoint(MULT_S[a], MULT_S[b], k);
  return r;
}
// [X^kx x Y^ky]^k on one site
S3 s_prod(const S3& X, int kx, const S3& Y, int ky, int k) {
  S3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int m = 0; m < 3; ++m)
        if (X.v[a][m] != 0.0 && Y.v[m][b] != 0.0)
          s += su2::same_space(MULT_S[a], MULT_S[m], MULT_S[b], kx, ky, k) * X.v[a][m] * Y.v[m][b];
      r.v[a][b] = std::fabs(s) < 1e-15 ? 0.0 : s;
    }
  return r;
}

struct SiteOps {
  S3 I, c, d, n, nn, A0, B[2], DD0;
  SiteOps() {
    I = s_ident();
    c = s_c();
    d = s_adj(c, 1);
    A0 = s_prod(c, 1, c, 1, 0);
    B[0] = s_prod(c, 1, d, 1, 0);
    B[1] = s_prod(c, 1, d, 1, 2);
    DD0 = s_prod(d, 1, d, 1, 0);
    n = B[0] * (-SQ2);          // E_oo = -sqrt(2) B^0_oo: diag(0, 1, 2)
    nn.v[2][2] = 1.0;           // n_up n_dn
  }
};
const SiteOps& site() {
  static const SiteOps s;
  return s;
}

// T_m of a single site o (m outside it): 1/2 h_mo d_o + (mo|oo) n_o d_o
S3 site_T(const Integrals& I, int m, int o) {
  const SiteOps& S = site();
  const double h = I.h[(size_t)m * I.L + o];
  const double v = I.V[(((size_t)m * I.L + o) * I.L + o) * I.L + o];
  S3 nd = s_prod(S.n, 0, S.d, 1, 1);
  return S.d * (0.5 * h) + nd * v;
}
// H of a single site: h_oo n + (oo|oo) n_up n_dn
S3 site_H(const Integrals& I, int o) {
  const SiteOps& S = site();
  const double h = I.h[(size_t)o * I.L + o];
  const double v = I.V[(((size_t)o * I.L + o) * I.L + o) * I.L + o];
  return S.n * h + S.nn * v;
}

inline double V(const Integrals& I, int p, int q, int r, int s) {
  const size_t L = (size_t)I.L;
  return I.V[((p * L + q) * L + r) * L + s];
}
// coefficient of B^k_kl in Q^k_ij (k2 = 2k)
inline double qcoef(const Integrals& I, int k2, int i, int j, int k, int l) {
  return k2 == 0 ? 2.0 * V(I, i, j, k, l) - V(I, i, l, k, j) : SQ3 * V(I, i, l, k, j);
}

// f(0..n-1) on up to 16 host threads (independent items); the first
// exception of any item is rethrown
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

// One contribution coef [O_B^k1 x o^k2]^k (left: block part first; right:
// site part first). src == nullptr: the block identity (k1 = 0); adj: the
// adjoint tensor of src. par: the operator of part 2 is odd (left: the site
// operator, right: the block operator).
struct C2 {
  const OpView* src;
  bool adj;
  S3 o;
  int k1, k2, k;
  double coef;
  bool par;
};
C2 mk(const OpView* src, bool adj, const S3& o, int k1, int k2, int k, double coef, bool par) {
  return C2{src, adj, o, k1, k2, k, coef, par};
}

struct Ctx2 {
  const EnvBlock& B;
  const Integrals& I;
  Enlarged& E;
  const ProdBasis& pb;
  struct Pending {
    Key key;
    bool odd;
    int k;
    std::vector<C2> cs;
  };
  std::vector<Pending> pending;
  Ctx2(const EnvBlock& b, const Integrals& i, Enlarged& e) : B(b), I(i), E(e), pb(e.pb) {}

  const OpView* get(Key k) const {
    auto it = B.ops.find(k);
    if (it == B.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  }

  std::vector<BRef> src_blocks(const OpView* src, bool adj) const {
    if (src) return adj ? adjoint_su2(*src, nullptr, &B.basis).blocks : src->blocks;
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

  // coef * [src (x) site matrix unit (a, b) of value val]^k on the enlarged basis
  void expand(const std::vector<BRef>& src, int a, int b, double val, int k1, int k2, int k, bool par,
              std::vector<BRef>& out) const {
    if (val == 0.0) return;
    for (const BRef& r0 : src) {
      const int Sr = B.basis.q[r0.r].s, Sc = B.basis.q[r0.c].s;
      for (int i = 0; i < NSITE; ++i) {
        if (mult_of(i) != a) continue;
        const int sr = pb.find(r0.r, i);
        if (sr < 0) continue;
        for (int i2 = 0; i2 < NSITE; ++i2) {
          if (mult_of(i2) != b) continue;
          const int sc = pb.find(r0.c, i2);
          if (sc < 0) continue;
          const int Jr = pb.sub_qn(sr).s, Jc = pb.sub_qn(sc).s;
          const double F = E.left ? su2::coupled(Sr, MULT_S[a], Jr, Sc, MULT_S[b], Jc, k1, k2, k)
                                  : su2::coupled(MULT_S[a], Sr, Jr, MULT_S[b], Sc, Jc, k2, k1, k);
          if (F == 0.0) continue;
          double sgn = 1.0;
          if (par) {
            if (E.left) { if (B.basis.q[r0.c].n & 1) sgn = -1.0; }
            else if (MULT_N[b] & 1) sgn = -1.0;
          }
          BRef r = r0;
          r.r = sr;
          r.c = sc;
          r.sc = r0.sc * val * F * sgn;
          out.push_back(r);
        }
      }
    }
  }

  void view(Key key, const std::vector<C2>& cs, bool odd, int k) {
    OpView v;
    v.odd = odd;
    v.k2 = k;
    for (const C2& c : cs) {
      const std::vector<BRef> src = src_blocks(c.src, c.adj);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) expand(src, a, b, c.coef * c.o.v[a][b], c.k1, c.k2, c.k, c.par, v.blocks);
    }
    if (!v.blocks.empty()) E.ops[key] = std::move(v);
  }

  void materialize(Key key, std::vector<C2>&& cs, bool odd, int k) { pending.push_back({key, odd, k, std::move(cs)}); }

  // Group every pending operator's contributions by (site matrix unit, ranks,
  // parity flag): a group with one block operator stays a reference, a group
  // with several is summed once into new storage on the block basis.
  struct Item { const OpView* src; bool adj; double coef; };
  struct Group { int a, b, k1, k2, k; bool par; std::vector<Item> items; };
  struct Plan { std::vector<Group> groups; };

  void finish(Executor& ex) {
    std::vector<Plan> plans(pending.size());
    parallel_for(pending.size(), [&](size_t n) {
      std::map<std::tuple<int, int, int, int, int, int>, int> gi;
      std::vector<std::unordered_map<uintptr_t, int>> where;
      auto& G = plans[n].groups;
      for (const C2& c : pending[n].cs) {
        if (c.coef == 0.0) continue;
        const uintptr_t id = reinterpret_cast<uintptr_t>(c.src) * 2 + (c.adj ? 1 : 0);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            const double x = c.o.v[a][b];
            if (x == 0.0) continue;
            auto key = std::make_tuple(a * 3 + b, c.k1, c.k2, c.k, c.par ? 1 : 0, 0);
            auto it = gi.find(key);
            int g;
            if (it == gi.end()) {
              g = (int)G.size();
              gi.emplace(key, g);
              G.push_back({a, b, c.k1, c.k2, c.k, c.par, {}});
              where.emplace_back();
            } else {
              g = it->second;
            }
            auto ins = where[g].emplace(id, (int)G[g].items.size());
            if (ins.second) G[g].items.push_back({c.src, c.adj, c.coef * x});
            else G[g].items[ins.first->second].coef += c.coef * x;
          }
      }
    });
    std::unordered_map<uintptr_t, std::vector<BRef>> blocks_of;
    for (auto& pl : plans)
      for (auto& g : pl.groups)
        for (auto& itm : g.items) {
          const uintptr_t id = reinterpret_cast<uintptr_t>(itm.src) * 2 + (itm.adj ? 1 : 0);
          if (!blocks_of.count(id)) blocks_of.emplace(id, src_blocks(itm.src, itm.adj));
        }
    auto blocks_ro = [&](const OpView* src, bool adj) -> const std::vector<BRef>& {
      return blocks_of.at(reinterpret_cast<uintptr_t>(src) * 2 + (adj ? 1 : 0));
    };
    // summed groups: destination blocks per group (offsets in order of first
    // appearance), problems in block-key order
    struct Mat {
      size_t n, g;
      std::map<std::pair<int, int>, std::pair<int64_t, std::pair<int, int>>> blk;
      int64_t size = 0, off = 0;
      size_t nseg = 0, seg0 = 0, prob0 = 0;
    };
    std::vector<Mat> mats;
    for (size_t n = 0; n < plans.size(); ++n)
      for (size_t g = 0; g < plans[n].groups.size(); ++g)
        if (plans[n].groups[g].items.size() >= 2) {
          mats.emplace_back();
          mats.back().n = n;
          mats.back().g = g;
        }
    parallel_for(mats.size(), [&](size_t mi) {
      Mat& mt = mats[mi];
      for (auto& itm : plans[mt.n].groups[mt.g].items)
        for (const BRef& b : blocks_ro(itm.src, itm.adj)) {
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
    if (nseg > (size_t)INT32_MAX) throw std::runtime_error("enlarge_su2: summation task list too long");
    uint64_t store = total ? ex.alloc(total) : 0;
    if (store) E.owned.push_back(store);
    Launch l;
    l.segs.resize(nseg);
    l.probs.resize(nprob);
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
        for (const BRef& b : blocks_ro(itm.src, itm.adj)) {
          key_of.push_back(kidx.at({b.r, b.c}));
          start[key_of.back() + 1]++;
        }
      for (size_t i = 0; i < kidx.size(); ++i) start[i + 1] += start[i];
      std::vector<size_t> pos(start.begin(), start.end() - 1);
      size_t e = 0;
      for (auto& itm : grp.items)
        for (const BRef& b : blocks_ro(itm.src, itm.adj)) {
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
    std::map<std::pair<size_t, size_t>, std::vector<BRef>> summed;
    for (size_t mi = 0; mi < mats.size(); ++mi) summed[{mats[mi].n, mats[mi].g}] = std::move(refs[mi]);
    if (!l.empty()) ex.run(l, 0, 0);
    std::vector<OpView> views(plans.size());
    parallel_for(plans.size(), [&](size_t n) {
      OpView& v = views[n];
      v.odd = pending[n].odd;
      v.k2 = pending[n].k;
      for (size_t g = 0; g < plans[n].groups.size(); ++g) {
        auto& grp = plans[n].groups[g];
        if (grp.items.size() >= 2) {
          expand(summed.at({n, g}), grp.a, grp.b, 1.0, grp.k1, grp.k2, grp.k, grp.par, v.blocks);
        } else if (grp.items.size() == 1) {
          auto& itm = grp.items[0];
          expand(blocks_ro(itm.src, itm.adj), grp.a, grp.b, itm.coef, grp.k1, grp.k2, grp.k, grp.par, v.blocks);
        }
      }
    });
    for (size_t n = 0; n < plans.size(); ++n)
      if (!views[n].blocks.empty()) E.ops[pending[n].key] = std::move(views[n]);
  }
};

}  // namespace

OpView adjoint_su2(const OpView& o, const ProdBasis* pb, const Basis* basis) {
  OpView t;
  t.odd = o.odd;
  t.k2 = o.k2;
  t.blocks.reserve(o.blocks.size());
  for (const BRef& b : o.blocks) {
    const int Sr = pb ? pb->sub_qn(b.r).s : basis->q[b.r].s;
    const int Sc = pb ? pb->sub_qn(b.c).s : basis->q[b.c].s;
    BRef x = b;
    std::swap(x.r, x.c);
    std::swap(x.rows, x.cols);
    x.tr = !b.tr;
    x.sc = b.sc * su2::adjoint(Sr, Sc, o.k2);
    t.blocks.push_back(x);
  }
  return t;
}

void enlarge_su2(const EnvBlock& B, const Integrals& I, Executor& ex, Enlarged& E, bool normal) {
  // normal: the enlarged block keeps the pair operators A^k, B^k of its own
  // orbitals; otherwise P^k, Q^k of the orbitals outside it. A block with
  // normal pairs may switch here (its pairs then form the block-block part of
  // P' and Q'); complementary pairs cannot become normal.
  if (normal && !B.normal) throw std::logic_error("enlarge_su2: complementary pairs cannot become normal");
  const int L = I.L;
  const bool left = B.left;
  E.left = left;
  E.normal = normal;
  E.ops.clear();
  E.pb = make_prod(B.basis, left);
  Ctx2 x(B, I, E);
  const SiteOps& S = site();
  const S3& I3 = S.I;
  // recoupling coefficients of the three-operator terms of T (all spins 1/2,
  // E_qr d_s = -sqrt(2) [[c_q x d_r]^0 x d_s]^1/2, operators numbered 0, 1, 2):
  //   pair (0, 2) coupled first, 1 last:  swap23_K = <((0 2)K, 1)|((0 1)0, 2)>
  //   pair (1, 2) coupled first, 0 apart: assoc_K  = <(0, (1 2)K)|((0 1)0, 2)>
  // with (-1)^k for the other coupling order of the pair and the single
  // operator; K = 2k doubled
  double sw[2], as[2];
  for (int k = 0; k < 2; ++k) {
    sw[k] = su2::swap23(1, 1, 1, 0, 2 * k, 1);
    as[k] = su2::assoc(1, 1, 1, 0, 2 * k, 1);
  }
  auto sgnk = [](int k) { return (k & 1) ? -1.0 : 1.0; };
  // the added site o, the block's orbitals [b0, b1), the orbitals outside the
  // enlarged block [u0, u1); on a right block the site part comes first, and
  // an even rank-k operator X and an odd spin-1/2 one Y couple as
  // [X x Y]^1/2 = (-1)^k [Y x X]^1/2 (they commute, Clebsch-Gordan symmetry)
  const int o = left ? B.cut : B.cut - 1;
  const int b0 = left ? 0 : o + 1, b1 = left ? o : L;
  const int u0 = left ? o + 1 : 0, u1 = left ? L : o;
  E.cut = left ? o + 1 : o;
  auto key2 = [](int f, int p, int q, int K) { return p <= q ? Key(f, p, q, K) : Key(f, q, p, K); };
  x.view(Key(F_I), {mk(nullptr, false, I3, 0, 0, 0, 1.0, false)}, false, 0);
  for (int p = b0; p < b1; ++p)
    if (auto C = x.get(Key(F_C, p))) x.view(Key(F_C, p), {mk(C, false, I3, 1, 0, 1, 1.0, !left)}, true, 1);
  x.view(Key(F_C, o), {mk(nullptr, false, S.c, 0, 1, 1, 1.0, left)}, true, 1);
  if (normal) {
    // A'^k, B'^k of the enlarged block's orbitals (p <= q): the block's own,
    // the block orbital with the site ([c_p x c_o], [c_p x d_o] on a left
    // block; [c_o x c_q], [c_o x d_q] on a right one) and the site's
    for (int k = 0; k < 2; ++k) {
      const int K = 2 * k;
      for (int p = b0; p < b1; ++p)
        for (int q = p; q < b1; ++q) {
          if (auto A = x.get(Key(F_A, p, q, K))) x.view(Key(F_A, p, q, K), {mk(A, false, I3, K, 0, K, 1.0, false)}, false, K);
          if (auto Bv = x.get(Key(F_B, p, q, K))) x.view(Key(F_B, p, q, K), {mk(Bv, false, I3, K, 0, K, 1.0, false)}, false, K);
        }
      for (int p = b0; p < b1; ++p)
        if (auto C = x.get(Key(F_C, p))) {
          if (left) {
            x.view(Key(F_A, p, o, K), {mk(C, false, S.c, 1, 1, K, 1.0, true)}, false, K);
            x.view(Key(F_B, p, o, K), {mk(C, false, S.d, 1, 1, K, 1.0, true)}, false, K);
          } else {
            x.view(Key(F_A, o, p, K), {mk(C, false, S.c, 1, 1, K, 1.0, true)}, false, K);
            x.view(Key(F_B, o, p, K), {mk(C, true, S.c, 1, 1, K, 1.0, true)}, false, K);
          }
        }
      x.view(Key(F_B, o, o, K), {mk(nullptr, false, S.B[k], 0, K, K, 1.0, false)}, false, K);
    }
    x.view(Key(F_A, o, o, 0), {mk(nullptr, false, S.A0, 0, 0, 0, 1.0, false)}, false, 0);
  }
  // T'_m for the orbitals m outside the enlarged block
  for (int m = u0; m < u1; ++m) {
    std::vector<C2> cs;
    if (auto T = x.get(Key(F_S, m))) cs.push_back(mk(T, false, I3, 1, 0, 1, 1.0, !left));
    cs.push_back(mk(nullptr, false, site_T(I, m, o), 0, 1, 1, 1.0, left));
    // one block operator, two on the site
    for (int q = b0; q < b1; ++q) {
      auto Cq = x.get(Key(F_C, q));
      if (!Cq) continue;
      // (b) q = r = o, s = q in the block: (mq|oo) [d_q x n_o]^1/2 (n has rank 0)
      cs.push_back(mk(Cq, true, S.n, 1, 0, 1, V(I, m, q, o, o), !left));
      // (e) r = s = o: (mo|qo) E_qo d_o = -sqrt(2) assoc_0 [c_q x [d_o x d_o]^0]^1/2
      // (left); on a right block reordered d_o d_o c_q (sign +1), tree ((1 2)0, 0)
      cs.push_back(mk(Cq, false, S.DD0, 1, 0, 1, -SQ2 * as[0] * V(I, m, o, q, o), !left));
      // (f) q = s = o: (mo|oq) E_oq d_o. Left: reordered d_q c_o d_o (sign -1),
      // tree (1, (0 2)K): -sqrt(2) (-1) (-1)^k swap23_K [d_q x B^K_oo]^1/2.
      // Right: reordered c_o d_o d_q (sign -1), tree ((0 2)K, 1): sqrt(2) swap23_K [B^K_oo x d_q]
      for (int k = 0; k < 2; ++k)
        cs.push_back(mk(Cq, true, S.B[k], 1, 2 * k, 1, SQ2 * (left ? sgnk(k) : 1.0) * sw[k] * V(I, m, o, o, q), !left));
    }
    // two block operators, one on the site
    for (int k = 0; k < 2; ++k) {
      const int K = 2 * k;
      if (B.normal) {
        // from the block's pairs, written block part first ([X x Y]); a right
        // block takes the site part first, hence the factor (-1)^k there
        const double rs = left ? 1.0 : sgnk(k);
        for (int p = b0; p < b1; ++p)
          for (int q = p; q < b1; ++q) {
            // (a) s = o: (mo|pq) E_pq d_o = -sqrt(2) [B^0_pq x d_o]; B^0_qp = adjoint(B^0_pq)
            // (c) r = o: (ms|qo) E_qo d_s, reordered c_q d_s d_o (sign -1), tree ((0 2)K, 1):
            //     -sqrt(2) (-1) swap23_K [B^K_qs x d_o]; B^K_sq = (-1)^k adjoint(B^K_qs)
            if (auto Bv = x.get(Key(F_B, p, q, K))) {
              double direct = SQ2 * sw[k] * V(I, m, q, p, o);   // (c) with (q, s) = (p, q)
              double adj = p != q ? SQ2 * sw[k] * sgnk(k) * V(I, m, p, q, o) : 0.0;   // (c) with (q, s) = (q, p)
              if (k == 0) {
                direct += -SQ2 * V(I, m, o, p, q);
                if (p != q) adj += -SQ2 * V(I, m, o, q, p);
              }
              cs.push_back(mk(Bv, false, S.d, K, 1, 1, rs * direct, left));
              if (adj != 0.0) cs.push_back(mk(Bv, true, S.d, K, 1, 1, rs * adj, left));
            }
            // (d) q = o: (ms|or) E_or d_s, reordered d_r d_s c_o (sign +1), tree ((1 2)K, 0):
            //     -sqrt(2) (-1)^k assoc_K [[d_r x d_s]^K x c_o]; [d_r x d_s]^K = -adjoint(A^K_rs),
            //     [d_s x d_r]^K = (-1)^k [d_r x d_s]^K
            if (auto A = x.get(Key(F_A, p, q, K))) {
              double w = V(I, m, q, o, p);                   // (r, s) = (p, q)
              if (p != q) w += sgnk(k) * V(I, m, p, o, q);   // (r, s) = (q, p)
              cs.push_back(mk(A, true, S.c, K, 1, 1, rs * SQ2 * sgnk(k) * as[k] * w, left));
            }
          }
      } else {
        // from the block's complementary pairs of (m, o):
        //   (a) + (c) = -1/sqrt(2) [d_o x Q^k_mo]^1/2,  (d) = -sqrt(2) assoc_K [c_o x P^K_mo]^1/2;
        // a left block stores (o, m) (o < m): Q^k_mo = (-1)^k adjoint(Q^k_om),
        // P^k_mo = (-1)^k P^k_om, and the block part comes first ((-1)^k again)
        if (auto Q = x.get(key2(F_Q, m, o, K))) cs.push_back(mk(Q, left, S.d, K, 1, 1, -1.0 / SQ2, left));
        if (auto P = x.get(key2(F_P, m, o, K))) cs.push_back(mk(P, false, S.c, K, 1, 1, -SQ2 * as[k], left));
      }
    }
    x.materialize(Key(F_S, m), std::move(cs), true, 1);
  }
  if (!normal) {
    // P'^k_pr, Q'^k_ij for p <= r, i <= j outside the enlarged block:
    //   P^k_pr = sum_{s,q} (pq|rs) [d_s x d_q]^k,  Q^k_ij = sum_{k,l} q^k_ijkl [c_k x d_l]^k
    // over the block's orbitals and the site; the block-block part is the
    // block's own P, Q, or (at the switch) formed from its A, B:
    //   [d_a x d_b]^k = -adjoint(A^k_ab), [d_b x d_a]^k = (-1)^k [d_a x d_b]^k (a != b),
    //   [c_b x d_a]^k = (-1)^k adjoint(B^k_ab)
    for (int k = 0; k < 2; ++k) {
      const int K = 2 * k;
      for (int p = u0; p < u1; ++p)
        for (int r = p; r < u1; ++r) {
          std::vector<C2> cs;
          if (!B.normal) {
            if (auto P = x.get(Key(F_P, p, r, K))) cs.push_back(mk(P, false, I3, K, 0, K, 1.0, false));
          } else {
            for (int a = b0; a < b1; ++a)
              for (int b = a; b < b1; ++b)
                if (auto A = x.get(Key(F_A, a, b, K))) {
                  const double w = V(I, p, b, r, a) + (a != b ? sgnk(k) * V(I, p, a, r, b) : 0.0);
                  if (w != 0.0) cs.push_back(mk(A, true, I3, K, 0, K, -w, false));
                }
          }
          if (k == 0) cs.push_back(mk(nullptr, false, S.DD0, 0, 0, 0, V(I, p, o, r, o), false));
          // one operator on the block (orbital a), one on the site: left
          // [d_a x d_o]^k with (po|ra) + (-1)^k (pa|ro); right [d_o x d_a]^k
          // with (pa|ro) + (-1)^k (po|ra)
          for (int a = b0; a < b1; ++a)
            if (auto Ca = x.get(Key(F_C, a))) {
              const double w = left ? V(I, p, o, r, a) + sgnk(k) * V(I, p, a, r, o)
                                    : V(I, p, a, r, o) + sgnk(k) * V(I, p, o, r, a);
              if (w != 0.0) cs.push_back(mk(Ca, true, S.d, 1, 1, K, w, true));
            }
          x.materialize(Key(F_P, p, r, K), std::move(cs), false, K);
        }
      for (int i = u0; i < u1; ++i)
        for (int j = i; j < u1; ++j) {
          std::vector<C2> cs;
          if (!B.normal) {
            if (auto Q = x.get(Key(F_Q, i, j, K))) cs.push_back(mk(Q, false, I3, K, 0, K, 1.0, false));
          } else {
            for (int a = b0; a < b1; ++a)
              for (int b = a; b < b1; ++b)
                if (auto Bv = x.get(Key(F_B, a, b, K))) {
                  const double w1 = qcoef(I, K, i, j, a, b);
                  if (w1 != 0.0) cs.push_back(mk(Bv, false, I3, K, 0, K, w1, false));
                  const double w2 = a != b ? sgnk(k) * qcoef(I, K, i, j, b, a) : 0.0;
                  if (w2 != 0.0) cs.push_back(mk(Bv, true, I3, K, 0, K, w2, false));
                }
          }
          cs.push_back(mk(nullptr, false, S.B[k], 0, K, K, qcoef(I, K, i, j, o, o), false));
          for (int a = b0; a < b1; ++a)
            if (auto Ca = x.get(Key(F_C, a))) {
              if (left) {
                // (k, l) = (a, o): q^k_ijao [c_a x d_o]^k; (o, a): q^k_ijoa [c_o x d_a]^k = (-1)^k q^k_ijoa [d_a x c_o]^k
                const double w1 = qcoef(I, K, i, j, a, o);
                if (w1 != 0.0) cs.push_back(mk(Ca, false, S.d, 1, 1, K, w1, true));
                const double w2 = sgnk(k) * qcoef(I, K, i, j, o, a);
                if (w2 != 0.0) cs.push_back(mk(Ca, true, S.c, 1, 1, K, w2, true));
              } else {
                // (k, l) = (o, a): q^k_ijoa [c_o x d_a]^k; (a, o): q^k_ijao [c_a x d_o]^k = (-1)^k q^k_ijao [d_o x c_a]^k
                const double w1 = qcoef(I, K, i, j, o, a);
                if (w1 != 0.0) cs.push_back(mk(Ca, true, S.c, 1, 1, K, w1, true));
                const double w2 = sgnk(k) * qcoef(I, K, i, j, a, o);
                if (w2 != 0.0) cs.push_back(mk(Ca, false, S.d, 1, 1, K, w2, true));
              }
            }
          x.materialize(Key(F_Q, i, j, K), std::move(cs), false, K);
        }
    }
  }
  // H' = H of the block + H of the site + the terms of H across the block | site cut
  {
    std::vector<C2> cs;
    if (auto H = x.get(Key(F_H))) cs.push_back(mk(H, false, I3, 0, 0, 0, 1.0, false));
    cs.push_back(mk(nullptr, false, site_H(I, o), 0, 0, 0, 1.0, false));
    // -sqrt(2) [c_p x T_p(site)]^0 over the block's orbitals and -sqrt(2) [T_o(block) x c_o]^0
    // (left; a right block writes the site part first), each with its Hermitian conjugate
    for (int p = b0; p < b1; ++p)
      if (auto C = x.get(Key(F_C, p))) {
        const S3 T = site_T(I, p, o);
        cs.push_back(mk(C, false, T, 1, 1, 0, -SQ2, true));
        cs.push_back(mk(C, true, s_adj(T, 1), 1, 1, 0, SQ2, true));
      }
    if (auto T = x.get(Key(F_S, o))) {
      cs.push_back(mk(T, false, S.c, 1, 1, 0, -SQ2, true));
      cs.push_back(mk(T, true, S.d, 1, 1, 0, SQ2, true));
    }
    if (B.normal) {
      // pairs of the block with P, Q of the site (the order of two even factors is free)
      for (int p = b0; p < b1; ++p)
        for (int r = p; r < b1; ++r) {
          // P^0_pr(o) = (po|ro) [d_o x d_o]^0 (P^1 of one site vanishes)
          if (auto A = x.get(Key(F_A, p, r, 0))) {
            const double coef = (p == r ? 0.5 : 1.0) * -1.0 * V(I, p, o, r, o);
            cs.push_back(mk(A, false, S.DD0, 0, 0, 0, coef, false));
            cs.push_back(mk(A, true, s_adj(S.DD0, 0), 0, 0, 0, coef, false));
          }
          for (int k = 0; k < 2; ++k)
            if (auto Bv = x.get(Key(F_B, p, r, 2 * k))) {
              // Q^k_pr(o) = q^k_proo B^k_oo
              const double qc = qcoef(I, 2 * k, p, r, o, o);
              cs.push_back(mk(Bv, false, S.B[k], 2 * k, 2 * k, 0, qc, false));
              if (p != r) cs.push_back(mk(Bv, true, s_adj(S.B[k], 2 * k), 2 * k, 2 * k, 0, qc, false));
            }
        }
    } else {
      // the block's P, Q of the site orbital with the site's pairs
      if (auto P = x.get(Key(F_P, o, o, 0))) {
        cs.push_back(mk(P, false, S.A0, 0, 0, 0, -0.5, false));
        cs.push_back(mk(P, true, s_adj(S.A0, 0), 0, 0, 0, -0.5, false));
      }
      for (int k = 0; k < 2; ++k)
        if (auto Q = x.get(Key(F_Q, o, o, 2 * k))) cs.push_back(mk(Q, false, S.B[k], 2 * k, 2 * k, 0, 1.0, false));
    }
    x.materialize(Key(F_H), std::move(cs), false, 0);
  }
  x.finish(ex);
}

std::vector<CenterTerm> center_terms_su2(const Enlarged& Lp, const Enlarged& Rp, const Integrals& I) {
  if (!Lp.left || Rp.left || Lp.cut != Rp.cut) throw std::logic_error("center_terms_su2: blocks do not meet");
  const int c = Lp.cut;   // L' = [0, c), R' = [c, L)
  const int L = I.L;
  std::vector<CenterTerm> terms;
  auto get = [](const Enlarged& E, Key k) -> const OpView* {
    auto it = E.ops.find(k);
    if (it == E.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  };
  const OpView* IL = get(Lp, Key(F_I));
  const OpView* IR = get(Rp, Key(F_I));
  auto add = [&](const OpView* a, bool at, const OpView* b, bool bt, double coef, int k2) {
    CenterTerm t{a, at, b, bt, coef};
    t.k2 = k2;
    terms.push_back(t);
  };
  if (auto h = get(Lp, Key(F_H))) add(h, false, IR, false, 1.0, 0);
  if (auto h = get(Rp, Key(F_H))) add(IL, false, h, false, 1.0, 0);
  if (I.ecore != 0.0) add(IL, false, IR, false, I.ecore, 0);
  for (int p = 0; p < c; ++p) {
    auto C = get(Lp, Key(F_C, p));
    auto T = get(Rp, Key(F_S, p));
    if (!C || !T) continue;
    add(C, false, T, false, -SQ2, 1);
    add(C, true, T, true, SQ2, 1);
  }
  for (int m = c; m < L; ++m) {
    auto T = get(Lp, Key(F_S, m));
    auto C = get(Rp, Key(F_C, m));
    if (!C || !T) continue;
    add(T, false, C, false, -SQ2, 1);
    add(T, true, C, true, SQ2, 1);
  }
  if (Lp.normal == Rp.normal) throw std::logic_error("center_terms_su2: exactly one enlarged block must hold normal pairs");
  // pair terms over the orbitals of the side with normal pairs; with normal
  // pairs on the right the factors are [P x A]^0 and [Q x B]^0, equal to
  // [A x P]^0 and [B x Q]^0 (even operators of equal rank coupled to 0), and
  // the spin sums of a+a+aa with both creators on one side give the same
  // coefficients whichever side that is
  const int n0 = Lp.normal ? 0 : c, n1 = Lp.normal ? c : L;
  const Enlarged& NE = Lp.normal ? Lp : Rp;   // normal pairs A, B
  const Enlarged& CE = Lp.normal ? Rp : Lp;   // complementary pairs P, Q
  auto add_pair = [&](const OpView* nrm, bool nt, const OpView* cmp, bool ct, double coef, int k2) {
    if (Lp.normal) add(nrm, nt, cmp, ct, coef, k2);
    else add(cmp, ct, nrm, nt, coef, k2);
  };
  for (int k = 0; k < 2; ++k) {
    const int K = 2 * k;
    const double ak = ((1 + k) & 1 ? -1.0 : 1.0) * std::sqrt(2.0 * k + 1.0);
    for (int p = n0; p < n1; ++p)
      for (int r = p; r < n1; ++r) {
        auto A = get(NE, Key(F_A, p, r, K));
        auto P = get(CE, Key(F_P, p, r, K));
        if (A && P) {
          const double coef = (p == r ? 0.5 : 1.0) * ak;
          add_pair(A, false, P, false, coef, K);
          add_pair(A, true, P, true, coef, K);
        }
        auto Bv = get(NE, Key(F_B, p, r, K));
        auto Q = get(CE, Key(F_Q, p, r, K));
        if (Bv && Q) {
          add_pair(Bv, false, Q, false, 1.0, K);
          if (p != r) add_pair(Bv, true, Q, true, 1.0, K);
        }
      }
  }
  return terms;
}

}  // namespace qd
