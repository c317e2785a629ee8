// Complementary-operator rules: how the operators of an enlarged block
// (block (x) site) are written in terms of the block's renormalized operators
// and exact single-site matrices.
//
// Spin-orbital form of the active-space Hamiltonian (k = 2p + sigma):
//   H = sum t_kl a+_k a_l + 1/2 sum w_ijkl a+_i a+_j a_k a_l,
//   t_kl = h_{p_k p_l} d(s_k, s_l),  w_ijkl = (p_i p_l | p_j p_k) d(s_i, s_l) d(s_j, s_k).
// Operators kept by a block at cut c (left = sites [0,c), right = [c,L)):
//   left : I, C_k = a+_k, A_kl = a+_k a+_l (k<l), B_kl = a+_k a_l   (k, l in block)
//          S_m (m outside), H
//   right: I, C_k (k in block), S_m (m outside, i.e. m < 2c),
//          P_ij = 1/2 sum_{kl in block} w_ijkl a_k a_l            (i<j<2c)
//          Q_il = sum_{jk in block} (w_ijkl - w_ijlk) a+_j a_k     (i,l<2c)
//          H
//   S^B_m = 1/2 sum_{j in B} t_mj a_j + sum_{jkl in B} w_mjkl a+_j a_k a_l.
// Decomposition at a cut L|R (normal pairs on the left):
//   H = H_L + H_R + sum_{i in L} (a+_i S^R_i - a_i (S^R_i)^+)
//     + sum_{m in R} (-S^L_m a+_m + (S^L_m)^+ a_m)
//     + 2 sum_{i<j in L} (A_ij P_ij + A_ij^+ P_ij^+) + sum_{il in L} B_il Q_il.
// A product O_X O_s on X (x) site acts as (O_X P_X^{p(O_s)}) (x) O_s; a
// product O_s O_Y on site (x) Y as (O_s P_s^{p(O_Y)}) (x) O_Y.
#include <algorithm>
#include <atomic>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>
#include <cmath>
#include <map>
#include <unordered_map>
#include <stdexcept>

#include "core.hpp"

namespace qd {

std::vector<Key> block_keys(bool left, int c, int L) {
  std::vector<Key> k;
  k.push_back(Key(F_I));
  if (left) {
    for (int a = 0; a < 2 * c; ++a) k.push_back(Key(F_C, a));
    for (int a = 0; a < 2 * c; ++a)
      for (int b = a + 1; b < 2 * c; ++b) k.push_back(Key(F_A, a, b));
    for (int a = 0; a < 2 * c; ++a)
      for (int b = 0; b < 2 * c; ++b) k.push_back(Key(F_B, a, b));
    for (int m = 2 * c; m < 2 * L; ++m) k.push_back(Key(F_S, m));
  } else {
    for (int a = 2 * c; a < 2 * L; ++a) k.push_back(Key(F_C, a));
    for (int a = 0; a < 2 * c; ++a)
      for (int b = a + 1; b < 2 * c; ++b) k.push_back(Key(F_P, a, b));
    for (int a = 0; a < 2 * c; ++a)
      for (int b = 0; b < 2 * c; ++b) k.push_back(Key(F_Q, a, b));
    for (int m = 0; m < 2 * c; ++m) k.push_back(Key(F_S, m));
  }
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
  Ctx(const EnvBlock& b, const Integrals& i, Enlarged& e) : B(b), I(i), E(e), pb(e.pb) {
    pending.reserve(16 + 8 * (size_t)i.L * i.L);  // complementary operators of one block
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
  void finish(Executor& ex) {
    const Monos& M = monos();
    struct Item { const OpView* src; bool T; double coef; };
    struct Group { Mat4 o; bool par; std::vector<Item> items; };
    struct Plan { std::vector<Group> groups; };
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
    // storage for summed groups
    int64_t total = 0;
    struct Mat { size_t n, g; std::map<std::pair<int, int>, std::pair<int64_t, std::pair<int, int>>> blk; };
    std::vector<Mat> mats;
    for (size_t n = 0; n < plans.size(); ++n)
      for (size_t g = 0; g < plans[n].groups.size(); ++g) {
        auto& grp = plans[n].groups[g];
        if (grp.items.size() < 2) continue;
        Mat mt{n, g, {}};
        for (auto& itm : grp.items)
          for (const BRef& b : blocks(itm.src, itm.T)) {
            auto key = std::make_pair(b.r, b.c);
            if (!mt.blk.count(key)) {
              mt.blk[key] = {total, {b.rows, b.cols}};
              total += (int64_t)b.rows * b.cols;
            }
          }
        mats.push_back(mt);
      }
    uint64_t store = total ? ex.alloc(total) : 0;
    if (store) E.owned.push_back(store);
    Launch l;
    {
      size_t nseg = 0, nprob = 0;
      for (auto& mt : mats) {
        nprob += mt.blk.size();
        for (auto& itm : plans[mt.n].groups[mt.g].items) nseg += blocks(itm.src, itm.T).size();
      }
      l.segs.reserve(nseg);
      l.probs.reserve(nprob);
    }
    std::map<std::pair<size_t, size_t>, std::vector<BRef>> summed;
    // block lists of every summed source, built here so that the parallel part
    // below only reads the cache
    for (auto& mt : mats)
      for (auto& itm : plans[mt.n].groups[mt.g].items) blocks(itm.src, itm.T);
    auto blocks_ro = [&](const OpView* src, bool T) -> const std::vector<BRef>& {
      return blocks_of.at(reinterpret_cast<uintptr_t>(src) * 2 + (T ? 1 : 0));
    };
    // each summed group's problems, segments (grouped by destination block in
    // key order, item order within a block) and block references, independently
    struct Part {
      std::vector<Seg> segs;
      std::vector<Prob> probs;
      std::vector<BRef> refs;
    };
    std::vector<Part> parts(mats.size());
    parallel_for(mats.size(), [&](size_t mi) {
      const Mat& mt = mats[mi];
      const auto& grp = plans[mt.n].groups[mt.g];
      Part& P = parts[mi];
      std::map<std::pair<int, int>, int> kidx;
      for (auto& kv : mt.blk) kidx.emplace(kv.first, (int)kidx.size());
      std::vector<std::pair<int, Seg>> tmp;
      for (auto& itm : grp.items)
        for (const BRef& b : blocks_ro(itm.src, itm.T)) {
          Seg sg;
          sg.a = 0; sg.abuf = B_ABS; sg.k = b.rows; sg.sc = itm.coef * b.sc;
          if (b.ident()) { sg.b = 0; sg.bbuf = B_ABS; }
          else { sg.b = b.ptr; sg.bbuf = B_ABS; sg.ldb = b.ld; sg.tb = b.tr ? 1 : 0; }
          tmp.push_back({kidx.at({b.r, b.c}), sg});
        }
      std::vector<int> start(kidx.size() + 1, 0);
      for (auto& e : tmp) start[e.first + 1]++;
      for (size_t i = 0; i < kidx.size(); ++i) start[i + 1] += start[i];
      P.segs.resize(tmp.size());
      {
        std::vector<int> pos(start.begin(), start.end() - 1);
        for (auto& e : tmp) P.segs[pos[e.first]++] = e.second;
      }
      int q = 0;
      for (auto& kv : mt.blk) {
        Prob pr;
        pr.c = store + 8ull * kv.second.first; pr.cbuf = B_ABS;
        pr.m = kv.second.second.first; pr.n = kv.second.second.second; pr.ldc = pr.n; pr.beta = 0;
        pr.seg0 = start[q];   // relative to this part; shifted when the parts are joined
        pr.nseg = start[q + 1] - start[q];
        ++q;
        P.probs.push_back(pr);
        BRef r;
        r.r = kv.first.first; r.c = kv.first.second; r.ptr = pr.c;
        r.rows = pr.m; r.cols = pr.n; r.ld = pr.n; r.tr = false; r.sc = 1.0;
        P.refs.push_back(r);
      }
    });
    for (size_t mi = 0; mi < mats.size(); ++mi) {
      const int base = (int)l.segs.size();
      for (Prob pr : parts[mi].probs) {
        pr.seg0 += base;
        l.probs.push_back(pr);
      }
      l.segs.insert(l.segs.end(), parts[mi].segs.begin(), parts[mi].segs.end());
      summed[{mats[mi].n, mats[mi].g}] = std::move(parts[mi].refs);
    }
    if (!l.empty()) ex.run(l, 0, 0);
    for (size_t n = 0; n < plans.size(); ++n) {
      OpView v;
      v.odd = pending[n].odd;
      for (size_t g = 0; g < plans[n].groups.size(); ++g) {
        auto& grp = plans[n].groups[g];
        if (grp.items.size() >= 2) {
          expand(summed[{n, g}], grp.o, 1.0, grp.par, v.blocks);
        } else if (grp.items.size() == 1) {
          auto& itm = grp.items[0];
          expand(blocks(itm.src, itm.T), grp.o, itm.coef, grp.par, v.blocks);
        }
      }
      if (!v.blocks.empty()) E.ops[pending[n].key] = v;
    }
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

void enlarge(const EnvBlock& B, const Integrals& I, Executor& ex, Enlarged& E, double* flops) {
  const int L = I.L;
  E.left = B.left;
  E.ops.clear();
  E.pb = make_prod(B.basis, B.left);
  Ctx x(B, I, E);
  const Mat4 I4 = Mat4::id();
  auto nonnull = [](const OpView* p) { return p != nullptr; };
  (void)nonnull;
  if (B.left) {
    const int c = B.cut;          // X = [0, c), site p = c
    E.cut = c + 1;
    const int sm[2] = {2 * c, 2 * c + 1};
    const int nx = 2 * c;
    x.view(Key(F_I), {C_(nullptr, false, I4, 1.0, false)}, false);
    for (int k = 0; k < nx; ++k)
      if (auto C = x.get(Key(F_C, k))) x.view(Key(F_C, k), {C_(C, false, I4, 1.0, false)}, true);
    for (int s = 0; s < 2; ++s) x.view(Key(F_C, sm[s]), {C_(nullptr, false, cre(s), 1.0, true)}, true);
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
    // S'_m, m outside the enlarged block
    for (int m = 2 * (c + 1); m < 2 * L; ++m) {
      std::vector<Contrib> cs;
      if (auto S = x.get(Key(F_S, m))) cs.push_back(C_(S, false, I4, 1.0, false));
      for (int j = 0; j < 2; ++j) cs.push_back(C_(nullptr, false, ann(j), 0.5 * I.t(m, sm[j]), true));
      for (int s = 0; s < 2; ++s) {
        const int l = sm[s];
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
      for (int i = 0; i < nx; ++i)
        for (int j = i + 1; j < nx; ++j)
          if (auto A = x.get(Key(F_A, i, j))) {
            Mat4 P;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) P = P + ann(a) * ann(b) * (0.5 * I.w(i, j, sm[a], sm[b]));
            cs.push_back(C_(A, false, P, 2.0, false));
            cs.push_back(C_(A, true, P.T(), 2.0, false));
          }
      for (int i = 0; i < nx; ++i)
        for (int l = 0; l < nx; ++l)
          if (auto Bil = x.get(Key(F_B, i, l))) {
            Mat4 Q;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) Q = Q + cre(a) * ann(b) * I.q(i, sm[a], sm[b], l);
            cs.push_back(C_(Bil, false, Q, 1.0, false));
          }
      x.materialize(Key(F_H), std::move(cs), false);
    }
  } else {
    const int c = B.cut - 1;      // site p = c, Y = [c+1, L)
    E.cut = c;
    const int mc = 2 * c;                     // complementary operators for modes < 2c
    const int sm[2] = {2 * c, 2 * c + 1};
    const int y0 = 2 * (c + 1);
    x.view(Key(F_I), {C_(nullptr, false, I4, 1.0, false)}, false);
    for (int s = 0; s < 2; ++s) x.view(Key(F_C, sm[s]), {C_(nullptr, false, cre(s), 1.0, false)}, true);
    for (int k = y0; k < 2 * L; ++k)
      if (auto C = x.get(Key(F_C, k))) x.view(Key(F_C, k), {C_(C, false, I4, 1.0, true)}, true);
    // P'_ij, i < j < 2c
    for (int i = 0; i < mc; ++i)
      for (int j = i + 1; j < mc; ++j) {
        std::vector<Contrib> cs;
        if (auto P = x.get(Key(F_P, i, j))) cs.push_back(C_(P, false, I4, 1.0, false));
        for (int s = 0; s < 2; ++s)
          for (int l = y0; l < 2 * L; ++l) {
            auto C = x.get(Key(F_C, l));
            if (!C) continue;
            double w = 0.5 * (I.w(i, j, sm[s], l) - I.w(i, j, l, sm[s]));
            if (w != 0.0) cs.push_back(C_(C, true, ann(s), w, true));
          }
        Mat4 P;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) P = P + ann(a) * ann(b) * (0.5 * I.w(i, j, sm[a], sm[b]));
        cs.push_back(C_(nullptr, false, P, 1.0, false));
        x.materialize(Key(F_P, i, j), std::move(cs), false);
      }
    // Q'_il, i, l < 2c
    for (int i = 0; i < mc; ++i)
      for (int l = 0; l < mc; ++l) {
        std::vector<Contrib> cs;
        if (auto Q = x.get(Key(F_Q, i, l))) cs.push_back(C_(Q, false, I4, 1.0, false));
        for (int s = 0; s < 2; ++s)
          for (int k = y0; k < 2 * L; ++k) {
            auto C = x.get(Key(F_C, k));
            if (!C) continue;
            double q1 = I.q(i, sm[s], k, l);    // (s,Y): a+_j(s) a_k(Y)
            if (q1 != 0.0) cs.push_back(C_(C, true, cre(s), q1, true));
            double q2 = -I.q(i, k, sm[s], l);   // (Y,s): a+_j(Y) a_k(s) = -a_k a+_j
            if (q2 != 0.0) cs.push_back(C_(C, false, ann(s), q2, true));
          }
        Mat4 Q;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) Q = Q + cre(a) * ann(b) * I.q(i, sm[a], sm[b], l);
        cs.push_back(C_(nullptr, false, Q, 1.0, false));
        x.materialize(Key(F_Q, i, l), std::move(cs), false);
      }
    // S'_m, m < 2c
    for (int m = 0; m < mc; ++m) {
      std::vector<Contrib> cs;
      if (auto S = x.get(Key(F_S, m))) cs.push_back(C_(S, false, I4, 1.0, true));
      Mat4 t1;
      for (int j = 0; j < 2; ++j) t1 = t1 + ann(j) * (0.5 * I.t(m, sm[j]));
      cs.push_back(C_(nullptr, false, t1, 1.0, false));
      for (int s = 0; s < 2; ++s) {
        if (auto P = x.get(Key(F_P, m, sm[s]))) cs.push_back(C_(P, false, cre(s), 2.0, false));
        if (auto Q = x.get(Key(F_Q, m, sm[s]))) cs.push_back(C_(Q, false, ann(s), 1.0, false));
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
      if (auto P = x.get(Key(F_P, sm[0], sm[1]))) {
        Mat4 A = cre(0) * cre(1);
        cs.push_back(C_(P, false, A, 2.0, false));
        cs.push_back(C_(P, true, A.T(), 2.0, false));
      }
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          if (auto Q = x.get(Key(F_Q, sm[a], sm[b]))) cs.push_back(C_(Q, false, cre(a) * ann(b), 1.0, false));
      x.materialize(Key(F_H), std::move(cs), false);
    }
  }
  x.finish(ex);
  (void)flops;
}

}  // namespace qd
