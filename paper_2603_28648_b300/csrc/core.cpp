// Layout, operator views, renormalization and H_eff task lists.
#include "core.hpp"
#include "su2.hpp"

#include <algorithm>
#include <atomic>
#include <exception>
#include <functional>
#include <mutex>
#include <thread>
#include <climits>
#include <cmath>
#include <stdexcept>
#include <tuple>
#include <unordered_map>

namespace qd {

const QN SITE_QN[NSITE] = {{0, 0}, {1, 1}, {1, -1}, {2, 0}};

void Basis::add(QN qq, int d) {
  if (!q.empty() && !(q.back() < qq)) throw std::runtime_error("Basis::add: labels must increase");
  idx[qq] = (int)q.size();
  q.push_back(qq);
  dim.push_back(d);
}

int64_t Basis::total() const {
  int64_t t = 0;
  for (int d : dim) t += d;
  return t;
}

QN ProdBasis::sub_qn(int s) const { return prod.q[subs[s].prod]; }
int ProdBasis::blk_parity(int s) const { return (blk->q[subs[s].blk].n & 1) ? -1 : 1; }
int ProdBasis::site_parity(int s) const { return (SITE_QN[subs[s].st].n & 1) ? -1 : 1; }

ProdBasis make_prod(const Basis& blk, bool left) {
  ProdBasis pb;
  pb.left = left;
  pb.blk = &blk;
  pb.prod.su2 = blk.su2;
  std::vector<std::tuple<QN, int, int, int>> items;  // label, first, second, (blk, st)
  for (int b = 0; b < blk.nsec(); ++b)
    for (int st = 0; st < NSITE; ++st) {
      QN q = blk.q[b] + SITE_QN[st];
      if (blk.su2 && q.s < 0) continue;   // a doublet couples a singlet to spin 1/2 only
      if (left) items.emplace_back(q, b, st, 0);
      else items.emplace_back(q, st, b, 0);
    }
  std::sort(items.begin(), items.end(), [](const auto& a, const auto& b) {
    if (std::get<0>(a) != std::get<0>(b)) return std::get<0>(a) < std::get<0>(b);
    if (std::get<1>(a) != std::get<1>(b)) return std::get<1>(a) < std::get<1>(b);
    return std::get<2>(a) < std::get<2>(b);
  });
  pb.subidx.assign(blk.nsec() * NSITE, -1);
  for (auto& it : items) {
    QN q = std::get<0>(it);
    int b = left ? std::get<1>(it) : std::get<2>(it);
    int st = left ? std::get<2>(it) : std::get<1>(it);
    int p = pb.prod.find(q);
    if (p < 0) {
      pb.prod.add(q, 0);
      p = pb.prod.nsec() - 1;
      pb.prod_subs.emplace_back();
    }
    Sub s;
    s.blk = b;
    s.st = st;
    s.prod = p;
    s.off = pb.prod.dim[p];
    s.dim = blk.dim[b];
    pb.prod.dim[p] += s.dim;
    pb.subidx[b * NSITE + st] = (int)pb.subs.size();
    pb.prod_subs[p].push_back((int)pb.subs.size());
    pb.subs.push_back(s);
  }
  return pb;
}

OpView transpose(const OpView& o) {
  OpView t;
  t.odd = o.odd;
  t.blocks.reserve(o.blocks.size());
  for (const BRef& b : o.blocks) {
    BRef x = b;
    std::swap(x.r, x.c);
    std::swap(x.rows, x.cols);
    x.tr = !b.tr;
    t.blocks.push_back(x);
  }
  return t;
}

double Integrals::t(int k, int l) const {
  if ((k & 1) != (l & 1)) return 0.0;
  return h[(k >> 1) * L + (l >> 1)];
}

double Integrals::w(int i, int j, int k, int l) const {
  // w_ijkl = (p_i p_l | p_j p_k) d(s_i, s_l) d(s_j, s_k)
  if ((i & 1) != (l & 1) || (j & 1) != (k & 1)) return 0.0;
  int64_t pi = i >> 1, pj = j >> 1, pk = k >> 1, pl = l >> 1;
  return V[((pi * L + pl) * L + pj) * L + pk];
}

Mat4 Mat4::id() {
  Mat4 m;
  for (int i = 0; i < 4; ++i) m(i, i) = 1.0;
  return m;
}
Mat4 Mat4::operator*(const Mat4& o) const {
  Mat4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += (*this)(i, k) * o(k, j);
      r(i, j) = s;
    }
  return r;
}
Mat4 Mat4::operator+(const Mat4& o) const {
  Mat4 r;
  for (int i = 0; i < 16; ++i) r.v[i] = v[i] + o.v[i];
  return r;
}
Mat4 Mat4::operator*(double s) const {
  Mat4 r;
  for (int i = 0; i < 16; ++i) r.v[i] = v[i] * s;
  return r;
}
Mat4 Mat4::T() const {
  Mat4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r(i, j) = (*this)(j, i);
  return r;
}
bool Mat4::zero() const {
  for (double x : v)
    if (x != 0.0) return false;
  return true;
}

Mat4 cre(int sigma) {
  Mat4 m;
  if (sigma == 0) {
    m(1, 0) = 1.0;   // a+_up |0> = |up>
    m(3, 2) = 1.0;   // a+_up |dn> = |updn>
  } else {
    m(2, 0) = 1.0;   // a+_dn |0> = |dn>
    m(3, 1) = -1.0;  // a+_dn |up> = -|updn>
  }
  return m;
}
Mat4 ann(int sigma) { return cre(sigma).T(); }

// ---------------------------------------------------------------------------
// Renormalization: O_new = U^T O U (left) or V O V^T (right), two stages.
// ---------------------------------------------------------------------------
namespace {
// f(0..n-1) on up to 16 host threads (items independent, each writing only its
// own results); the first exception of any item is rethrown
void parallel_for_ops(size_t n, const std::function<void(size_t)>& f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const unsigned nt = (unsigned)std::min<size_t>(std::min(hw, 16u), n / 16);
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
}  // namespace

void renormalize(const Enlarged& E, const Basis& nb, const std::vector<int>& nb_of_prod,
                 uint64_t tensor, const std::vector<int64_t>& toff, Executor& ex,
                 EnvBlock& out, int64_t tmp_budget, double* flops) {
  const ProdBasis& pb = E.pb;
  const bool left = E.left;
  out.left = left;
  out.normal = E.normal;
  out.basis = nb;
  out.ops.clear();
  // storage plan: every output block is allocated in one buffer
  struct OutBlk { int nq, nq2; int64_t off; };
  std::map<Key, std::map<std::pair<int, int>, int64_t>> layout;
  int64_t total = 0;
  for (auto& kv : E.ops) {
    if (kv.first.f == F_I) continue;  // the identity is never stored
    auto& lay = layout[kv.first];
    for (const BRef& b : kv.second.blocks) {
      int q = pb.subs[b.r].prod, q2 = pb.subs[b.c].prod;
      int nq = nb_of_prod[q], nq2 = nb_of_prod[q2];
      if (nq < 0 || nq2 < 0) continue;
      auto key = std::make_pair(nq, nq2);
      if (!lay.count(key)) {
        lay[key] = total;
        if (!E.batched) total += (int64_t)nb.dim[nq] * nb.dim[nq2];
      }
    }
    if (E.batched)  // sector order: operators with the same blocks get the same offsets
      for (auto& e : lay) {
        e.second = total;
        total += (int64_t)nb.dim[e.first.first] * nb.dim[e.first.second];
      }
  }
  uint64_t store = total ? ex.alloc(total) : 0;
  if (store) {
    out.owned.push_back(store);
    out.owned_n.push_back(total);
  }
  auto sub_ptr = [&](int s) -> uint64_t {
    const Sub& S = pb.subs[s];
    int nq = nb_of_prod[S.prod];
    if (left) return tensor + 8ull * (toff[S.prod] + (int64_t)S.off * nb.dim[nq]);
    return tensor + 8ull * (toff[S.prod] + S.off);
  };
  // Every stored operator (key order) is O' = U^T O U per output block: stage
  // 1 writes O U of each stored block reference to scratch, stage 2 sums U^T
  // times those (or U^T U_c for identity references) into the output block.
  // The operators are taken in chunks whose scratch fits the budget; each
  // operator's segments are built independently, then joined in order.
  struct OpPlan {
    const Key* key;
    const OpView* op;
    int64_t tbase;            // scratch offset of the operator in its chunk
    int chunk;
    std::vector<Seg> s1segs, s2segs;
    std::vector<Prob> s1probs, s2probs;   // seg0 relative to the operator's segments
    double fl1 = 0, fl2 = 0;
    OpView nv;
  };
  std::vector<OpPlan> ops;
  std::vector<int64_t> chunk_tmp;
  {
    int64_t tused = 0;
    int chunk = 0;
    for (auto& kv : E.ops) {
      if (kv.first.f == F_I) continue;
      int64_t need = 0;
      for (const BRef& b : kv.second.blocks) {
        int nq2 = nb_of_prod[pb.subs[b.c].prod];
        if (nq2 < 0 || nb_of_prod[pb.subs[b.r].prod] < 0 || b.ident()) continue;
        need += (int64_t)b.rows * nb.dim[nq2];
      }
      if (tused && tused + need > tmp_budget) {
        chunk_tmp.push_back(tused);
        ++chunk;
        tused = 0;
      }
      ops.emplace_back();
      OpPlan& o = ops.back();
      o.key = &kv.first;
      o.op = &kv.second;
      o.tbase = tused;
      o.chunk = chunk;
      tused += need;
    }
    chunk_tmp.push_back(tused);
  }
  parallel_for_ops(ops.size(), [&](size_t oi) {
    OpPlan& o = ops[oi];
    const OpView& op = *o.op;
    const auto& lay = layout.at(*o.key);
    o.nv.odd = op.odd;
    o.nv.k2 = op.k2;
    int64_t tused = o.tbase;
    // (output block, segment) pairs, grouped by output block below in the
    // order they were produced
    std::vector<std::pair<std::pair<int, int>, Seg>> segs;
    segs.reserve(op.blocks.size());
    for (const BRef& b : op.blocks) {
      const Sub& Sr = pb.subs[b.r];
      const Sub& Sc = pb.subs[b.c];
      int nq = nb_of_prod[Sr.prod], nq2 = nb_of_prod[Sc.prod];
      if (nq < 0 || nq2 < 0) continue;
      int dq = nb.dim[nq], dq2 = nb.dim[nq2];
      int pq = pb.prod.dim[Sr.prod], pq2 = pb.prod.dim[Sc.prod];
      Seg g;
      g.sc = b.sc;
      g.k = Sr.dim;
      if (left) {  // U_r^T (op U_c)
        g.a = sub_ptr(b.r); g.abuf = B_ABS; g.lda = dq; g.ta = 1;
      } else {     // V_r (op V_c^T)
        g.a = sub_ptr(b.r); g.abuf = B_ABS; g.lda = pq; g.ta = 0;
      }
      if (b.ident()) {
        if (left) { g.b = sub_ptr(b.c); g.bbuf = B_ABS; g.ldb = dq2; g.tb = 0; }
        else { g.b = sub_ptr(b.c); g.bbuf = B_ABS; g.ldb = pq2; g.tb = 1; }
      } else {
        Prob p;
        p.c = (uint64_t)tused; p.cbuf = B_TMP;
        p.m = b.rows; p.n = dq2; p.ldc = dq2; p.beta = 0;
        p.seg0 = (int)o.s1segs.size(); p.nseg = 1;
        Seg h;
        h.a = b.ptr; h.abuf = B_ABS; h.lda = b.ld; h.ta = b.tr ? 1 : 0;
        h.b = sub_ptr(b.c); h.bbuf = B_ABS; h.k = b.cols;
        if (left) { h.ldb = dq2; h.tb = 0; } else { h.ldb = pq2; h.tb = 1; }
        o.s1segs.push_back(h);
        o.s1probs.push_back(p);
        o.fl1 += 2.0 * p.m * p.n * h.k;
        g.b = (uint64_t)tused; g.bbuf = B_TMP; g.ldb = dq2; g.tb = 0;
        tused += (int64_t)b.rows * dq2;
      }
      segs.push_back({{nq, nq2}, g});
      o.fl2 += 2.0 * dq * dq2 * g.k;
    }
    std::stable_sort(segs.begin(), segs.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    o.s2segs.reserve(segs.size());
    for (size_t si = 0; si < segs.size();) {
      const std::pair<int, int> key = segs[si].first;
      int nq = key.first, nq2 = key.second;
      Prob p;
      p.c = store + 8ull * lay.at(key); p.cbuf = B_ABS;
      p.m = nb.dim[nq]; p.n = nb.dim[nq2]; p.ldc = p.n; p.beta = 0;
      p.seg0 = (int)o.s2segs.size();
      while (si < segs.size() && segs[si].first == key) o.s2segs.push_back(segs[si++].second);
      p.nseg = (int)o.s2segs.size() - p.seg0;
      o.s2probs.push_back(p);
      BRef r;
      r.r = nq; r.c = nq2; r.ptr = p.c; r.rows = p.m; r.cols = p.n; r.ld = p.n; r.tr = false; r.sc = 1.0;
      o.nv.blocks.push_back(r);
    }
  });
  // join each chunk in operator order (offsets by prefix sums, copies in
  // parallel) and run it
  double fl = 0;
  Launch s1, s2;
  struct Off { size_t s1s, s1p, s2s, s2p; };
  std::vector<Off> off(ops.size());
  for (size_t oi = 0; oi < ops.size();) {
    const int chunk = ops[oi].chunk;
    const size_t o0 = oi;
    Off t{0, 0, 0, 0};
    for (; oi < ops.size() && ops[oi].chunk == chunk; ++oi) {
      const OpPlan& o = ops[oi];
      off[oi] = t;
      t.s1s += o.s1segs.size(); t.s1p += o.s1probs.size();
      t.s2s += o.s2segs.size(); t.s2p += o.s2probs.size();
    }
    if (t.s1s > (size_t)INT32_MAX || t.s2s > (size_t)INT32_MAX)
      throw std::runtime_error("renormalize: task list too long");
    s1.clear();
    s2.clear();
    s1.segs.resize(t.s1s); s1.probs.resize(t.s1p);
    s2.segs.resize(t.s2s); s2.probs.resize(t.s2p);
    parallel_for_ops(oi - o0, [&](size_t j) {
      OpPlan& o = ops[o0 + j];
      const Off& f = off[o0 + j];
      std::copy(o.s1segs.begin(), o.s1segs.end(), s1.segs.begin() + f.s1s);
      std::copy(o.s2segs.begin(), o.s2segs.end(), s2.segs.begin() + f.s2s);
      for (size_t k = 0; k < o.s1probs.size(); ++k) {
        Prob p = o.s1probs[k];
        p.seg0 += (int)f.s1s;
        s1.probs[f.s1p + k] = p;
      }
      for (size_t k = 0; k < o.s2probs.size(); ++k) {
        Prob p = o.s2probs[k];
        p.seg0 += (int)f.s2s;
        s2.probs[f.s2p + k] = p;
      }
      std::vector<Seg>().swap(o.s1segs);
      std::vector<Seg>().swap(o.s2segs);
    });
    for (size_t j = o0; j < oi; ++j) {
      s1.flops += ops[j].fl1;
      s2.flops += ops[j].fl2;
      out.ops[*ops[j].key] = std::move(ops[j].nv);
    }
    if (s1.empty() && s2.empty()) continue;
    if (chunk_tmp[chunk]) ex.tmp(chunk_tmp[chunk]);
    if (!s1.empty()) ex.run(s1, 0, 0);
    if (!s2.empty()) ex.run(s2, 0, 0);
    fl += s1.flops + s2.flops;
  }
  if (flops) *flops += fl;
}

// ---------------------------------------------------------------------------
// Two-site wavefunction layout and H_eff psi plan.
// ---------------------------------------------------------------------------
PsiLayout make_psi_layout(const ProdBasis& Lp, const ProdBasis& Rp, QN target) {
  PsiLayout lay;
  const Basis& X = *Lp.blk;
  const Basis& Y = *Rp.blk;
  lay.su2 = X.su2;
  lay.target = target;
  lay.nl = Lp.nsub();
  lay.nr = Rp.nsub();
  lay.by_sub.assign((size_t)lay.nl * lay.nr, -1);
  for (int x = 0; x < X.nsec(); ++x)
    for (int i = 0; i < NSITE; ++i)
      for (int j = 0; j < NSITE; ++j)
        for (int y = 0; y < Y.nsec(); ++y) {
          if (lay.su2) {
            // SU(2): the multiplets (x i) J_a and (j y) J_b couple to the target spin
            const int ls = Lp.find(x, i), rs = Rp.find(y, j);
            if (ls < 0 || rs < 0) continue;
            const QN a = Lp.sub_qn(ls), b = Rp.sub_qn(rs);
            if (a.n + b.n != target.n || std::abs(a.s - b.s) > target.s || a.s + b.s < target.s) continue;
          } else {
            QN t = X.q[x] + SITE_QN[i] + SITE_QN[j] + Y.q[y];
            if (t != target) continue;
          }
          PsiLayout::Blk b;
          b.x = x; b.i = i; b.j = j; b.y = y;
          b.lsub = Lp.find(x, i);
          b.rsub = Rp.find(y, j);
          b.rows = X.dim[x];
          b.cols = Y.dim[y];
          b.off = lay.size;
          lay.size += (int64_t)b.rows * b.cols;
          lay.by_sub[(size_t)b.lsub * lay.nr + b.rsub] = (int)lay.blks.size();
          lay.blks.push_back(b);
        }
  return lay;
}

std::vector<CenterTerm> center_terms(const Enlarged& Lp, const Enlarged& Rp, const Integrals& I) {
  const int c = Lp.cut;  // L' = [0, c), R' = [c, L)
  const int L = I.L;
  std::vector<CenterTerm> terms;
  auto get = [](const Enlarged& E, Key k) -> const OpView* {
    auto it = E.ops.find(k);
    if (it == E.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  };
  const OpView* IL = get(Lp, Key(F_I));
  const OpView* IR = get(Rp, Key(F_I));
  // H = H_L' + H_R' + e_core
  if (auto h = get(Lp, Key(F_H))) terms.push_back({h, false, IR, false, 1.0});
  if (auto h = get(Rp, Key(F_H))) terms.push_back({IL, false, h, false, 1.0});
  if (I.ecore != 0.0) terms.push_back({IL, false, IR, false, I.ecore});
  // sum_{i in L'} ( a+_i S^R_i - a_i (S^R_i)^+ )
  for (int i = 0; i < 2 * c; ++i) {
    auto C = get(Lp, Key(F_C, i));
    auto S = get(Rp, Key(F_S, i));
    if (!C || !S) continue;
    terms.push_back({C, false, S, false, 1.0});
    terms.push_back({C, true, S, true, -1.0});
  }
  // sum_{m in R'} ( -S^L_m a+_m + (S^L_m)^+ a_m )
  for (int m = 2 * c; m < 2 * L; ++m) {
    auto S = get(Lp, Key(F_S, m));
    auto C = get(Rp, Key(F_C, m));
    if (!C || !S) continue;
    terms.push_back({S, false, C, false, -1.0});
    terms.push_back({S, true, C, true, 1.0});
  }
  if (Lp.normal == Rp.normal)
    throw std::logic_error("center_terms: exactly one enlarged block must hold normal pairs");
  if (Lp.normal) {
    // 2 sum_{i<j in L'} (A_ij P_ij + A_ij^+ P_ij^+) + sum_{il in L'} B_il Q_il
    for (int i = 0; i < 2 * c; ++i)
      for (int j = i + 1; j < 2 * c; ++j) {
        auto A = get(Lp, Key(F_A, i, j));
        auto P = get(Rp, Key(F_P, i, j));
        if (!A || !P) continue;
        terms.push_back({A, false, P, false, 2.0});
        terms.push_back({A, true, P, true, 2.0});
      }
    for (int i = 0; i < 2 * c; ++i)
      for (int l = 0; l < 2 * c; ++l) {
        auto B = get(Lp, Key(F_B, i, l));
        auto Q = get(Rp, Key(F_Q, i, l));
        if (!B || !Q) continue;
        terms.push_back({B, false, Q, false, 1.0});
      }
  } else {
    // normal pairs on the right (both pair products are even, so the order of
    // the factors is free): 2 sum_{i<j in R'} (P_ij A_ij + P_ij^+ A_ij^+)
    // + sum_{jk in R'} Q_jk B_jk, with P, Q of L' indexed by modes of R'
    for (int i = 2 * c; i < 2 * L; ++i)
      for (int j = i + 1; j < 2 * L; ++j) {
        auto P = get(Lp, Key(F_P, i, j));
        auto A = get(Rp, Key(F_A, i, j));
        if (!A || !P) continue;
        terms.push_back({P, false, A, false, 2.0});
        terms.push_back({P, true, A, true, 2.0});
      }
    for (int j = 2 * c; j < 2 * L; ++j)
      for (int k = 2 * c; k < 2 * L; ++k) {
        auto Q = get(Lp, Key(F_Q, j, k));
        auto B = get(Rp, Key(F_B, j, k));
        if (!B || !Q) continue;
        terms.push_back({Q, false, B, false, 1.0});
      }
  }
  return terms;
}

HeffPlan plan_heff(const Enlarged& Lp, const Enlarged& Rp, const PsiLayout& lay,
                   const Integrals& I, int64_t tmp_budget) {
  return plan_terms(Lp, Rp, lay, lay.su2 ? center_terms_su2(Lp, Rp, I) : center_terms(Lp, Rp, I), tmp_budget);
}

namespace {
// SU(2): reduced-element factor of the scalar coupling [O_L^k x O_R^k]^0 between
// the two-site multiplets (a b) S and (a' b') S (1 in U(1))
double pair_factor(const PsiLayout& lay, const ProdBasis& LB, const ProdBasis& RB, int k2, int la, int lap, int rb,
                   int rbp) {
  if (!lay.su2) return 1.0;
  return su2::coupled(LB.sub_qn(la).s, RB.sub_qn(rb).s, lay.target.s, LB.sub_qn(lap).s, RB.sub_qn(rbp).s,
                      lay.target.s, k2, k2, 0);
}
}  // namespace

OpView site_op_view(const Enlarged& E, const Mat4& o, bool par) {
  OpView v;
  const Basis& B = *E.pb.blk;
  for (int x = 0; x < B.nsec(); ++x)
    for (int i = 0; i < NSITE; ++i)
      for (int j = 0; j < NSITE; ++j) {
        double val = o(i, j);
        if (val == 0.0) continue;
        BRef r;
        r.r = E.pb.find(x, i);
        r.c = E.pb.find(x, j);
        r.ptr = 0;
        r.rows = r.cols = r.ld = B.dim[x];
        double sg = 1.0;
        if (par) sg = E.left ? ((B.q[x].n & 1) ? -1.0 : 1.0) : ((SITE_QN[j].n & 1) ? -1.0 : 1.0);
        r.sc = val * sg;
        v.blocks.push_back(r);
      }
  return v;
}

HeffPlan plan_terms(const Enlarged& Lp, const Enlarged& Rp, const PsiLayout& lay,
                    const std::vector<CenterTerm>& terms, int64_t tmp_budget) {
  HeffPlan plan;
  plan.nterms = (int)terms.size();

  const ProdBasis& LB = Lp.pb;
  Launch s1, s2;
  // (psi block, segment) pairs of the current chunk, emitted grouped by
  // block in index order (a counting sort keeps the order within a block)
  std::vector<std::pair<int, Seg>> out;
  std::vector<int> cnt(lay.blks.size() + 1);
  std::vector<Seg> sorted;
  std::unordered_map<uint64_t, int64_t> blocks_read;  // storage address -> elements
  auto note = [&](const BRef& b) {
    if (b.ident()) return;
    int64_t& e = blocks_read[b.ptr];
    e = std::max<int64_t>(e, (int64_t)b.rows * b.cols);
  };
  int64_t tused = 0;
  auto flush = [&]() {
    if (out.empty() && s1.empty()) return;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (auto& e : out) cnt[e.first + 1]++;
    for (size_t bi = 0; bi < lay.blks.size(); ++bi) cnt[bi + 1] += cnt[bi];
    sorted.resize(out.size());
    {
      std::vector<int> pos(cnt.begin(), cnt.end() - 1);
      for (auto& e : out) sorted[pos[e.first]++] = e.second;
    }
    s2.segs.reserve(s2.segs.size() + sorted.size());
    for (size_t bi = 0; bi < lay.blks.size(); ++bi) {
      const int n = cnt[bi + 1] - cnt[bi];
      if (n == 0) continue;
      const auto& pbk = lay.blks[bi];
      Prob p;
      p.c = (uint64_t)pbk.off; p.cbuf = B_SIG;
      p.m = pbk.rows; p.n = pbk.cols; p.ldc = pbk.cols; p.beta = 1;
      p.seg0 = (int)s2.segs.size(); p.nseg = n;
      s2.segs.insert(s2.segs.end(), sorted.begin() + cnt[bi], sorted.begin() + cnt[bi + 1]);
      s2.probs.push_back(p);
    }
    plan.flops += s1.flops + s2.flops;
    plan.stage1.push_back(std::move(s1));
    plan.stage2.push_back(std::move(s2));
    plan.tmp_elems = std::max(plan.tmp_elems, tused);
    s1 = Launch();
    s2 = Launch();
    out.clear();
    tused = 0;
  };
  const ProdBasis& RB = Rp.pb;
  for (const CenterTerm& t : terms) {
    OpView Lv = t.LT ? (lay.su2 ? adjoint_su2(*t.L, &LB, nullptr) : transpose(*t.L)) : *t.L;
    OpView Rv = t.RT ? (lay.su2 ? adjoint_su2(*t.R, &RB, nullptr) : transpose(*t.R)) : *t.R;
    std::map<int, std::vector<const BRef*>> lby;  // col sub -> blocks
    for (const BRef& b : Lv.blocks) lby[b.c].push_back(&b);
    int64_t need = 0;
    for (const BRef& bR : Rv.blocks) {
      if (bR.ident()) continue;
      for (auto& kv : lby) {
        const int it = lay.find(kv.first, bR.c);
        if (it >= 0) need += (int64_t)lay.blks[it].rows * bR.rows;
      }
    }
    if (tused && tused + need > tmp_budget) flush();
    for (const BRef& bR : Rv.blocks) {
      for (auto& kv : lby) {
        int cL = kv.first;
        const int it = lay.find(cL, bR.c);
        if (it < 0) continue;
        note(bR);
        const auto& pin = lay.blks[it];
        int par = 1;
        if (Rv.odd) par = (LB.prod.q[LB.subs[cL].prod].n & 1) ? -1 : 1;
        const double bsc = t.coef * bR.sc * par;
        uint64_t Tb;
        int Tbuf, ldT = bR.rows;
        if (bR.ident()) {
          Tb = (uint64_t)pin.off; Tbuf = B_PSI; ldT = pin.cols;
        } else {
          Prob p;
          p.c = (uint64_t)tused; p.cbuf = B_TMP;
          p.m = pin.rows; p.n = bR.rows; p.ldc = bR.rows; p.beta = 0;
          p.seg0 = (int)s1.segs.size(); p.nseg = 1;
          p.osc = bsc;
          Seg h;
          h.a = (uint64_t)pin.off; h.abuf = B_PSI; h.lda = pin.cols; h.ta = 0;
          h.b = bR.ptr; h.bbuf = B_ABS; h.ldb = bR.ld; h.tb = bR.tr ? 0 : 1;
          h.k = bR.cols;
          s1.segs.push_back(h);
          s1.probs.push_back(p);
          s1.flops += 2.0 * p.m * p.n * h.k;
          Tb = (uint64_t)tused; Tbuf = B_TMP;
          tused += (int64_t)p.m * p.n;
        }

        for (const BRef* bL : kv.second) {
          const int ot = lay.find(bL->r, bR.r);
          if (ot < 0) continue;
          note(*bL);
          Seg g;
          if (bL->ident()) { g.a = 0; g.abuf = B_ABS; g.lda = 0; g.ta = 0; }
          else { g.a = bL->ptr; g.abuf = B_ABS; g.lda = bL->ld; g.ta = bL->tr ? 1 : 0; }
          g.b = Tb; g.bbuf = Tbuf; g.ldb = ldT; g.tb = 0;
          g.k = bL->cols;
          // the SU(2) coupling factor goes with the left reference (for S = 0 it
          // depends on the left reference alone, so the left views are not duplicated)
          g.asc = bL->sc * pair_factor(lay, LB, RB, t.k2, bL->r, bL->c, bR.r, bR.c);
          g.sc = bsc * g.asc;
          g.bsc = bsc;
          if (g.asc == 0.0) continue;
          out.push_back({ot, g});
          if (!bL->ident()) s2.flops += 2.0 * bL->rows * bR.rows * (double)bL->cols;
        }
      }
    }
  }
  flush();
  double e = 2.0 * (double)lay.size;
  for (auto& kv : blocks_read) e += (double)kv.second;
  plan.bytes = 8.0 * e;
  return plan;
}

Launch plan_diag(const Enlarged& Lp, const Enlarged& Rp, const PsiLayout& lay, const Integrals& I,
                 uint64_t ones) {
  // diag H_eff[(x,i,j,y)][a][b] = sum_t c_t dL[a] dR[b] over terms whose left and
  // right blocks are diagonal blocks: rank-1 segments (K = 1) with strided
  // diagonals (leading dimension ld + 1) or a vector of ones for identities
  std::vector<CenterTerm> terms = lay.su2 ? center_terms_su2(Lp, Rp, I) : center_terms(Lp, Rp, I);
  std::vector<std::pair<int, Seg>> out;  // (psi block, segment), grouped by block below
  const ProdBasis& LB = Lp.pb;
  const ProdBasis& RB = Rp.pb;
  for (const CenterTerm& t : terms) {
    OpView Lv = t.LT ? (lay.su2 ? adjoint_su2(*t.L, &LB, nullptr) : transpose(*t.L)) : *t.L;
    OpView Rv = t.RT ? (lay.su2 ? adjoint_su2(*t.R, &RB, nullptr) : transpose(*t.R)) : *t.R;
    std::map<int, std::vector<const BRef*>> ldiag, rdiag;
    for (const BRef& b : Lv.blocks) if (b.r == b.c) ldiag[b.r].push_back(&b);
    for (const BRef& b : Rv.blocks) if (b.r == b.c) rdiag[b.r].push_back(&b);
    for (auto& lk : ldiag)
      for (auto& rk : rdiag) {
        const int it = lay.find(lk.first, rk.first);
        if (it < 0) continue;
        int par = 1;
        if (Rv.odd) par = (LB.prod.q[LB.subs[lk.first].prod].n & 1) ? -1 : 1;
        for (const BRef* bl : lk.second)
          for (const BRef* br : rk.second) {
            Seg g;
            g.k = 1;
            if (bl->ident()) { g.a = ones; g.lda = 1; } else { g.a = bl->ptr; g.lda = bl->ld + 1; }
            g.abuf = B_ABS; g.ta = 0;
            if (br->ident()) { g.b = ones; g.ldb = 1; } else { g.b = br->ptr; g.ldb = br->ld + 1; }
            g.bbuf = B_ABS; g.tb = 1;
            g.sc = t.coef * bl->sc * br->sc * par * pair_factor(lay, LB, RB, t.k2, lk.first, lk.first, rk.first, rk.first);
            if (g.sc == 0.0) continue;
            out.push_back({it, g});
          }
      }
  }
  Launch l;
  std::stable_sort(out.begin(), out.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  l.segs.reserve(out.size());
  for (size_t i = 0; i < out.size();) {
    const int bi = out[i].first;
    const auto& b = lay.blks[bi];
    Prob p;
    p.c = (uint64_t)b.off; p.cbuf = B_SIG;
    p.m = b.rows; p.n = b.cols; p.ldc = b.cols; p.beta = 1;
    p.seg0 = (int)l.segs.size();
    while (i < out.size() && out[i].first == bi) l.segs.push_back(out[i++].second);
    p.nseg = (int)l.segs.size() - p.seg0;
    l.probs.push_back(p);
  }
  (void)I;
  return l;
}

}  // namespace qd
