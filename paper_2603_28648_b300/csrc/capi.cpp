// C ABI: context, integral and MPS import, environment build, H_eff psi.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qcdmrg.h"
#include "core.hpp"
#include "kernels.hpp"

using namespace qd;

struct qcdmrg_ctx {
  Backend be;
  int device = 0;
  int64_t tmp_budget = 0;
  Integrals I;
  bool have_int = false;
  int N = 0, two_s = 0;
  bool have_target = false;
  // MPS
  int L = 0, center = -1;
  std::vector<Basis> bonds;                      // 0..L (center+1 unused)
  std::vector<uint64_t> site;                    // device storage per site
  std::vector<std::vector<int64_t>> site_off;    // per product sector (-1: absent)
  std::vector<std::vector<int>> site_nb;         // product sector -> new bond sector
  std::vector<double> psi0;
  // environment
  bool have_env = false;
  std::vector<EnvBlock> lenv, renv;
  Enlarged Lp, Rp;
  PsiLayout lay;
  HeffPlan plan;
  std::vector<std::pair<int, int>> prepared;      // (stage1, stage2) handles
  uint64_t dpsi = 0, dsig = 0;
  qcdmrg_stats_t st{};
  std::string err;

  ~qcdmrg_ctx() { free_env(); free_mps(); if (dpsi) be.ex->release(dpsi); if (dsig) be.ex->release(dsig); delete be.ex; }
  void free_env() {
    if (!be.ex) return;
    for (auto& e : lenv) for (auto p : e.owned) be.ex->release(p);
    for (auto& e : renv) for (auto p : e.owned) be.ex->release(p);
    for (auto p : Lp.owned) be.ex->release(p);
    for (auto p : Rp.owned) be.ex->release(p);
    lenv.clear(); renv.clear();
    Lp = Enlarged(); Rp = Enlarged();
    if (be.pr) be.pr->drop_prepared();
    prepared.clear();
    have_env = false;
  }
  void free_mps() {
    if (!be.ex) return;
    for (auto p : site) if (p) be.ex->release(p);
    site.clear();
    center = -1;
  }
};

namespace {

struct Fail {
  int code;
  std::string msg;
};

template <class F>
int guard(qcdmrg_ctx* c, F&& f) {
  if (!c) return QCDMRG_EINVAL;
  try {
    c->err.clear();
    return f();
  } catch (const Fail& e) {
    c->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return QCDMRG_ENOMEM;
  } catch (const std::runtime_error& e) {
    c->err = e.what();
    std::string m = e.what();
    if (m.find("out of memory") != std::string::npos) return QCDMRG_ENOMEM;
    return QCDMRG_ECUDA;
  }
}

EnvBlock vacuum(bool left, int cut) {
  EnvBlock b;
  b.left = left;
  b.cut = cut;
  b.basis.add(QN{0, 0}, 1);
  return b;
}

}  // namespace

extern "C" {

int qcdmrg_create(qcdmrg_ctx** out, const qcdmrg_config* cfg) {
  if (!out || !cfg) return QCDMRG_EINVAL;
  *out = nullptr;
  if (cfg->symmetry != QCDMRG_U1) return QCDMRG_EINVAL;
  auto* c = new qcdmrg_ctx();
  try {
    c->device = cfg->device;
    c->be = make_backend(cfg->device);
    double gb = cfg->tmp_budget_gb > 0 ? cfg->tmp_budget_gb : 2.0;
    c->tmp_budget = (int64_t)(gb * 1e9 / 8);
  } catch (const std::exception& e) {
    delete c;
    return QCDMRG_ECUDA;
  }
  *out = c;
  return QCDMRG_OK;
}

int qcdmrg_destroy(qcdmrg_ctx* ctx) {
  if (!ctx) return QCDMRG_EINVAL;
  delete ctx;
  return QCDMRG_OK;
}

const char* qcdmrg_last_error(const qcdmrg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int qcdmrg_load_integrals(qcdmrg_ctx* ctx, int L, const double* h, const double* V, double e_core) {
  return guard(ctx, [&]() {
    if (L < 2 || !h || !V) throw Fail{QCDMRG_EINVAL, "L must be >= 2 and h, V non-null"};
    if (!std::isfinite(e_core)) throw Fail{QCDMRG_EINVAL, "e_core is not finite"};
    size_t n2 = (size_t)L * L, n4 = n2 * n2;
    for (size_t i = 0; i < n2; ++i)
      if (!std::isfinite(h[i])) throw Fail{QCDMRG_EINVAL, "h has non-finite entries"};
    for (int p = 0; p < L; ++p)
      for (int q = 0; q < L; ++q)
        if (std::fabs(h[p * L + q] - h[q * L + p]) > 1e-12 * (1 + std::fabs(h[p * L + q])))
          throw Fail{QCDMRG_EINVAL, "h is not symmetric"};
    for (size_t i = 0; i < n4; ++i)
      if (!std::isfinite(V[i])) throw Fail{QCDMRG_EINVAL, "V has non-finite entries"};
    ctx->free_env();
    ctx->free_mps();
    ctx->I.L = L;
    ctx->I.h.assign(h, h + n2);
    ctx->I.V.assign(V, V + n4);
    ctx->I.ecore = e_core;
    ctx->have_int = true;
    return QCDMRG_OK;
  });
}

int qcdmrg_set_target(qcdmrg_ctx* ctx, int N, int two_s) {
  return guard(ctx, [&]() {
    if (N < 0 || ((N + two_s) & 1)) throw Fail{QCDMRG_EINVAL, "N and 2Sz must have equal parity"};
    if (ctx->have_int && (N > 2 * ctx->I.L || std::abs(two_s) > N))
      throw Fail{QCDMRG_EINVAL, "target outside the Fock space"};
    ctx->free_env();
    ctx->N = N;
    ctx->two_s = two_s;
    ctx->have_target = true;
    return QCDMRG_OK;
  });
}

int qcdmrg_import_mps(qcdmrg_ctx* ctx, const qcdmrg_mps_desc* d, const double* data, size_t n) {
  return guard(ctx, [&]() {
    if (!ctx->have_int || !ctx->have_target) throw Fail{QCDMRG_ESTATE, "load integrals and target first"};
    if (!d || !data || !d->bond_nsec || !d->bond_sec) throw Fail{QCDMRG_EINVAL, "null argument"};
    const int L = d->L;
    if (L != ctx->I.L) throw Fail{QCDMRG_EINVAL, "MPS length differs from the integrals"};
    if (d->center < 0 || d->center + 1 >= L) throw Fail{QCDMRG_EINVAL, "centre out of range"};
    ctx->free_env();
    ctx->free_mps();
    std::vector<Basis> bonds(L + 1);
    int pos = 0;
    for (int b = 0; b <= L; ++b) {
      int ns = d->bond_nsec[b];
      if (ns < 0) throw Fail{QCDMRG_EINVAL, "negative sector count"};
      for (int s = 0; s < ns; ++s) {
        QN q{d->bond_sec[3 * pos], d->bond_sec[3 * pos + 1]};
        int dim = d->bond_sec[3 * pos + 2];
        ++pos;
        if (dim <= 0) throw Fail{QCDMRG_EINVAL, "sector dimension must be positive"};
        if (bonds[b].nsec() && !(bonds[b].q.back() < q))
          throw Fail{QCDMRG_EINVAL, "sector labels must increase within a bond"};
        bonds[b].add(q, dim);
      }
    }
    const int c = d->center;
    if (bonds[0].nsec() != 1 || bonds[0].q[0] != QN{0, 0} || bonds[0].dim[0] != 1)
      throw Fail{QCDMRG_EINVAL, "bond 0 must be the vacuum"};
    if (bonds[L].nsec() != 1 || bonds[L].q[0] != QN{0, 0} || bonds[L].dim[0] != 1)
      throw Fail{QCDMRG_EINVAL, "bond L (right block of no sites) must be the vacuum"};
    size_t off = 0;
    ctx->site.assign(L, 0);
    ctx->site_off.assign(L, {});
    ctx->site_nb.assign(L, {});
    auto take_site = [&](int p, const Basis& from, bool left, const Basis& to) {
      ProdBasis pb = make_prod(from, left);
      std::vector<int64_t> so(pb.prod.nsec(), -1);
      std::vector<int> nb(pb.prod.nsec(), -1);
      int64_t tot = 0;
      for (int q = 0; q < pb.prod.nsec(); ++q) {
        int t = to.find(pb.prod.q[q]);
        if (t < 0) continue;
        if (to.dim[t] > pb.prod.dim[q]) throw Fail{QCDMRG_EINVAL, "bond sector larger than its product space"};
        so[q] = tot;
        nb[q] = t;
        tot += (int64_t)pb.prod.dim[q] * to.dim[t];
      }
      for (int t = 0; t < to.nsec(); ++t)
        if (pb.prod.find(to.q[t]) < 0) throw Fail{QCDMRG_EINVAL, "bond sector not reachable from its neighbour"};
      if (off + tot > n) throw Fail{QCDMRG_EINVAL, "MPS data shorter than its layout"};
      uint64_t dev = ctx->be.ex->alloc(tot);
      ctx->be.ex->upload(dev, data + off, tot);
      off += tot;
      ctx->site[p] = dev;
      ctx->site_off[p] = so;
      ctx->site_nb[p] = nb;
    };
    for (int p = 0; p < c; ++p) take_site(p, bonds[p], true, bonds[p + 1]);
    for (int p = c + 2; p < L; ++p) take_site(p, bonds[p + 1], false, bonds[p]);
    // psi
    ProdBasis Lp = make_prod(bonds[c], true), Rp = make_prod(bonds[c + 2], false);
    PsiLayout lay = make_psi_layout(Lp, Rp, QN{ctx->N, ctx->two_s});
    if (off + lay.size != n) throw Fail{QCDMRG_EINVAL, "MPS data length does not match its layout"};
    ctx->psi0.assign(data + off, data + off + lay.size);
    ctx->bonds = bonds;
    ctx->L = L;
    ctx->center = c;
    return QCDMRG_OK;
  });
}

int qcdmrg_init_mps(qcdmrg_ctx* ctx, int D, uint64_t seed, int center) {
  return guard(ctx, [&]() {
    if (!ctx->have_int || !ctx->have_target) throw Fail{QCDMRG_ESTATE, "load integrals and target first"};
    const int L = ctx->I.L;
    if (D < 1) throw Fail{QCDMRG_EINVAL, "D must be positive"};
    if (center < 0 || center + 1 >= L) throw Fail{QCDMRG_EINVAL, "centre out of range"};
    ctx->free_env();
    ctx->free_mps();
    auto st = mps_structure(L, ctx->N, ctx->two_s, D);
    for (int b = 1; b < L; ++b)
      if (st[b].empty()) throw Fail{QCDMRG_EINVAL, "target not reachable: empty bond"};
    std::vector<Basis> bonds(L + 1);
    for (int b = 0; b <= center; ++b)
      for (auto& kv : st[b]) bonds[b].add(kv.first, kv.second);
    for (int b = center + 2; b <= L; ++b)
      for (auto& kv : st[L - b]) bonds[b].add(kv.first, kv.second);
    Executor& ex = *ctx->be.ex;
    ctx->site.assign(L, 0);
    ctx->site_off.assign(L, {});
    ctx->site_nb.assign(L, {});
    auto mix = [](uint64_t a, uint64_t b) {
      uint64_t x = a ^ (b + 0x9E3779B97F4A7C15ull + (a << 6) + (a >> 2));
      x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
      x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
      return x ^ (x >> 31);
    };
    for (int p = 0; p < L; ++p) {
      if (p == center || p == center + 1) continue;
      const bool left = p < center;
      const Basis& from = left ? bonds[p] : bonds[p + 1];
      const Basis& to = left ? bonds[p + 1] : bonds[p];
      ProdBasis pb = make_prod(from, left);
      std::vector<int64_t> so(pb.prod.nsec(), -1);
      std::vector<int> nb(pb.prod.nsec(), -1);
      int64_t tot = 0, maxblk = 0;
      for (int q = 0; q < pb.prod.nsec(); ++q) {
        int t = to.find(pb.prod.q[q]);
        if (t < 0) continue;
        so[q] = tot;
        nb[q] = t;
        int64_t sz = (int64_t)pb.prod.dim[q] * to.dim[t];
        tot += sz;
        maxblk = std::max(maxblk, sz);
      }
      uint64_t dev = ex.alloc(tot);
      uint64_t scratch = left ? ex.alloc(maxblk) : 0;
      for (int q = 0; q < pb.prod.nsec(); ++q) {
        if (nb[q] < 0) continue;
        int rows = pb.prod.dim[q], d = to.dim[nb[q]];
        uint64_t sd = mix(mix(seed, (uint64_t)p), (uint64_t)q);
        if (left) {
          // orthonormal columns of a rows x d matrix, stored row-major
          ex.randn(scratch, (int64_t)rows * d, sd);
          ex.orthonormal_cols(scratch, rows, d);
          Launch l;
          Prob pr;
          pr.c = dev + 8ull * so[q]; pr.m = rows; pr.n = d; pr.ldc = d; pr.nseg = 1;
          Seg g;
          g.a = 0; g.b = scratch; g.ldb = rows; g.tb = 1; g.k = rows;
          l.segs.push_back(g);
          l.probs.push_back(pr);
          ex.run(l, 0, 0);
        } else {
          // orthonormal rows of a d x cols matrix = orthonormal columns of its
          // column-major transpose
          uint64_t dst = dev + 8ull * so[q];
          ex.randn(dst, (int64_t)rows * d, sd);
          ex.orthonormal_cols(dst, rows, d);
        }
      }
      if (scratch) ex.release(scratch);
      ctx->site[p] = dev;
      ctx->site_off[p] = so;
      ctx->site_nb[p] = nb;
    }
    ProdBasis Lp = make_prod(bonds[center], true), Rp = make_prod(bonds[center + 2], false);
    PsiLayout lay = make_psi_layout(Lp, Rp, QN{ctx->N, ctx->two_s});
    uint64_t tp = ex.alloc(std::max<int64_t>(1, lay.size));
    ex.randn(tp, lay.size, mix(seed, 0xC0FFEEull));
    double nrm = std::sqrt(ex.dot(tp, tp, lay.size));
    ex.scale(tp, 1.0 / nrm, lay.size);
    ctx->psi0.resize(lay.size);
    ex.download(ctx->psi0.data(), tp, lay.size);
    ex.release(tp);
    ctx->bonds = bonds;
    ctx->L = L;
    ctx->center = center;
    return QCDMRG_OK;
  });
}

int qcdmrg_get_bond(const qcdmrg_ctx* cctx, int bond, int* nsec, int* sec, int cap) {
  qcdmrg_ctx* ctx = const_cast<qcdmrg_ctx*>(cctx);
  return guard(ctx, [&]() {
    if (ctx->center < 0) throw Fail{QCDMRG_ESTATE, "no MPS"};
    if (bond < 0 || bond > ctx->L || !nsec) throw Fail{QCDMRG_EINVAL, "bad bond"};
    const Basis& b = ctx->bonds[bond];
    *nsec = b.nsec();
    if (sec) {
      if (cap < 3 * b.nsec()) throw Fail{QCDMRG_EINVAL, "sector buffer too small"};
      for (int i = 0; i < b.nsec(); ++i) {
        sec[3 * i] = b.q[i].n;
        sec[3 * i + 1] = b.q[i].s;
        sec[3 * i + 2] = b.dim[i];
      }
    }
    return QCDMRG_OK;
  });
}

int qcdmrg_get_psi(const qcdmrg_ctx* cctx, double* out, size_t n) {
  qcdmrg_ctx* ctx = const_cast<qcdmrg_ctx*>(cctx);
  return guard(ctx, [&]() {
    if (ctx->center < 0) throw Fail{QCDMRG_ESTATE, "no MPS"};
    if (!out || n != ctx->psi0.size()) throw Fail{QCDMRG_EINVAL, "output size differs from the wavefunction"};
    std::copy(ctx->psi0.begin(), ctx->psi0.end(), out);
    return QCDMRG_OK;
  });
}

int qcdmrg_build_env(qcdmrg_ctx* ctx) {
  return guard(ctx, [&]() {
    if (ctx->center < 0) throw Fail{QCDMRG_ESTATE, "import an MPS first"};
    auto t0 = std::chrono::steady_clock::now();
    ctx->free_env();
    Executor& ex = *ctx->be.ex;
    const int L = ctx->L, c = ctx->center;
    double fl = 0;
    EnvBlock left = vacuum(true, 0);
    for (int p = 0; p < c; ++p) {
      Enlarged E;
      enlarge(left, ctx->I, ex, E, &fl);
      EnvBlock nb;
      nb.cut = p + 1;
      renormalize(E, ctx->bonds[p + 1], ctx->site_nb[p], ctx->site[p], ctx->site_off[p], ex, nb,
                  ctx->tmp_budget, &fl);
      for (auto q : E.owned) ex.release(q);
      for (auto q : left.owned) ex.release(q);
      left = nb;
    }
    EnvBlock right = vacuum(false, L);
    for (int p = L - 1; p >= c + 2; --p) {
      Enlarged E;
      enlarge(right, ctx->I, ex, E, &fl);
      EnvBlock nb;
      nb.cut = p;
      renormalize(E, ctx->bonds[p], ctx->site_nb[p], ctx->site[p], ctx->site_off[p], ex, nb,
                  ctx->tmp_budget, &fl);
      for (auto q : E.owned) ex.release(q);
      for (auto q : right.owned) ex.release(q);
      right = nb;
    }
    ctx->lenv.push_back(left);
    ctx->renv.push_back(right);
    enlarge(ctx->lenv.back(), ctx->I, ex, ctx->Lp, &fl);
    enlarge(ctx->renv.back(), ctx->I, ex, ctx->Rp, &fl);
    ctx->lay = make_psi_layout(ctx->Lp.pb, ctx->Rp.pb, QN{ctx->N, ctx->two_s});
    if (ctx->lay.size != (int64_t)ctx->psi0.size()) throw Fail{QCDMRG_EINVAL, "wavefunction layout mismatch"};
    ctx->plan = plan_heff(ctx->Lp, ctx->Rp, ctx->lay, ctx->I, ctx->tmp_budget);
    ex.tmp(std::max<int64_t>(1, ctx->plan.tmp_elems));
    for (size_t k = 0; k < ctx->plan.stage1.size(); ++k)
      ctx->prepared.emplace_back(ctx->be.pr->prepare(ctx->plan.stage1[k]),
                                 ctx->be.pr->prepare(ctx->plan.stage2[k]));
    if (ctx->dpsi) ex.release(ctx->dpsi);
    if (ctx->dsig) ex.release(ctx->dsig);
    ctx->dpsi = ex.alloc(ctx->lay.size);
    ctx->dsig = ex.alloc(ctx->lay.size);
    ctx->have_env = true;
    auto t1 = std::chrono::steady_clock::now();
    ctx->st.env_flops = fl;
    ctx->st.env_seconds = std::chrono::duration<double>(t1 - t0).count();
    ctx->st.heff_flops = ctx->plan.flops;
    ctx->st.psi_size = ctx->lay.size;
    ctx->st.nterms = ctx->plan.nterms;
    ctx->st.nlaunch = 2 * (int)ctx->plan.stage1.size();
    return QCDMRG_OK;
  });
}

int qcdmrg_psi_size(const qcdmrg_ctx* ctx, size_t* n) {
  if (!ctx || !n) return QCDMRG_EINVAL;
  if (ctx->center < 0) return QCDMRG_ESTATE;
  *n = ctx->psi0.size();
  return QCDMRG_OK;
}

static void heff_dev(qcdmrg_ctx* ctx, uint64_t psi, uint64_t sig, void* stream, int prec) {
  PreparedRunner& pr = *ctx->be.pr;
  pr.zero_async(sig, ctx->lay.size, stream);
  for (auto& h : ctx->prepared) {
    pr.run_prepared(h.first, psi, sig, stream, prec);
    pr.run_prepared(h.second, psi, sig, stream, prec);
  }
}

static bool valid_precision(int p) {
  return p == QCDMRG_FP64 || p == QCDMRG_TF32 || p == QCDMRG_BF16 || p == QCDMRG_BF16X3;
}

int qcdmrg_apply_heff(qcdmrg_ctx* ctx, int precision, const double* psi, double* sigma) {
  return guard(ctx, [&]() {
    if (!ctx->have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!valid_precision(precision)) throw Fail{QCDMRG_EINVAL, "unknown precision"};
    if (!psi || !sigma) throw Fail{QCDMRG_EINVAL, "null argument"};
    Executor& ex = *ctx->be.ex;
    ex.upload(ctx->dpsi, psi, ctx->lay.size);
    auto t0 = std::chrono::steady_clock::now();
    void* st = ctx->be.pr->stream();
    heff_dev(ctx, ctx->dpsi, ctx->dsig, st, precision);
    ctx->be.pr->sync(st);
    if (ctx->be.pr->take_error()) throw Fail{QCDMRG_ETIMEOUT, "a tensor-core kernel wait gave up"};
    auto t1 = std::chrono::steady_clock::now();
    ctx->st.heff_seconds = std::chrono::duration<double>(t1 - t0).count();
    ex.download(sigma, ctx->dsig, ctx->lay.size);
    return QCDMRG_OK;
  });
}

int qcdmrg_apply_heff_dev(qcdmrg_ctx* ctx, int precision, const void* psi, void* sigma, void* stream) {
  return guard(ctx, [&]() {
    if (!ctx->have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!valid_precision(precision)) throw Fail{QCDMRG_EINVAL, "unknown precision"};
    if (!psi || !sigma || psi == sigma) throw Fail{QCDMRG_EINVAL, "psi and sigma must be distinct device arrays"};
    heff_dev(ctx, (uint64_t)psi, (uint64_t)sigma, stream, precision);
    return QCDMRG_OK;
  });
}

int qcdmrg_check_device(qcdmrg_ctx* ctx) {
  return guard(ctx, [&]() {
    if (ctx->be.pr->take_error()) throw Fail{QCDMRG_ETIMEOUT, "a tensor-core kernel wait gave up"};
    return QCDMRG_OK;
  });
}

int qcdmrg_stats(const qcdmrg_ctx* ctx, qcdmrg_stats_t* out) {
  if (!ctx || !out) return QCDMRG_EINVAL;
  *out = ctx->st;
  out->device_bytes = ctx->be.pr ? ctx->be.pr->bytes_allocated() : 0;
  return QCDMRG_OK;
}

}  // extern "C"
