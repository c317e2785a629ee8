// C ABI: context, integral and MPS import, environment build, H_eff psi.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qcdmrg.h"
#include "configs.hpp"
#include "entanglement.hpp"
#include "orbitals.hpp"
#include "core.hpp"
#include "engine.hpp"
#include "kernels.hpp"
#include "noalloc.hpp"
#include "graph.hpp"

using namespace qd;

struct qcdmrg_ctx {
  Backend be;
  Engine eng;
  int device = 0;
  bool have_int = false, have_target = false;
  uint64_t dpsi = 0, dsig = 0;   // host-API staging buffers
  int64_t staged = 0;
  qcdmrg_stats_t st{};
  std::string err;
  ~qcdmrg_ctx() {
    if (!be.ex) return;
    eng.clear();
    eng.ex = nullptr;  // the engine must not touch the executor after it is deleted
    eng.pr = nullptr;
    if (dpsi) be.ex->release(dpsi);
    if (dsig) be.ex->release(dsig);
    delete be.ex;
  }
  void staging(int64_t n) {
    if (n <= staged && dpsi) return;
    if (dpsi) be.ex->release(dpsi);
    if (dsig) be.ex->release(dsig);
    dpsi = be.ex->alloc(std::max<int64_t>(1, n));
    dsig = be.ex->alloc(std::max<int64_t>(1, n));
    staged = n;
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
  } catch (const StateError& e) {
    c->err = e.what();
    return QCDMRG_ESTATE;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return QCDMRG_ENOMEM;
  } catch (const std::runtime_error& e) {
    c->err = e.what();
    std::string m = e.what();
    if (m.find("out of memory") != std::string::npos) return QCDMRG_ENOMEM;
    return QCDMRG_ECUDA;
  } catch (const std::invalid_argument& e) {
    c->err = e.what();
    return QCDMRG_EINVAL;
  } catch (const std::exception& e) {
    c->err = e.what();
    return QCDMRG_EINTERNAL;
  } catch (...) {
    c->err = "unknown exception";
    return QCDMRG_EINTERNAL;
  }
}

// host-only calls (no context): exceptions become status codes at the C boundary
template <class F>
int host_guard(F&& f) {
  try {
    return f();
  } catch (const std::invalid_argument&) {
    return QCDMRG_EINVAL;
  } catch (const std::bad_alloc&) {
    return QCDMRG_ENOMEM;
  } catch (...) {
    return QCDMRG_EINTERNAL;
  }
}

// Gamma averaged over the 8 index permutations that leave (pq|rs) invariant
std::vector<double> permutation_average(const std::vector<double>& G, int L) {
  auto at = [L](int p, int q, int r, int s) { return (((size_t)p * L + q) * L + r) * L + s; };
  std::vector<double> A(G.size());
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q)
      for (int r = 0; r < L; ++r)
        for (int s = 0; s < L; ++s)
          A[at(p, q, r, s)] = (G[at(p, q, r, s)] + G[at(q, p, r, s)] + G[at(p, q, s, r)] + G[at(q, p, s, r)] +
                               G[at(r, s, p, q)] + G[at(s, r, p, q)] + G[at(r, s, q, p)] + G[at(s, r, q, p)]) /
                              8.0;
  return A;
}

}  // namespace

extern "C" {

int qcdmrg_create(qcdmrg_ctx** out, const qcdmrg_config* cfg) {
  if (!out || !cfg) return QCDMRG_EINVAL;
  *out = nullptr;
  if (cfg->symmetry != QCDMRG_U1 && cfg->symmetry != QCDMRG_SU2) return QCDMRG_EINVAL;
  // the configuration is checked before any CUDA call
  if (!(cfg->hbm_budget_gb >= 0) || !(cfg->tmp_budget_gb >= 0) || cfg->pair_switch < 0 || cfg->sum_gemm < -1 ||
      cfg->sum_gemm > 1 || cfg->tile_chunk < 0 || cfg->tile_chunk > 65536)
    return QCDMRG_EINVAL;
  auto* c = new qcdmrg_ctx();
  try {
    c->device = cfg->device;
    c->be = make_backend(cfg->device);
    double gb = cfg->tmp_budget_gb > 0 ? cfg->tmp_budget_gb : 2.0;
    c->eng.ex = c->be.ex;
    c->eng.pr = c->be.pr;
    c->eng.tmp_budget = (int64_t)(gb * 1e9 / 8);
    c->eng.hbm_budget = (int64_t)(cfg->hbm_budget_gb * 1e9);
    c->eng.autotune = cfg->autotune_off == 0;
    c->eng.pair_switch = cfg->pair_switch;
    c->eng.su2 = cfg->symmetry == QCDMRG_SU2;
    c->eng.device = cfg->device;
    c->eng.sum_gemm = cfg->sum_gemm;
    c->eng.tcfg.chunk = cfg->tile_chunk;
  } catch (const std::invalid_argument&) {
    delete c;
    return QCDMRG_EINVAL;
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
    ctx->eng.clear();
    ctx->eng.I.L = L;
    ctx->eng.I.h.assign(h, h + n2);
    ctx->eng.I.V.assign(V, V + n4);
    ctx->eng.I.ecore = e_core;
    ctx->have_int = true;
    return QCDMRG_OK;
  });
}

int qcdmrg_set_target(qcdmrg_ctx* ctx, int N, int two_s) {
  return guard(ctx, [&]() {
    if (N < 0 || ((N + two_s) & 1)) throw Fail{QCDMRG_EINVAL, "N and 2Sz must have equal parity"};
    if (ctx->eng.su2 && two_s < 0) throw Fail{QCDMRG_EINVAL, "2S must not be negative"};
    if (ctx->have_int && (N > 2 * ctx->eng.I.L || std::abs(two_s) > N))
      throw Fail{QCDMRG_EINVAL, "target outside the Fock space"};
    ctx->eng.clear();
    ctx->eng.N = N;
    ctx->eng.two_s = two_s;
    ctx->have_target = true;
    return QCDMRG_OK;
  });
}

int qcdmrg_import_mps(qcdmrg_ctx* ctx, const qcdmrg_mps_desc* d, const double* data, size_t n) {
  return guard(ctx, [&]() {
    if (!ctx->have_int || !ctx->have_target) throw Fail{QCDMRG_ESTATE, "load integrals and target first"};
    if (!d || !data || !d->bond_nsec || !d->bond_sec) throw Fail{QCDMRG_EINVAL, "null argument"};
    Engine& E = ctx->eng;
    const int L = d->L;
    if (L != E.I.L) throw Fail{QCDMRG_EINVAL, "MPS length differs from the integrals"};
    if (d->center < 0 || d->center + 1 >= L) throw Fail{QCDMRG_EINVAL, "centre out of range"};
    E.clear();
    std::vector<Basis> bonds(L + 1);
    for (auto& b : bonds) b.su2 = E.su2;
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
    E.site.assign(L, 0);
    E.site_off.assign(L, {});
    E.site_nb.assign(L, {});
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
      E.site[p] = dev;
      E.site_off[p] = so;
      E.site_nb[p] = nb;
    };
    for (int p = 0; p < c; ++p) take_site(p, bonds[p], true, bonds[p + 1]);
    for (int p = c + 2; p < L; ++p) take_site(p, bonds[p + 1], false, bonds[p]);
    // psi
    ProdBasis Lp = make_prod(bonds[c], true), Rp = make_prod(bonds[c + 2], false);
    PsiLayout lay = make_psi_layout(Lp, Rp, QN{E.N, E.two_s});
    if (off + lay.size != n) throw Fail{QCDMRG_EINVAL, "MPS data length does not match its layout"};
    E.bonds = bonds;
    E.L = L;
    E.center = c;
    E.set_psi_host(std::vector<double>(data + off, data + off + lay.size));
    return QCDMRG_OK;
  });
}

namespace {

// The current MPS in the layout qcdmrg_import_mps reads: sector triples of
// bonds 0..center and center+2..L (bond center+1 has none), the left site
// tensors U_q, the right site tensors V_q (product-sector order), then psi.
struct HostMps {
  int L = 0, center = -1;
  std::vector<int> nsec, sec;
  std::vector<double> data;
};

HostMps export_host(qcdmrg_ctx* ctx) {
  Engine& E = ctx->eng;
  if (E.center < 0) throw Fail{QCDMRG_ESTATE, "no MPS"};
  HostMps M;
  M.L = E.L;
  M.center = E.center;
  const int L = E.L, c = E.center;
  for (int b = 0; b <= L; ++b) {
    const bool have = b <= c || b >= c + 2;
    const Basis& B = E.bonds[b];
    M.nsec.push_back(have ? B.nsec() : 0);
    if (!have) continue;
    for (int i = 0; i < B.nsec(); ++i) {
      M.sec.push_back(B.q[i].n);
      M.sec.push_back(B.q[i].s);
      M.sec.push_back(B.dim[i]);
    }
  }
  auto put_site = [&](int p, const Basis& from, bool left, const Basis& to) {
    ProdBasis pb = make_prod(from, left);
    for (int q = 0; q < pb.prod.nsec(); ++q) {
      const int t = to.find(pb.prod.q[q]);
      if (t < 0) continue;
      if (q >= (int)E.site_off[p].size() || E.site_off[p][q] < 0)
        throw Fail{QCDMRG_ESTATE, "site tensor without a stored sector"};
      const int64_t cnt = (int64_t)pb.prod.dim[q] * to.dim[t];
      const size_t at = M.data.size();
      M.data.resize(at + (size_t)cnt);
      ctx->be.ex->download(M.data.data() + at, E.site[p] + 8ull * (uint64_t)E.site_off[p][q], cnt);
    }
  };
  for (int p = 0; p < c; ++p) put_site(p, E.bonds[p], true, E.bonds[p + 1]);
  for (int p = c + 2; p < L; ++p) put_site(p, E.bonds[p + 1], false, E.bonds[p]);
  std::vector<double> psi = E.get_psi_host();
  M.data.insert(M.data.end(), psi.begin(), psi.end());
  return M;
}

}  // namespace

int qcdmrg_export_mps(qcdmrg_ctx* ctx, int* L, int* center, int* bond_nsec, int* bond_sec, int sec_cap,
                      double* data, size_t cap, int* n_sec, size_t* n_data) {
  return guard(ctx, [&]() {
    HostMps M = export_host(ctx);
    if (L) *L = M.L;
    if (center) *center = M.center;
    if (n_sec) *n_sec = (int)(M.sec.size() / 3);
    if (n_data) *n_data = M.data.size();
    if (bond_nsec) std::copy(M.nsec.begin(), M.nsec.end(), bond_nsec);
    if (bond_sec) {
      if (sec_cap < (int)M.sec.size()) throw Fail{QCDMRG_EINVAL, "sector buffer too small"};
      std::copy(M.sec.begin(), M.sec.end(), bond_sec);
    }
    if (data) {
      if (cap < M.data.size()) throw Fail{QCDMRG_EINVAL, "data buffer too small"};
      std::copy(M.data.begin(), M.data.end(), data);
    }
    return QCDMRG_OK;
  });
}

int qcdmrg_checkpoint(qcdmrg_ctx* ctx, const char* path) {
  return guard(ctx, [&]() {
    if (!path) throw Fail{QCDMRG_EINVAL, "null path"};
    if (!ctx->have_int || !ctx->have_target) throw Fail{QCDMRG_ESTATE, "no integrals or target"};
    HostMps M = export_host(ctx);
    const Engine& E = ctx->eng;
    FILE* f = std::fopen(path, "wb");
    if (!f) throw Fail{QCDMRG_EIO, std::string("cannot open ") + path};
    const char magic[8] = {'Q', 'C', 'D', 'M', 'R', 'G', 'C', '1'};
    const int64_t hdr[7] = {E.I.L, E.N, E.two_s, M.center, (int64_t)M.nsec.size(), (int64_t)M.sec.size(),
                            (int64_t)M.data.size()};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int64_t), 7, f) == 7 &&
              std::fwrite(&E.I.ecore, sizeof(double), 1, f) == 1 &&
              std::fwrite(E.I.h.data(), sizeof(double), E.I.h.size(), f) == E.I.h.size() &&
              std::fwrite(E.I.V.data(), sizeof(double), E.I.V.size(), f) == E.I.V.size() &&
              std::fwrite(M.nsec.data(), sizeof(int), M.nsec.size(), f) == M.nsec.size() &&
              std::fwrite(M.sec.data(), sizeof(int), M.sec.size(), f) == M.sec.size() &&
              std::fwrite(M.data.data(), sizeof(double), M.data.size(), f) == M.data.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) throw Fail{QCDMRG_EIO, std::string("write failed: ") + path};
    return QCDMRG_OK;
  });
}

int qcdmrg_restore(qcdmrg_ctx* ctx, const char* path) {
  if (!ctx) return QCDMRG_EINVAL;
  int rc = guard(ctx, [&]() {
    if (!path) throw Fail{QCDMRG_EINVAL, "null path"};
    return QCDMRG_OK;
  });
  if (rc != QCDMRG_OK) return rc;
  std::vector<double> h, V, data;
  std::vector<int> nsec, sec;
  int64_t hdr[7] = {0, 0, 0, 0, 0, 0, 0};
  double ecore = 0.0;
  rc = guard(ctx, [&]() {
    FILE* f = std::fopen(path, "rb");
    if (!f) throw Fail{QCDMRG_EIO, std::string("cannot open ") + path};
    char magic[8];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "QCDMRGC1", 8) == 0 &&
              std::fread(hdr, sizeof(int64_t), 7, f) == 7;
    const int64_t L = hdr[0];
    ok = ok && L >= 2 && L <= 512 && hdr[4] == L + 1 && hdr[5] >= 0 && hdr[5] % 3 == 0 && hdr[5] <= (int64_t)1 << 30 &&
         hdr[6] >= 0 && hdr[6] <= (int64_t)1 << 40;
    if (ok) {
      h.resize((size_t)(L * L));
      V.resize((size_t)(L * L * L * L));
      nsec.resize((size_t)hdr[4]);
      sec.resize((size_t)hdr[5]);
      data.resize((size_t)hdr[6]);
      ok = std::fread(&ecore, sizeof(double), 1, f) == 1 &&
           std::fread(h.data(), sizeof(double), h.size(), f) == h.size() &&
           std::fread(V.data(), sizeof(double), V.size(), f) == V.size() &&
           std::fread(nsec.data(), sizeof(int), nsec.size(), f) == nsec.size() &&
           std::fread(sec.data(), sizeof(int), sec.size(), f) == sec.size() &&
           std::fread(data.data(), sizeof(double), data.size(), f) == data.size();
    }
    std::fclose(f);
    if (!ok) throw Fail{QCDMRG_EIO, std::string("not a qcdmrg checkpoint or truncated: ") + path};
    return QCDMRG_OK;
  });
  if (rc != QCDMRG_OK) return rc;
  rc = qcdmrg_load_integrals(ctx, (int)hdr[0], h.data(), V.data(), ecore);
  if (rc == QCDMRG_OK) rc = qcdmrg_set_target(ctx, (int)hdr[1], (int)hdr[2]);
  if (rc == QCDMRG_OK) {
    qcdmrg_mps_desc d{(int)hdr[0], (int)hdr[3], nsec.data(), sec.data()};
    rc = qcdmrg_import_mps(ctx, &d, data.data(), data.size());
  }
  return rc;
}

int qcdmrg_init_mps(qcdmrg_ctx* ctx, int D, uint64_t seed, int center) {
  return guard(ctx, [&]() {
    if (!ctx->have_int || !ctx->have_target) throw Fail{QCDMRG_ESTATE, "load integrals and target first"};
    Engine& E = ctx->eng;
    const int L = E.I.L;
    if (D < 1) throw Fail{QCDMRG_EINVAL, "D must be positive"};
    if (center < 0 || center + 1 >= L) throw Fail{QCDMRG_EINVAL, "centre out of range"};
    E.clear();
    auto st = mps_structure(L, E.N, E.two_s, D, E.su2);
    for (int b = 1; b < L; ++b)
      if (st[b].empty()) throw Fail{QCDMRG_EINVAL, "target not reachable: empty bond"};
    std::vector<Basis> bonds(L + 1);
    for (auto& b : bonds) b.su2 = E.su2;
    for (int b = 0; b <= center; ++b)
      for (auto& kv : st[b]) bonds[b].add(kv.first, kv.second);
    for (int b = center + 2; b <= L; ++b)
      for (auto& kv : st[L - b]) bonds[b].add(kv.first, kv.second);
    Executor& ex = *ctx->be.ex;
    E.site.assign(L, 0);
    E.site_off.assign(L, {});
    E.site_nb.assign(L, {});
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
      E.site[p] = dev;
      E.site_off[p] = so;
      E.site_nb[p] = nb;
    }
    ProdBasis Lp = make_prod(bonds[center], true), Rp = make_prod(bonds[center + 2], false);
    PsiLayout lay = make_psi_layout(Lp, Rp, QN{E.N, E.two_s});
    uint64_t tp = ex.alloc(std::max<int64_t>(1, lay.size));
    ex.randn(tp, lay.size, mix(seed, 0xC0FFEEull));
    double nrm = std::sqrt(ex.dot(tp, tp, lay.size));
    if (!(nrm > 0)) throw Fail{QCDMRG_EINVAL, "empty two-site wavefunction"};
    ex.scale(tp, 1.0 / nrm, lay.size);
    E.bonds = bonds;
    E.L = L;
    E.center = center;
    E.dpsi = tp;
    return QCDMRG_OK;
  });
}

int qcdmrg_get_bond(const qcdmrg_ctx* cctx, int bond, int* nsec, int* sec, int cap) {
  qcdmrg_ctx* ctx = const_cast<qcdmrg_ctx*>(cctx);
  return guard(ctx, [&]() {
    if (ctx->eng.center < 0) throw Fail{QCDMRG_ESTATE, "no MPS"};
    if (bond < 0 || bond > ctx->eng.L || !nsec) throw Fail{QCDMRG_EINVAL, "bad bond"};
    const Basis& b = ctx->eng.bonds[bond];
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
    if (ctx->eng.center < 0) throw Fail{QCDMRG_ESTATE, "no MPS"};
    std::vector<double> h = ctx->eng.get_psi_host();
    if (!out || n != h.size()) throw Fail{QCDMRG_EINVAL, "output size differs from the wavefunction"};
    std::copy(h.begin(), h.end(), out);
    return QCDMRG_OK;
  });
}

int qcdmrg_set_psi(qcdmrg_ctx* ctx, const double* psi, size_t n) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (E.center < 0) throw Fail{QCDMRG_ESTATE, "no MPS"};
    ProdBasis a = make_prod(E.bonds[E.center], true), b = make_prod(E.bonds[E.center + 2], false);
    int64_t sz = make_psi_layout(a, b, QN{E.N, E.two_s}).size;
    if (!psi || (int64_t)n != sz) throw Fail{QCDMRG_EINVAL, "input size differs from the wavefunction"};
    ctx->be.ex->upload(E.dpsi, psi, sz);
    return QCDMRG_OK;
  });
}

int qcdmrg_build_env(qcdmrg_ctx* ctx) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (E.center < 0) throw Fail{QCDMRG_ESTATE, "import or initialise an MPS first"};
    E.build_env();
    ctx->st.env_flops = E.env_flops;
    ctx->st.env_seconds = E.env_seconds;
    ctx->st.heff_flops = E.plan.flops;
    ctx->st.heff_bytes = E.plan.bytes;
    ctx->st.psi_size = E.lay.size;
    ctx->st.nterms = E.plan.nterms;
    ctx->st.nlaunch = 2 * (int)E.plan.stage1.size();
    return QCDMRG_OK;
  });
}

int qcdmrg_psi_size(const qcdmrg_ctx* ctx, size_t* n) {
  if (!ctx || !n) return QCDMRG_EINVAL;
  if (ctx->eng.center < 0) return QCDMRG_ESTATE;
  ProdBasis a = make_prod(ctx->eng.bonds[ctx->eng.center], true);
  ProdBasis b = make_prod(ctx->eng.bonds[ctx->eng.center + 2], false);
  *n = (size_t)make_psi_layout(a, b, QN{ctx->eng.N, ctx->eng.two_s}).size;
  return QCDMRG_OK;
}

int qcdmrg_psi_layout(const qcdmrg_ctx* cctx, int* blocks, int cap, int* nblocks, size_t* nelem) {
  qcdmrg_ctx* ctx = const_cast<qcdmrg_ctx*>(cctx);
  return guard(ctx, [&]() {
    const Engine& E = ctx->eng;
    if (E.center < 0) throw Fail{QCDMRG_ESTATE, "no MPS"};
    const Basis& X = E.bonds[E.center];
    const Basis& Y = E.bonds[E.center + 2];
    ProdBasis a = make_prod(X, true), b = make_prod(Y, false);
    PsiLayout lay = make_psi_layout(a, b, QN{E.N, E.two_s});
    if (nblocks) *nblocks = (int)lay.blks.size();
    if (nelem) *nelem = (size_t)lay.size;
    if (blocks) {
      if (cap < 8 * (int)lay.blks.size()) throw Fail{QCDMRG_EINVAL, "block buffer too small"};
      int k = 0;
      for (const auto& bk : lay.blks) {
        blocks[k++] = X.q[bk.x].n;
        blocks[k++] = X.q[bk.x].s;
        blocks[k++] = bk.i;
        blocks[k++] = bk.j;
        blocks[k++] = Y.q[bk.y].n;
        blocks[k++] = Y.q[bk.y].s;
        blocks[k++] = bk.rows;
        blocks[k++] = bk.cols;
      }
    }
    return QCDMRG_OK;
  });
}

int qcdmrg_energy_grad(qcdmrg_ctx* ctx, double* energy, double* dpsi, double* gamma1, double* gamma2) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (gamma1 && E.center != E.L - 2)
      throw Fail{QCDMRG_ESTATE, "the one-particle density matrix needs the centre at (L-2, L-1)"};
    Executor& ex = *ctx->be.ex;
    const int64_t n = E.lay.size;
    uint64_t sig = ex.alloc(std::max<int64_t>(1, n));
    double e = 0.0;
    try {
      E.heff(E.dpsi, sig, ctx->be.pr->stream(), 0);
      const double nn = ex.dot(E.dpsi, E.dpsi, n);
      if (!(nn > 0)) throw Fail{QCDMRG_EINVAL, "zero wavefunction"};
      e = ex.dot(E.dpsi, sig, n) / nn;
      if (dpsi) {
        // dE/dpsi = 2 (H psi - E psi) / <psi|psi>
        ex.axpby(sig, -e, E.dpsi, 1.0, n);
        ex.scale(sig, 2.0 / nn, n);
        ex.download(dpsi, sig, n);
      }
    } catch (...) {
      ex.release(sig);
      throw;
    }
    ex.release(sig);
    if (energy) *energy = e;
    if (gamma1) {
      std::vector<double> g = E.rdm1();
      std::copy(g.begin(), g.end(), gamma1);
    }
    if (gamma2) {
      // environment-build probes while they are affordable, the centre walk
      // (averaged over the 8 permutations of (pq|rs)) beyond
      std::vector<double> g = E.L <= 10 ? E.rdm2() : permutation_average(E.rdm2_sweep(), E.L);
      std::copy(g.begin(), g.end(), gamma2);
    }
    return QCDMRG_OK;
  });
}

static bool valid_precision(int p) {
  return p == QCDMRG_FP64 || p == QCDMRG_TF32 || p == QCDMRG_BF16 || p == QCDMRG_BF16X3;
}

int qcdmrg_apply_heff(qcdmrg_ctx* ctx, int precision, const double* psi, double* sigma) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!valid_precision(precision)) throw Fail{QCDMRG_EINVAL, "unknown precision"};
    if (!psi || !sigma) throw Fail{QCDMRG_EINVAL, "null argument"};
    Executor& ex = *ctx->be.ex;
    ctx->staging(E.lay.size);
    ex.upload(ctx->dpsi, psi, E.lay.size);
    auto t0 = std::chrono::steady_clock::now();
    void* st = ctx->be.pr->stream();
    E.heff(ctx->dpsi, ctx->dsig, st, precision);
    ctx->be.pr->sync(st);
    auto t1 = std::chrono::steady_clock::now();
    if (ctx->be.pr->take_error()) throw Fail{QCDMRG_ETIMEOUT, "a tensor-core kernel wait gave up"};
    ctx->st.heff_seconds = std::chrono::duration<double>(t1 - t0).count();
    ex.download(sigma, ctx->dsig, E.lay.size);
    return QCDMRG_OK;
  });
}

int qcdmrg_apply_heff_dev(qcdmrg_ctx* ctx, int precision, const void* psi, void* sigma, void* stream) {
  return guard(ctx, [&]() {
    if (!ctx->eng.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!valid_precision(precision)) throw Fail{QCDMRG_EINVAL, "unknown precision"};
    if (!psi || !sigma || psi == sigma) throw Fail{QCDMRG_EINVAL, "psi and sigma must be distinct device arrays"};
    ctx->eng.heff((uint64_t)psi, (uint64_t)sigma, stream, precision);
    return QCDMRG_OK;
  });
}

int qcdmrg_apply_heff_noalloc(qcdmrg_ctx* ctx, const void* psi, void* sigma, void* stream) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!psi || !sigma || psi == sigma) throw Fail{QCDMRG_EINVAL, "psi and sigma must be distinct device arrays"};
    if (E.plan.tmp_elems > NOALLOC_SCRATCH_DOUBLES)
      throw Fail{QCDMRG_EINVAL, "this H_eff needs " + std::to_string(E.plan.tmp_elems) +
                                    " doubles of scratch; the fixed array holds " +
                                    std::to_string(NOALLOC_SCRATCH_DOUBLES) +
                                    " (use qcdmrg_apply_heff_dev, or a smaller tmp_budget_gb)"};
    heff_noalloc(E, ctx->device, (uint64_t)psi, (uint64_t)sigma, stream);
    return QCDMRG_OK;
  });
}

static DavOpts dav_opts(const qcdmrg_dav_opts* o) {
  DavOpts d;
  if (!o) return d;
  if (o->tol > 0) d.tol = o->tol;
  if (o->max_iter > 0) d.max_iter = o->max_iter;
  if (o->m_max > 0) d.m_max = o->m_max;
  d.policy = o->policy;
  d.precision = o->precision;
  if (o->tau1 > 0) d.tau1 = o->tau1;
  if (o->tau2 > 0) d.tau2 = o->tau2;
  return d;
}

int qcdmrg_rdm1(qcdmrg_ctx* ctx, double* gamma) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!gamma) throw Fail{QCDMRG_EINVAL, "null argument"};
    std::vector<double> g = E.rdm1();
    std::copy(g.begin(), g.end(), gamma);
    return QCDMRG_OK;
  });
}

int qcdmrg_rdm2(qcdmrg_ctx* ctx, double* gamma2) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!gamma2) throw Fail{QCDMRG_EINVAL, "null argument"};
    std::vector<double> g = E.rdm2();
    std::copy(g.begin(), g.end(), gamma2);
    return QCDMRG_OK;
  });
}

int qcdmrg_rdm2_sweep(qcdmrg_ctx* ctx, double* gamma2) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!gamma2) throw Fail{QCDMRG_EINVAL, "null argument"};
    std::vector<double> g = E.rdm2_sweep();
    std::copy(g.begin(), g.end(), gamma2);
    return QCDMRG_OK;
  });
}

int qcdmrg_orbital_rdm(qcdmrg_ctx* ctx, double* rho) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!rho) throw Fail{QCDMRG_EINVAL, "null argument"};
    std::vector<double> r = E.orbital_rdm2();
    std::copy(r.begin(), r.end(), rho);
    return QCDMRG_OK;
  });
}

int qcdmrg_orbital_entanglement(int L, const double* rho, double* s1, double* mutual) {
  return host_guard([&]() {
    if (L < 2 || !rho || !mutual) return QCDMRG_EINVAL;
    for (size_t k = 0; k < (size_t)L * L * 256; ++k)
      if (!std::isfinite(rho[k])) return QCDMRG_EINVAL;
    orbital_entanglement(L, rho, s1, mutual);
    return QCDMRG_OK;
  });
}

int qcdmrg_fiedler_order(int L, const double* mutual, int* order, double* fiedler) {
  return host_guard([&]() {
    if (L < 2 || !mutual || !order) return QCDMRG_EINVAL;
    for (int i = 0; i < L; ++i)
      for (int j = 0; j <= i; ++j) {
        const double a = mutual[(size_t)i * L + j], b = mutual[(size_t)j * L + i];
        if (!std::isfinite(a) || !std::isfinite(b) || std::fabs(a - b) > 1e-12 * std::max(1.0, std::fabs(a)))
          return QCDMRG_EINVAL;
      }
    fiedler_order(L, mutual, order, fiedler);
    return QCDMRG_OK;
  });
}

namespace {

bool symmetric_finite(int L, const double* m) {
  for (int i = 0; i < L; ++i)
    for (int j = 0; j <= i; ++j) {
      const double a = m[(size_t)i * L + j], b = m[(size_t)j * L + i];
      if (!std::isfinite(a) || !std::isfinite(b) || std::fabs(a - b) > 1e-12 * std::max(1.0, std::fabs(a)))
        return false;
    }
  return true;
}

bool permutation(int L, const int* order) {
  std::vector<char> seen(L, 0);
  for (int k = 0; k < L; ++k) {
    if (order[k] < 0 || order[k] >= L || seen[order[k]]) return false;
    seen[order[k]] = 1;
  }
  return true;
}

}  // namespace

int qcdmrg_ordering_cost(int L, const double* mutual, const int* order, double eta, double* cost) {
  return host_guard([&]() {
    if (L < 2 || !mutual || !order || !cost || !std::isfinite(eta) || !(eta > 0)) return QCDMRG_EINVAL;
    if (!symmetric_finite(L, mutual) || !permutation(L, order)) return QCDMRG_EINVAL;
    *cost = ordering_cost(L, mutual, order, eta);
    return QCDMRG_OK;
  });
}

int qcdmrg_refine_order(int L, const double* mutual, double eta, int* order, int max_swaps, int* swaps) {
  return host_guard([&]() {
    if (L < 2 || !mutual || !order || !std::isfinite(eta) || !(eta > 0) || max_swaps < 0) return QCDMRG_EINVAL;
    if (!symmetric_finite(L, mutual) || !permutation(L, order)) return QCDMRG_EINVAL;
    const int n = refine_order(L, mutual, eta, order, max_swaps);
    if (swaps) *swaps = n;
    return QCDMRG_OK;
  });
}

int qcdmrg_heff_diag(qcdmrg_ctx* ctx, double* out, size_t n) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (!out || n != (size_t)E.lay.size) throw Fail{QCDMRG_EINVAL, "output size differs from the wavefunction"};
    ctx->be.ex->download(out, E.ddiag, E.lay.size);
    return QCDMRG_OK;
  });
}

int qcdmrg_davidson(qcdmrg_ctx* ctx, const qcdmrg_dav_opts* o, double* energy, double* resid, int* iters) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (o && (!valid_precision(o->precision) || o->policy < 0 || o->policy > 1))
      throw Fail{QCDMRG_EINVAL, "bad Davidson options"};
    const auto t0 = std::chrono::steady_clock::now();
    DavResult r = E.davidson(dav_opts(o));
    ctx->st.dav_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < 4; ++k) ctx->st.dav_hpsi[k] = r.hpsi[k];
    ctx->st.dav_energy_mixed = r.energy_mixed;
    if (energy) *energy = r.energy;
    if (resid) *resid = r.resid;
    if (iters) *iters = r.iters;
    return r.converged ? QCDMRG_OK : QCDMRG_ENOTCONV;
  });
}

int qcdmrg_truncate(qcdmrg_ctx* ctx, int D, int dir, double* trunc_err) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (D < 1 || (dir != 1 && dir != -1)) throw Fail{QCDMRG_EINVAL, "D >= 1 and dir = +1 or -1"};
    if ((dir > 0 && E.center + 2 >= E.L) || (dir < 0 && E.center == 0))
      throw Fail{QCDMRG_EINVAL, "the centre cannot move further in that direction"};
    double e = E.truncate_move(D, dir, 0.0);
    if (trunc_err) *trunc_err = e;
    return QCDMRG_OK;
  });
}

int qcdmrg_truncate_dbss(qcdmrg_ctx* ctx, int D_min, int D_max, double eps, int dir, double* trunc_err,
                         int* kept) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (D_min < 1 || D_max < D_min || !(eps > 0.0) || (dir != 1 && dir != -1))
      throw Fail{QCDMRG_EINVAL, "1 <= D_min <= D_max, eps > 0 and dir = +1 or -1"};
    if ((dir > 0 && E.center + 2 >= E.L) || (dir < 0 && E.center == 0))
      throw Fail{QCDMRG_EINVAL, "the centre cannot move further in that direction"};
    int nk = 0;
    double e = E.truncate_move(D_max, dir, 0.0, eps, D_min, &nk);
    if (trunc_err) *trunc_err = e;
    if (kept) *kept = nk;
    return QCDMRG_OK;
  });
}

int qcdmrg_extrapolate(const double* x, const double* energy, int n, int degree, double* coef) {
  return host_guard([&]() {
    // least-squares polynomial E(x) = coef[0] + coef[1] x + ... + coef[degree] x^degree
    // through the n points; x is scaled to [-1, 1] for the normal equations, whose
    // (degree + 1)^2 system is solved by Gaussian elimination with partial pivoting
    if (!x || !energy || !coef || degree < 1 || degree > 3 || n < degree + 1) return QCDMRG_EINVAL;
    double xs = 0;
    for (int i = 0; i < n; ++i) {
      if (!std::isfinite(x[i]) || !std::isfinite(energy[i])) return QCDMRG_EINVAL;
      xs = std::max(xs, std::fabs(x[i]));
    }
    if (!(xs > 0)) return QCDMRG_EINVAL;
    const int m = degree + 1;
    long double A[4][5] = {};
    for (int i = 0; i < n; ++i) {
      long double p[4];
      p[0] = 1;
      for (int k = 1; k < m; ++k) p[k] = p[k - 1] * (x[i] / xs);
      for (int r = 0; r < m; ++r) {
        for (int c = 0; c < m; ++c) A[r][c] += p[r] * p[c];
        A[r][m] += p[r] * energy[i];
      }
    }
    for (int c = 0; c < m; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (std::fabs((double)A[r][c]) > std::fabs((double)A[piv][c])) piv = r;
      if (!(std::fabs((double)A[piv][c]) > 0)) return QCDMRG_EINVAL;   // points do not fix the polynomial
      for (int k = 0; k <= m; ++k) std::swap(A[c][k], A[piv][k]);
      for (int r = 0; r < m; ++r) {
        if (r == c) continue;
        const long double f = A[r][c] / A[c][c];
        for (int k = c; k <= m; ++k) A[r][k] -= f * A[c][k];
      }
    }
    double sc = 1.0;
    for (int k = 0; k < m; ++k) {
      coef[k] = (double)(A[k][m] / A[k][k]) / sc;
      sc *= xs;
    }
    return QCDMRG_OK;
  });
}

int qcdmrg_active_space(int n, int ncore, int nact, const double* h, const double* V, double* e_core,
                        double* h_act, double* V_act) {
  return host_guard([&]() {
    if (n < 1 || ncore < 0 || nact < 1 || ncore + nact > n || !h || !V || !e_core || !h_act || !V_act)
      return QCDMRG_EINVAL;
    active_space(n, ncore, nact, h, V, e_core, h_act, V_act);
    return QCDMRG_OK;
  });
}

int qcdmrg_orbital_gradient(int n, int ncore, int nact, const double* h, const double* V, const double* gamma1,
                            const double* gamma2, double* grad) {
  return host_guard([&]() {
    if (n < 1 || ncore < 0 || nact < 1 || ncore + nact > n || !h || !V || !gamma1 || !gamma2 || !grad)
      return QCDMRG_EINVAL;
    orbital_gradient(n, ncore, nact, h, V, gamma1, gamma2, grad);
    return QCDMRG_OK;
  });
}

int qcdmrg_orbital_hessian_diag(int n, int ncore, int nact, const double* h, const double* V, const double* gamma1,
                                const double* gamma2, double* hdiag) {
  return host_guard([&]() {
    if (n < 1 || ncore < 0 || nact < 1 || ncore + nact > n || !h || !V || !gamma1 || !gamma2 || !hdiag)
      return QCDMRG_EINVAL;
    orbital_hessian_diag(n, ncore, nact, h, V, gamma1, gamma2, hdiag);
    return QCDMRG_OK;
  });
}

int qcdmrg_rotate_orbitals(int n, const double* kappa, const double* h, const double* V, double* U, double* h_out,
                           double* V_out) {
  return host_guard([&]() {
    if (n < 1 || !kappa || !h || !V || !h_out || !V_out) return QCDMRG_EINVAL;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q <= p; ++q) {
        const double a = kappa[(size_t)p * n + q], b = kappa[(size_t)q * n + p];
        if (!std::isfinite(a) || std::fabs(a + b) > 1e-12 * std::max(1.0, std::fabs(a))) return QCDMRG_EINVAL;
      }
    std::vector<double> u((size_t)n * n);
    expm_antisym(n, kappa, u.data());
    rotate_integrals(n, u.data(), h, V, h_out, V_out);
    if (U) std::copy(u.begin(), u.end(), U);
    return QCDMRG_OK;
  });
}

int qcdmrg_move_center(qcdmrg_ctx* ctx, int target) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
    if (target < 0 || target + 1 >= E.L) throw Fail{QCDMRG_EINVAL, "centre out of range"};
    while (E.center > target) E.truncate_move(1 << 30, -1, 1e-28);
    while (E.center < target) E.truncate_move(1 << 30, +1, 1e-28);
    return QCDMRG_OK;
  });
}

namespace {

void check_sweep_opts(const Engine& E, const qcdmrg_sweep_opts* o) {
  if (!E.have_env) throw Fail{QCDMRG_ESTATE, "build_env first"};
  if (!o || o->D < 1) throw Fail{QCDMRG_EINVAL, "sweep options with D >= 1 required"};
  if (o->trunc_eps < 0.0 || (o->trunc_eps > 0.0 && (o->D_min < 1 || o->D_min > o->D)))
    throw Fail{QCDMRG_EINVAL, "dynamic selection needs 1 <= D_min <= D"};
}

// one two-site optimisation of a sweep: Davidson at the centre, then the
// truncation that moves the centre by dir
void sweep_step(Engine& E, const qcdmrg_sweep_opts* o, const DavOpts& dop, int dir, qcdmrg_sweep_report& R,
                bool& conv) {
  DavResult r = E.davidson(dop);
  conv = conv && r.converged;
  for (int k = 0; k < 4; ++k) R.n_hpsi[k] += r.hpsi[k];
  R.energy = r.energy;
  R.energy_mixed = r.energy_mixed;
  R.n_steps++;
  int nk = 0;
  double e = E.truncate_move(o->D, dir, 0.0, o->trunc_eps, o->D_min, &nk);
  R.max_trunc_err = std::max(R.max_trunc_err, e);
  R.max_D = std::max(R.max_D, nk);
}

}  // namespace

int qcdmrg_sweep(qcdmrg_ctx* ctx, const qcdmrg_sweep_opts* o, qcdmrg_sweep_report* rep) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    check_sweep_opts(E, o);
    if (E.L < 3) throw Fail{QCDMRG_EINVAL, "sweeps need L >= 3"};
    auto t0 = std::chrono::steady_clock::now();
    while (E.center > 0) E.truncate_move(1 << 30, -1, 1e-28);
    DavOpts dop = dav_opts(&o->dav);
    qcdmrg_sweep_report R{};
    bool conv = true;
    for (int l = 0; l < E.L - 2; ++l) sweep_step(E, o, dop, +1, R, conv);
    for (int l = E.L - 2; l > 0; --l) sweep_step(E, o, dop, -1, R, conv);
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = R;
    ctx->st.heff_flops = E.plan.flops;
    ctx->st.heff_bytes = E.plan.bytes;
    ctx->st.psi_size = E.lay.size;
    return conv ? QCDMRG_OK : QCDMRG_ENOTCONV;
  });
}

int qcdmrg_sweep_left(qcdmrg_ctx* ctx, const qcdmrg_sweep_opts* o, qcdmrg_sweep_report* rep) {
  return guard(ctx, [&]() {
    Engine& E = ctx->eng;
    check_sweep_opts(E, o);
    auto t0 = std::chrono::steady_clock::now();
    DavOpts dop = dav_opts(&o->dav);
    qcdmrg_sweep_report R{};
    bool conv = true;
    while (E.center > 0) sweep_step(E, o, dop, -1, R, conv);
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = R;
    return conv ? QCDMRG_OK : QCDMRG_ENOTCONV;
  });
}

int qcdmrg_select_configs(int symmetry, int L, int N, int two_s, const double* h, const double* V, int nmax,
                          uint8_t* steps, double* energy, int* count) {
  if ((symmetry != QCDMRG_U1 && symmetry != QCDMRG_SU2) || L < 2 || L > 4096 || nmax < 1 || !h || !V ||
      !steps || !count)
    return QCDMRG_EINVAL;
  return host_guard([&]() {
    std::vector<uint8_t> st;
    std::vector<double> en;
    const int m = select_configs(L, symmetry == QCDMRG_SU2, N, two_s, h, V, nmax, st, en);
    std::copy(st.begin(), st.end(), steps);
    if (energy) std::copy(en.begin(), en.end(), energy);
    *count = m;
    return QCDMRG_OK;
  });
}

int qcdmrg_config_mps(int symmetry, int L, int N, int two_s, int n, const uint8_t* steps, const double* coef,
                      int* center, int* bond_nsec, int* bond_sec, int sec_cap, double* data, size_t cap,
                      int* n_sec, size_t* n_data) {
  if ((symmetry != QCDMRG_U1 && symmetry != QCDMRG_SU2) || L < 2 || n < 1 || !steps || !coef)
    return QCDMRG_EINVAL;
  return host_guard([&]() {
    ImportArrays A;
    configs_to_mps(L, symmetry == QCDMRG_SU2, N, two_s, n, steps, coef, A);
    if ((bond_sec && sec_cap < (int)A.sec.size()) || (data && cap < A.data.size())) return QCDMRG_EINVAL;
    if (center) *center = A.center;
    if (n_sec) *n_sec = (int)(A.sec.size() / 3);
    if (n_data) *n_data = A.data.size();
    if (bond_nsec) std::copy(A.nsec.begin(), A.nsec.end(), bond_nsec);
    if (bond_sec) std::copy(A.sec.begin(), A.sec.end(), bond_sec);
    if (data) std::copy(A.data.begin(), A.data.end(), data);
    return QCDMRG_OK;
  });
}

int qcdmrg_check_device(qcdmrg_ctx* ctx) {
  return guard(ctx, [&]() {
    if (ctx->be.pr->take_error()) throw Fail{QCDMRG_ETIMEOUT, "a tensor-core kernel wait gave up"};
    return QCDMRG_OK;
  });
}

struct qcdmrg_graph {
  HeffGraph* g = nullptr;
};

int qcdmrg_graph_create(qcdmrg_ctx* const* ctxs, int n, int precision, const void* const* psi,
                        void* const* sigma, qcdmrg_graph** out) {
  if (!ctxs || n < 1 || !psi || !sigma || !out) return QCDMRG_EINVAL;
  *out = nullptr;
  if (!valid_precision(precision)) return QCDMRG_EINVAL;
  std::vector<Engine*> eng;
  std::vector<uint64_t> ps, ss;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !psi[i] || !sigma[i] || psi[i] == sigma[i]) return QCDMRG_EINVAL;
    if (!ctxs[i]->eng.have_env) return QCDMRG_ESTATE;
    if (ctxs[i]->device != ctxs[0]->device) return QCDMRG_EINVAL;
    eng.push_back(&ctxs[i]->eng);
    ps.push_back((uint64_t)psi[i]);
    ss.push_back((uint64_t)sigma[i]);
  }
  try {
    auto* g = new qcdmrg_graph();
    g->g = graph_create(eng, ps, ss, precision);
    *out = g;
  } catch (const std::exception& e) {
    ctxs[0]->err = e.what();
    return QCDMRG_ECUDA;
  }
  return QCDMRG_OK;
}

int qcdmrg_graph_launch(qcdmrg_graph* g, void* stream) {
  if (!g || !g->g) return QCDMRG_EINVAL;
  try {
    graph_launch(g->g, stream);
  } catch (const std::exception&) {
    return QCDMRG_ECUDA;
  }
  return QCDMRG_OK;
}

int qcdmrg_graph_info(const qcdmrg_graph* g, double* flops, int* nodes) {
  if (!g || !g->g) return QCDMRG_EINVAL;
  if (flops) *flops = graph_flops(g->g);
  if (nodes) *nodes = graph_nodes(g->g);
  return QCDMRG_OK;
}

int qcdmrg_graph_destroy(qcdmrg_graph* g) {
  if (!g) return QCDMRG_EINVAL;
  graph_destroy(g->g);
  delete g;
  return QCDMRG_OK;
}

int qcdmrg_stats(const qcdmrg_ctx* ctx, qcdmrg_stats_t* out) {
  if (!ctx || !out) return QCDMRG_EINVAL;
  *out = ctx->st;
  out->device_bytes = ctx->be.pr ? ctx->be.pr->bytes_allocated() : 0;
  out->live_bytes = ctx->be.ex ? ctx->be.ex->live_bytes() : 0;
  out->h2d_bytes = ctx->eng.h2d_bytes;
  out->tile_kmax = ctx->eng.tcfg.kmax;
  out->tile_width = ctx->eng.tcfg.width;
  out->tile_chunk = ctx->eng.tcfg.chunk;
  out->tile_passes = ctx->eng.tiled_passes;
  out->tile_t_bytes = ctx->eng.tiled_t_plane;
  out->tunes = ctx->eng.tunes;
  out->tune_seconds = ctx->eng.tune_seconds;
  out->d2h_bytes = ctx->eng.d2h_bytes;
  out->evictions = ctx->eng.evictions;
  out->restores = ctx->eng.restores;
  out->copy_wait_seconds = ctx->be.ex ? ctx->be.ex->copies_wait_seconds() : 0.0;
  for (int c = 0; c < 4; ++c) out->f64_tiles[c] = 0;
  out->f64_split_tiles = 0;
  if (ctx->be.pr && ctx->eng.have_env)
    for (auto& h : ctx->eng.prepared)
      for (int hh : {h.first, h.second}) {
        int64_t c[5];
        ctx->be.pr->tile_counts(hh, c);
        for (int k = 0; k < 4; ++k) out->f64_tiles[k] += c[k];
        out->f64_split_tiles += c[4];
      }
  return QCDMRG_OK;
}

}  // extern "C"
