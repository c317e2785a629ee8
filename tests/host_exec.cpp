// Test-only host execution of the library's H_eff task lists, without a GPU.
//
// The library's host planner (rules, renormalization, H_eff task lists, tiled
// work items) runs unchanged with an executor that keeps every buffer in host
// memory and executes each segmented-GEMM task list with plain loops. The
// driver imports an MPS (the C-ABI import layout), builds the environment,
// applies the FP64 task lists to psi, and separately evaluates the tiled work
// items of the tensor-core path in FP64 (views, panels, term scalars, T tiles,
// no bf16 rounding), so that both plans can be compared with the oracle.
//
// Every launch is checked against the buffers it addresses. The environment
// variable HOST_EXEC_PAIR_SWITCH sets the cut of the normal/complementary switch,
// HOST_EXEC_SUM_GEMM the form of the operator sums (1 GEMM, -1 block by block).
//
// usage: host_exec in.bin out.bin                       (one H_eff psi, both plans)
//        host_exec in.bin out.bin sweep D nsweeps tol     (full FP64 sweeps)
//        host_exec in.bin out.bin rdm1                    (1-RDM, centre at L-2)
//        host_exec in.bin out.bin rdm2sweep               (2-RDM by the centre walk, then
//                                                          psi and sigma at the centre)
//        host_exec in.bin out.bin orbrdm                  (two-orbital density matrices,
//                                                          L*L blocks of 256, then psi, sigma)
//        host_exec in.bin out.bin warmup D nsweeps tol    (half sweep left from the
//                                                          imported centre, then sweeps)
//        host_exec in.bin out.bin sweeprdm D nsweeps tol  (sweeps, then the two-orbital
//                                                          density matrices)
//        host_exec in.bin out.bin sweepgamma D nsweeps tol (sweeps, then the 2-RDM by the
//                                                          walk of the centre)
//   in : int64 L, N, two_sz, center, nsec_len (= L+1), sec_len, data_len;
//        h (L*L), V (L^4) doubles; bond_nsec, bond_sec int32; data doubles
//   out: sigma of the FP64 task lists, then sigma of the tiled work items; or
//        the energy of the last optimisation of each sweep (the sweeps start by
//        moving the centre to bond 0, as qcdmrg_sweep does)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "engine.hpp"
#include "tiled.hpp"

using namespace qd;

namespace {

struct HostEx : Executor {
  std::map<uint64_t, std::vector<double>> bufs;  // base address -> storage
  uint64_t tmp_base = 0;
  int64_t tmp_n = 0, live = 0;
  uint64_t alloc(int64_t n) override {
    std::vector<double> v((size_t)std::max<int64_t>(1, n), 0.0);
    const uint64_t p = reinterpret_cast<uint64_t>(v.data());
    live += (int64_t)v.size() * 8;
    bufs[p] = std::move(v);
    return p;
  }
  void release(uint64_t p) override {
    auto it = bufs.find(p);
    if (it != bufs.end()) {
      live -= (int64_t)it->second.size() * 8;
      bufs.erase(it);
    }
  }
  int64_t size_of(uint64_t p) const {
    auto it = bufs.find(p);
    return it == bufs.end() ? 0 : (int64_t)it->second.size();
  }
  uint64_t tmp(int64_t n) override {
    if (n > tmp_n) {
      if (tmp_base) release(tmp_base);
      tmp_base = alloc(n);
      tmp_n = n;
    }
    return tmp_base;
  }
  static double* ptr(uint64_t p) { return reinterpret_cast<double*>(p); }
  // the elements [q, q + last] must lie inside one live allocation
  void inside(const double* q, int64_t last, const char* what) const {
    const uint64_t a = reinterpret_cast<uint64_t>(q);
    auto it = bufs.upper_bound(a);
    if (last < 0 || it == bufs.begin()) throw std::runtime_error(std::string("task list: ") + what + " outside every buffer");
    --it;
    const int64_t first = (int64_t)(a - it->first);
    if (first % 8 || first / 8 + last >= (int64_t)it->second.size())
      throw std::runtime_error(std::string("task list: ") + what + " past the end of its buffer");
  }
  void exec(const Launch& l, uint64_t psi, uint64_t sig) {
    const uint64_t base[4] = {0, psi, sig, tmp_base};
    auto res = [&](uint64_t v, int buf) { return buf == 0 ? ptr(v) : ptr(base[buf] + v * 8); };
    for (const Prob& p : l.probs) {
      if (p.m <= 0 || p.n <= 0 || p.ldc < p.n) throw std::runtime_error("task list: empty or malformed problem");
      if (p.seg0 < 0 || p.nseg < 0 || p.seg0 + p.nseg > (int)l.segs.size()) throw std::runtime_error("task list: segment range");
      inside(res(p.c, p.cbuf), (int64_t)(p.m - 1) * p.ldc + p.n - 1, "C");
      std::vector<double> acc((size_t)p.m * p.n, 0.0);
      for (int s = p.seg0; s < p.seg0 + p.nseg; ++s) {
        const Seg& g = l.segs[s];
        const bool aid = g.a == 0 && g.abuf == 0, bid = g.b == 0 && g.bbuf == 0;
        if (aid) {
          if (bid) {
            for (int r = 0; r < std::min(p.m, p.n); ++r) acc[(size_t)r * p.n + r] += g.sc;
          } else {
            const double* B = res(g.b, g.bbuf);
            inside(B, g.tb ? (int64_t)(p.n - 1) * g.ldb + p.m - 1 : (int64_t)(p.m - 1) * g.ldb + p.n - 1, "B of a gather");
            for (int r = 0; r < p.m; ++r)
              for (int c = 0; c < p.n; ++c)
                acc[(size_t)r * p.n + c] += g.sc * (g.tb ? B[(size_t)c * g.ldb + r] : B[(size_t)r * g.ldb + c]);
          }
          continue;
        }
        if (bid) throw std::runtime_error("task list: identity B with a stored A");
        const double* A = res(g.a, g.abuf);
        const double* B = res(g.b, g.bbuf);
        if (g.k <= 0) throw std::runtime_error("task list: empty segment");
        inside(A, g.ta ? (int64_t)(g.k - 1) * g.lda + p.m - 1 : (int64_t)(p.m - 1) * g.lda + g.k - 1, "A");
        inside(B, g.tb ? (int64_t)(p.n - 1) * g.ldb + g.k - 1 : (int64_t)(g.k - 1) * g.ldb + p.n - 1, "B");
        for (int r = 0; r < p.m; ++r)
          for (int k = 0; k < g.k; ++k) {
            const double a = g.sc * (g.ta ? A[(size_t)k * g.lda + r] : A[(size_t)r * g.lda + k]);
            if (a == 0.0) continue;
            for (int c = 0; c < p.n; ++c)
              acc[(size_t)r * p.n + c] += a * (g.tb ? B[(size_t)c * g.ldb + k] : B[(size_t)k * g.ldb + c]);
          }
      }
      double* C = res(p.c, p.cbuf);
      for (int r = 0; r < p.m; ++r)
        for (int c = 0; c < p.n; ++c) {
          double& d = C[(size_t)r * p.ldc + c];
          d = p.beta ? d + acc[(size_t)r * p.n + c] : acc[(size_t)r * p.n + c];
        }
    }
  }
  void run(const Launch& l, uint64_t psi, uint64_t sig) override { exec(l, psi, sig); }
  void upload(uint64_t dst, const double* h, int64_t n) override { std::memcpy(ptr(dst), h, (size_t)n * 8); }
  void download(double* h, uint64_t src, int64_t n) override { std::memcpy(h, ptr(src), (size_t)n * 8); }
  void zero(uint64_t p, int64_t n) override { std::fill(ptr(p), ptr(p) + n, 0.0); }
  void randn(uint64_t, int64_t, uint64_t) override { throw std::runtime_error("not needed"); }
  void orthonormal_cols(uint64_t, int, int) override { throw std::runtime_error("not needed"); }
  double dot(uint64_t x, uint64_t y, int64_t n) override {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += ptr(x)[i] * ptr(y)[i];
    return s;
  }
  void scale(uint64_t x, double a, int64_t n) override {
    for (int64_t i = 0; i < n; ++i) ptr(x)[i] *= a;
  }
  void axpby(uint64_t y, double a, uint64_t x, double b, int64_t n) override {
    for (int64_t i = 0; i < n; ++i) ptr(y)[i] = a * ptr(x)[i] + b * ptr(y)[i];
  }
  void precond(uint64_t t, uint64_t r, uint64_t d, double theta, double fl, int64_t n) override {
    for (int64_t i = 0; i < n; ++i) {
      double den = ptr(d)[i] - theta;
      if (std::fabs(den) < fl) den = den < 0 ? -fl : fl;
      ptr(t)[i] = ptr(r)[i] / den;
    }
  }
  // symmetric eigendecomposition by cyclic Jacobi rotations: A (n x n,
  // column-major) becomes the eigenvectors, w the ascending eigenvalues
  void eigh(uint64_t a, int n, double* w) override {
    double* A = ptr(a);
    std::vector<double> M((size_t)n * n), Vv((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) M[(size_t)i * n + j] = 0.5 * (A[(size_t)j * n + i] + A[(size_t)i * n + j]);
    for (int i = 0; i < n; ++i) Vv[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
      double off = 0, tot = 0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          const double x = M[(size_t)i * n + j] * M[(size_t)i * n + j];
          tot += x;
          if (i != j) off += x;
        }
      if (off <= 1e-30 * std::max(tot, 1e-300)) break;
      for (int p = 0; p < n; ++p)
        for (int q = p + 1; q < n; ++q) {
          const double apq = M[(size_t)p * n + q];
          if (apq == 0.0) continue;
          const double app = M[(size_t)p * n + p], aqq = M[(size_t)q * n + q];
          const double tau = (aqq - app) / (2.0 * apq);
          const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
          const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
          for (int k = 0; k < n; ++k) {  // rows p, q
            const double mpk = M[(size_t)p * n + k], mqk = M[(size_t)q * n + k];
            M[(size_t)p * n + k] = c * mpk - s * mqk;
            M[(size_t)q * n + k] = s * mpk + c * mqk;
          }
          for (int k = 0; k < n; ++k) {  // columns p, q
            const double mkp = M[(size_t)k * n + p], mkq = M[(size_t)k * n + q];
            M[(size_t)k * n + p] = c * mkp - s * mkq;
            M[(size_t)k * n + q] = s * mkp + c * mkq;
          }
          for (int k = 0; k < n; ++k) {
            const double vkp = Vv[(size_t)k * n + p], vkq = Vv[(size_t)k * n + q];
            Vv[(size_t)k * n + p] = c * vkp - s * vkq;
            Vv[(size_t)k * n + q] = s * vkp + c * vkq;
          }
        }
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return M[(size_t)x * n + x] < M[(size_t)y * n + y]; });
    for (int j = 0; j < n; ++j) {
      w[j] = M[(size_t)ord[j] * n + ord[j]];
      for (int i = 0; i < n; ++i) A[(size_t)j * n + i] = Vv[(size_t)i * n + ord[j]];
    }
  }
  void copy(uint64_t d, uint64_t s, int64_t n) override { std::memcpy(ptr(d), ptr(s), (size_t)n * 8); }
  uint64_t host_alloc(int64_t) override { throw std::runtime_error("not needed"); }
  void host_free(uint64_t) override {}
  void d2h(uint64_t, uint64_t, int64_t) override {}
  void h2d_async(uint64_t, uint64_t, int64_t) override {}
  void copies_join() override {}
  double copies_wait_seconds() override { return 0.0; }
  int64_t live_bytes() const override { return live; }
};

struct HostRunner : PreparedRunner {
  HostEx* ex;
  std::vector<Launch> prepared;
  explicit HostRunner(HostEx* e) : ex(e) {}
  int prepare(const Launch& l) override {
    prepared.push_back(l);
    return (int)prepared.size() - 1;
  }
  void drop_prepared() override { prepared.clear(); }
  void run_prepared(int h, uint64_t psi, uint64_t sig, void*, int prec) override {
    if (prec != 0) throw std::runtime_error("host execution runs the FP64 task lists only");
    ex->exec(prepared.at(h), psi, sig);
  }
  int take_error() override { return 0; }
  const void* prepared_handle(int) const override { return nullptr; }
  void tile_counts(int, int64_t c[5]) const override { for (int i = 0; i < 5; ++i) c[i] = 0; }
  void* stream() override { return nullptr; }
  void sync(void*) override {}
  void zero_async(uint64_t p, int64_t n, void*) override { ex->zero(p, n); }
  int64_t bytes_allocated() const override { return ex->live; }
  // The BF16 forms are emulated for the Davidson policy tests: the FP64 task
  // lists of the centre (prepared in stage order), then every element of sigma perturbed by a relative
  // amount uniform in [-u, u] (u = 2^-9 for BF16, 2^-18 for the split form),
  // from a counter-based hash of the element and of the call.
  int planes = 0;
  uint64_t calls = 0;
  void prepare_tiled(const TiledPlan&, int p) override { planes = p; }
  void set_tiled_items(const TiledPlan&) override {}
  int tiled_planes() const override { return planes; }
  double time_tiled(uint64_t, uint64_t, int, int) override { return 0.0; }
  void run_tiled(uint64_t psi, uint64_t sig, void*, int prec) override {
    for (const Launch& l : prepared) ex->exec(l, psi, sig);
    const double u = prec == 2 ? std::ldexp(1.0, -9) : std::ldexp(1.0, -18);
    double* s = reinterpret_cast<double*>(sig);
    const int64_t n = ex->size_of(sig);
    ++calls;
    for (int64_t i = 0; i < n; ++i) {
      uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull ^ (calls * 0xBF58476D1CE4E5B9ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double r = (double)(z >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
      s[i] *= 1.0 + u * (2.0 * r - 1.0);
    }
  }
};

// value of element (r, c) of a view (scaled, possibly transposed, or a scaled identity)
double view_at(const TView& v, int r, int c, const double* psi) {
  if (r >= v.rows || c >= v.cols) return 0.0;
  if (v.src == 0 && v.buf == 0) return r == c ? v.scale : 0.0;
  const double* s = v.buf ? psi + v.src : reinterpret_cast<const double*>(v.src);
  return v.scale * (v.tr ? s[(size_t)c * v.ld + r] : s[(size_t)r * v.ld + c]);
}

// sigma of the tiled work items evaluated in FP64
std::vector<double> tiled_sigma(const HeffPlan& plan, const PsiLayout& lay, const double* psi, const TileCfg& cfg,
                                int64_t tbudget, int* npasses) {
  const TiledPlan T = plan_tiled(plan, lay, cfg, tbudget);
  if (npasses) *npasses = T.npasses();
  std::map<int64_t, const TView*> A, B, Ps;  // arena offset of a view -> view
  for (auto& v : T.avw) A[v.dst] = &v;
  for (auto& v : T.bvw) B[v.dst] = &v;
  for (auto& v : T.psivw) Ps[v.dst] = &v;
  std::vector<double> sig((size_t)lay.size, 0.0);
  // pass by pass: the T arena offsets of a pass are its own (rebased), so the
  // T_t of one pass are forgotten before the next pass writes its own
  for (int pass = 0; pass < T.npasses(); ++pass) {
  std::map<int64_t, std::vector<double>> Tt;  // T arena offset -> T_t^T (ntot x mtot, row-major)
  std::map<int64_t, int> Tcols;
  for (int ii = T.pass1[pass]; ii < T.pass1[pass + 1]; ++ii) {
    const K1Item& it = T.i1[ii];
    const int c8 = tiled_c8(it.k);
    const TView* pv = Ps.at(it.b - (int64_t)it.np * (TP_B / 8) * c8 * 128);
    for (int vi = it.v0; vi < it.v0 + it.nv; ++vi) {
      const K1View& w = T.v1[vi];
      const TView* rv = B.at(w.a - (int64_t)w.mp * (TP_A / 8) * c8 * 128);
      auto& M = Tt[w.tout];
      if (M.empty()) {
        M.assign((size_t)w.ntot * it.mtot, 0.0);
        Tcols[w.tout] = it.mtot;
      }
      for (int r = 0; r < w.mrows; ++r) {
        const int R = w.mp * TP_A + r;
        for (int x = 0; x < it.nrows; ++x) {
          const int X = it.np * TP_B + x;
          double s = 0;
          for (int y = 0; y < it.k; ++y) s += view_at(*rv, R, y, psi) * view_at(*pv, X, y, psi);
          M[(size_t)R * it.mtot + X] = w.osc * s;
        }
      }
    }
  }
  for (int ii = T.pass2[pass]; ii < T.pass2[pass + 1]; ++ii) {
    const K2Item& it = T.i2[ii];
    for (int s = it.s0; s < it.s1; ++s) {
      const K2Seg& g = T.s2[s];
      const TView* av = A.at(g.a);
      const auto& M = Tt.at(g.b);
      const int K = Tcols.at(g.b);
      for (int r = 0; r < it.mrows; ++r)
        for (int c = 0; c < it.nrows; ++c) {
          const int R = it.mp * TP_A + r, C = it.np * TP_B + c;
          double acc = 0;
          for (int k = 0; k < g.k; ++k) acc += view_at(*av, R, k, psi) * M[(size_t)C * K + k];
          sig[(size_t)it.out + (size_t)R * it.ldc + C] += acc;
        }
    }
  }
  }
  return sig;
}

template <class T>
void rd(FILE* f, T* p, size_t n) {
  if (std::fread(p, sizeof(T), n, f) != n) throw std::runtime_error("short input");
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  try {
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) throw std::runtime_error("cannot open input");
    int64_t hd[7];
    rd(f, hd, 7);
    const int L = (int)hd[0];
    std::vector<double> h((size_t)L * L), V((size_t)L * L * L * L), data((size_t)hd[6]);
    std::vector<int> nsec((size_t)hd[4]), sec((size_t)hd[5]);
    rd(f, h.data(), h.size());
    rd(f, V.data(), V.size());
    rd(f, nsec.data(), nsec.size());
    rd(f, sec.data(), sec.size());
    rd(f, data.data(), data.size());
    std::fclose(f);

    HostEx ex;
    HostRunner pr(&ex);
    Engine E;
    E.ex = &ex;
    E.pr = &pr;
    E.tmp_budget = (int64_t)(2e9 / 8);
    if (const char* sw = std::getenv("HOST_EXEC_PAIR_SWITCH")) E.pair_switch = std::atoi(sw);
    if (const char* sg = std::getenv("HOST_EXEC_SUM_GEMM")) E.sum_gemm = std::atoi(sg);
    E.I.L = L;
    E.I.h = h;
    E.I.V = V;
    E.N = (int)hd[1];
    E.two_s = (int)hd[2];
    const int c = (int)hd[3];
    if (const char* s2 = std::getenv("HOST_EXEC_SU2")) E.su2 = std::atoi(s2) != 0;
    // import, as the C ABI does: bond sectors, site tensors per product sector, psi
    std::vector<Basis> bonds(L + 1);
    for (auto& b : bonds) b.su2 = E.su2;
    int pos = 0;
    for (int b = 0; b <= L; ++b)
      for (int s = 0; s < nsec[b]; ++s, ++pos) bonds[b].add(QN{sec[3 * pos], sec[3 * pos + 1]}, sec[3 * pos + 2]);
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
        const int t = to.find(pb.prod.q[q]);
        if (t < 0) continue;
        so[q] = tot;
        nb[q] = t;
        tot += (int64_t)pb.prod.dim[q] * to.dim[t];
      }
      const uint64_t dev = ex.alloc(tot);
      ex.upload(dev, data.data() + off, tot);
      off += (size_t)tot;
      E.site[p] = dev;
      E.site_off[p] = so;
      E.site_nb[p] = nb;
    };
    for (int p = 0; p < c; ++p) take_site(p, bonds[p], true, bonds[p + 1]);
    for (int p = c + 2; p < L; ++p) take_site(p, bonds[p + 1], false, bonds[p]);
    E.bonds = bonds;
    E.L = L;
    E.center = c;
    E.set_psi_host(std::vector<double>(data.begin() + (long)off, data.end()));
    E.build_env();
    if (argc >= 7 && std::string(argv[3]) == "sweep") {
      const int D = std::atoi(argv[4]), nsw = std::atoi(argv[5]);
      DavOpts o;
      o.tol = std::atof(argv[6]);
      // optional dynamic block-state selection: eps and D_min
      const double eps = argc >= 8 ? std::atof(argv[7]) : 0.0;
      const int dmin = argc >= 9 ? std::atoi(argv[8]) : 1;
      while (E.center > 0) E.truncate_move(1 << 30, -1, 1e-28);
      std::vector<double> energies;
      int maxk = 0, sumk = 0;
      for (int sw = 0; sw < nsw; ++sw) {
        double e = 0.0;
        for (int l = 0; l < L - 2; ++l) {
          e = E.davidson(o).energy;
          int k = 0;
          E.truncate_move(D, +1, 0.0, eps, dmin, &k);
          maxk = std::max(maxk, k);
          sumk += k;
        }
        for (int l = L - 2; l > 0; --l) {
          e = E.davidson(o).energy;
          int k = 0;
          E.truncate_move(D, -1, 0.0, eps, dmin, &k);
          maxk = std::max(maxk, k);
          sumk += k;
        }
        energies.push_back(e);
      }
      if (eps > 0.0) {
        energies.push_back((double)maxk);
        energies.push_back((double)sumk);
      }
      FILE* o2 = std::fopen(argv[2], "wb");
      if (!o2) throw std::runtime_error("cannot open output");
      std::fwrite(energies.data(), 8, energies.size(), o2);
      std::fclose(o2);
      return 0;
    }
    if (argc >= 7 && std::string(argv[3]) == "sweepgamma") {
      // nsw sweeps (fixed D), then the 2-RDM by the walk; out: the last energy, then Gamma
      const int D = std::atoi(argv[4]), nsw = std::atoi(argv[5]);
      DavOpts o;
      o.tol = std::atof(argv[6]);
      while (E.center > 0) E.truncate_move(1 << 30, -1, 1e-28);
      double e = 0.0;
      for (int sw = 0; sw < nsw; ++sw) {
        for (int l = 0; l < L - 2; ++l) {
          e = E.davidson(o).energy;
          E.truncate_move(D, +1, 0.0);
        }
        for (int l = L - 2; l > 0; --l) {
          e = E.davidson(o).energy;
          E.truncate_move(D, -1, 0.0);
        }
      }
      const std::vector<double> g = E.rdm2_sweep();
      FILE* o11 = std::fopen(argv[2], "wb");
      if (!o11) throw std::runtime_error("cannot open output");
      std::fwrite(&e, 8, 1, o11);
      std::fwrite(g.data(), 8, g.size(), o11);
      std::fclose(o11);
      return 0;
    }
    if (argc >= 7 && std::string(argv[3]) == "sweeprdm") {
      // nsw sweeps (as in "sweep", fixed D), then the two-orbital density matrices of
      // the final state; out: one energy per sweep, then L*L blocks of 256
      const int D = std::atoi(argv[4]), nsw = std::atoi(argv[5]);
      DavOpts o;
      o.tol = std::atof(argv[6]);
      while (E.center > 0) E.truncate_move(1 << 30, -1, 1e-28);
      std::vector<double> out;
      for (int sw = 0; sw < nsw; ++sw) {
        double e = 0.0;
        for (int l = 0; l < L - 2; ++l) {
          e = E.davidson(o).energy;
          E.truncate_move(D, +1, 0.0);
        }
        for (int l = L - 2; l > 0; --l) {
          e = E.davidson(o).energy;
          E.truncate_move(D, -1, 0.0);
        }
        out.push_back(e);
      }
      const std::vector<double> r = E.orbital_rdm2();
      out.insert(out.end(), r.begin(), r.end());
      FILE* o10 = std::fopen(argv[2], "wb");
      if (!o10) throw std::runtime_error("cannot open output");
      std::fwrite(out.data(), 8, out.size(), o10);
      std::fclose(o10);
      return 0;
    }
    if (argc >= 7 && std::string(argv[3]) == "warmup") {
      // the warm-up half sweep from the imported centre to (0, 1) (as qcdmrg_sweep_left),
      // then nsw full sweeps (as qcdmrg_sweep); out: the energy of the first solve, the
      // energy at the end of the half sweep, then one energy per full sweep
      const int D = std::atoi(argv[4]), nsw = std::atoi(argv[5]);
      DavOpts o;
      o.tol = std::atof(argv[6]);
      std::vector<double> energies;
      double e = 0.0;
      bool first = true;
      while (E.center > 0) {
        e = E.davidson(o).energy;
        if (first) energies.push_back(e);
        first = false;
        E.truncate_move(D, -1, 0.0);
      }
      energies.push_back(e);
      for (int sw = 0; sw < nsw; ++sw) {
        for (int l = 0; l < L - 2; ++l) {
          e = E.davidson(o).energy;
          E.truncate_move(D, +1, 0.0);
        }
        for (int l = L - 2; l > 0; --l) {
          e = E.davidson(o).energy;
          E.truncate_move(D, -1, 0.0);
        }
        energies.push_back(e);
      }
      FILE* o9 = std::fopen(argv[2], "wb");
      if (!o9) throw std::runtime_error("cannot open output");
      std::fwrite(energies.data(), 8, energies.size(), o9);
      std::fclose(o9);
      return 0;
    }
    if (argc >= 4 && std::string(argv[3]) == "davidson") {
      // FP64 Davidson and the mixed policy (emulated BF16 forms) from the same start
      const std::vector<double> psi0 = E.get_psi_host();
      DavOpts o;
      o.tol = 1e-8;
      DavResult r0, r1;
      if (std::getenv("HOST_EXEC_MIXED_FIRST")) {
        o.policy = 1;
        r1 = E.davidson(o);
        E.set_psi_host(psi0);
        o.policy = 0;
        r0 = E.davidson(o);
      } else {
        r0 = E.davidson(o);
        E.set_psi_host(psi0);
        o.policy = 1;
        r1 = E.davidson(o);
      }
      std::vector<double> out = {r0.energy, r1.energy, r0.resid, r1.resid, (double)r0.converged,
                                 (double)r1.converged, (double)r0.hpsi[0], (double)r1.hpsi[0], (double)r1.hpsi[2],
                                 (double)r1.hpsi[3], r1.energy_mixed};
      FILE* o5 = std::fopen(argv[2], "wb");
      if (!o5) throw std::runtime_error("cannot open output");
      std::fwrite(out.data(), 8, out.size(), o5);
      std::fclose(o5);
      return 0;
    }
    if (argc >= 5 && std::string(argv[3]) == "moveto") {
      // exact centre moves to sites (t, t+1) for each t of a comma-separated
      // list in turn, then psi and sigma at the last one
      std::string ts = argv[4];
      size_t pos = 0;
      while (pos <= ts.size()) {
        const size_t e = ts.find(',', pos);
        const int t = std::atoi(ts.substr(pos, e == std::string::npos ? std::string::npos : e - pos).c_str());
        while (E.center > t) E.truncate_move(1 << 30, -1, 1e-28);
        while (E.center < t) E.truncate_move(1 << 30, +1, 1e-28);
        if (e == std::string::npos) break;
        pos = e + 1;
      }
      const int64_t n2 = E.lay.size;
      const uint64_t sg2 = ex.alloc(n2);
      E.heff(E.dpsi, sg2, nullptr, 0);
      std::vector<double> ps((size_t)n2), sv((size_t)n2);
      ex.download(ps.data(), E.dpsi, n2);
      ex.download(sv.data(), sg2, n2);
      FILE* o7 = std::fopen(argv[2], "wb");
      if (!o7) throw std::runtime_error("cannot open output");
      std::fwrite(ps.data(), 8, ps.size(), o7);
      std::fwrite(sv.data(), 8, sv.size(), o7);
      std::fclose(o7);
      return 0;
    }
    if (argc >= 4 && std::string(argv[3]) == "rdm2sweep") {
      const std::vector<double> g = E.rdm2_sweep();
      FILE* o4 = std::fopen(argv[2], "wb");
      if (!o4) throw std::runtime_error("cannot open output");
      std::fwrite(g.data(), 8, g.size(), o4);
      // then sigma at the centre the walk returned to, to check that the state is unchanged
      const int64_t n2 = E.lay.size;
      const uint64_t sg2 = ex.alloc(n2);
      E.heff(E.dpsi, sg2, nullptr, 0);
      std::vector<double> ps((size_t)n2), sv((size_t)n2);
      ex.download(ps.data(), E.dpsi, n2);
      ex.download(sv.data(), sg2, n2);
      std::fwrite(ps.data(), 8, ps.size(), o4);
      std::fwrite(sv.data(), 8, sv.size(), o4);
      std::fclose(o4);
      return 0;
    }
    if (argc >= 4 && std::string(argv[3]) == "orbrdm") {
      const std::vector<double> g = E.orbital_rdm2();
      FILE* o8 = std::fopen(argv[2], "wb");
      if (!o8) throw std::runtime_error("cannot open output");
      std::fwrite(g.data(), 8, g.size(), o8);
      // then psi and sigma at the centre the walk returned to
      const int64_t n8 = E.lay.size;
      const uint64_t sg8 = ex.alloc(n8);
      E.heff(E.dpsi, sg8, nullptr, 0);
      std::vector<double> ps8((size_t)n8), sv8((size_t)n8);
      ex.download(ps8.data(), E.dpsi, n8);
      ex.download(sv8.data(), sg8, n8);
      std::fwrite(ps8.data(), 8, ps8.size(), o8);
      std::fwrite(sv8.data(), 8, sv8.size(), o8);
      ex.release(sg8);
      std::fclose(o8);
      return 0;
    }
    if (argc >= 4 && std::string(argv[3]) == "rdm2") {
      const std::vector<double> g = E.rdm2();
      FILE* o6 = std::fopen(argv[2], "wb");
      if (!o6) throw std::runtime_error("cannot open output");
      std::fwrite(g.data(), 8, g.size(), o6);
      std::fclose(o6);
      return 0;
    }
    if (argc >= 4 && std::string(argv[3]) == "rdm1") {
      const std::vector<double> g = E.rdm1();
      FILE* o3 = std::fopen(argv[2], "wb");
      if (!o3) throw std::runtime_error("cannot open output");
      std::fwrite(g.data(), 8, g.size(), o3);
      std::fclose(o3);
      return 0;
    }
    const int64_t n = E.lay.size;
    if ((size_t)n != data.size() - off) throw std::runtime_error("psi layout differs from the input");
    const uint64_t sig = ex.alloc(n);
    E.heff(E.dpsi, sig, nullptr, 0);
    std::vector<double> s64((size_t)n);
    ex.download(s64.data(), sig, n);
    TileCfg cfg;
    cfg.kmax = 8;  // small: many split stage-2 items
    cfg.width = 128;
    int64_t tb = 0;
    if (const char* e = std::getenv("HOST_EXEC_T_BUDGET")) tb = std::atoll(e);
    int npasses = 1;
    std::vector<double> st = tiled_sigma(E.plan, E.lay, reinterpret_cast<const double*>(E.dpsi), cfg, tb, &npasses);
    std::fprintf(stderr, "heff_flops=%.0f\n", E.plan.flops);
    std::fprintf(stderr, "tiled_passes=%d\n", npasses);
    FILE* o = std::fopen(argv[2], "wb");
    if (!o) throw std::runtime_error("cannot open output");
    std::fwrite(s64.data(), 8, s64.size(), o);
    std::fwrite(st.data(), 8, st.size(), o);
    std::fclose(o);
  } catch (const std::exception& e) {
    std::fprintf(stderr, "host_exec: %s\n", e.what());
    return 1;
  }
  return 0;
}
