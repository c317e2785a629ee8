// Sweep engine: environment build, H_eff psi, Davidson with FP64 control and a
// precision policy, density-matrix truncation, renormalization and the
// two-site wavefunction transformation that moves the centre.
#include "engine.hpp"
#include "su2.hpp"
#include "su2expand.hpp"

#include <algorithm>
#include <climits>
#include <deque>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <stdexcept>
#include <array>
#include <tuple>

namespace qd {

namespace {

constexpr double TIE_REL = 1e-8;  // relative width of a group of equal weights at the cut
// density-matrix eigenvalues at or below this are rounding noise (absolute
// error ~1e-16 of the unit trace) and are always discarded
constexpr double WEIGHT_FLOOR = 1e-14;

EnvBlock vacuum(bool left, int cut, bool su2) {
  EnvBlock b;
  b.left = left;
  b.cut = cut;
  b.basis.su2 = su2;
  b.basis.add(QN{0, 0}, 1);
  return b;
}

// Jacobi eigensolver for the small symmetric subspace matrix (n <= 64):
// eigenvalues ascending in w, eigenvectors as columns of V (n x n, row-major).
void small_eigh(const std::vector<double>& A0, int n, std::vector<double>& w, std::vector<double>& V) {
  std::vector<double> A(A0);
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        double th = 0.5 * std::atan2(2 * apq, aqq - app);
        double c = std::cos(th), s = std::sin(th);
        for (int k = 0; k < n; ++k) {
          double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
  w.resize(n);
  std::vector<double> W((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]];
    for (int k = 0; k < n; ++k) W[(size_t)k * n + j] = V[(size_t)k * n + ord[j]];
  }
  V.swap(W);
}

// site multiplet of a coupling channel (SU(2)): 0 |0>, 1 the doublet, 2 |updn>
inline int site_mult(int ch) { return ch == 0 ? 0 : (ch == 3 ? 2 : 1); }
const int SITE_MULT_S[3] = {0, 1, 0};

Prob copy_prob(uint64_t dst, int m, int n, int ldc, int seg0) {
  Prob p;
  p.c = dst; p.cbuf = B_ABS; p.m = m; p.n = n; p.ldc = ldc; p.beta = 0; p.seg0 = seg0; p.nseg = 1;
  return p;
}

}  // namespace

void Engine::free_block(EnvBlock& b) {
  if (!b.evicted)
    for (auto p : b.owned) ex->release(p);
  for (auto h : b.host) ex->host_free(h);
  b.owned.clear();
  b.owned_n.clear();
  b.host.clear();
  b.evicted = false;
  b.ops.clear();
}

void Engine::evict(EnvBlock& b) {
  if (b.evicted || b.owned.empty()) return;
  ex->copies_join();   // no copy of this block may be in flight
  for (auto h : b.host) ex->host_free(h);
  b.host.clear();
  for (size_t k = 0; k < b.owned.size(); ++k) {
    uint64_t h = ex->host_alloc(b.owned_n[k]);
    ex->d2h(h, b.owned[k], b.owned_n[k]);
    d2h_bytes += 8 * b.owned_n[k];
    ex->release(b.owned[k]);
    b.host.push_back(h);
  }
  b.evicted = true;
  ++evictions;
}

void Engine::restore_async(EnvBlock& b) {
  if (!b.evicted) return;
  for (size_t k = 0; k < b.owned.size(); ++k) {
    const uint64_t old = b.owned[k], n = (uint64_t)b.owned_n[k];
    const uint64_t nw = ex->alloc(b.owned_n[k]);
    ex->h2d_async(nw, b.host[k], b.owned_n[k]);
    h2d_bytes += 8 * b.owned_n[k];
    for (auto& kv : b.ops)
      for (BRef& r : kv.second.blocks)
        if (r.ptr >= old && r.ptr < old + 8 * n) r.ptr = nw + (r.ptr - old);
    b.owned[k] = nw;
  }
  b.evicted = false;
  ++restores;
  // host copies are freed once the copies are joined (ensure_resident)
}

void Engine::ensure_resident(EnvBlock& b) {
  if (b.evicted) restore_async(b);
  ex->copies_join();
  for (auto h : b.host) ex->host_free(h);
  b.host.clear();
}

void Engine::enforce_budget_build(int cut, bool left) {
  if (hbm_budget <= 0) return;
  // during the environment build only the newest block of each side is needed
  while (ex->live_bytes() > hbm_budget) {
    EnvBlock* far = nullptr;
    if (left) {
      for (auto& kv : lenv)
        if (kv.first < cut && !kv.second.evicted && !kv.second.owned.empty()) { far = &kv.second; break; }
    } else {
      for (auto it = renv.rbegin(); it != renv.rend(); ++it)
        if (it->first > cut && !it->second.evicted && !it->second.owned.empty()) { far = &it->second; break; }
    }
    if (!far) break;
    evict(*far);
  }
}

void Engine::enforce_budget() {
  if (hbm_budget <= 0) return;
  // candidates: blocks not needed by the centre or the next move, farthest first
  while (ex->live_bytes() > hbm_budget) {
    EnvBlock* far = nullptr;
    int dist = -1;
    for (auto& kv : lenv) {
      int d = center - kv.first;
      if (kv.first < center - 1 && !kv.second.evicted && !kv.second.owned.empty() && d > dist) {
        dist = d;
        far = &kv.second;
      }
    }
    for (auto& kv : renv) {
      int d = kv.first - (center + 2);
      if (kv.first > center + 3 && !kv.second.evicted && !kv.second.owned.empty() && d > dist) {
        dist = d;
        far = &kv.second;
      }
    }
    if (!far) break;
    evict(*far);
  }
}

void Engine::free_enlarged(Enlarged& e) {
  for (auto p : e.owned) ex->release(p);
  e.owned.clear();
  e.ops.clear();
}

void Engine::clear_env() {
  if (!ex) return;
  for (auto& kv : lenv) free_block(kv.second);
  for (auto& kv : renv) free_block(kv.second);
  lenv.clear();
  renv.clear();
  free_enlarged(Lp);
  free_enlarged(Rp);
  if (pr) pr->drop_prepared();
  prepared.clear();
  if (ddiag) ex->release(ddiag);
  ddiag = 0;
  have_env = false;
}

void Engine::clear() {
  if (!ex) return;
  clear_env();
  for (auto p : site)
    if (p) ex->release(p);
  site.clear();
  if (dpsi) ex->release(dpsi);
  dpsi = 0;
  if (dones) ex->release(dones);
  dones = 0;
  ones_n = 0;
  center = -1;
}

void Engine::set_psi_host(const std::vector<double>& h) {
  if (dpsi) ex->release(dpsi);
  dpsi = ex->alloc(std::max<size_t>(1, h.size()));
  ex->upload(dpsi, h.data(), (int64_t)h.size());
}

std::vector<double> Engine::get_psi_host() {
  ProdBasis a = make_prod(bonds[center], true), b = make_prod(bonds[center + 2], false);
  PsiLayout l = make_psi_layout(a, b, QN{N, two_s});
  std::vector<double> h(l.size);
  if (l.size) ex->download(h.data(), dpsi, l.size);
  return h;
}

void Engine::build_env() {
  auto t0 = std::chrono::steady_clock::now();
  clear_env();
  double fl = 0;
  lenv[0] = vacuum(true, 0, su2);
  lenv[0].normal = normal_at(true, 0);
  for (int p = 0; p < center; ++p) {
    Enlarged E;
    E.batched = batched_sums();
    if (su2) enlarge_su2(lenv[p], I, *ex, E, normal_at(true, p + 1));
    else enlarge(lenv[p], I, *ex, E, &fl, normal_at(true, p + 1));
    EnvBlock nb;
    nb.cut = p + 1;
    renormalize(E, bonds[p + 1], site_nb[p], site[p], site_off[p], *ex, nb, tmp_budget, &fl);
    free_enlarged(E);
    lenv[p + 1] = nb;
    enforce_budget_build(p + 1, true);
  }
  renv[L] = vacuum(false, L, su2);
  renv[L].normal = normal_at(false, L);
  for (int p = L - 1; p >= center + 2; --p) {
    Enlarged E;
    E.batched = batched_sums();
    E.local = keep_local && !su2;
    if (su2) enlarge_su2(renv[p + 1], I, *ex, E, normal_at(false, p));
    else enlarge(renv[p + 1], I, *ex, E, &fl, normal_at(false, p));
    EnvBlock nb;
    nb.cut = p;
    renormalize(E, bonds[p], site_nb[p], site[p], site_off[p], *ex, nb, tmp_budget, &fl);
    free_enlarged(E);
    renv[p] = nb;
    enforce_budget_build(p, false);
  }
  env_flops = fl;
  prepare_center();
  env_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void Engine::prepare_center() {
  free_enlarged(Lp);
  free_enlarged(Rp);
  if (pr) pr->drop_prepared();
  prepared.clear();
  double fl = 0;
  ensure_resident(lenv.at(center));
  ensure_resident(renv.at(center + 2));
  Lp.batched = Rp.batched = batched_sums();
  if (su2) {
    enlarge_su2(lenv.at(center), I, *ex, Lp, normal_at(true, center + 1));
    enlarge_su2(renv.at(center + 2), I, *ex, Rp, normal_at(false, center + 1));
  } else {
    enlarge(lenv.at(center), I, *ex, Lp, &fl, normal_at(true, center + 1));
    enlarge(renv.at(center + 2), I, *ex, Rp, &fl, normal_at(false, center + 1));
  }
  lay = make_psi_layout(Lp.pb, Rp.pb, QN{N, two_s});
  plan = plan_heff(Lp, Rp, lay, I, tmp_budget);
  ex->tmp(std::max<int64_t>(1, plan.tmp_elems));
  for (size_t k = 0; k < plan.stage1.size(); ++k) {
    // stage 1 of a chunk is prepared before its stage 2 (runners may replay in handle order)
    const int h1 = pr->prepare(plan.stage1[k]);
    const int h2 = pr->prepare(plan.stage2[k]);
    prepared.emplace_back(h1, h2);
  }
  int64_t mx = 1;
  for (int d : lenv.at(center).basis.dim) mx = std::max<int64_t>(mx, d);
  for (int d : renv.at(center + 2).basis.dim) mx = std::max<int64_t>(mx, d);
  if (mx > ones_n) {
    if (dones) ex->release(dones);
    std::vector<double> one(mx, 1.0);
    dones = ex->alloc(mx);
    ex->upload(dones, one.data(), mx);
    ones_n = mx;
  }
  diag_launch = plan_diag(Lp, Rp, lay, I, dones);
  if (ddiag) ex->release(ddiag);
  ddiag = ex->alloc(std::max<int64_t>(1, lay.size));
  ex->run(diag_launch, 0, ddiag);
  have_env = true;
}

void Engine::heff(uint64_t psi, uint64_t sig, void* stream, int prec) {
  pr->zero_async(sig, lay.size, stream);
  if (prec == 2 || prec == 3) {
    // BF16 forms: bf16 operand mirrors fed to the tensor cores by bulk copies
    // the mixed Davidson policy prepares the three planes of the split once:
    // the BF16 form reads plane 0, which is the same round-to-nearest bf16
    const int planes = (prec == 3 || mixed_planes) ? 3 : 1;
    if (pr->tiled_planes() < planes) {
      TiledPlan tp = plan_tiled(plan, lay, tcfg);
      tiled_tbudget = tiled_t_bytes(planes, tp);
      if (tiled_tbudget > 0) tp = plan_tiled(plan, lay, tcfg, tiled_tbudget);
      tiled_passes = tp.npasses();
      tiled_t_plane = tp.tbytes;
      pr->prepare_tiled(tp, planes);
      pr->set_tiled_chunk(tcfg.chunk);
      if (autotune) {
        tune_tiled(psi, sig, prec);
        pr->zero_async(sig, lay.size, stream);
      }
    }
    pr->run_tiled(psi, sig, stream, prec);
    return;
  }
  for (auto& h : prepared) {
    pr->run_prepared(h.first, psi, sig, stream, prec);
    pr->run_prepared(h.second, psi, sig, stream, prec);
  }
}

// T arena of the tiled path: one pass when the operand mirrors and every T_t
// of the product fit the free device memory with a 4 GB margin (for the
// Davidson vectors and the other work of a step); otherwise the T_t are split
// into passes of the bytes left. QCDMRG_TILED_T_BYTES (bytes of one plane)
// sets the budget instead, to exercise the passes on small problems.
int64_t Engine::tiled_t_bytes(int planes, const TiledPlan& full) {
  if (const char* e = std::getenv("QCDMRG_TILED_T_BYTES")) {
    const long long v = std::atoll(e);
    if (v > 0) return (int64_t)v;
  }
  const int64_t free = pr->free_device_bytes();
  if (free == INT64_MAX) return 0;
  const int64_t margin = (int64_t)4 << 30;
  const int64_t mirrors = (full.abytes + full.bbytes + full.psibytes) * planes;
  if (mirrors + full.tbytes * planes + margin <= free) return 0;
  const int64_t left = (free - margin - mirrors) / planes;
  if (left < ((int64_t)64 << 20))
    throw std::runtime_error("tiled path: the bf16 operand mirrors leave no room for the stage-1 intermediates");
  return left;
}

// Autotuner of the bf16 tensor-core path. Phase 1 times every candidate
// work-item shape on this centre's task lists (the operand mirrors stay; only
// the items change); phase 2 times chunk byte targets of the kernels with the
// best items (no re-planning: the target is a kernel argument). The choice is
// cached per device and problem class: precision, psi size to a factor of two,
// and two coarse features of the block-size histogram (flops per psi element,
// which grows with the typical block dimension, and the number of stage-2
// problems, to a factor of two each), so the centres of a sweep at the same
// bond dimension and block structure are tuned once or twice, not at every step.
void Engine::tune_tiled(uint64_t psi, uint64_t sig, int prec) {
  static std::mutex mu;
  static std::map<std::array<int, 5>, TileCfg> cache;
  auto lg2 = [](double v) {
    int l = 0;
    while (v > 1.0 && l < 62) {
      v *= 0.5;
      ++l;
    }
    return l;
  };
  size_t nprob2 = 0;
  for (const Launch& l : plan.stage2) nprob2 += l.probs.size();
  const std::array<int, 5> key = {device, prec, lg2((double)lay.size), lg2(plan.flops / std::max<int64_t>(1, lay.size)),
                                  lg2((double)nprob2)};
  auto same_items = [](const TileCfg& a, const TileCfg& b) { return a.kmax == b.kmax && a.width == b.width; };
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      if (!same_items(it->second, tcfg)) pr->set_tiled_items(plan_tiled(plan, lay, it->second, tiled_tbudget));
      tcfg = it->second;
      pr->set_tiled_chunk(tcfg.chunk);
      return;
    }
  }
  auto t0 = std::chrono::steady_clock::now();
  // BF16x3 keeps the FP32 accumulation of one item to K <= 4096
  std::vector<TileCfg> cands = {{4096, TP_B, 0}, {1024, TP_B, 0}, {4096, 128, 0}, {1024, 128, 0}};
  if (prec != 3) cands.push_back({1 << 30, TP_B, 0});
  TileCfg loaded = tcfg, best = tcfg;
  pr->set_tiled_chunk(0);
  double tbest = 1e30;
  for (const TileCfg& c : cands) {
    if (!same_items(c, loaded)) {
      pr->set_tiled_items(plan_tiled(plan, lay, c, tiled_tbudget));
      loaded = c;
    }
    const double t = pr->time_tiled(psi, sig, prec, 2);
    if (t < tbest) {
      tbest = t;
      best = c;
    }
  }
  if (!same_items(best, loaded)) pr->set_tiled_items(plan_tiled(plan, lay, best, tiled_tbudget));
  for (int chunk : {32768, 49152, 65536}) {
    pr->set_tiled_chunk(chunk);
    const double t = pr->time_tiled(psi, sig, prec, 2);
    if (t < tbest) {
      tbest = t;
      best.chunk = chunk;
    }
  }
  pr->set_tiled_chunk(best.chunk);
  tcfg = best;
  {
    std::lock_guard<std::mutex> g(mu);
    cache[key] = best;
  }
  ++tunes;
  tune_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

DavResult Engine::davidson(const DavOpts& o) {
  // QCDMRG_DAV_TRACE=1 prints every iteration to stderr
  static const bool trace = std::getenv("QCDMRG_DAV_TRACE") && std::atoi(std::getenv("QCDMRG_DAV_TRACE")) != 0;
  DavResult R;
  const int64_t n = lay.size;
  if (n == 0) throw std::runtime_error("empty wavefunction");
  const int mmax = std::max(2, std::min(o.m_max, 64));
  void* st = pr->stream();
  std::vector<uint64_t> V(mmax), W(mmax);
  for (int k = 0; k < mmax; ++k) {
    V[k] = ex->alloc(n);
    W[k] = ex->alloc(n);
  }
  uint64_t x = ex->alloc(n), w = ex->alloc(n), r = ex->alloc(n), t = ex->alloc(n);
  uint64_t xp = ex->alloc(n), wp = ex->alloc(n);   // previous Ritz pair (restart)
  bool have_prev = false;
  auto cleanup = [&]() {
    for (int k = 0; k < mmax; ++k) {
      ex->release(V[k]);
      ex->release(W[k]);
    }
    ex->release(x); ex->release(w); ex->release(r); ex->release(t);
    ex->release(xp); ex->release(wp);
  };
  try {
    int prec = o.policy ? 2 : o.precision;   // policy 1 starts in BF16
    mixed_planes = o.policy != 0;
    // policy 1 after the BF16x3 phase: FP64 residual correction. Each outer
    // check applies H once in FP64 to the normalised Ritz vector (energy and
    // residual from that product); if the residual is above tol, the FP64 pair
    // (x, H x) restarts the subspace and BF16x3 products expand it (inner
    // iterations) until the mixed residual has fallen by REFINE_DROP, stalls, or
    // REFINE_MAX inner products were spent; then the next FP64 check. The
    // mixed products only have to resolve the correction, so their rounding
    // error enters relative to the residual, not to H psi.
    bool refine = false, w0_exact = false;
    double outer_rn = 0.0;
    int inner = 0;
    constexpr double REFINE_DROP = 0.03;
    const int REFINE_MAX = mmax - 2;   // inner products between checks (no restart in between)
    // rounding floors of the residual: the reduced forms compute H psi to a
    // relative accuracy of about 2^-9 (BF16) and 2^-17 (three-term split, its
    // FP32 accumulation included), so their residuals cannot fall much below
    // that fraction of |theta|
    const double FLOOR_BF16 = 8.0 * std::ldexp(1.0, -9), FLOOR_X3 = 8.0 * std::ldexp(1.0, -17);
    auto apply = [&](uint64_t in, uint64_t out) {
      heff(in, out, st, prec);
      pr->sync(st);
      if (pr->take_error()) throw std::runtime_error("tensor-core kernel wait gave up");
      R.hpsi[prec]++;
    };
    ex->copy(V[0], dpsi, n);
    double nrm = std::sqrt(ex->dot(V[0], V[0], n));
    if (nrm == 0) throw std::runtime_error("zero initial vector");
    ex->scale(V[0], 1.0 / nrm, n);
    apply(V[0], W[0]);
    int m = 1;
    std::vector<double> Hs((size_t)mmax * mmax, 0.0);
    Hs[0] = ex->dot(V[0], W[0], n);
    // classical Gram-Schmidt against V[0..k), twice (one batched dot and one
    // batched update per pass)
    auto orth = [&](uint64_t tv, int k) {
      std::vector<double> c(k);
      for (int pass = 0; pass < 2; ++pass) {
        ex->mdot(V.data(), k, tv, n, c.data());
        for (double& v : c) v = -v;
        ex->mcombine(tv, V.data(), c.data(), k, 1.0, n);
      }
    };
    double theta = Hs[0];
    std::vector<double> phase_res;   // residuals of the current precision phase
    for (int it = 0; it < o.max_iter; ++it) {
      R.iters = it + 1;
      std::vector<double> hs((size_t)m * m), ev, vec;
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) hs[(size_t)i * m + j] = 0.5 * (Hs[(size_t)i * mmax + j] + Hs[(size_t)j * mmax + i]);
      small_eigh(hs, m, ev, vec);
      theta = ev[0];
      if (it > 0) {
        ex->copy(xp, x, n);
        ex->copy(wp, w, n);
        have_prev = true;
      }
      {
        std::vector<double> y(m);
        for (int k = 0; k < m; ++k) y[k] = vec[(size_t)k * m + 0];
        ex->mcombine(x, V.data(), y.data(), m, 0.0, n);
        ex->mcombine(w, W.data(), y.data(), m, 0.0, n);
      }
      ex->copy(r, w, n);
      ex->axpby(r, -theta, x, 1.0, n);
      double rn = std::sqrt(ex->dot(r, r, n));
      R.resid = rn;
      R.energy = theta;
      int nprec = prec;
      phase_res.push_back(rn);
      if (trace) std::fprintf(stderr, "davidson it %d prec %d refine %d m %d theta %.12f resid %.3e\n", it, prec,
                              (int)refine, m, theta, rn);
      bool check = false;   // FP64 outer check of the refinement
      if (o.policy) {
        // a reduced-precision phase ends at its threshold, at its rounding
        // floor, or when its residual has stopped falling (no 10 % drop in 8
        // iterations)
        const size_t np = phase_res.size();
        const bool stalled = np > 8 && rn > 0.9 * phase_res[np - 9];
        const double at = std::fabs(theta);
        if (!refine) {
          if (prec == 2 && (rn < o.tau1 || rn < FLOOR_BF16 * at || stalled)) nprec = 3;
          if (prec == 3 && (rn < o.tau2 || rn < FLOOR_X3 * at || stalled || rn < o.tol)) check = true;
          if (prec == 2 && rn < o.tol) check = true;
        } else if (inner > 0 && (rn < REFINE_DROP * outer_rn || rn < o.tol || stalled || inner >= REFINE_MAX)) {
          check = true;
        }
      }
      if (check) {
        if (!refine) R.energy_mixed = theta;
        refine = true;
        prec = 3;
        phase_res.clear();
        inner = 0;
        double xn = std::sqrt(ex->dot(x, x, n));
        ex->copy(V[0], x, n);
        ex->scale(V[0], 1.0 / xn, n);
        {
          const int keep = prec;
          prec = 0;
          apply(V[0], W[0]);       // the FP64 product of the check
          prec = keep;
        }
        m = 1;
        Hs[0] = ex->dot(V[0], W[0], n);
        w0_exact = true;
        outer_rn = -1.0;           // set from the exact residual at the top of the loop
        have_prev = false;
        continue;
      }
      if (refine && outer_rn < 0.0) {
        // first pass after a check: x = V0 and w = W0 = H x in FP64, so theta and
        // rn are the exact Rayleigh quotient and residual
        outer_rn = rn;
        if (rn < o.tol) {
          R.converged = true;
          break;
        }
      }
      if (refine) ++inner;
      if (nprec != prec) {  // restart from the Ritz vector with the new precision
        if (prec == 3) R.energy_mixed = theta;
        prec = nprec;
        w0_exact = false;
        phase_res.clear();
        double xn = std::sqrt(ex->dot(x, x, n));
        ex->copy(V[0], x, n);
        ex->scale(V[0], 1.0 / xn, n);
        apply(V[0], W[0]);
        m = 1;
        Hs[0] = ex->dot(V[0], W[0], n);
        have_prev = false;
        continue;
      }
      if (!o.policy && rn < o.tol) {
        R.converged = true;
        break;
      }
      // correction vector: preconditioned residual, orthogonalised twice
      ex->precond(t, r, ddiag, theta, o.floor, n);
      orth(t, m);
      double tn = std::sqrt(ex->dot(t, t, n));
      if (!(tn > 1e-14)) {  // no new direction: take the residual itself
        ex->copy(t, r, n);
        orth(t, m);
        tn = std::sqrt(ex->dot(t, t, n));
        if (!(tn > 1e-14)) { R.converged = rn < o.tol; break; }
      }
      if (m == mmax) {  // restart: keep the Ritz vector and the previous one
        w0_exact = false;
        double xn = std::sqrt(ex->dot(x, x, n));
        ex->copy(V[0], x, n);
        ex->scale(V[0], 1.0 / xn, n);
        ex->copy(W[0], w, n);
        ex->scale(W[0], 1.0 / xn, n);
        m = 1;
        Hs[0] = ex->dot(V[0], W[0], n);
        if (have_prev) {  // V1 = xp - (V0.xp) V0 normalised; W1 by the same combination
          double c = ex->dot(V[0], xp, n);
          ex->copy(V[1], xp, n);
          ex->axpby(V[1], -c, V[0], 1.0, n);
          ex->copy(W[1], wp, n);
          ex->axpby(W[1], -c, W[0], 1.0, n);
          double c2 = ex->dot(V[0], V[1], n);   // second pass
          ex->axpby(V[1], -c2, V[0], 1.0, n);
          ex->axpby(W[1], -c2, W[0], 1.0, n);
          double vn = std::sqrt(ex->dot(V[1], V[1], n));
          if (vn > 1e-3) {  // W1 by cancellation is only accurate when V1 is well conditioned
            ex->scale(V[1], 1.0 / vn, n);
            ex->scale(W[1], 1.0 / vn, n);
            double h01 = ex->dot(V[0], W[1], n), h11 = ex->dot(V[1], W[1], n);
            Hs[1] = h01;
            Hs[(size_t)mmax] = h01;
            Hs[(size_t)mmax + 1] = h11;
            m = 2;
          }
        }
        orth(t, m);
        tn = std::sqrt(ex->dot(t, t, n));
      }
      ex->copy(V[m], t, n);
      ex->scale(V[m], 1.0 / tn, n);
      apply(V[m], W[m]);
      {
        // after an FP64 check W0 = H V0 is exact: the coupling of V0 with a new
        // direction is taken as V_m . (H V0) (H symmetric), whose error does not
        // swamp the small true coupling the way V0 . (H V_m) in BF16x3 would
        std::vector<double> col(m + 1);
        ex->mdot(V.data(), m + 1, W[m], n, col.data());
        if (w0_exact) col[0] = ex->dot(V[m], W[0], n);
        for (int i = 0; i <= m; ++i) {
          Hs[(size_t)i * mmax + m] = col[i];
          Hs[(size_t)m * mmax + i] = col[i];
        }
      }
      ++m;
    }
    // store the normalised Ritz vector as the new wavefunction
    double xn = std::sqrt(ex->dot(x, x, n));
    ex->copy(dpsi, x, n);
    ex->scale(dpsi, 1.0 / xn, n);
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
  return R;
}

double Engine::truncate_move(int D, int dir, double drop_below, double eps, int Dmin, int* kept) {
  // a negative drop_below keeps every weight above the rounding noise of its
  // own sector's eigenvalues (exact moves for measurements); otherwise weights
  // at the global rounding floor are always dropped
  const bool exact = drop_below < 0;
  drop_below = exact ? 0.0 : std::max(drop_below, WEIGHT_FLOOR);
  const QN target{N, two_s};
  const ProdBasis& LB = Lp.pb;
  const ProdBasis& RB = Rp.pb;
  // sector matrices: moving right, Psi_q [rows of L' sector q, columns of every
  // R' sector coupled with q to the target]; moving left, Psi_r [rows of every
  // L' sector coupled with r, columns of R' sector r]. In U(1) each sector has
  // one partner; in SU(2) an L' multiplet of spin S_a couples with R'
  // multiplets of every spin |S_a - S| .. S_a + S, and the density matrix of
  // the multiplets of a sector, Psi_q Psi_q^T, sums over all of them (the
  // weight of a multiplet is that of all its M components).
  auto couples = [&](QN a, QN b) {
    if (!su2) return a + b == target;
    return a.n + b.n == target.n && std::abs(a.s - b.s) <= target.s && a.s + b.s >= target.s;
  };
  struct Sec { int key; int rows, cols; int64_t off, roff; std::map<int, int> poff; };
  std::vector<Sec> secs;
  const ProdBasis& KB = dir > 0 ? LB : RB;   // the side that is truncated
  const ProdBasis& OB = dir > 0 ? RB : LB;   // its partners
  std::vector<int> sec_of(KB.prod.nsec(), -1);
  int64_t tot = 0, rtot = 0;
  for (int kq = 0; kq < KB.prod.nsec(); ++kq) {
    Sec s;
    s.key = kq;
    int pdim = 0;
    for (int oq = 0; oq < OB.prod.nsec(); ++oq)
      if (dir > 0 ? couples(KB.prod.q[kq], OB.prod.q[oq]) : couples(OB.prod.q[oq], KB.prod.q[kq])) {
        s.poff[oq] = pdim;
        pdim += OB.prod.dim[oq];
      }
    if (s.poff.empty()) continue;
    s.rows = dir > 0 ? KB.prod.dim[kq] : pdim;
    s.cols = dir > 0 ? pdim : KB.prod.dim[kq];
    s.off = tot;
    s.roff = rtot;
    const int ne = KB.prod.dim[kq];
    tot += (int64_t)s.rows * s.cols;
    rtot += (int64_t)ne * ne;
    sec_of[kq] = (int)secs.size();
    secs.push_back(s);
  }
  uint64_t Psi = ex->alloc(std::max<int64_t>(1, tot));
  uint64_t Rho = ex->alloc(std::max<int64_t>(1, rtot));
  {
    Launch g;
    for (const auto& b : lay.blks) {
      const Sub& sl = LB.subs[b.lsub];
      const Sub& sr = RB.subs[b.rsub];
      const Sec& s = secs.at(sec_of[dir > 0 ? sl.prod : sr.prod]);
      const int64_t r0 = dir > 0 ? sl.off : s.poff.at(sl.prod) + sl.off;
      const int64_t c0 = dir > 0 ? s.poff.at(sr.prod) + sr.off : sr.off;
      Seg e;
      e.a = 0; e.b = dpsi + 8ull * b.off; e.ldb = b.cols; e.k = b.rows;
      g.probs.push_back(copy_prob(Psi + 8ull * (s.off + r0 * s.cols + c0), b.rows, b.cols, s.cols, (int)g.segs.size()));
      g.segs.push_back(e);
    }
    ex->run(g, 0, 0);
    Launch h;
    for (const auto& s : secs) {
      Seg e;
      uint64_t P = Psi + 8ull * s.off;
      if (dir > 0) {  // rho = Psi Psi^T
        e.a = P; e.lda = s.cols; e.ta = 0; e.b = P; e.ldb = s.cols; e.tb = 1; e.k = s.cols;
        h.probs.push_back(copy_prob(Rho + 8ull * s.roff, s.rows, s.rows, s.rows, (int)h.segs.size()));
      } else {        // rho = Psi^T Psi
        e.a = P; e.lda = s.cols; e.ta = 1; e.b = P; e.ldb = s.cols; e.tb = 0; e.k = s.rows;
        h.probs.push_back(copy_prob(Rho + 8ull * s.roff, s.cols, s.cols, s.cols, (int)h.segs.size()));
      }
      h.segs.push_back(e);
    }
    ex->run(h, 0, 0);
  }
  // eigen-decompositions and the global selection of the D largest weights
  std::vector<std::vector<double>> lam(secs.size());
  std::vector<std::tuple<double, QN, int, int>> cand;  // (-lambda, left label, index in sector (desc), sector)
  for (size_t k = 0; k < secs.size(); ++k) {
    int ne = dir > 0 ? secs[k].rows : secs[k].cols;
    lam[k].resize(ne);
    ex->eigh(Rho + 8ull * secs[k].roff, ne, lam[k].data());
    // ties are ordered by the left label (the truncated side's partner label in U(1))
    const QN lab = dir > 0 || su2 ? KB.prod.q[secs[k].key] : target - KB.prod.q[secs[k].key];
    for (int j = 0; j < ne; ++j) cand.emplace_back(-lam[k][ne - 1 - j], lab, j, (int)k);
  }
  std::sort(cand.begin(), cand.end(), [](const auto& a, const auto& b) {
    if (std::get<0>(a) != std::get<0>(b)) return std::get<0>(a) < std::get<0>(b);
    if (std::get<1>(a) != std::get<1>(b)) return std::get<1>(a) < std::get<1>(b);
    return std::get<2>(a) < std::get<2>(b);
  });
  if (eps > 0.0) {
    // dynamic block-state selection: tail[j] = sum of the weights from j on
    const int n = (int)cand.size();
    std::vector<double> tail(n + 1, 0.0);
    for (int j = n - 1; j >= 0; --j) tail[j] = tail[j + 1] + std::max(0.0, -std::get<0>(cand[j]));
    int De = std::min(D, n);
    for (int d = std::max(1, Dmin); d <= std::min(D, n); ++d)
      if (tail[d] <= eps) {
        De = d;
        break;
      }
    D = std::max(1, De);
  }
  // weights equal up to rounding (within TIE_REL of the D-th) are kept or
  // dropped together: a group straddling the cut is dropped (spin-flip pairs
  // of Sz = 0 states carry equal weights; rounding must not pick one)
  double above = -1.0;
  if ((int)cand.size() > D && D > 0) {
    const double lc = -std::get<0>(cand[D - 1]), ln = -std::get<0>(cand[D]);
    if (ln >= lc - TIE_REL * lc) above = lc + TIE_REL * lc;
  }
  std::vector<int> keep(secs.size(), 0);
  double disc = 0;
  int nk = 0;
  // exact moves: eigenvalues of a sector's density matrix carry an absolute
  // rounding error of about n eps lambda_max(sector); anything below 8 times
  // that is not distinguishable from zero and is dropped
  std::vector<double> noise(secs.size(), 0.0);
  if (exact)
    for (size_t k = 0; k < secs.size(); ++k) {
      double mx = 0.0;
      for (double v : lam[k]) mx = std::max(mx, v);
      noise[k] = 8.0 * (double)lam[k].size() * 2.220446049250313e-16 * mx;
    }
  for (auto& c : cand) {
    double l = -std::get<0>(c);
    if (nk < D && l > drop_below && l > noise[std::get<3>(c)] && l > above) {
      keep[std::get<3>(c)]++;
      ++nk;
    } else {
      disc += std::max(0.0, l);
    }
  }
  if (nk == 0) throw std::runtime_error("truncation kept no state");
  if (kept) *kept = nk;
  // new bond basis
  Basis nb;
  nb.su2 = su2;
  std::vector<int> nb_of_sec(secs.size(), -1);
  {
    std::vector<std::pair<QN, int>> lab;
    for (size_t k = 0; k < secs.size(); ++k)
      if (keep[k]) lab.push_back({KB.prod.q[secs[k].key], (int)k});
    std::sort(lab.begin(), lab.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (auto& x : lab) {
      nb_of_sec[x.second] = nb.nsec();
      nb.add(x.first, keep[x.second]);
    }
  }
  // new site tensor
  const ProdBasis& PB = dir > 0 ? LB : RB;
  std::vector<int64_t> toff(PB.prod.nsec(), -1);
  std::vector<int> tnb(PB.prod.nsec(), -1);
  int64_t ttot = 0;
  for (size_t k = 0; k < secs.size(); ++k) {
    if (!keep[k]) continue;
    int q = secs[k].key;
    int ne = dir > 0 ? secs[k].rows : secs[k].cols;
    toff[q] = ttot;
    tnb[q] = nb_of_sec[k];
    ttot += (int64_t)ne * keep[k];
  }
  uint64_t T = ex->alloc(std::max<int64_t>(1, ttot));
  {
    Launch g;
    for (size_t k = 0; k < secs.size(); ++k) {
      if (!keep[k]) continue;
      int q = secs[k].key;
      int ne = dir > 0 ? secs[k].rows : secs[k].cols;
      int d = keep[k];
      uint64_t ev = Rho + 8ull * (secs[k].roff + (int64_t)(ne - d) * ne);  // last d eigenvectors
      Seg e;
      e.a = 0; e.b = ev; e.ldb = ne; e.k = dir > 0 ? ne : d;
      if (dir > 0) {  // U_q[r][k] = evec_k[r]: transpose of the column-major block
        e.tb = 1;
        g.probs.push_back(copy_prob(T + 8ull * toff[q], ne, d, d, (int)g.segs.size()));
      } else {        // V_q[k][c] = evec_k[c]: same memory order
        e.tb = 0;
        g.probs.push_back(copy_prob(T + 8ull * toff[q], d, ne, ne, (int)g.segs.size()));
      }
      g.segs.push_back(e);
    }
    ex->run(g, 0, 0);
  }
  double fl = 0;
  // C = U^T Psi (right move) or Psi V^T (left move)
  std::vector<int64_t> coff(secs.size(), -1);
  int64_t ctot = 0;
  for (size_t k = 0; k < secs.size(); ++k) {
    if (!keep[k]) continue;
    coff[k] = ctot;
    ctot += (int64_t)keep[k] * (dir > 0 ? secs[k].cols : secs[k].rows);
  }
  uint64_t Cb = ex->alloc(std::max<int64_t>(1, ctot));
  {
    Launch g;
    for (size_t k = 0; k < secs.size(); ++k) {
      if (!keep[k]) continue;
      const Sec& s = secs[k];
      int q = s.key;
      int d = keep[k];
      Seg e;
      uint64_t P = Psi + 8ull * s.off, U = T + 8ull * toff[q];
      if (dir > 0) {
        e.a = U; e.lda = d; e.ta = 1; e.b = P; e.ldb = s.cols; e.tb = 0; e.k = s.rows;
        g.probs.push_back(copy_prob(Cb + 8ull * coff[k], d, s.cols, s.cols, (int)g.segs.size()));
      } else {
        e.a = P; e.lda = s.cols; e.ta = 0; e.b = U; e.ldb = s.cols; e.tb = 1; e.k = s.cols;
        g.probs.push_back(copy_prob(Cb + 8ull * coff[k], s.rows, d, d, (int)g.segs.size()));
      }
      g.segs.push_back(e);
    }
    ex->run(g, 0, 0);
  }
  const int c = center;
  // new block and new centre
  if (dir > 0) {
    EnvBlock blk;
    blk.cut = c + 1;
    renormalize(Lp, nb, tnb, T, toff, *ex, blk, tmp_budget, &fl);
    site[c] = T;
    site_off[c] = toff;
    site_nb[c] = tnb;
    bonds[c + 1] = nb;
    lenv[c + 1] = blk;
    // psi'(x', i', j', y') = C[x' rows, (i', y) cols] V_{c+2}[y, (j', y')]; in SU(2) the
    // sum runs over the channels of the old R' sub-block (s, y) whose site multiplet is
    // that of i', each recoupled from |x', (s y) J_old; S> to |(x' s) J_a, y; S>
    ProdBasis nL = make_prod(bonds[c + 1], true), nR = make_prod(bonds[c + 3], false);
    PsiLayout nl = make_psi_layout(nL, nR, target);
    ProdBasis R3 = make_prod(bonds[c + 3], false);
    uint64_t np = ex->alloc(std::max<int64_t>(1, nl.size));
    std::vector<int> sec_of_nb(nb.nsec(), -1);
    for (size_t k = 0; k < secs.size(); ++k)
      if (nb_of_sec[k] >= 0) sec_of_nb[nb_of_sec[k]] = (int)k;
    Launch g;
    for (const auto& b : nl.blks) {
      const int r = R3.find(b.y, b.j);                // product sub (j', y') of site c+2
      const int rp = R3.subs[r].prod;
      const int y = bonds[c + 2].find(R3.prod.q[rp]);
      if (y < 0) continue;
      const int k = sec_of_nb[b.x];
      const Sec& s = secs.at(k);
      Prob p = copy_prob(np + 8ull * b.off, b.rows, b.cols, b.cols, (int)g.segs.size());
      p.nseg = 0;
      for (int ch = 0; ch < NSITE; ++ch) {
        if (su2 ? site_mult(ch) != site_mult(b.i) : ch != b.i) continue;
        const int sR = RB.find(y, ch);                  // old R' sub (s, y)
        if (sR < 0) continue;
        auto po = s.poff.find(RB.subs[sR].prod);
        if (po == s.poff.end()) continue;
        double w = 1.0;
        if (su2) {
          const int Ja = nL.sub_qn(nL.find(b.x, b.i)).s, Jold = RB.sub_qn(sR).s;
          w = su2::assoc(nb.q[b.x].s, SITE_MULT_S[site_mult(ch)], bonds[c + 2].q[y].s, Ja, Jold, target.s);
          if (w == 0.0) continue;
        }
        Seg e;
        e.a = Cb + 8ull * (coff[k] + po->second + RB.subs[sR].off); e.lda = s.cols; e.ta = 0;
        e.b = site[c + 2] + 8ull * (site_off[c + 2][rp] + R3.subs[r].off); e.ldb = R3.prod.dim[rp]; e.tb = 0;
        e.k = bonds[c + 2].dim[y];
        e.sc = w;
        g.segs.push_back(e);
        ++p.nseg;
      }
      if (p.nseg) g.probs.push_back(p);
    }
    ex->zero(np, std::max<int64_t>(1, nl.size));
    ex->run(g, 0, 0);
    ex->release(site[c + 2]);
    site[c + 2] = 0;
    free_block(renv.at(c + 2));
    renv.erase(c + 2);
    bonds[c + 2] = Basis();
    ex->release(dpsi);
    dpsi = np;
    center = c + 1;
  } else {
    EnvBlock blk;
    blk.cut = c + 1;
    renormalize(Rp, nb, tnb, T, toff, *ex, blk, tmp_budget, &fl);
    site[c + 1] = T;
    site_off[c + 1] = toff;
    site_nb[c + 1] = tnb;
    bonds[c + 1] = nb;
    renv[c + 1] = blk;
    // psi'(x', i', j', y') = U_{c-1}[(x', i') rows -> x] C[(x, j') rows, y' cols]; in SU(2)
    // over the channels of the old L' sub-block (x, s) whose site multiplet is that of
    // j', each recoupled from |(x s) J_old, y'; S> to |x, (s y') J_b; S>
    ProdBasis nL = make_prod(bonds[c - 1], true), nR = make_prod(bonds[c + 1], false);
    PsiLayout nl = make_psi_layout(nL, nR, target);
    ProdBasis L1 = make_prod(bonds[c - 1], true);
    uint64_t np = ex->alloc(std::max<int64_t>(1, nl.size));
    std::vector<int> sec_of_nb(nb.nsec(), -1);
    for (size_t k = 0; k < secs.size(); ++k)
      if (nb_of_sec[k] >= 0) sec_of_nb[nb_of_sec[k]] = (int)k;
    Launch g;
    for (const auto& b : nl.blks) {
      const int u = L1.find(b.x, b.i);                // product sub (x', i') of site c-1
      const int up = L1.subs[u].prod;
      const int x = bonds[c].find(L1.prod.q[up]);
      if (x < 0) continue;
      const int k = sec_of_nb[b.y];
      const Sec& s = secs.at(k);
      const int d = keep[k];
      Prob p = copy_prob(np + 8ull * b.off, b.rows, b.cols, b.cols, (int)g.segs.size());
      p.nseg = 0;
      for (int ch = 0; ch < NSITE; ++ch) {
        if (su2 ? site_mult(ch) != site_mult(b.j) : ch != b.j) continue;
        const int sL = LB.find(x, ch);                  // old L' sub (x, s)
        if (sL < 0) continue;
        auto po = s.poff.find(LB.subs[sL].prod);
        if (po == s.poff.end()) continue;
        double w = 1.0;
        if (su2) {
          const int Jb = nR.sub_qn(nR.find(b.y, b.j)).s, Jold = LB.sub_qn(sL).s;
          w = su2::assoc(bonds[c].q[x].s, SITE_MULT_S[site_mult(ch)], nb.q[b.y].s, Jold, Jb, target.s);
          if (w == 0.0) continue;
        }
        Seg e;
        e.a = site[c - 1] + 8ull * (site_off[c - 1][up] + (int64_t)L1.subs[u].off * bonds[c].dim[x]);
        e.lda = bonds[c].dim[x]; e.ta = 0;
        e.b = Cb + 8ull * (coff[k] + (po->second + (int64_t)LB.subs[sL].off) * d); e.ldb = d; e.tb = 0;
        e.k = bonds[c].dim[x];
        e.sc = w;
        g.segs.push_back(e);
        ++p.nseg;
      }
      if (p.nseg) g.probs.push_back(p);
    }
    ex->zero(np, std::max<int64_t>(1, nl.size));
    ex->run(g, 0, 0);
    ex->release(site[c - 1]);
    site[c - 1] = 0;
    free_block(lenv.at(c));
    lenv.erase(c);
    bonds[c] = Basis();
    ex->release(dpsi);
    dpsi = np;
    center = c - 1;
  }
  ex->release(Psi);
  ex->release(Rho);
  ex->release(Cb);
  env_flops += fl;
  prepare_center();
  enforce_budget();
  // prefetch the block the next move in this direction will need
  if (dir > 0) {
    auto it = renv.find(center + 3);
    if (it != renv.end() && it->second.evicted) restore_async(it->second);
  } else {
    auto it = lenv.find(center - 1);
    if (it != lenv.end() && it->second.evicted) restore_async(it->second);
  }
  return disc;
}

double Engine::expect(const std::vector<CenterTerm>& terms) {
  HeffPlan pl = plan_terms(Lp, Rp, lay, terms, tmp_budget);
  ex->tmp(std::max<int64_t>(1, pl.tmp_elems));
  uint64_t tau = ex->alloc(std::max<int64_t>(1, lay.size));
  for (size_t k = 0; k < pl.stage1.size(); ++k) {
    ex->run(pl.stage1[k], dpsi, tau);
    ex->run(pl.stage2[k], dpsi, tau);
  }
  double v = ex->dot(dpsi, tau, lay.size);
  ex->release(tau);
  return v;
}

std::vector<double> Engine::rdm1() {
  // (SU(2): rdm1_su2, after the same rebuild when the blocks at the centre hold
  // complementary pairs on the left.)
  // At the centre (L-2, L-1) the left enlarged block L' holds the normal
  // operators a+_k a_l of every spin-orbital of sites 0..L-2, and the right
  // enlarged block is the last site alone, so every E_pq is a product of
  // stored operators:
  //   p, q < L-1 : B_{p s, q s} (x) 1
  //   p < L-1 = q: (a+_p)_L' (a_q)_R'
  //   q < L-1 = p: a+_p a_q = -(a_q)_L' (a+_p)_R'
  //   p = q = L-1: 1 (x) a+_p a_p on the last site
  if (center != L - 2) throw StateError("the one-particle density matrix needs the centre at (L-2, L-1)");
  if (!Lp.normal) {
    // the blocks at this centre hold complementary pairs on the left: rebuild
    // the environment with normal pairs on the left (the MPS is unchanged),
    // take the density matrix there, and restore the switched environment
    const int saved = pair_switch;
    pair_switch = 0;
    std::vector<double> g;
    try {
      build_env();
      g = rdm1();
    } catch (...) {
      pair_switch = saved;
      build_env();
      throw;
    }
    pair_switch = saved;
    build_env();
    return g;
  }
  if (su2) return rdm1_su2();
  const double nrm = ex->dot(dpsi, dpsi, lay.size);
  auto get = [](const Enlarged& E, Key k) -> const OpView* {
    auto it = E.ops.find(k);
    if (it == E.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  };
  const OpView* IL = get(Lp, Key(F_I));
  const OpView* IR = get(Rp, Key(F_I));
  const int last = L - 1;
  std::vector<double> g((size_t)L * L, 0.0);
  std::vector<OpView> site_ops;
  site_ops.reserve(2);
  for (int s = 0; s < 2; ++s) site_ops.push_back(site_op_view(Rp, cre(s) * ann(s), false));
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q) {
      std::vector<CenterTerm> t;
      for (int s = 0; s < 2; ++s) {
        const int kp = 2 * p + s, kq = 2 * q + s;
        if (p < last && q < last) {
          if (auto B = get(Lp, Key(F_B, kp, kq))) t.push_back({B, false, IR, false, 1.0});
        } else if (p < last) {
          auto C = get(Lp, Key(F_C, kp));
          auto Cr = get(Rp, Key(F_C, kq));
          if (C && Cr) t.push_back({C, false, Cr, true, 1.0});
        } else if (q < last) {
          auto C = get(Lp, Key(F_C, kq));
          auto Cr = get(Rp, Key(F_C, kp));
          if (C && Cr) t.push_back({C, true, Cr, false, -1.0});
        } else {
          t.push_back({IL, false, &site_ops[s], false, 1.0});
        }
      }
      if (!t.empty()) g[(size_t)p * L + q] = expect(t) / nrm;
    }
  return g;
}

std::vector<double> Engine::rdm1_su2() {
  // SU(2): gamma_pq = <E_pq> with E_pq = -sqrt(2) [c_p x d_q]^0. At the centre
  // (L-2, L-1) the left enlarged block holds B^0_pq = [c_p x d_q]^0 for p <= q
  // of its orbitals and c_p; the right enlarged block is the last orbital:
  //   p <= q < L-1 : -sqrt(2) [B^0_pq x 1]^0
  //   p < L-1 = q  : -sqrt(2) [c_p x d_q]^0, d_q the adjoint tensor of c_q on the right
  //   p = q = L-1  : N - sum of the other diagonal elements (Tr gamma = N)
  // gamma is symmetric (real state, E_qp = E_pq^+).
  if (center != L - 2) throw StateError("the one-particle density matrix needs the centre at (L-2, L-1)");
  const double nrm = ex->dot(dpsi, dpsi, lay.size);
  auto get = [](const Enlarged& E, Key k) -> const OpView* {
    auto it = E.ops.find(k);
    if (it == E.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  };
  const OpView* IR = get(Rp, Key(F_I));
  const int last = L - 1;
  const double sq2 = std::sqrt(2.0);
  std::vector<double> g((size_t)L * L, 0.0);
  for (int p = 0; p < last; ++p)
    for (int q = p; q < L; ++q) {
      CenterTerm t{nullptr, false, nullptr, false, -sq2};
      if (q < last) {
        t.L = get(Lp, Key(F_B, p, q, 0));
        t.R = IR;
        t.k2 = 0;
      } else {
        t.L = get(Lp, Key(F_C, p));
        t.R = get(Rp, Key(F_C, q));
        t.RT = true;
        t.k2 = 1;
      }
      if (!t.L || !t.R) continue;
      const double v = expect({t}) / nrm;
      g[(size_t)p * L + q] = g[(size_t)q * L + p] = v;
    }
  double tr = 0.0;
  for (int p = 0; p < last; ++p) tr += g[(size_t)p * L + p];
  g[(size_t)last * L + last] = N - tr;
  return g;
}

std::vector<double> Engine::rdm2_sweep() {
  if (su2) return rdm2_sweep_su2();
  // Gamma_pqrs = sum over spins sigma, tau of <a+_{p sigma} a+_{r tau} a_{s tau} a_{q sigma}>,
  // each element measured at the one centre (s1, s2 = s1 + 1) where its four
  // operators split into at most two on the left block (stored C, A, B), any
  // number on each of the two sites (exact 4x4 products) and at most one on
  // the right block (stored C): with o1 <= o2 <= o3 <= o4 the sorted orbitals,
  // s2 = max(o3, 1). The centre walks the chain once by exact moves (every
  // weight above its sector's rounding noise kept, so the state is not
  // changed at first order as it would be by dropping weights at the global
  // floor); afterwards the MPS and its environment are restored as they were.
  if (!have_env) throw StateError("build_env first");
  if (pair_switch > 0) {
    // the walk reads normal pairs from every left block
    const int saved = pair_switch;
    pair_switch = 0;
    std::vector<double> g;
    try {
      build_env();
      g = rdm2_sweep();
    } catch (...) {
      pair_switch = saved;
      build_env();
      throw;
    }
    pair_switch = saved;
    build_env();
    return g;
  }
  const size_t L4 = (size_t)L * L * L * L;
  auto at = [&](int p, int q, int r, int s) { return (((size_t)p * L + q) * L + r) * L + s; };
  // representatives of {pqrs, rspq, qpsr, srqp} (equal for a real state), by centre
  std::vector<std::vector<std::array<int, 4>>> todo(L - 1);
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q)
      for (int r = 0; r < L; ++r)
        for (int s = 0; s < L; ++s) {
          const std::array<int, 4> t{p, q, r, s};
          if (std::array<int, 4>{r, s, p, q} < t || std::array<int, 4>{q, p, s, r} < t ||
              std::array<int, 4>{s, r, q, p} < t)
            continue;
          std::array<int, 4> o = t;
          std::sort(o.begin(), o.end());
          todo[std::max(o[2], 1) - 1].push_back(t);
        }
  std::vector<double> G(L4, 0.0);
  auto get = [](const EnvBlock& B, Key k) -> const OpView* {
    auto it = B.ops.find(k);
    if (it == B.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  };
  // the MPS before the walk, restored exactly afterwards (the walk re-gauges it)
  const MpsSnapshot snap = snapshot();
  try {
  while (center > 0) truncate_move(1 << 30, -1, -1.0);
  for (int s1 = 0; s1 <= L - 2; ++s1) {
    if (s1 > 0) truncate_move(1 << 30, +1, -1.0);
    const int s2 = s1 + 1;
    const EnvBlock& LB = lenv.at(s1);
    const EnvBlock& RB = renv.at(s2 + 1);
    const int64_t n = lay.size;
    const double nrm = ex->dot(dpsi, dpsi, n);
    if (!(nrm > 0)) throw std::runtime_error("zero wavefunction");
    uint64_t tau = ex->alloc(std::max<int64_t>(1, n));
    try {
      for (const auto& t : todo[s1]) {
        std::deque<OpView> views;
        std::vector<CenterTerm> terms;
        for (int sg = 0; sg < 2; ++sg)
          for (int tu = 0; tu < 2; ++tu) {
            struct Op { bool cre; int mode, orb; };
            const Op ops[4] = {{true, 2 * t[0] + sg, t[0]}, {true, 2 * t[2] + tu, t[2]},
                               {false, 2 * t[3] + tu, t[3]}, {false, 2 * t[1] + sg, t[1]}};
            if (ops[0].mode == ops[1].mode || ops[2].mode == ops[3].mode) continue;
            int grp[4];
            for (int i = 0; i < 4; ++i) grp[i] = ops[i].orb < s1 ? 0 : ops[i].orb == s1 ? 1 : ops[i].orb == s2 ? 2 : 3;
            int inv = 0;
            for (int i = 0; i < 4; ++i)
              for (int j = i + 1; j < 4; ++j) inv += grp[i] > grp[j];
            std::vector<Op> g[4];
            for (int i = 0; i < 4; ++i) g[grp[i]].push_back(ops[i]);
            if (g[3].size() > 1 || g[0].size() > 2) throw std::logic_error("rdm2_sweep: element at the wrong centre");
            Mat4 m1 = Mat4::id(), m2 = Mat4::id();
            for (const Op& o : g[1]) m1 = m1 * (o.cre ? cre(o.mode & 1) : ann(o.mode & 1));
            for (const Op& o : g[2]) m2 = m2 * (o.cre ? cre(o.mode & 1) : ann(o.mode & 1));
            // left block: identity, C_k / C_k^T, or a pair in operator order
            std::vector<Contrib> xl;
            const bool par1 = g[1].size() & 1;
            auto add = [&](const OpView* src, bool T, double c) {
              Contrib x;
              x.src = src; x.srcT = T; x.o = m1; x.coef = c; x.par = par1;
              xl.push_back(x);
            };
            if (g[0].empty()) {
              add(nullptr, false, 1.0);
            } else if (g[0].size() == 1) {
              if (auto C = get(LB, Key(F_C, g[0][0].mode))) add(C, !g[0][0].cre, 1.0);
            } else {
              const Op a = g[0][0], b = g[0][1];
              const int k1 = a.mode, k2 = b.mode;
              if (a.cre && b.cre) {          // a+_k1 a+_k2
                if (auto A = get(LB, Key(F_A, std::min(k1, k2), std::max(k1, k2)))) add(A, false, k1 < k2 ? 1.0 : -1.0);
              } else if (!a.cre && !b.cre) { // a_k1 a_k2 = (a+_k2 a+_k1)^T
                if (auto A = get(LB, Key(F_A, std::min(k1, k2), std::max(k1, k2)))) add(A, true, k2 < k1 ? 1.0 : -1.0);
              } else if (a.cre) {            // a+_k1 a_k2
                if (auto B = get(LB, Key(F_B, k1, k2))) add(B, false, 1.0);
              } else {                       // a_k1 a+_k2 = d_k1k2 - a+_k2 a_k1
                if (auto B = get(LB, Key(F_B, k2, k1))) add(B, false, -1.0);
                if (k1 == k2) add(nullptr, false, 1.0);
              }
            }
            if (xl.empty()) continue;
            const OpView* rsrc = nullptr;
            bool rT = false;
            if (g[3].size() == 1) {
              rsrc = get(RB, Key(F_C, g[3][0].mode));
              if (!rsrc) continue;
              rT = !g[3][0].cre;
            }
            Contrib yr;
            yr.src = rsrc; yr.srcT = rT; yr.o = m2; yr.coef = 1.0; yr.par = g[3].size() & 1;
            views.push_back(product_view(LB, I, Lp, xl, (g[0].size() + g[1].size()) & 1));
            const OpView* X = &views.back();
            views.push_back(product_view(RB, I, Rp, {yr}, (g[2].size() + g[3].size()) & 1));
            const OpView* Y = &views.back();
            if (X->empty() || Y->empty()) continue;
            terms.push_back({X, false, Y, false, (inv & 1) ? -1.0 : 1.0});
          }
        double v = 0.0;
        if (!terms.empty()) {
          HeffPlan pl = plan_terms(Lp, Rp, lay, terms, tmp_budget);
          ex->tmp(std::max<int64_t>(1, pl.tmp_elems));
          ex->zero(tau, n);
          for (size_t k = 0; k < pl.stage1.size(); ++k) {
            ex->run(pl.stage1[k], dpsi, tau);
            ex->run(pl.stage2[k], dpsi, tau);
          }
          v = ex->dot(dpsi, tau, n) / nrm;
        }
        const int p = t[0], q = t[1], r = t[2], s = t[3];
        G[at(p, q, r, s)] = G[at(r, s, p, q)] = G[at(q, p, s, r)] = G[at(s, r, q, p)] = v;
      }
    } catch (...) {
      ex->release(tau);
      throw;
    }
    ex->release(tau);
  }
  } catch (...) {
    restore(snap);
    throw;
  }
  restore(snap);
  return G;
}

Engine::MpsSnapshot Engine::snapshot() {
  MpsSnapshot sn;
  sn.center = center;
  sn.bonds = bonds;
  sn.off = site_off;
  sn.nb = site_nb;
  sn.site.resize(L);
  for (int p = 0; p < L; ++p) {
    if (!site[p]) continue;
    const bool left = p < center;
    const ProdBasis pb = make_prod(left ? bonds[p] : bonds[p + 1], left);
    const Basis& to = left ? bonds[p + 1] : bonds[p];
    int64_t n = 0;
    for (int q = 0; q < pb.prod.nsec(); ++q)
      if (site_off[p][q] >= 0) n = std::max<int64_t>(n, site_off[p][q] + (int64_t)pb.prod.dim[q] * to.dim[site_nb[p][q]]);
    sn.site[p].resize((size_t)n);
    if (n) ex->download(sn.site[p].data(), site[p], n);
  }
  sn.psi = get_psi_host();
  return sn;
}

void Engine::restore(const MpsSnapshot& sn) {
  clear_env();
  for (auto& t : site)
    if (t) ex->release(t);
  site.assign(L, 0);
  for (int p = 0; p < L; ++p) {
    if (sn.site[p].empty()) continue;
    site[p] = ex->alloc((int64_t)sn.site[p].size());
    ex->upload(site[p], sn.site[p].data(), (int64_t)sn.site[p].size());
  }
  bonds = sn.bonds;
  site_off = sn.off;
  site_nb = sn.nb;
  center = sn.center;
  set_psi_host(sn.psi);
  build_env();
}

std::vector<double> Engine::on_m_expansion(const std::function<std::vector<double>(Engine&)>& f, int two_m) {
  if (!have_env) throw StateError("build_env first");
  if (two_m == INT_MIN) two_m = two_s;
  MpsSnapshot sn = snapshot();
  SU2Mps in;
  in.L = L;
  in.center = center;
  in.N = N;
  in.two_s = two_s;
  in.bonds = std::move(sn.bonds);
  in.site_off = std::move(sn.off);
  in.site_nb = std::move(sn.nb);
  in.site = std::move(sn.site);
  in.psi = std::move(sn.psi);
  U1Mps out;
  expand_mps_su2(in, out, two_m);
  Engine U;
  U.ex = ex;
  U.pr = pr;
  U.I = I;
  U.N = N;
  U.two_s = two_m;
  U.L = L;
  U.su2 = false;
  U.device = device;
  U.tmp_budget = tmp_budget;
  U.hbm_budget = hbm_budget;
  U.autotune = autotune;
  U.bonds = out.bonds;
  U.site.assign(L, 0);
  U.site_off = out.site_off;
  U.site_nb = out.site_nb;
  std::vector<double> r;
  auto done = [&]() {
    U.clear();
    U.ex = nullptr;   // its destructor must not drop the runner's lists again
    U.pr = nullptr;
    // the U(1) engine's centre replaced this engine's prepared task lists
    prepare_center();
  };
  try {
    for (int p = 0; p < L; ++p) {
      if (p == center || p == center + 1) continue;
      U.site[p] = ex->alloc((int64_t)out.site[p].size());
      ex->upload(U.site[p], out.site[p].data(), (int64_t)out.site[p].size());
    }
    U.center = center;
    U.set_psi_host(out.psi);
    U.build_env();
    r = f(U);
  } catch (...) {
    done();
    throw;
  }
  done();
  return r;
}

std::vector<double> Engine::rdm2_sweep_su2() {
  return on_m_expansion([](Engine& U) { return U.rdm2_sweep(); });
}

std::vector<double> Engine::orbital_rdm2() {
  if (!have_env) throw StateError("build_env first");
  if (su2) {
    // rho_ij of one component depends on M; the average over the multiplet
    // does not (it is what the spin-free entropies of the state are made of)
    std::vector<double> avg((size_t)L * L * 256, 0.0);
    for (int m = -two_s; m <= two_s; m += 2) {
      const std::vector<double> r = on_m_expansion([](Engine& U) { return U.orbital_rdm2(); }, m);
      for (size_t k = 0; k < avg.size(); ++k) avg[k] += r[k] / (two_s + 1);
    }
    return avg;
  }
  std::vector<double> R((size_t)L * L * 256, 0.0);
  // the MPS before the walk, restored exactly afterwards
  const MpsSnapshot snap = snapshot();
  auto put_back = [&]() {
    keep_local = false;
    restore(snap);
  };
  static const int NOCC[4] = {0, 1, 1, 2};
  static const int SZ2[4] = {0, 1, -1, 0};
  auto unit = [](int u) {
    Mat4 m;
    m(u / 4, u % 4) = 1.0;
    return m;
  };
  auto get = [](const EnvBlock& B, Key k) -> const OpView* {
    auto it = B.ops.find(k);
    if (it == B.ops.end() || it->second.empty()) return nullptr;
    return &it->second;
  };
  try {
    while (center > 0) truncate_move(1 << 30, -1, -1.0);
    keep_local = true;
    build_env();   // right blocks with the matrix units of their orbitals
    for (int s1 = 0; s1 <= L - 2; ++s1) {
      if (s1 > 0) truncate_move(1 << 30, +1, -1.0);
      const int s2 = s1 + 1;
      const EnvBlock& LB = lenv.at(s1);
      const EnvBlock& RB = renv.at(s2 + 1);
      const double nrm = ex->dot(dpsi, dpsi, lay.size);
      if (!(nrm > 0)) throw std::runtime_error("zero wavefunction");
      for (int j = s2; j < L; ++j)
        for (int u = 0; u < 16; ++u)
          for (int v = 0; v < 16; ++v) {
            const int dn = NOCC[u / 4] - NOCC[u % 4] + NOCC[v / 4] - NOCC[v % 4];
            const int ds = SZ2[u / 4] - SZ2[u % 4] + SZ2[v / 4] - SZ2[v % 4];
            if (dn != 0 || ds != 0) continue;
            const bool ou = (NOCC[u / 4] + NOCC[u % 4]) & 1, ov = (NOCC[v / 4] + NOCC[v % 4]) & 1;
            Contrib xl;
            xl.src = nullptr; xl.srcT = false; xl.o = unit(u); xl.coef = 1.0; xl.par = ou;
            Contrib yr;
            yr.srcT = false; yr.coef = 1.0;
            if (j == s2) {
              yr.src = nullptr; yr.o = unit(v); yr.par = false;
            } else {
              yr.src = get(RB, Key(F_L, j, v));
              if (!yr.src) continue;
              yr.o = Mat4::id(); yr.par = ov;
            }
            OpView X = product_view(LB, I, Lp, {xl}, ou);
            OpView Y = product_view(RB, I, Rp, {yr}, ov);
            if (X.empty() || Y.empty()) continue;
            const double val = expect({CenterTerm{&X, false, &Y, false, 1.0}}) / nrm;
            // In the basis with orbitals i, j first, E_u(i) = |s_i><r_i| (x) 1 and
            // E_v(j) = P_i^odd(v) (x) |s_j><r_j| (the fermion string of orbital j's
            // operators crosses orbital i), so <E_u E_v> = (-1)^(n(r_i) odd(v))
            // rho_ij[(r_i r_j), (s_i s_j)] with rho_ij = Tr_rest |Psi><Psi|,
            // u = 4 s_i + r_i, v = 4 s_j + r_j
            const int r = 4 * (u % 4) + (v % 4), sc = 4 * (u / 4) + (v / 4);
            const double sg = ((NOCC[u % 4] & 1) && ov) ? -1.0 : 1.0;
            R[((size_t)s1 * L + j) * 256 + (size_t)r * 16 + sc] = sg * val;
          }
    }
  } catch (...) {
    put_back();
    throw;
  }
  put_back();
  return R;
}

std::vector<double> Engine::rdm2() {
  // Either symmetry: the probes only rebuild the environment with other integrals
  // and read <H_eff>; Gamma is the spin-summed (spin-free) 2-RDM in both.
  // At fixed MPS the energy is linear in V: with h = 0, e_core = 0 and V the
  // unit tensor on one permutation orbit {pqrs, qprs, pqsr, qpsr, rspq, srpq,
  // rsqp, srqp}, <H_eff> = 1/2 sum over the orbit's distinct elements of
  // Gamma. Each element of the orbit receives the orbit average.
  if (!have_env) throw StateError("build_env first");
  const int64_t n = lay.size;
  const double nrm = ex->dot(dpsi, dpsi, n);
  if (!(nrm > 0)) throw std::runtime_error("zero wavefunction");
  const Integrals saved = I;
  const size_t L4 = (size_t)L * L * L * L;
  auto at = [&](int p, int q, int r, int s) { return (((size_t)p * L + q) * L + r) * L + s; };
  std::vector<double> G(L4, 0.0);
  uint64_t sig = ex->alloc(std::max<int64_t>(1, n));
  try {
    I.h.assign((size_t)L * L, 0.0);
    I.ecore = 0.0;
    for (int p = 0; p < L; ++p)
      for (int q = 0; q < L; ++q)
        for (int r = 0; r < L; ++r)
          for (int s = 0; s < L; ++s) {
            const std::array<std::array<int, 4>, 8> perm = {{{p, q, r, s}, {q, p, r, s}, {p, q, s, r}, {q, p, s, r},
                                                             {r, s, p, q}, {s, r, p, q}, {r, s, q, p}, {s, r, q, p}}};
            std::vector<std::array<int, 4>> orbit(perm.begin(), perm.end());
            std::sort(orbit.begin(), orbit.end());
            orbit.erase(std::unique(orbit.begin(), orbit.end()), orbit.end());
            if (orbit.front() != perm[0]) continue;  // not the orbit's smallest member
            I.V.assign(L4, 0.0);
            for (auto& e : orbit) I.V[at(e[0], e[1], e[2], e[3])] = 1.0;
            build_env();
            heff(dpsi, sig, pr->stream(), 0);
            const double e = ex->dot(dpsi, sig, n) / nrm;
            for (auto& x : orbit) G[at(x[0], x[1], x[2], x[3])] = 2.0 * e / (double)orbit.size();
          }
  } catch (...) {
    I = saved;
    ex->release(sig);
    build_env();
    throw;
  }
  I = saved;
  ex->release(sig);
  build_env();
  return G;
}

}  // namespace qd
