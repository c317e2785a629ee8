// Host-side check of the library's task lists, without a GPU.
//
// Builds the environment of a random-structure MPS with a recording executor
// (device addresses are handed out by a bump allocator and every allocation is
// remembered; nothing is computed), then checks that every FP64 segment, every
// tiled work item, view and segment of the tensor-core path stays inside the
// buffer it addresses, that no work item is empty, and that the algorithmic
// flop counts of the FP64 and tiled plans agree. An out-of-range offset in a
// plan would be an out-of-bounds access on the GPU.
//
// usage: planner_check L N D   (2Sz = N mod 2, centre bond L/2 - 1)
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <string>

#include "engine.hpp"
#include "tiled.hpp"

using namespace qd;

namespace {

int fails = 0;
void fail(const std::string& m) {
  if (fails < 20) std::fprintf(stderr, "FAIL: %s\n", m.c_str());
  ++fails;
}

struct RecEx : Executor {
  uint64_t next = 1ull << 40;
  std::map<uint64_t, int64_t> alloc_bytes;  // base -> bytes
  uint64_t tmp_base = 0;
  int64_t tmp_n = 0;
  int64_t live = 0;
  std::map<uint64_t, int64_t> cur;  // allocations not yet released
  int64_t cur_live = 0, peak = 0;
  uint64_t alloc(int64_t n) override {
    const uint64_t p = next;
    const int64_t b = std::max<int64_t>(8, n * 8);
    next += ((b + 255) / 256) * 256 + 256;
    alloc_bytes[p] = b;
    live += b;
    cur[p] = b;
    cur_live += b;
    peak = std::max(peak, cur_live);
    return p;
  }
  void release(uint64_t p) override {
    auto it = cur.find(p);
    if (it == cur.end()) return;
    cur_live -= it->second;
    cur.erase(it);
  }
  uint64_t tmp(int64_t n) override {
    if (n > tmp_n) {
      tmp_base = alloc(n);
      tmp_n = n;
    }
    return tmp_base;
  }
  // [addr, addr + bytes) inside one recorded allocation
  bool inside(uint64_t addr, int64_t bytes) const {
    auto it = alloc_bytes.upper_bound(addr);
    if (it == alloc_bytes.begin()) return false;
    --it;
    return addr >= it->first && addr + (uint64_t)bytes <= it->first + (uint64_t)it->second;
  }
  // every launch the host planner hands over (renormalization, enlargement
  // sums, the GEMM-form sums): each problem's C and each segment's A and B
  // must lie inside one allocation (psi and sigma buffers, scratch or stored)
  int64_t launches_checked = 0;
  void run(const Launch& l, uint64_t psi, uint64_t sig) override {
    ++launches_checked;
    const uint64_t base[4] = {0, psi, sig, tmp_base};
    auto addr = [&](uint64_t v, int buf) { return buf == 0 ? v : base[buf] + v * 8; };
    for (size_t pi = 0; pi < l.probs.size(); ++pi) {
      const Prob& p = l.probs[pi];
      if (p.m <= 0 || p.n <= 0 || p.ldc < p.n || p.seg0 < 0 || p.nseg < 0 ||
          (size_t)p.seg0 + p.nseg > l.segs.size()) {
        fail("launch problem " + std::to_string(pi) + " malformed");
        continue;
      }
      if (!inside(addr(p.c, p.cbuf), 8 * ((int64_t)(p.m - 1) * p.ldc + p.n))) fail("launch C out of bounds");
      for (int si = p.seg0; si < p.seg0 + p.nseg; ++si) {
        const Seg& g = l.segs[si];
        const bool aid = g.a == 0 && g.abuf == 0, bid = g.b == 0 && g.bbuf == 0;
        if (aid) {
          if (!bid) {
            const int64_t last = g.tb ? (int64_t)(p.n - 1) * g.ldb + p.m - 1 : (int64_t)(p.m - 1) * g.ldb + p.n - 1;
            if (!inside(addr(g.b, g.bbuf), 8 * (last + 1))) fail("launch gathered B out of bounds");
          }
          continue;
        }
        if (bid || g.k <= 0) { fail("launch segment malformed"); continue; }
        const int64_t la = g.ta ? (int64_t)(g.k - 1) * g.lda + p.m - 1 : (int64_t)(p.m - 1) * g.lda + g.k - 1;
        const int64_t lb = g.tb ? (int64_t)(p.n - 1) * g.ldb + g.k - 1 : (int64_t)(g.k - 1) * g.ldb + p.n - 1;
        if (!inside(addr(g.a, g.abuf), 8 * (la + 1))) fail("launch A out of bounds");
        if (!inside(addr(g.b, g.bbuf), 8 * (lb + 1))) fail("launch B out of bounds");
      }
    }
  }
  void upload(uint64_t, const double*, int64_t) override {}
  void download(double* h, uint64_t, int64_t n) override { std::fill(h, h + n, 0.0); }
  void zero(uint64_t, int64_t) override {}
  void randn(uint64_t, int64_t, uint64_t) override {}
  void orthonormal_cols(uint64_t, int, int) override {}
  double dot(uint64_t, uint64_t, int64_t) override { return 1.0; }
  void scale(uint64_t, double, int64_t) override {}
  void axpby(uint64_t, double, uint64_t, double, int64_t) override {}
  void precond(uint64_t, uint64_t, uint64_t, double, double, int64_t) override {}
  void eigh(uint64_t, int, double*) override {}
  void copy(uint64_t, uint64_t, int64_t) override {}
  uint64_t host_alloc(int64_t) override { return 0; }
  void host_free(uint64_t) override {}
  void d2h(uint64_t, uint64_t, int64_t) override {}
  void h2d_async(uint64_t, uint64_t, int64_t) override {}
  void copies_join() override {}
  double copies_wait_seconds() override { return 0.0; }
  int64_t live_bytes() const override { return live; }
};

struct NullRunner : PreparedRunner {
  int n = 0;
  int prepare(const Launch&) override { return n++; }
  void drop_prepared() override {}
  void run_prepared(int, uint64_t, uint64_t, void*, int) override {}
  int take_error() override { return 0; }
  const void* prepared_handle(int) const override { return nullptr; }
  void tile_counts(int, int64_t c[5]) const override { for (int i = 0; i < 5; ++i) c[i] = 0; }
  void* stream() override { return nullptr; }
  void sync(void*) override {}
  void zero_async(uint64_t, int64_t, void*) override {}
  int64_t bytes_allocated() const override { return 0; }
  void prepare_tiled(const TiledPlan&, int) override {}
  void set_tiled_items(const TiledPlan&) override {}
  int tiled_planes() const override { return 0; }
  double time_tiled(uint64_t, uint64_t, int, int) override { return 0.0; }
  void run_tiled(uint64_t, uint64_t, void*, int) override {}
};

// extent in elements of a rows x cols operand with leading dimension ld,
// stored transposed when tr
int64_t extent(int rows, int cols, int ld, int tr) {
  if (rows <= 0 || cols <= 0) return 0;
  return tr ? (int64_t)(cols - 1) * ld + rows : (int64_t)(rows - 1) * ld + cols;
}

void check_fp64(const HeffPlan& P, const PsiLayout& lay, const RecEx& ex) {
  auto buf_ok = [&](uint64_t a, int buf, int64_t elems, const char* what) {
    if (elems <= 0) return;
    bool ok = false;
    if (buf == B_ABS) ok = ex.inside(a, elems * 8);
    else if (buf == B_PSI || buf == B_SIG) ok = (int64_t)a + elems <= lay.size;
    else if (buf == B_TMP) ok = (int64_t)a + elems <= P.tmp_elems;
    if (!ok) fail(std::string("fp64 plan: ") + what + " out of its buffer");
  };
  for (size_t c = 0; c < P.stage1.size(); ++c)
    for (const Launch* L : {&P.stage1[c], &P.stage2[c]}) {
      for (const Prob& p : L->probs) {
        if (p.nseg <= 0) fail("fp64 plan: problem without segments");
        if (p.seg0 < 0 || p.seg0 + p.nseg > (int)L->segs.size()) fail("fp64 plan: segment range");
        buf_ok(p.c, p.cbuf, extent(p.m, p.n, p.ldc, 0), "output");
        for (int s = p.seg0; s < p.seg0 + p.nseg && s < (int)L->segs.size(); ++s) {
          const Seg& g = L->segs[s];
          if (g.k <= 0) fail("fp64 plan: segment without K");
          if (!(g.a == 0 && g.abuf == B_ABS)) buf_ok(g.a, g.abuf, extent(p.m, g.k, g.lda, g.ta), "A operand");
          if (!(g.b == 0 && g.bbuf == B_ABS)) buf_ok(g.b, g.bbuf, extent(g.k, p.n, g.ldb, g.tb), "B operand");
        }
      }
    }
}

void check_tiled(const HeffPlan& P, const PsiLayout& lay, const RecEx& ex, const TileCfg& cfg, int64_t tbudget = 0) {
  const TiledPlan T = plan_tiled(P, lay, cfg, tbudget);
  // passes: item ranges cover both stages in order, and every T_t a stage-2
  // segment reads is written by a stage-1 view of the same pass
  if (T.pass1.size() < 2 || T.pass1.size() != T.pass2.size() || T.pass1.front() != 0 || T.pass2.front() != 0 ||
      T.pass1.back() != (int)T.i1.size() || T.pass2.back() != (int)T.i2.size())
    fail("tiled passes do not cover the items");
  for (int p = 0; p + 1 < (int)T.pass1.size(); ++p) {
    if (T.pass1[p + 1] < T.pass1[p] || T.pass2[p + 1] < T.pass2[p]) fail("tiled pass ranges out of order");
    std::set<int64_t> written;
    for (int i = T.pass1[p]; i < T.pass1[p + 1]; ++i)
      for (int v = T.i1[i].v0; v < T.i1[i].v0 + T.i1[i].nv; ++v) written.insert(T.v1[v].tout);
    for (int i = T.pass2[p]; i < T.pass2[p + 1]; ++i)
      for (int sg = T.i2[i].s0; sg < T.i2[i].s1; ++sg)
        if (!written.count(T.s2[sg].b)) fail("stage-2 segment reads a T tile its pass does not write");
  }
  if (tbudget == 0 && T.npasses() != 1) fail("unbounded tiled plan with more than one pass");
  if (std::getenv("PLANNER_TILED_STATS") && cfg.kmax == 4096 && cfg.width == 256) {
    // MMA work of both stages (M = 128 rows per A panel, N = the B panel rows rounded to 16,
    // K rounded to 16) against the algorithmic flops; chunks of 64 K per MMA group
    double mma1 = 0, mma2 = 0, kch1 = 0, kch2 = 0;
    for (const K1Item& it : T.i1)
      for (int v = it.v0; v < it.v0 + it.nv; ++v) {
        const int nm = 16 * ((it.nrows + 15) / 16), kk = 16 * ((it.k + 15) / 16);
        mma1 += 2.0 * 128 * nm * kk;
        kch1 += (kk + 63) / 64;
      }
    for (const K2Item& it : T.i2)
      for (int sg = it.s0; sg < it.s1; ++sg) {
        const int nm = 16 * ((it.nrows + 15) / 16), kk = 16 * ((T.s2[sg].k + 15) / 16);
        mma2 += 2.0 * 128 * nm * kk;
        kch2 += (kk + 63) / 64;
      }
    std::printf("tiled: stage1 items %zu views %zu, stage2 items %zu segs %zu; MMA flops %.3f + %.3f TFLOP for %.3f "
                "useful (padding %.2fx); K chunks of 64: %.0f + %.0f; arenas A %.2f B %.2f psi %.3f T %.2f GB/plane\n",
                T.i1.size(), T.v1.size(), T.i2.size(), T.s2.size(), mma1 / 1e12, mma2 / 1e12, T.flops / 1e12,
                (mma1 + mma2) / T.flops, kch1, kch2, T.abytes / 1e9, T.bbytes / 1e9, T.psibytes / 1e9,
                T.tbytes / 1e9);
  }
  if (std::getenv("PLANNER_CHUNK_STATS") && cfg.kmax == 4096 && cfg.width == 256) {
    // chunks the tiled kernel's producer issues per product, for a fixed K depth per
    // chunk (KC) or one chosen per item so that a chunk holds about `target` bytes
    for (int np : {1, 3}) {
      const int KC = np == 1 ? 64 : 32;
      for (int target : {0, 32768, 49152, 65536}) {
        auto depth = [&](int per8) {
          if (target == 0) return KC;
          const int c = std::min(256, std::max(KC, 16 * (target / (2 * per8))));
          return c;
        };
        double c1 = 0, c2 = 0;
        for (const K1Item& it : T.i1) {
          int pa = 0;
          for (int v = it.v0; v < it.v0 + it.nv; ++v) pa += T.v1[v].pa8;
          const int kc = depth(np * (pa + it.pb8) * 128);
          const int kp = tiled_c8(it.k) * 8;
          c1 += (kp + kc - 1) / kc;
        }
        for (const K2Item& it : T.i2) {
          const int pa8 = (it.mrows + 7) / 8, pb8 = (it.nrows + 7) / 8;
          const int kc = depth(np * (pa8 + pb8) * 128);
          int packed = 0, bytes = 0;
          for (int sg = it.s0; sg < it.s1; ++sg) {
            const int kp = tiled_c8(T.s2[sg].k) * 8;
            if (kp == 0) continue;
            if (kp > kc) {
              c2 += (kp + kc - 1) / kc;
              continue;
            }
            const int b = np * (pa8 + pb8) * (kp / 8) * 128;
            if (packed == 0 || packed == 16 || bytes + b > std::max(32768, target)) {
              c2 += 1;
              packed = 0;
              bytes = 0;
            }
            ++packed;
            bytes += b;
          }
        }
        std::printf("chunks: planes %d target %d: stage 1 %.0f, stage 2 %.0f\n", np, target, c1, c2);
      }
    }
  }
  if (T.flops != P.flops) fail("tiled plan: flop count differs from the FP64 plan");
  // conversion views
  auto views_ok = [&](const std::vector<TView>& vs, int64_t arena, const char* what) {
    for (const TView& v : vs) {
      if (v.rows <= 0 || v.cols <= 0) fail(std::string("tiled view without rows or columns: ") + what);
      if (v.dst < 0 || v.dst + tiled_bytes(v.rows, v.cols, v.panel) > arena)
        fail(std::string("tiled view past its arena: ") + what);
      if (v.src == 0 && v.buf == 0) continue;  // scaled identity
      const int64_t e = extent(v.rows, v.cols, v.ld, v.tr);
      if (v.buf == 1 ? (int64_t)v.src + e > lay.size : !ex.inside(v.src, e * 8))
        fail(std::string("tiled view source out of its buffer: ") + what);
    }
  };
  views_ok(T.avw, T.abytes, "left");
  views_ok(T.bvw, T.bbytes, "right");
  views_ok(T.psivw, T.psibytes, "psi");
  // stage 1
  int64_t nviews = 0;
  for (const K1Item& it : T.i1) {
    if (it.nv <= 0 || it.nv > 16) fail("stage-1 item with 0 or more than 16 views");
    if (it.k <= 0 || it.nrows <= 0 || it.nrows > TP_B) fail("stage-1 item shape");
    const int c8 = tiled_c8(it.k);
    if (it.pb8 != (it.nrows + 7) / 8) fail("stage-1 psi panel core rows");
    if (it.b + (int64_t)it.pb8 * c8 * 128 > T.psibytes) fail("stage-1 psi panel past the psi arena");
    int cols = 0;
    for (int v = it.v0; v < it.v0 + it.nv; ++v) {
      if (v < 0 || v >= (int)T.v1.size()) {
        fail("stage-1 view index");
        continue;
      }
      const K1View& w = T.v1[v];
      ++nviews;
      if (w.mrows <= 0 || w.mrows > TP_A || w.pa8 != (w.mrows + 7) / 8) fail("stage-1 view rows");
      if (w.a + (int64_t)w.pa8 * c8 * 128 > T.bbytes) fail("stage-1 view panel past the right arena");
      if (w.tcol % 16 || w.tcol != cols) fail("stage-1 accumulator columns not packed in order");
      cols = w.tcol + 16 * ((it.nrows + 15) / 16);
      if (cols > 256) fail("stage-1 accumulator columns beyond 256");
      if (w.mp * TP_A + w.mrows > w.ntot) fail("stage-1 view rows beyond T rows");
      if (w.tout < 0 || w.tout + tiled_bytes(w.ntot, it.mtot, TP_B) > T.tbytes) fail("stage-1 T tile past the T arena");
      if (it.np * TP_B + it.nrows > it.mtot) fail("stage-1 psi panel beyond the psi block rows");
    }
  }
  if (nviews != (int64_t)T.v1.size()) fail("stage-1 views not covered exactly once");
  // stage 2
  std::vector<int> seen(T.s2.size(), 0);
  for (const K2Item& it : T.i2) {
    if (it.s1 <= it.s0) fail("stage-2 item without segments");
    if (it.mrows <= 0 || it.mrows > TP_A || it.nrows <= 0 || it.nrows > TP_B) fail("stage-2 tile shape");
    const int64_t last = it.out + (int64_t)(it.mp * TP_A + it.mrows - 1) * it.ldc + it.np * TP_B + it.nrows;
    if (it.out < 0 || last > lay.size) fail("stage-2 tile past sigma");
    const int pa8 = (it.mrows + 7) / 8, pb8 = (it.nrows + 7) / 8;
    for (int s = it.s0; s < it.s1; ++s) {
      if (s < 0 || s >= (int)T.s2.size()) {
        fail("stage-2 segment index");
        continue;
      }
      seen[s]++;
      const K2Seg& g = T.s2[s];
      if (g.k <= 0) fail("stage-2 segment without K");
      const int c8 = tiled_c8(g.k);
      if (g.a + (int64_t)it.mp * (TP_A / 8) * c8 * 128 + (int64_t)pa8 * c8 * 128 > T.abytes)
        fail("stage-2 left view panel past the left arena");
      if (g.b + (int64_t)it.np * (TP_B / 8) * c8 * 128 + (int64_t)pb8 * c8 * 128 > T.tbytes)
        fail("stage-2 T panel past the T arena");
    }
  }
  // every segment is used by the tiles of its sigma block: same count for all
  // segments of a block, at least once
  for (size_t s = 0; s < seen.size(); ++s)
    if (seen[s] < 1) fail("stage-2 segment never used");
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 4) {
    std::fprintf(stderr, "usage: planner_check L N D [pair_switch [sum_gemm [su2]]]\n");
    return 2;
  }
  const int L = std::atoi(argv[1]), N = std::atoi(argv[2]), D = std::atoi(argv[3]);
  const bool su2 = argc > 6 && std::atoi(argv[6]) != 0;
  const int two_s = su2 ? 0 : N % 2;
  RecEx ex;
  NullRunner pr;
  Engine E;
  E.ex = &ex;
  E.pr = &pr;
  E.N = N;
  E.two_s = two_s;
  E.L = L;
  E.su2 = su2;
  E.tmp_budget = (int64_t)(2e9 / 8);
  if (argc > 4) E.pair_switch = std::atoi(argv[4]);
  if (argc > 5) E.sum_gemm = std::atoi(argv[5]);
  E.I.L = L;
  E.I.h.assign((size_t)L * L, 0.0);
  E.I.V.assign((size_t)L * L * L * L, 0.0);
  // generic symmetric integrals (every coupling present)
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q) E.I.h[(size_t)p * L + q] = 0.1 + 0.01 * ((p + q) % 7);
  for (int p = 0; p < L; ++p)
    for (int q = 0; q < L; ++q)
      for (int r = 0; r < L; ++r)
        for (int s = 0; s < L; ++s) {
          const int a = std::min(p, q) * L + std::max(p, q), b = std::min(r, s) * L + std::max(r, s);
          E.I.V[(((size_t)p * L + q) * L + r) * L + s] = 0.01 + 1e-3 * ((std::min(a, b) * 31 + std::max(a, b) * 17) % 97);
        }
  const int center = L / 2 - 1;
  auto st = mps_structure(L, N, two_s, D, su2);
  std::vector<Basis> bonds(L + 1);
  for (auto& b : bonds) b.su2 = su2;
  for (int b = 0; b <= center; ++b)
    for (auto& kv : st[b]) bonds[b].add(kv.first, kv.second);
  for (int b = center + 2; b <= L; ++b)
    for (auto& kv : st[L - b]) bonds[b].add(kv.first, kv.second);
  E.site.assign(L, 0);
  E.site_off.assign(L, {});
  E.site_nb.assign(L, {});
  for (int p = 0; p < L; ++p) {
    if (p == center || p == center + 1) continue;
    const bool left = p < center;
    const Basis& from = left ? bonds[p] : bonds[p + 1];
    const Basis& to = left ? bonds[p + 1] : bonds[p];
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
    E.site[p] = ex.alloc(std::max<int64_t>(1, tot));
    E.site_off[p] = so;
    E.site_nb[p] = nb;
  }
  E.bonds = bonds;
  E.center = center;
  {
    ProdBasis a = make_prod(bonds[center], true), b = make_prod(bonds[center + 2], false);
    PsiLayout l = make_psi_layout(a, b, QN{N, two_s});
    E.dpsi = ex.alloc(std::max<int64_t>(1, l.size));
  }
  E.build_env();
  check_fp64(E.plan, E.lay, ex);
  for (int kmax : {1024, 4096, 1 << 30})
    for (int width : {128, 256}) {
      TileCfg cfg;
      cfg.kmax = kmax;
      cfg.width = width;
      check_tiled(E.plan, E.lay, ex, cfg);
      if (kmax == 4096 && width == 256) {
        // T arena split into about five passes
        const int64_t tb = plan_tiled(E.plan, E.lay, cfg).tbytes;
        check_tiled(E.plan, E.lay, ex, cfg, std::max<int64_t>(1, tb / 5));
      }
    }
  {
    // executed (padded) FP64 flops of the centre product: tiles of 64 or 32 (least
    // padding), K of each segment rounded up to 16
    auto tsz = [](int d) { return ((d + 63) / 64) * 64 <= ((d + 31) / 32) * 32 ? 64 : 32; };
    double exec_fl = 0, useful = 0, exec_k = 0, exec_k8 = 0, exec_16 = 0, exec_w = 0;
    for (auto* Lv : {&E.plan.stage1, &E.plan.stage2})
      for (const Launch& l : *Lv) {
        useful += l.flops;
        for (const Prob& p : l.probs) {
          const int tm = tsz(p.m), tn = tsz(p.n);
          const double tiles = (double)((p.m + tm - 1) / tm) * ((p.n + tn - 1) / tn);
          for (int k = 0; k < p.nseg; ++k) {
            const Seg& g = l.segs[p.seg0 + k];
            if (g.a == 0 && g.abuf == 0) continue;
            exec_fl += tiles * 2.0 * tm * tn * 16.0 * ((g.k + 15) / 16);
            exec_k += tiles * 2.0 * tm * tn * g.k;
            exec_k8 += tiles * 2.0 * tm * tn * 8.0 * ((g.k + 7) / 8);
            const int tm2 = 16 * ((p.m + 15) / 16) <= 64 ? 16 * ((p.m + 15) / 16) : tm;
            const int tn2 = 16 * ((p.n + 15) / 16) <= 64 ? 16 * ((p.n + 15) / 16) : tn;
            const double tiles2 = (double)((p.m + tm2 - 1) / tm2) * ((p.n + tn2 - 1) / tn2);
            exec_16 += tiles2 * 2.0 * tm2 * tn2 * 8.0 * ((g.k + 7) / 8);
            // warps skip 16-row x (tn/2)-column regions outside the problem; K exact
            for (int m0 = 0; m0 < p.m; m0 += tm)
              for (int n0 = 0; n0 < p.n; n0 += tn) {
                const int rm = std::min(tm, p.m - m0), rn = std::min(tn, p.n - n0);
                const int wc = tn / 2;
                exec_w += 2.0 * (16.0 * ((rm + 15) / 16)) * (wc * ((rn + wc - 1) / wc)) * g.k;
              }
          }
        }
      }
    if (std::getenv("PLANNER_REGION_STATS")) {
      // FP64 executed by warp regions of rh x rw outputs (exact K), per region shape
      // and with the best shape chosen per problem; and at 8 x 8 granularity
      const int shapes[3][2] = {{16, 32}, {8, 64}, {32, 16}};
      double ex[3] = {0, 0, 0}, best = 0, fine = 0;
      for (auto* Lv : {&E.plan.stage1, &E.plan.stage2})
        for (const Launch& l : *Lv)
          for (const Prob& p : l.probs) {
            double kk = 0;
            for (int k = 0; k < p.nseg; ++k) {
              const Seg& g = l.segs[p.seg0 + k];
              if (!(g.a == 0 && g.abuf == 0)) kk += g.k;
            }
            const int tm = tsz(p.m), tn = tsz(p.n);
            double e3[3] = {0, 0, 0};
            for (int m0 = 0; m0 < p.m; m0 += tm)
              for (int n0 = 0; n0 < p.n; n0 += tn) {
                const int rm = std::min(tm, p.m - m0), rn = std::min(tn, p.n - n0);
                for (int sh = 0; sh < 3; ++sh) {
                  const int rh = shapes[sh][0], rw = shapes[sh][1];
                  e3[sh] += 2.0 * (rh * ((rm + rh - 1) / rh)) * (rw * ((rn + rw - 1) / rw)) * kk;
                }
              }
            for (int sh = 0; sh < 3; ++sh) ex[sh] += e3[sh];
            best += std::min(e3[0], std::min(e3[1], e3[2]));
            fine += 2.0 * (8.0 * ((p.m + 7) / 8)) * (8.0 * ((p.n + 7) / 8)) * kk;
          }
      std::printf("fp64 regions: useful/executed 16x32 %.3f, 8x64 %.3f, 32x16 %.3f, best per problem %.3f, "
                  "8x8 %.3f\n", useful / ex[0], useful / ex[1], useful / ex[2], useful / best, useful / fine);
    }
    std::printf("fp64 padding: useful %.3f TFLOP, executed %.3f TFLOP, efficiency %.3f (exact K %.3f, K by 8 %.3f, "
                "tiles by 16 up to 64 and K by 8 %.3f, warp skipping %.3f)\n", useful / 1e12, exec_fl / 1e12,
                useful / exec_fl, useful / exec_k, useful / exec_k8, useful / exec_16, useful / exec_w);
  }
  int64_t lp = 0, rp = 0;
  for (uint64_t a : E.Lp.owned) lp += ex.alloc_bytes.at(a);
  for (uint64_t a : E.Rp.owned) rp += ex.alloc_bytes.at(a);
  std::printf("centre enlarged blocks: left %.2f GB (%zu ops), right %.2f GB (%zu ops)\n", lp / 1e9, E.Lp.ops.size(),
              rp / 1e9, E.Rp.ops.size());
  int64_t env = 0;
  for (auto& kv : E.lenv)
    for (int64_t n : kv.second.owned_n) env += 8 * n;
  for (auto& kv : E.renv)
    for (int64_t n : kv.second.owned_n) env += 8 * n;
  std::printf("L=%d N=%d D=%d psi=%lld terms=%d gflop=%.4f launches=%lld fails=%d peak_gb=%.2f live_gb=%.2f env_gb=%.2f "
              "heff_gb=%.3f env_tflop=%.2f\n", L, N, D, (long long)E.lay.size, E.plan.nterms, E.plan.flops / 1e9,
              (long long)ex.launches_checked, fails, ex.peak / 1e9, ex.cur_live / 1e9, env / 1e9, E.plan.bytes / 1e9,
              E.env_flops / 1e12);
  std::printf("heff plan: flops=%.17g bytes=%.17g\n", E.plan.flops, E.plan.bytes);
  return fails ? 1 : 0;
}
