// Work items of the bulk-copy-fed tensor-core H_eff psi (see tiled.hpp), derived
// from the FP64 task lists of the same product.
#include "tiled.hpp"

#include <cstring>
#include <map>
#include <stdexcept>
#include <tuple>
#include <unordered_map>

namespace qd {

namespace {

using VKey = std::tuple<uint64_t, int, int, int, int, int, double>;  // src, buf, ld, tr, rows, cols, scale

inline uint64_t mix(uint64_t h, uint64_t v) {
  // splitmix64 finaliser of the running value
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  h ^= h >> 30;
  h *= 0xbf58476d1ce4e5b9ull;
  h ^= h >> 27;
  h *= 0x94d049bb133111ebull;
  return h ^ (h >> 31);
}
struct VKeyHash {
  size_t operator()(const VKey& k) const {
    uint64_t sb = 0;
    const double sc = std::get<6>(k);
    if (sc != 0.0) std::memcpy(&sb, &sc, 8);   // +0 and -0 compare equal: one hash
    uint64_t h = mix(0, std::get<0>(k));
    h = mix(h, ((uint64_t)(uint32_t)std::get<1>(k) << 32) | (uint32_t)std::get<2>(k));
    h = mix(h, ((uint64_t)(uint32_t)std::get<3>(k) << 32) | (uint32_t)std::get<4>(k));
    h = mix(h, (uint64_t)(uint32_t)std::get<5>(k));
    return (size_t)mix(h, sb);
  }
};
struct PairHash {
  size_t operator()(const std::pair<int64_t, double>& k) const {
    uint64_t sb = 0;
    if (k.second != 0.0) std::memcpy(&sb, &k.second, 8);
    return (size_t)mix(mix(0, (uint64_t)k.first), sb);
  }
};

// views are deduplicated through a hash index; offsets follow insertion order,
// so the arenas do not depend on the index's iteration order
struct Arena {
  std::vector<TView>* views;
  int64_t* bytes;
  int panel;
  std::unordered_map<VKey, int64_t, VKeyHash> index;
  int64_t add(uint64_t src, int buf, int ld, int tr, int rows, int cols, double scale) {
    VKey k{src, buf, ld, tr, rows, cols, scale};
    auto it = index.find(k);
    if (it != index.end()) return it->second;
    TView v{src, buf, rows, cols, ld, tr, panel, scale, *bytes};
    views->push_back(v);
    index[k] = *bytes;
    *bytes += tiled_bytes(rows, cols, panel);
    return v.dst;
  }
};

struct TProd {       // one T_t: psi block x right view
  int blk;
  int64_t b, tout;
  int n, k;
  double osc;
};

struct SigBlk {
  int64_t out;
  int m, n, ldc;
  std::vector<K2Seg> segs;
  std::vector<int> tp;   // the T_t of each segment
};

inline int round16(int x) { return 16 * ((x + 15) / 16); }

}  // namespace

TiledPlan plan_tiled(const HeffPlan& plan, const PsiLayout& lay, const TileCfg& cfg, int64_t tbudget) {
  const int kmax = cfg.kmax;
  TiledPlan P;
  P.flops = plan.flops;
  P.psi_elems = lay.size;
  Arena psi{&P.psivw, &P.psibytes, TP_B, {}};
  Arena am{&P.avw, &P.abytes, TP_A, {}};
  Arena bm{&P.bvw, &P.bbytes, TP_A, {}};
  std::unordered_map<int64_t, int> blk_of_off;
  std::vector<int64_t> psi_off(lay.blks.size());
  for (size_t i = 0; i < lay.blks.size(); ++i) {
    const auto& b = lay.blks[i];
    // every work item of the kernels needs at least one K step: an empty
    // block would leave an accumulator that no MMA completes
    if (b.rows <= 0 || b.cols <= 0) throw std::runtime_error("tiled plan: empty psi block");
    blk_of_off[b.off] = (int)i;
    psi_off[i] = psi.add((uint64_t)b.off, 1, b.cols, 0, b.rows, b.cols, 1.0);
  }
  auto blk_at = [&](int64_t off) {
    auto it = blk_of_off.find(off);
    if (it == blk_of_off.end()) throw std::runtime_error("tiled plan: psi block not found");
    return it->second;
  };

  std::vector<TProd> tps;
  {
    size_t n1 = 0, n2 = 0;
    for (const Launch& l : plan.stage1) n1 += l.probs.size();
    for (const Launch& l : plan.stage2) n2 += l.segs.size();
    tps.reserve(n1 + n2 / 8 + 16);
  }
  auto add_t = [&](int blk, int64_t b, int n, int k, double osc) {
    tps.push_back({blk, b, P.tbytes, n, k, osc});
    P.tbytes += tiled_bytes(n, lay.blks[blk].rows, TP_B);  // transposed: n rows, K = psi rows
    return (int)tps.size() - 1;
  };
  std::unordered_map<std::pair<int64_t, double>, int, PairHash> copies;  // (psi offset, scalar) -> T_t of psi itself
  std::unordered_map<int64_t, int> sig_of;
  std::vector<SigBlk> sig;

  for (size_t c = 0; c < plan.stage1.size(); ++c) {
    const Launch& L1 = plan.stage1[c];
    const Launch& L2 = plan.stage2[c];
    std::unordered_map<uint64_t, int> t_of;  // FP64 stage-1 output offset of this chunk -> T_t
    t_of.reserve(L1.probs.size());
    for (const Prob& p : L1.probs) {
      const Seg& h = L1.segs[p.seg0];
      const int blk = blk_at((int64_t)h.a);
      if (lay.blks[blk].rows != p.m || lay.blks[blk].cols != h.k)
        throw std::runtime_error("tiled plan: stage-1 shape");
      const int64_t b = bm.add(h.b, 0, h.ldb, h.tb ? 0 : 1, p.n, h.k, 1.0);
      t_of[p.c] = add_t(blk, b, p.n, h.k, p.osc);
    }
    for (const Prob& p : L2.probs) {
      auto it = sig_of.find((int64_t)p.c);
      int si;
      if (it == sig_of.end()) {
        si = (int)sig.size();
        sig_of[(int64_t)p.c] = si;
        sig.push_back({(int64_t)p.c, p.m, p.n, p.ldc, {}, {}});
      } else {
        si = it->second;
      }
      for (int s = 0; s < p.nseg; ++s) {
        const Seg& g = L2.segs[p.seg0 + s];
        int tp;
        if (g.bbuf == B_TMP) {
          auto jt = t_of.find(g.b);
          if (jt == t_of.end()) throw std::runtime_error("tiled plan: stage-1 output not found");
          tp = jt->second;
          if (tps[tp].osc != g.bsc) throw std::runtime_error("tiled plan: stage-1 scalar differs between users");
        } else if (g.bbuf == B_PSI) {
          auto key = std::make_pair((int64_t)g.b, g.bsc);
          auto jt = copies.find(key);
          if (jt != copies.end()) {
            tp = jt->second;
          } else {
            const int blk = blk_at((int64_t)g.b);
            const int n = lay.blks[blk].cols;
            tp = add_t(blk, bm.add(0, 0, 0, 0, n, n, 1.0), n, n, g.bsc);
            copies[key] = tp;
          }
        } else {
          throw std::runtime_error("tiled plan: unexpected stage-2 operand");
        }
        if (tps[tp].n != p.n || lay.blks[tps[tp].blk].rows != g.k)
          throw std::runtime_error("tiled plan: stage-2 shape");
        // the left reference scalar (sign included) is folded into its view
        const int64_t a = (g.a == 0 && g.abuf == B_ABS) ? am.add(0, 0, 0, 0, p.m, g.k, g.asc)
                                                         : am.add(g.a, 0, g.lda, g.ta, p.m, g.k, g.asc);
        if (g.k <= 0) throw std::runtime_error("tiled plan: stage-2 segment without K");
        sig[si].segs.push_back({a, tps[tp].tout, g.k, 0});
        sig[si].tp.push_back(tp);
      }
    }
  }

  // passes: T_t in creation order, a new pass when the next one would take
  // the pass beyond the budget; offsets rebased to the pass start
  std::vector<int> tpass(tps.size(), 0);
  int npass = 1;
  if (tbudget > 0 && P.tbytes > tbudget) {
    int64_t start = 0, top = 0;
    for (size_t i = 0; i < tps.size(); ++i) {
      const int64_t sz = tiled_bytes(tps[i].n, lay.blks[tps[i].blk].rows, TP_B);
      if (tps[i].tout + sz - start > tbudget && tps[i].tout > start) {
        start = tps[i].tout;
        ++npass;
      }
      tpass[i] = npass - 1;
      tps[i].tout -= start;
      top = std::max(top, tps[i].tout + sz);
    }
    P.tbytes = top;
    for (SigBlk& sb : sig)
      for (size_t k = 0; k < sb.segs.size(); ++k) sb.segs[k].b = tps[sb.tp[k]].tout;
  }
  // stage 1: T_t grouped by psi block, blocks ordered by right then left
  // sector so that consecutive items reuse the same right views from L2; an
  // item holds views while their accumulator columns fit the width and their
  // rows fit the 256 A rows of a chunk
  std::vector<std::vector<int>> by_blk(lay.blks.size());
  for (int i = 0; i < (int)tps.size(); ++i) by_blk[tps[i].blk].push_back(i);
  std::vector<int> order(lay.blks.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    return std::make_pair(lay.blks[x].rsub, lay.blks[x].lsub) < std::make_pair(lay.blks[y].rsub, lay.blks[y].lsub);
  });
  P.pass1.assign(1, 0);
  for (int pass = 0; pass < npass; ++pass) {
  for (int blk : order) {
    if (by_blk[blk].empty()) continue;
    bool any = false;
    for (int tp : by_blk[blk]) any = any || tpass[tp] == pass;
    if (!any) continue;
    const auto& pb = lay.blks[blk];
    const int c8 = tiled_c8(pb.cols);
    for (int np = 0; np * TP_B < pb.rows; ++np) {
      const int nrows = std::min(TP_B, pb.rows - np * TP_B);
      const int nm = round16(nrows);
      K1Item it{};
      it.b = psi_off[blk] + (int64_t)np * (TP_B / 8) * c8 * 128;
      it.pb8 = (nrows + 7) / 8;
      it.nrows = nrows;
      it.k = pb.cols;
      it.np = np;
      it.mtot = pb.rows;
      it.v0 = (int)P.v1.size();
      it.nv = 0;
      int col = 0, rows = 0;
      for (int tp : by_blk[blk]) {
        if (tpass[tp] != pass) continue;
        const TProd& t = tps[tp];
        for (int mp = 0; mp * TP_A < t.n; ++mp) {
          const int mrows = std::min(TP_A, t.n - mp * TP_A);
          const int r8 = 8 * ((mrows + 7) / 8);
          if (it.nv && (col + nm > std::max(cfg.width, nm) || rows + r8 > 2 * TP_A || it.nv == 16)) {
            P.i1.push_back(it);
            it.v0 = (int)P.v1.size();
            it.nv = 0;
            col = 0;
            rows = 0;
          }
          K1View v{};
          v.a = t.b + (int64_t)mp * (TP_A / 8) * c8 * 128;
          v.tout = t.tout;
          v.osc = t.osc;
          v.pa8 = r8 / 8;
          v.mrows = mrows;
          v.tcol = col;
          v.mp = mp;
          v.ntot = t.n;
          P.v1.push_back(v);
          it.nv++;
          col += nm;
          rows += r8;
        }
      }
      if (it.nv) P.i1.push_back(it);
    }
  }
  P.pass1.push_back((int)P.i1.size());
  }

  // stage 2: per pass, the segments of each sigma block in that pass, ranges
  // of summed K <= kmax, costliest first; a block split over several ranges
  // or passes adds with atomics
  P.pass2.assign(1, 0);
  for (int pass = 0; pass < npass; ++pass) {
    std::vector<std::pair<double, K2Item>> items;
    for (const SigBlk& sb : sig) {
      if (sb.segs.empty()) continue;
      bool here = false, elsewhere = false;
      for (int tp : sb.tp) {
        if (tpass[tp] == pass) here = true;
        else elsewhere = true;
      }
      if (!here) continue;
      std::vector<std::pair<int, int>> ranges;
      int s0 = (int)P.s2.size(), ks = 0;
      for (size_t k = 0; k < sb.segs.size(); ++k) {
        if (tpass[sb.tp[k]] != pass) continue;
        const K2Seg& g = sb.segs[k];
        const int s = (int)P.s2.size();
        if (s > s0 && ks + g.k > kmax) {
          ranges.push_back({s0, s});
          s0 = s;
          ks = 0;
        }
        ks += g.k;
        P.s2.push_back(g);
      }
      ranges.push_back({s0, (int)P.s2.size()});
      const int split = (ranges.size() > 1 || elsewhere) ? 1 : 0;
      for (int mp = 0; mp * TP_A < sb.m; ++mp)
        for (int np = 0; np * TP_B < sb.n; ++np)
          for (auto& r : ranges) {
            K2Item it{};
            it.out = sb.out;
            it.ldc = sb.ldc;
            it.mrows = std::min(TP_A, sb.m - mp * TP_A);
            it.nrows = std::min(TP_B, sb.n - np * TP_B);
            it.mp = mp;
            it.np = np;
            it.s0 = r.first;
            it.s1 = r.second;
            it.split = split;
            double cost = 0;
            for (int s = r.first; s < r.second; ++s) cost += P.s2[s].k + 16;
            items.push_back({cost * round16(it.nrows), it});
          }
    }
    std::stable_sort(items.begin(), items.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (auto& x : items) P.i2.push_back(x.second);
    P.pass2.push_back((int)P.i2.size());
  }
  return P;
}

}  // namespace qd
