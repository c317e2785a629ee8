// Tiled BF16 operands and work items of the bulk-copy-fed tensor-core H_eff psi.
//
// H_eff psi runs in two stages, both summed over the operator-product terms t:
//   stage 1: T_t = s_t psi_blk O_R^T   (one per term, right block reference, psi block)
//   stage 2: sigma_blk += O_L T_t       (every left block reference of the term)
// Every operand is stored once in bf16 (one plane, or three planes hi/mid/lo
// for the three-term split) in the K-major core-matrix layout that
// tcgen05.mma reads from shared memory: 8 x 8 bf16 core matrices of 128
// contiguous bytes; rows in panels (128 rows for A operands, 256 for B
// operands), each panel stored core column by core column; rows padded to 8
// and K to 16 with zeros. The bytes one K chunk of one panel needs are then a
// single contiguous range, copied to shared memory by one cp.async.bulk.
// Stage 1 writes T_t transposed (rows = columns of the sigma block, K = rows
// of the psi block) in the same layout, ready to be the B operand of stage 2.
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

#include "core.hpp"

#ifdef __CUDACC__
#define QD_HD __host__ __device__
#else
#define QD_HD
#endif

namespace qd {

constexpr int TP_A = 128;  // panel rows of A operands (MMA M)
constexpr int TP_B = 256;  // panel rows of B operands (largest MMA N)

// 16-byte core columns of a K extent, padded to a multiple of 16 elements
QD_HD inline int tiled_c8(int cols) { return 2 * ((cols + 15) / 16); }

// bytes of one plane of a tiled rows x cols operand with panel height P
inline int64_t tiled_bytes(int rows, int cols, int P) {
  int64_t r8 = 0;
  for (int p = 0; p < rows; p += P) r8 += (std::min(P, rows - p) + 7) / 8;
  return r8 * tiled_c8(cols) * 128;
}

// One operand to convert from FP64: view(r, c) = scale * src[r * ld + c]
// (tr: src[c * ld + r]); src == 0 with buf 0: scale * identity.
struct TView {
  uint64_t src;     // byte address (buf 0) or element offset into psi (buf 1)
  int buf;          // 0 absolute, 1 psi
  int rows, cols, ld, tr;
  int panel;        // TP_A or TP_B
  double scale;
  int64_t dst;      // byte offset in its arena (plane 0)
};

// Stage 1 computes T_t transposed directly, T_t^T = O_R psi_blk^T: the A
// operand is a right view (M = its rows, panel of 128), the B operand the psi
// block (N = its rows, panel of 256, K = its columns). An item is one psi panel
// times several views, each its own MMA into its own accumulator columns, so
// that accumulator lane = row of T_t^T and the epilogue stores 16-byte rows.
struct K1View {
  int64_t a;        // right-view arena offset of the view's panel
  int64_t tout;     // T arena offset of T_t^T (ntot rows, K = mtot)
  double osc;       // s_t: term coefficient x reference scalar x fermion parity
  int pa8, mrows;   // core rows and valid rows of the view panel
  int tcol;         // first accumulator column (multiple of 16)
  int mp, ntot;     // view panel index, rows of the view (rows of T_t^T)
  int pad;
};
struct K1Item {
  int64_t b;        // psi arena offset of the psi panel
  int pb8, nrows;   // core rows and valid rows of the psi panel
  int k;            // K = columns of the psi block
  int np, mtot;     // psi panel index, rows of the psi block (K of T_t^T)
  int v0, nv;       // views
  int pad;
};

// Stage 2. An item is one 128-row x up-to-256-column tile of one sigma block,
// summing O_L T_t over a range of segments (split items add with atomics).
struct K2Seg {
  int64_t a, b;     // A arena offset of the left reference view, T arena offset of T_t
  int k, neg;       // K; neg: negate the product (unused: scalars are folded into the views)
};
struct K2Item {
  int64_t out;      // element offset of the sigma block
  int ldc, mrows, nrows, mp, np;
  int s0, s1, split;
};

struct TiledPlan {
  std::vector<TView> avw, bvw, psivw;   // left views (A role), right views (A role), psi (B role)
  int64_t abytes = 0, bbytes = 0, psibytes = 0, tbytes = 0;
  int64_t psi_elems = 0;                // elements of psi and sigma
  std::vector<K1View> v1;
  std::vector<K1Item> i1;
  std::vector<K2Seg> s2;
  std::vector<K2Item> i2;
  // passes: the T_t of pass p occupy the T arena together (offsets rebased to
  // its start), stage-1 items [pass1[p], pass1[p+1]) write them and stage-2
  // items [pass2[p], pass2[p+1]) read them; the arena holds the largest pass
  std::vector<int> pass1, pass2;
  double flops = 0;                     // algorithmic, same count as the FP64 plan
  int npasses() const { return (int)pass1.size() - 1; }
};

// Work-item shape, picked per problem-size class by the autotuner.
//   kmax : summed K of one stage-2 item before a sigma block's segments are
//          split over several items (more parallelism, FP64 atomics)
//   width: accumulator columns of one stage-1 item (views side by side)
//   chunk: chunk byte target of the kernels (0: fixed K depth per chunk; the
//          items do not depend on it)
struct TileCfg {
  int kmax = 4096;
  int width = TP_B;
  int chunk = 0;
};

// The operand arenas (views, offsets, sizes) do not depend on the TileCfg,
// only the work items do. tbudget (bytes of one plane, 0: unlimited) bounds
// the T arena: the T_t are split into passes in creation order, each pass
// within the budget (a single T_t larger than it makes a pass of its own).
// A sigma block whose segments fall in several passes adds with atomics.
TiledPlan plan_tiled(const HeffPlan& plan, const PsiLayout& lay, const TileCfg& cfg, int64_t tbudget = 0);

}  // namespace qd
