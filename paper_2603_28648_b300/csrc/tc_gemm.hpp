// Device task-list records shared by the FP64 and tcgen05 segmented GEMMs.
#pragma once
#include <cuda_runtime.h>

namespace qd {

struct GSeg {
  unsigned long long a, b;   // a == 0 && abuf == 0: A = I (and B = I if also b == 0 && bbuf == 0)
  int lda, ldb, k;
  unsigned char abuf, bbuf, ta, tb;
  double sc;
};
struct GProb {
  unsigned long long c;
  int m, n, ldc, beta, seg0, nseg, cbuf, pad;
};
// One work item: tile (m0, n0) of a problem over segments [s0, s1). A problem
// split over several segment ranges is accumulated with FP64 atomics; every
// output that is split is zero-initialised or has beta = 1.
struct GTile {
  int prob, m0, n0, s0, s1, split;
};
struct Bases {
  unsigned long long b[4];   // 0: absolute, 1: psi, 2: sigma, 3: scratch
};
using TcSeg = GSeg;
using TcProb = GProb;
using TcTile = GTile;
using TcBases = Bases;

enum TcMode : int { TC_TF32 = 3 };
constexpr int TC_TILE = 128;

// Launch the tcgen05 kernel of the given mode (TF32) over 128x128 tiles. err (device
// int) is set to 1 if a bounded wait gave up.
cudaError_t launch_tc(int mode, const TcProb* P, const TcSeg* S, const TcTile* T, int nt, TcBases B,
                      int* err, cudaStream_t st);

}  // namespace qd
