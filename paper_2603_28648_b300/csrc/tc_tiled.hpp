// Launchers of the bulk-copy-fed tensor-core H_eff psi kernels (tc_tiled.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tiled.hpp"

namespace qd {

constexpr int TT_BF16 = 0;    // one bf16 plane, one MMA per K step
constexpr int TT_BF16X3 = 1;  // three bf16 planes, six MMAs per K step

// FP64 views -> tiled bf16 planes (plane q at dst + q * plane_bytes);
// psi_base resolves views with buf == 1
cudaError_t launch_tile_views(const TView* views, int nviews, uint8_t* dst, int64_t plane_bytes, int planes,
                              const double* psi_base, cudaStream_t st);

// chunk_bytes: 0 moves a fixed K depth per chunk (64 for BF16, 32 for BF16x3);
// a positive value (at most 65536) deepens the chunks of small panels until a
// chunk holds about that many bytes (at most 256 K elements per chunk)

// Stage 1: T_t^T from the right views and psi (T arena pads must be zero)
cudaError_t launch_tiled_stage1(int mode, const K1Item* items, int nitems, const K1View* views,
                                const uint8_t* psi_arena, int64_t psi_plane, const uint8_t* r_arena,
                                int64_t r_plane, uint8_t* t_arena, int64_t t_plane, int chunk_bytes, int grid,
                                int* err, cudaStream_t st);

// Stage 2: sigma += O_L T_t (sigma zeroed by the caller)
cudaError_t launch_tiled_stage2(int mode, const K2Item* items, int nitems, const K2Seg* segs,
                                const uint8_t* a_arena, int64_t a_plane, const uint8_t* t_arena,
                                int64_t t_plane, double* sigma, int chunk_bytes, int grid, int* err,
                                cudaStream_t st);

}  // namespace qd
