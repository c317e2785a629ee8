// Backend interface shared by the C ABI and the CUDA executor.
#pragma once
#include <cuda_runtime.h>

#include "core.hpp"
#include "tiled.hpp"

namespace qd {

// Launch lists uploaded once and replayed on any psi / sigma pair.
struct PreparedRunner {
  virtual ~PreparedRunner() {}
  virtual int prepare(const Launch& l) = 0;
  virtual void drop_prepared() = 0;
  // precision: 0 FP64 (CUDA cores), 1 TF32, 2 BF16, 3 BF16x3 (tcgen05)
  virtual void run_prepared(int handle, uint64_t psi, uint64_t sig, void* stream, int precision) = 0;
  // returns and clears the device error flag of the tensor-core kernels
  virtual int take_error() = 0;
  // opaque device task list of a prepared launch (for the no-allocation path)
  virtual const void* prepared_handle(int handle) const = 0;
  // FP64 work items of a prepared launch: tiles per shape class (64x64, 64x32,
  // 32x64, 32x32) in counts[0..3], split-K tiles (FP64 atomics) in counts[4]
  virtual void tile_counts(int handle, int64_t counts[5]) const = 0;
  virtual void* stream() = 0;
  virtual void sync(void* stream) = 0;
  virtual void zero_async(uint64_t p, int64_t n, void* stream) = 0;
  virtual int64_t bytes_allocated() const = 0;
  // bulk-copy-fed tensor-core path (BF16, BF16x3): bf16 operand mirrors with one or
  // three planes and the work items of both stages (dropped with the prepared
  // launches); tiled_planes() is 0 when nothing is prepared
  virtual void prepare_tiled(const TiledPlan& plan, int planes) = 0;
  // replaces the work items only (same arenas: another TileCfg of the same plan)
  virtual void set_tiled_items(const TiledPlan& plan) = 0;
  // chunk byte target of the tiled kernels (0: fixed K depth per chunk)
  virtual void set_tiled_chunk(int bytes) { (void)bytes; }
  virtual int tiled_planes() const = 0;
  // device bytes free now, counting the tiled path's current arenas as free (the
  // tiled path sizes its T arena from it when it prepares a centre, which
  // releases those arenas first)
  virtual int64_t free_device_bytes() const { return INT64_MAX; }
  // device seconds of one H_eff psi on the tiled path (mean of reps, after one warm-up)
  virtual double time_tiled(uint64_t psi, uint64_t sig, int precision, int reps) = 0;
  // sigma must be zero; precision 2 (BF16) or 3 (BF16x3)
  virtual void run_tiled(uint64_t psi, uint64_t sig, void* stream, int precision) = 0;
};

struct Backend {
  Executor* ex = nullptr;
  PreparedRunner* pr = nullptr;
};

// Creates the CUDA backend on a device (throws std::runtime_error on failure).
Backend make_backend(int device);

// Runs one prepared launch with the FP64 kernel, scratch base given by the caller.
cudaError_t launch_f64_prepared(const void* handle, uint64_t psi, uint64_t sig, uint64_t scratch,
                                cudaStream_t st);

}  // namespace qd
