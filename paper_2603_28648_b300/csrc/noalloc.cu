// H_eff psi without any allocation inside the call.
//
// Some callers cannot allocate device memory at the moment they need an
// H_eff psi: code that runs while a CUDA graph is being captured (where
// cudaMalloc is not allowed), code that shares the GPU with a framework whose
// caching allocator already holds all free memory, and solvers with a fixed
// memory budget that must not grow during iterations. qcdmrg_apply_heff_noalloc
// serves them: it runs the same FP64 task lists as qcdmrg_apply_heff_dev but
// keeps the stage-1 intermediates (psi blocks times right operator blocks) in
// the fixed device array below instead of the context's scratch buffer, and
// calls no allocating routine.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits. All calls share it and it keeps
// the contents of the last call; two calls whose kernels overlap on the GPU
// (different streams, or different contexts on one device) race on it.
// Nothing in it needs to start at zero: each intermediate is written by its
// stage-1 problem before any stage-2 problem reads it.
#include <cuda_runtime.h>

#include <mutex>
#include <stdexcept>
#include <string>

#include "kernels.hpp"
#include "noalloc.hpp"

namespace qd {

static __device__ __align__(256) double noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

namespace {
std::mutex g_mu;
uint64_t g_addr[64] = {0};  // device address of the array per device ordinal
}  // namespace

uint64_t noalloc_scratch_address() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    throw std::runtime_error("CUDA: no current device for the no-allocation scratch");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw std::runtime_error(std::string("CUDA: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    g_addr[dev] = reinterpret_cast<uint64_t>(p);
  }
  return g_addr[dev];
}

}  // namespace qd

#include "engine.hpp"

namespace qd {

namespace {
// makes `device` current for the call and gives the caller's current device
// back on every exit path
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) throw std::runtime_error(std::string("CUDA: ") + cudaGetErrorString(e));
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace

void heff_noalloc(Engine& E, int device, uint64_t psi, uint64_t sig, void* stream) {
  DeviceGuard guard(device);
  // a launch error left pending by earlier, unrelated work on this thread is
  // cleared here, so that the status of this call reports its own launches
  (void)cudaGetLastError();
  const uint64_t scratch = noalloc_scratch_address();
  cudaError_t e;
  cudaStream_t st = (cudaStream_t)stream;
  e = cudaMemsetAsync(reinterpret_cast<void*>(sig), 0, (size_t)E.lay.size * 8, st);
  if (e != cudaSuccess) throw std::runtime_error(std::string("CUDA: ") + cudaGetErrorString(e));
  for (auto& h : E.prepared) {
    e = launch_f64_prepared(E.pr->prepared_handle(h.first), psi, sig, scratch, st);
    if (e == cudaSuccess) e = launch_f64_prepared(E.pr->prepared_handle(h.second), psi, sig, scratch, st);
    if (e != cudaSuccess) throw std::runtime_error(std::string("CUDA: ") + cudaGetErrorString(e));
  }
}

}  // namespace qd
