// Fixed device scratch for the no-allocation H_eff psi entry point.
#pragma once
#include <cstdint>

namespace qd {

// 4 Mi doubles = 32 MiB per device.
constexpr int64_t NOALLOC_SCRATCH_DOUBLES = 4ll * 1024 * 1024;

// Device address of the scratch array on the current device; the first call
// per device looks it up (cudaGetSymbolAddress) with that device current.
uint64_t noalloc_scratch_address();

struct Engine;
// FP64 H_eff psi of the engine's centre with the fixed scratch array; enqueued
// on stream; allocates nothing.
void heff_noalloc(Engine& E, int device, uint64_t psi, uint64_t sig, void* stream);

}  // namespace qd
