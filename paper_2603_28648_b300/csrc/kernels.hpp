// Backend interface shared by the C ABI and the CUDA executor.
#pragma once
#include "core.hpp"

namespace qd {

// Launch lists uploaded once and replayed on any psi / sigma pair.
struct PreparedRunner {
  virtual ~PreparedRunner() {}
  virtual int prepare(const Launch& l) = 0;
  virtual void drop_prepared() = 0;
  virtual void run_prepared(int handle, uint64_t psi, uint64_t sig, void* stream) = 0;
  virtual void* stream() = 0;
  virtual void sync(void* stream) = 0;
  virtual void zero_async(uint64_t p, int64_t n, void* stream) = 0;
  virtual int64_t bytes_allocated() const = 0;
};

struct Backend {
  Executor* ex = nullptr;
  PreparedRunner* pr = nullptr;
};

// Creates the CUDA backend on a device (throws std::runtime_error on failure).
Backend make_backend(int device);

}  // namespace qd
