// Launch accounting shared by every translation unit: construct a KernelTimer
// on the launching stream right before a launch; it counts the launch and,
// when timing is enabled, brackets it with CUDA events on that stream.
#pragma once

#include <cuda_runtime.h>

namespace sg {
class KernelTimer {
 public:
  KernelTimer(const char* name, cudaStream_t st);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  cudaEvent_t a_ = nullptr;
  cudaEvent_t b_ = nullptr;
};
}  // namespace sg

// Launches `call` (a kernel<<<...>>>(...) expression) under a KernelTimer.
#define SG_TIMED(name, stream, call) \
  do {                               \
    ::sg::KernelTimer _kt(name, stream); \
    call;                            \
  } while (0)
