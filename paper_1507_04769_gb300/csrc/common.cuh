// Shared host/device helpers of the sparse grid characteristics library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/sg.h"

namespace sg {

// Thread-local last-error message (defined in api.cu).
void set_error(const std::string& msg);
void clear_error();

inline int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

inline int cuda_fail(cudaError_t e, const char* where) {
  return fail(SG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SG_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return ::sg::cuda_fail(_e, #expr); \
  } while (0)

// Checks that the launch queued without error.
#define SG_LAUNCH_CHECK(name)                                   \
  do {                                                          \
    cudaError_t _e = cudaGetLastError();                        \
    if (_e != cudaSuccess) return ::sg::cuda_fail(_e, name);    \
  } while (0)

// Lets `func` launch with `bytes` of dynamic shared memory.  Above the default
// 48 KB the cap is raised to the most the device allows (less the kernel's
// static shared memory), always to the same value: host threads that launch
// the same kernel with different sizes concurrently can then never lower the
// cap below another thread's launch.
template <typename F>
inline cudaError_t ensure_dynamic_smem(F* func, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(func));
  if (e != cudaSuccess) return e;
  const int cap = optin - static_cast<int>(fa.sharedSizeBytes);
  if (static_cast<long long>(bytes) > cap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(func), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              cap);
}

// The device blocks of grid and surplus handles come from a library-owned
// stream-ordered pool per device that keeps up to 1 GiB of freed blocks, so
// building and freeing a handle every step costs no cudaMalloc/cudaFree.
// block_free synchronises the device first (a handle's last use may be on
// any stream), as cudaFree does.
cudaError_t block_alloc(void** p, size_t bytes, cudaStream_t st);
void block_free(void* p);

constexpr int kMaxDim = 8;
constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace sg
