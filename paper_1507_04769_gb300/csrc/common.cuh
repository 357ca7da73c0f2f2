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

constexpr int kMaxDim = 8;
constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace sg
