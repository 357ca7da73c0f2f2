// Fifth-generation tensor-core helpers shared by the tcgen05 kernels:
// shared-memory matrix descriptors (no swizzle, K-major core matrices),
// bounded mbarrier waits and the TF32 splitting of FP32 values.
#pragma once

#include <cstdint>

namespace sg {

constexpr unsigned kTcSpinLimit = 1u << 24;     // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// byte offset (between the two core matrices along K), stride-dimension byte
// offset (between consecutive 8-row groups), fixed version bits 0b001 at 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
  d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;   // base offset 0, relative LBO, swizzle mode 0 (none)
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Split of x into TF32 parts: hi = x rounded to the nearest TF32 value (ties
// away from zero: half an ulp of the 10-bit mantissa added to the magnitude,
// the 13 low bits cleared), lo = x - hi (exact in FP32, Sterbenz) rounded the
// same way.  Both have zero low bits, so the tensor cores read them as given.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = __uint_as_float((__float_as_uint(__fsub_rn(x, hi)) + 0x1000u) & 0xFFFFE000u);
}

// Instruction descriptor for kind::tf32: D = F32, A = B = TF32, both K-major,
// M x N with M = 128 (or 64) and N a multiple of 16 up to 256.
__device__ __forceinline__ uint32_t idesc_tf32_mn(int m, int n) {
  uint32_t d = 0;
  d |= 1u << 4;                        // D format F32
  d |= 2u << 7;                        // A format TF32
  d |= 2u << 10;                       // B format TF32
  d |= static_cast<uint32_t>(n >> 3) << 17;
  d |= static_cast<uint32_t>(m >> 4) << 24;
  return d;
}

}  // namespace sg
