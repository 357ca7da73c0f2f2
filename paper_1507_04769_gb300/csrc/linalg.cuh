// Warp-cooperative dense elimination on small matrices held in shared memory.
#pragma once

#include <cuda_runtime.h>

namespace sg {

// Correctly rounded reciprocal: the value of 1 / x without the division's
// slow path.
__device__ __forceinline__ float lin_recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double lin_recip(double x) { return __drcp_rn(x); }

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// Gaussian elimination with partial pivoting on the first NP columns of an
// R x C row-major matrix M (row stride C) held in shared memory, by one warp.
// Rows are swapped physically; multipliers are left in the eliminated
// columns; rows NP..R-1 end up with zeros (multipliers) in columns 0..NP-1,
// i.e. they hold the Schur complement in columns NP..C-1.  Ties in the pivot
// search go to the lowest row index.  Returns false if a pivot column was
// entirely zero (or non-finite); elimination then continues with a zero
// multiplier so no NaN is produced.
template <typename T, int R, int C, int NP>
__device__ bool warp_eliminate(T* M, int lane) {
  bool ok = true;
#pragma unroll 1
  for (int k = 0; k < NP; ++k) {
    T bv = T(-1);
    int br = k;
    for (int r = k + lane; r < R; r += 32) {
      T v = tabs(M[r * C + k]);
      if (v > bv) {
        bv = v;
        br = r;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, bv, off);
      int orow = __shfl_xor_sync(0xffffffffu, br, off);
      if (ov > bv || (ov == bv && orow < br)) {
        bv = ov;
        br = orow;
      }
    }
    const bool good = bv > T(0) && bv < T(INFINITY);
    ok = ok && good;
    if (br != k) {
      for (int c = k + lane; c < C; c += 32) {
        T a = M[k * C + c];
        M[k * C + c] = M[br * C + c];
        M[br * C + c] = a;
      }
    }
    __syncwarp();
    const T inv = good ? lin_recip(M[k * C + k]) : T(0);
    for (int r = k + 1 + lane; r < R; r += 32) M[r * C + k] *= inv;
    __syncwarp();
    const int nr = R - k - 1, nc = C - k - 1;
    const int total = nr * nc;
    if (total > 0) {
      const int q = 32 / nc, rem = 32 % nc;
      int r = lane / nc, c = lane % nc;
      for (int e = lane; e < total; e += 32) {
        const int rr = k + 1 + r, cc = k + 1 + c;
        M[rr * C + cc] -= M[rr * C + k] * M[k * C + cc];
        c += rem;
        r += q;
        if (c >= nc) {
          c -= nc;
          ++r;
        }
      }
    }
    __syncwarp();
  }
  return ok;
}

// Deterministic warp sum / max (fixed butterfly order).
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    T o = __shfl_xor_sync(0xffffffffu, v, off);
    v = (o > v || o != o) ? o : v;
  }
  return v;
}

}  // namespace sg
