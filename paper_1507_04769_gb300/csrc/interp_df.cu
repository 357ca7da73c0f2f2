// FP64-accurate evaluation of the sparse-grid interpolant on the FP32 pipe.
//
// GB300 issues FP32 arithmetic at 64x its FP64 rate, so this path carries
// every quantity as an unevaluated pair of floats (hi + lo, about 48
// significant bits):
//   * products by the FMA-based exact product (two_prod) plus cross terms,
//   * sums by Knuth's exact two_sum,
//   * reciprocals by one Newton correction of the FP32 reciprocal,
// all with explicitly rounded intrinsics so that no step is contracted.  The
// contraction sum_m phi_m w_m is the compensated dot product of Ogita, Rump
// and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005):
// exact products and sums feed the leading float, every rounding error goes
// to a second float, and every 64 nodes the pair is folded into an FP64
// accumulator, so the error grows with the block length, not with M.
#include "common.cuh"
#include "diag.cuh"
#include "basis.cuh"
#include "interp.cuh"

namespace sg {

constexpr int kFoldBlock = 64;     // nodes per FP64 fold of the compensated sums
constexpr int kChunk = 128;        // nodes staged in shared memory at a time

// Node loop of the pair-of-floats evaluation.  Every node has exactly A table
// factors (padded with table entry 0, the exact constant 1), so the loop has
// no data-dependent branch.  Offsets and surpluses of kChunk nodes are staged
// in shared memory by the whole block with coalesced loads.
template <int K, int A>
__global__ void __launch_bounds__(kEvalThreads) k_eval_df32(EvalArgs e, int d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tab = reinterpret_cast<float2*>(smem_raw);
  const int nf = e.nf;
  float2* wch = tab + size_t(d) * nf * kEvalThreads;                 // kChunk x K
  uint16_t* och = reinterpret_cast<uint16_t*>(wch + kChunk * K);    // kChunk x A
  const int tid = threadIdx.x;
  const int64_t q = blockIdx.x * int64_t(kEvalThreads) + tid;
  const bool live = q < e.Q;
  for (int dim = 0; dim < d; ++dim) {
    const double u = live ? (e.xq[q * d + dim] - e.lo[dim]) / e.width[dim] : 0.5;
    basis_row_df(u, e.level, e.xfdf, tab + (dim * nf) * kEvalThreads + tid, kEvalThreads);
  }
  double total[K];
  float ah[K], al[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    total[c] = 0.0;
    ah[c] = 0.0f;
    al[c] = 0.0f;
  }
  auto T = [&](int off) {
    const float2 v = tab[off * kEvalThreads + tid];
    return df{v.x, v.y};
  };
  int since_fold = 0;
  for (int64_t m0 = 0; m0 < e.M; m0 += kChunk) {
    const int cn = e.M - m0 < kChunk ? static_cast<int>(e.M - m0) : kChunk;
    __syncthreads();   // tables written / previous chunk consumed
    for (int x = tid; x < cn * K; x += kEvalThreads) wch[x] = e.Wdf[m0 * K + x];
    for (int x = tid; x < cn * A; x += kEvalThreads) {
      const int nn = x / A, j = x % A;
      och[x] = e.ops[(m0 + nn) * kMaxDim + j];
    }
    __syncthreads();
#pragma unroll 2
    for (int nn = 0; nn < cn; ++nn) {
      df phi = T(och[nn * A]);
#pragma unroll
      for (int j = 1; j < A; ++j) phi = df_mul(phi, T(och[nn * A + j]));
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const float2 wc = wch[nn * K + c];
        const float p = __fmul_rn(phi.hi, wc.x);
        const float pe = __fmaf_rn(phi.hi, wc.x, -p);
        const float t = __fadd_rn(__fmaf_rn(phi.hi, wc.y, __fmul_rn(phi.lo, wc.x)), pe);
        const float s = __fadd_rn(ah[c], p);
        const float bb = __fsub_rn(s, ah[c]);
        const float se = __fadd_rn(__fsub_rn(ah[c], __fsub_rn(s, bb)), __fsub_rn(p, bb));
        ah[c] = s;
        al[c] = __fadd_rn(al[c], __fadd_rn(se, t));
      }
      if (++since_fold == kFoldBlock) {
        since_fold = 0;
#pragma unroll
        for (int c = 0; c < K; ++c) {
          total[c] += static_cast<double>(ah[c]) + static_cast<double>(al[c]);
          ah[c] = 0.0f;
          al[c] = 0.0f;
        }
      }
    }
  }
  if (live) {
#pragma unroll
    for (int c = 0; c < K; ++c)
      e.out[q * K + c] = total[c] + (static_cast<double>(ah[c]) + static_cast<double>(al[c]));
  }
}

template <int K>
static int launch_df32_k(const EvalArgs& e, int d, int A, cudaStream_t st) {
  const size_t smem = sizeof(float2) * d * e.nf * kEvalThreads + sizeof(float2) * kChunk * K +
                      sizeof(uint16_t) * kChunk * kMaxDim;
  if (smem > 220 * 1024) return fail(SG_EUNSUPPORTED, "sg_eval_feedback: grid level too high for the DF32 kernel");
  const unsigned blocks = static_cast<unsigned>(ceil_div(e.Q, kEvalThreads));
#define SG_DF_A(AA)                                                                                  \
  case AA:                                                                                           \
    SG_CUDA_TRY(cudaFuncSetAttribute(k_eval_df32<K, AA>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     static_cast<int>(smem)));                                       \
    SG_TIMED("k_eval_df32", st, (k_eval_df32<K, AA><<<blocks, kEvalThreads, smem, st>>>(e, d)));     \
    break;
  switch (A) {
    SG_DF_A(1)
    SG_DF_A(2)
    SG_DF_A(3)
    SG_DF_A(4)
    SG_DF_A(5)
    SG_DF_A(6)
    SG_DF_A(7)
    SG_DF_A(8)
    default: return fail(SG_EINVAL, "sg_eval_feedback: bad active-dimension count");
  }
#undef SG_DF_A
  SG_LAUNCH_CHECK("k_eval_df32");
  return SG_OK;
}

int eval_df32(const EvalArgs& e, int d, cudaStream_t st) {
  const int A = e.amax < 1 ? 1 : e.amax;
  switch (e.k) {
    case 1: return launch_df32_k<1>(e, d, A, st);
    case 2: return launch_df32_k<2>(e, d, A, st);
    case 3: return launch_df32_k<3>(e, d, A, st);
    case 4: return launch_df32_k<4>(e, d, A, st);
    case 6: return launch_df32_k<6>(e, d, A, st);
    default: return fail(SG_EUNSUPPORTED, "sg_eval_feedback: SG_EVAL_DF32 supports k = 1, 2, 3, 4, 6");
  }
}

// Splits FP64 values into (hi, lo) float pairs.
__global__ void k_split_df(int64_t n, const double* __restrict__ src, float2* __restrict__ dst) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const df v = df_from(src[i]);
  dst[i] = make_float2(v.hi, v.lo);
}

int split_df(int64_t n, const double* src, float2* dst, cudaStream_t st) {
  if (n <= 0) return SG_OK;
  SG_TIMED("k_split_df", st, (k_split_df<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(n, src, dst)));
  SG_LAUNCH_CHECK("k_split_df");
  return SG_OK;
}

}  // namespace sg
