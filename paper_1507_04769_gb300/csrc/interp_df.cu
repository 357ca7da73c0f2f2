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

constexpr int kFoldBlock = 64;     // nodes per FP64 fold of the compensated sums (per thread)
constexpr int kDfWarps = 6;        // warps per block
constexpr int kDfThreads = 32 * kDfWarps;
constexpr int kDfChunk = 256;      // nodes staged in shared memory at a time
// surplus pairs per staged node: K rounded up to even, so a node's pairs are
// read as 16-byte words
template <int K>
constexpr int df_kp() { return (K + 1) & ~1; }

// Product of a pair with a pair, left unnormalised: the result (p, e) has
// p = fl(a.hi b.hi) and e = the exact rounding error of p plus the cross
// terms, so p + e carries the product to about 2^-46 relative.  Skipping the
// renormalisation is safe because |e| stays below about 2^-22 |p| and every
// consumer (the next product, the compensated dot) treats hi and lo only
// through products and exact sums.
__device__ __forceinline__ df df_mul_raw(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}

struct DfAcc {
  double total;
  float ah, al;
};

// Nodes [n0, n1) of the staged chunk with exactly A active factors; this
// thread's node stream takes those with index = stream (mod NS).  off_s:
// byte offsets of the node's table rows (kMaxDim slots), w_s: K surplus
// pairs per node.
template <int K, int A, int NS>
__device__ __forceinline__ void df_group(const unsigned char* __restrict__ tab_q, const uint32_t* __restrict__ off_s,
                                         const float2* __restrict__ w_s, int n0, int n1, int stream,
                                         DfAcc (&acc)[K], int& since_fold) {
  int nn = n0 + ((stream - n0) % NS + NS) % NS;
  int left = nn < n1 ? (n1 - nn + NS - 1) / NS : 0;
  while (left > 0) {
    // a run of nodes up to the next fold, with no per-node fold test
    const int run = left < kFoldBlock - since_fold ? left : kFoldBlock - since_fold;
#pragma unroll 2
    for (int r = 0; r < run; ++r, nn += NS) {
      df phi = {1.0f, 0.0f};
      if constexpr (A > 0) {
        uint32_t o[A];
        if constexpr (A <= 4) {
          const uint4 v = *reinterpret_cast<const uint4*>(off_s + nn * kMaxDim);
          const uint32_t t[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int a = 0; a < A; ++a) o[a] = t[a];
        } else {
          const uint4 v0 = *reinterpret_cast<const uint4*>(off_s + nn * kMaxDim);
          const uint4 v1 = *reinterpret_cast<const uint4*>(off_s + nn * kMaxDim + 4);
          const uint32_t t[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
          for (int a = 0; a < A; ++a) o[a] = t[a];
        }
        const float2 f0 = *reinterpret_cast<const float2*>(tab_q + o[0]);
        phi = {f0.x, f0.y};
#pragma unroll
        for (int a = 1; a < A; ++a) {
          const float2 f = *reinterpret_cast<const float2*>(tab_q + o[a]);
          phi = df_mul_raw(phi, {f.x, f.y});
        }
      }
      float2 wv[df_kp<K>()];
#pragma unroll
      for (int h = 0; h < df_kp<K>() / 2; ++h) {
        const float4 v = reinterpret_cast<const float4*>(w_s + nn * df_kp<K>())[h];
        wv[2 * h] = make_float2(v.x, v.y);
        wv[2 * h + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const float2 wc = wv[c];
        // p = fl(phi.hi w.hi); t = its exact rounding error plus the cross
        // terms (the unnormalised product of df_mul_raw)
        const float p = __fmul_rn(phi.hi, wc.x);
        float t = __fmaf_rn(phi.hi, wc.x, -p);
        t = __fmaf_rn(phi.hi, wc.y, t);
        t = __fmaf_rn(phi.lo, wc.x, t);
        // Knuth's two_sum of the running sum and p
        const float s = __fadd_rn(acc[c].ah, p);
        const float bb = __fsub_rn(s, acc[c].ah);
        const float se = __fadd_rn(__fsub_rn(acc[c].ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        acc[c].ah = s;
        acc[c].al = __fadd_rn(acc[c].al, __fadd_rn(se, t));
      }
    }
    left -= run;
    since_fold += run;
    if (since_fold == kFoldBlock) {
      since_fold = 0;
#pragma unroll
      for (int c = 0; c < K; ++c) {
        acc[c].total += static_cast<double>(acc[c].ah) + static_cast<double>(acc[c].al);
        acc[c].ah = 0.0f;
        acc[c].al = 0.0f;
      }
    }
  }
}

// Block = QB queries x NS = kDfWarps * 32 / QB node streams: lane q % QB of
// the block evaluates query q over the nodes of its stream.  The d x nf basis
// table of each query (pairs) is built once in shared memory and shared by
// the block's streams; the streams' partial sums are added in FP64 in a
// fixed order.  Nodes come in the evaluation order, grouped by their number
// of active dimensions A, so every group runs a loop with a fixed-length
// product.  QB = 32 for the usual levels; 16 or 8 when the d x nf tables of
// 32 queries do not fit in shared memory (high levels).
template <int K, int QB>
__global__ void __launch_bounds__(kDfThreads) k_eval_df32(EvalArgs e, int d) {
  constexpr int NS = kDfThreads / QB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nf = e.nf;
  const int tab_bytes = d * nf * QB * static_cast<int>(sizeof(float2));
  float2* tab = reinterpret_cast<float2*>(smem_raw);                                  // [d*nf][QB]
  uint32_t* off_s = reinterpret_cast<uint32_t*>(smem_raw + tab_bytes);                 // [kDfChunk][kMaxDim]
  float2* w_s = reinterpret_cast<float2*>(off_s + kDfChunk * kMaxDim);                 // [kDfChunk][df_kp<K>]
  const int tid = threadIdx.x;
  const int ql = tid % QB, stream = tid / QB;
  const int64_t qbase = blockIdx.x * int64_t(QB);

  // basis tables: (query, dim) tasks over the block
  for (int task = tid; task < QB * d; task += kDfThreads) {
    const int tq = task % QB, dim = task / QB;
    const int64_t q = qbase + tq;
    const double u = q < e.Q ? (e.xq[q * d + dim] - e.lo[dim]) / e.width[dim] : 0.5;
    basis_row_df(u, e.level, e.xfdf, tab + (dim * nf) * QB + tq, QB);
  }
  const unsigned char* tab_q = reinterpret_cast<const unsigned char*>(tab + ql);

  DfAcc acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = {0.0, 0.0f, 0.0f};
  int since_fold = 0;
  for (int64_t m0 = 0; m0 < e.M; m0 += kDfChunk) {
    const int cn = e.M - m0 < kDfChunk ? static_cast<int>(e.M - m0) : kDfChunk;
    __syncthreads();   // tables written / previous chunk consumed
    for (int x = tid; x < cn * kMaxDim; x += kDfThreads) {
      const int nn = x / kMaxDim, j = x % kMaxDim;
      // table row (dim * nf + id) -> byte offset within the query column
      off_s[x] = static_cast<uint32_t>(e.ops[(m0 + nn) * kMaxDim + j]) * (QB * sizeof(float2));
    }
    for (int x = tid; x < cn * K; x += kDfThreads) w_s[(x / K) * df_kp<K>() + x % K] = e.Wdf[m0 * K + x];
    __syncthreads();
    // groups of equal active-dimension count that meet this chunk
    for (int a = 0; a <= kMaxDim; ++a) {
      const int64_t g0 = e.grp[a] > m0 ? e.grp[a] : m0;
      const int64_t g1 = e.grp[a + 1] < m0 + cn ? e.grp[a + 1] : m0 + cn;
      if (g0 >= g1) continue;
      const int n0 = static_cast<int>(g0 - m0), n1 = static_cast<int>(g1 - m0);
      switch (a) {
        case 0: df_group<K, 0, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        case 1: df_group<K, 1, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        case 2: df_group<K, 2, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        case 3: df_group<K, 3, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        case 4: df_group<K, 4, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        case 5: df_group<K, 5, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        case 6: df_group<K, 6, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        case 7: df_group<K, 7, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
        default: df_group<K, 8, NS>(tab_q, off_s, w_s, n0, n1, stream, acc, since_fold); break;
      }
    }
  }
  // streams' partial sums, added in stream order
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_raw);   // [NS][QB][K], over the tables
#pragma unroll
  for (int c = 0; c < K; ++c)
    red[(stream * QB + ql) * K + c] = acc[c].total + (static_cast<double>(acc[c].ah) + static_cast<double>(acc[c].al));
  __syncthreads();
  if (tid < QB) {
    const int64_t q = qbase + tid;
    if (q < e.Q) {
#pragma unroll
      for (int c = 0; c < K; ++c) {
        double v = red[tid * K + c];
        for (int st = 1; st < NS; ++st) v += red[(st * QB + tid) * K + c];
        e.out[q * K + c] = v;
      }
    }
  }
}

template <int K, int QB>
static size_t df32_smem(const EvalArgs& e, int d) {
  const size_t tab = sizeof(float2) * d * e.nf * QB;
  const size_t red = sizeof(double) * kDfThreads * K;
  return (tab > red ? tab : red) + sizeof(uint32_t) * kDfChunk * kMaxDim + sizeof(float2) * kDfChunk * df_kp<K>();
}

template <int K, int QB>
static int launch_df32_kq(const EvalArgs& e, int d, size_t smem, cudaStream_t st) {
  const unsigned blocks = static_cast<unsigned>(ceil_div(e.Q, QB));
  SG_CUDA_TRY(ensure_dynamic_smem(k_eval_df32<K, QB>, smem));
  SG_TIMED("k_eval_df32", st, (k_eval_df32<K, QB><<<blocks, kDfThreads, smem, st>>>(e, d)));
  SG_LAUNCH_CHECK("k_eval_df32");
  return SG_OK;
}

template <int K>
static int launch_df32_k(const EvalArgs& e, int d, cudaStream_t st) {
  constexpr size_t kLimit = 220 * 1024;
  if (df32_smem<K, 32>(e, d) <= kLimit) return launch_df32_kq<K, 32>(e, d, df32_smem<K, 32>(e, d), st);
  if (df32_smem<K, 16>(e, d) <= kLimit) return launch_df32_kq<K, 16>(e, d, df32_smem<K, 16>(e, d), st);
  if (df32_smem<K, 8>(e, d) <= kLimit) return launch_df32_kq<K, 8>(e, d, df32_smem<K, 8>(e, d), st);
  return fail(SG_EUNSUPPORTED, "sg_eval_feedback: grid level too high for the DF32 kernel");
}

int eval_df32(const EvalArgs& e, int d, cudaStream_t st) {
  switch (e.k) {
    case 1: return launch_df32_k<1>(e, d, st);
    case 2: return launch_df32_k<2>(e, d, st);
    case 3: return launch_df32_k<3>(e, d, st);
    case 4: return launch_df32_k<4>(e, d, st);
    case 6: return launch_df32_k<6>(e, d, st);
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
