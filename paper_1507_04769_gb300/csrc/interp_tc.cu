// Split-TF32 evaluation of the interpolant contraction on the fifth-generation
// tensor cores (tcgen05, accumulator in tensor memory).
//
// u = Phi W with Phi (queries x nodes) generated on the fly and W (nodes x k)
// the surpluses.  With Phi = Phi_hi + Phi_lo and W = W_hi + W_lo split into
// TF32 parts, u ~ Phi_hi W_hi + Phi_hi W_lo + Phi_lo W_hi (the 3xTF32 scheme):
// one accumulator D (128 rows x 16 columns, FP32) receives
//   Phi_hi x [W_hi | W_lo | 0]  and  Phi_lo x [W_hi | 0 | 0],
// so that u = D[:, 0:k] + D[:, k:2k] (k <= 8 outputs).
//
// One CTA (8 warps) per 128 queries; threads t and t + 128 own query row t,
// each for one K-step of 8 nodes.  Per chunk of 16 nodes the threads write
// their rows of Phi_hi and Phi_lo into shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix), thread 0 issues
// 2 x 2 MMAs of shape M=128, N=16, K=8 and commits them to an mbarrier; the
// next chunk is written into the other buffer while the tensor cores work.  Every wait on an mbarrier has an iteration
// limit: on timeout the kernel records an error flag, writes NaN outputs,
// releases its tensor memory and returns.
#include "common.cuh"
#include "diag.cuh"
#include "interp.cuh"

namespace sg {

constexpr int kTcRows = 128;          // queries per CTA (= MMA M)
constexpr int kTcThreads = 256;       // two threads per query row
constexpr int kTcN = 16;              // MMA N (2k <= 16)
constexpr int kTcChunk = 16;          // nodes per chunk (2 MMA K-steps of 8, one per thread of a row)
constexpr int kTcAStep = kTcRows * 32;          // bytes of one K-step of A (128 rows x 8 tf32)
constexpr int kTcABytes = 2 * kTcAStep;         // one chunk of Phi_hi or Phi_lo: 8 KB
constexpr int kTcBStep = kTcN * 32;             // bytes of one K-step of B (16 rows x 8 tf32)
constexpr int kTcBBytes = 2 * kTcBStep;         // one chunk of one B matrix: 1 KB
constexpr int kTcBPack = 2 * kTcBBytes / 4;     // floats per chunk of [B1 | B2]
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

// Instruction descriptor for kind::tf32: D = F32, A = B = TF32, both K-major,
// N = 16, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32() {
  uint32_t d = 0;
  d |= 1u << 4;                        // D format F32
  d |= 2u << 7;                        // A format TF32
  d |= 2u << 10;                       // B format TF32
  d |= static_cast<uint32_t>(kTcN >> 3) << 17;
  d |= static_cast<uint32_t>(kTcRows >> 4) << 24;
  return d;
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

// FP32 barycentric basis values (same construction as the FP64 basis_row).
__device__ void basis_row_f32(float u, int level, const double* __restrict__ xf, float* tab, int stride) {
  tab[0] = 1.0f;
  if (level == 0) return;
  const int fine_n = 1 << level;
  float rinv[kMaxFine + 1];
  int hit = -1;
  for (int p = 0; p <= fine_n; ++p) {
    const float diff = u - static_cast<float>(xf[p]);
    if (diff == 0.0f) hit = p;
    rinv[p] = diff == 0.0f ? 0.0f : 1.0f / diff;
  }
  int id = 1;
  for (int l = 2; l <= level + 1; ++l) {
    const int n = 1 << (l - 1);
    const int sf = fine_n / n;
    const bool exact = hit >= 0 && (hit % sf) == 0;
    float den = 0.0f;
    if (!exact)
      for (int m = 0; m <= n; ++m) {
        float wm = (m & 1) ? -1.0f : 1.0f;
        if (m == 0 || m == n) wm *= 0.5f;
        den += wm * rinv[m * sf];
      }
    const float inv = exact ? 0.0f : 1.0f / den;
    const int cnt = l == 2 ? 2 : (n >> 1);
    for (int j = 0; j < cnt; ++j) {
      const int m = l == 2 ? j * n : 2 * j + 1;
      float v;
      if (exact) {
        v = (m * sf == hit) ? 1.0f : 0.0f;
      } else {
        float wm = (m & 1) ? -1.0f : 1.0f;
        if (m == 0 || m == n) wm *= 0.5f;
        v = wm * rinv[m * sf] * inv;
      }
      tab[(id + j) * stride] = v;
    }
    id += cnt;
  }
}

struct TcArgs {
  EvalArgs e;
  int d;
  const float* bpack;   // nchunks x kTcBPack
  int nchunks;
  int* err;
};

__global__ void __launch_bounds__(kTcThreads) k_eval_tf32x3(TcArgs t) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const EvalArgs& e = t.e;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kTcRows - 1), half = tid / kTcRows;
  const int64_t q = blockIdx.x * int64_t(kTcRows) + row;
  const bool live = q < e.Q;
  const int nf = e.nf;
  // layout: A buffers (2 x [hi, lo]) | B buffers (2 x [B1, B2]) | tables | barriers
  unsigned char* abuf = smem;                                        // 2 * 2 * kTcABytes
  unsigned char* bbuf = abuf + 4 * kTcABytes;                        // 2 * 2 * kTcBBytes
  float* tab = reinterpret_cast<float*>(bbuf + 4 * kTcBBytes);       // d * nf * kTcRows
  uint64_t* bars = reinterpret_cast<uint64_t*>(tab + size_t(t.d) * nf * kTcRows);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2);

  // the two threads of a row share the dimensions of its 1-D tables
  for (int dim = half; dim < t.d; dim += 2) {
    const double u = live ? (e.xq[q * t.d + dim] - e.lo[dim]) / e.width[dim] : 0.5;
    basis_row_f32(static_cast<float>(u), e.level, e.xf, tab + (dim * nf) * kTcRows + row, kTcRows);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_holder)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_holder;
  const uint32_t idesc = idesc_tf32();
  bool ok = true;
  uint32_t phase[2] = {0u, 0u};

  for (int c = 0; c < t.nchunks; ++c) {
    const int buf = c & 1;
    if (c >= 2) {
      // the MMAs that read this buffer two chunks ago must have finished
      ok = ok && mbar_wait(smem_u32(&bars[buf]), phase[buf]);
      phase[buf] ^= 1u;
    }
    unsigned char* ahi = abuf + (2 * buf) * kTcABytes;
    unsigned char* alo = ahi + kTcABytes;
    // this thread's K-step (8 nodes) of row `row`, as two 16-byte core-matrix
    // rows: element (r, k) of K-step s at
    //   s * kTcAStep + ((r / 8) * 2 + (k % 8) / 4) * 128 + (r % 8) * 16 + (k % 4) * 4
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      float hv[4], lv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t m = int64_t(c) * kTcChunk + half * 8 + c2 * 4 + j;
        float phi = 0.0f;
        if (m < e.M) {
          const uint16_t* o = e.ops + m * kMaxDim;
          phi = tab[o[0] * kTcRows + row];
          for (int a = 1; a < e.amax; ++a) phi *= tab[o[a] * kTcRows + row];
        }
        hv[j] = tf32_round(phi);
        lv[j] = tf32_round(phi - hv[j]);
      }
      const int off = half * kTcAStep + ((row / 8) * 2 + c2) * 128 + (row % 8) * 16;
      *reinterpret_cast<float4*>(ahi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
      *reinterpret_cast<float4*>(alo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
    }
    // the chunk of [B1 | B2], pre-packed in the same layout
    const float4* src = reinterpret_cast<const float4*>(t.bpack + size_t(c) * kTcBPack);
    float4* dst = reinterpret_cast<float4*>(bbuf + (2 * buf) * kTcBBytes);
    for (int x = tid; x < kTcBPack / 4; x += kTcThreads) dst[x] = src[x];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a_hi = smem_u32(ahi), a_lo = smem_u32(alo);
      const uint32_t b1 = smem_u32(bbuf + (2 * buf) * kTcBBytes), b2 = b1 + kTcBBytes;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint64_t da_hi = smem_desc(a_hi + s * kTcAStep, 128, 256);
        const uint64_t da_lo = smem_desc(a_lo + s * kTcAStep, 128, 256);
        const uint64_t db1 = smem_desc(b1 + s * kTcBStep, 128, 256);
        const uint64_t db2 = smem_desc(b2 + s * kTcBStep, 128, 256);
        const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da_hi), "l"(db1), "r"(idesc), "r"(acc));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da_lo), "l"(db2), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bars[buf])));
    }
  }
  // the last commit covers every MMA issued before it
  if (t.nchunks > 0) {
    const int lb = (t.nchunks - 1) & 1;
    ok = ok && mbar_wait(smem_u32(&bars[lb]), phase[lb]);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = 0.0f;
  if (warp < 4) {
    // warp w reads accumulator rows (tensor-memory lanes) 32w .. 32w + 31
    const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
  }
  const bool all_ok = __syncthreads_and(ok);
  if (live && half == 0) {
    for (int cix = 0; cix < e.k; ++cix) {
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j == cix) hi = v[j];
        if (j == e.k + cix) lo = v[j];
      }
      e.out[q * e.k + cix] = all_ok ? static_cast<double>(hi) + static_cast<double>(lo) : NAN;
    }
  }
  if (!all_ok && tid == 0) atomicExch(t.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// [B1 | B2] per chunk: B1 = [W_hi | W_lo | 0], B2 = [W_hi | 0 | 0] (16 columns),
// element (n, node kk of the chunk) of one matrix at
//   (kk / 8) * 128 + ((n / 8) * 2 + (kk % 8) / 4) * 32 + (n % 8) * 4 + kk % 4   (floats)
__global__ void k_pack_tf32(int64_t M, int k, int nchunks, const double* __restrict__ W, float* __restrict__ bp) {
  const int64_t x = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (x >= int64_t(nchunks) * kTcChunk * kTcN) return;
  const int n = static_cast<int>(x % kTcN);
  const int64_t node = x / kTcN;
  const int c = static_cast<int>(node / kTcChunk), kk = static_cast<int>(node % kTcChunk);
  float b1 = 0.f, b2 = 0.f;
  if (node < M) {
    if (n < k) {
      const float hi = tf32_round(static_cast<float>(W[node * k + n]));
      b1 = hi;
      b2 = hi;
    } else if (n < 2 * k) {
      const double w = W[node * k + (n - k)];
      const float hi = tf32_round(static_cast<float>(w));
      b1 = tf32_round(static_cast<float>(w - static_cast<double>(hi)));
    }
  }
  const int off = (kk / 8) * 128 + ((n / 8) * 2 + (kk % 8) / 4) * 32 + (n % 8) * 4 + kk % 4;
  bp[size_t(c) * kTcBPack + off] = b1;
  bp[size_t(c) * kTcBPack + kTcBBytes / 4 + off] = b2;
}

size_t tf32_pack_floats(int64_t M, int k) {
  if (k > kTcN / 2) return 0;   // the tensor-core path serves k <= 8
  return size_t(ceil_div(M, kTcChunk)) * kTcBPack;
}

// s->bpack (tf32_pack_floats(M, k) floats) and s->tc_err come with the
// surplus's allocation.
int pack_tf32(sg_surplus* s, cudaStream_t st) {
  if (s->k > kTcN / 2) return SG_OK;   // the tensor-core path serves k <= 8
  const int nchunks = static_cast<int>(ceil_div(s->M, kTcChunk));
  s->tc_chunks = nchunks;
  cudaError_t e;
  if ((e = cudaMemsetAsync(s->tc_err, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "pack_tf32: memset");
  const int64_t total = int64_t(nchunks) * kTcChunk * kTcN;
  SG_TIMED("k_pack_tf32", st,
           (k_pack_tf32<<<static_cast<unsigned>(ceil_div(total, 256)), 256, 0, st>>>(s->M, s->k, nchunks, s->Ws,
                                                                                   s->bpack)));
  SG_LAUNCH_CHECK("k_pack_tf32");
  return SG_OK;
}

int eval_tf32x3(const EvalArgs& e, const sg_surplus* s, cudaStream_t st) {
  if (!s->bpack) return fail(SG_EUNSUPPORTED, "sg_eval_feedback: SG_EVAL_TF32X3 needs k <= 8");
  TcArgs t{};
  t.e = e;
  t.d = s->d;
  t.bpack = s->bpack;
  t.nchunks = s->tc_chunks;
  t.err = s->tc_err;
  const size_t smem = 4 * kTcABytes + 4 * kTcBBytes + sizeof(float) * s->d * s->nf * kTcRows + 64;
  if (smem > 227 * 1024) return fail(SG_EUNSUPPORTED, "sg_eval_feedback: grid level too high for TF32X3");
  SG_CUDA_TRY(ensure_dynamic_smem(k_eval_tf32x3, static_cast<int>(smem)));
  const unsigned blocks = static_cast<unsigned>(ceil_div(e.Q, kTcRows));
  SG_TIMED("k_eval_tf32x3", st, (k_eval_tf32x3<<<blocks, kTcThreads, smem, st>>>(t)));
  SG_LAUNCH_CHECK("k_eval_tf32x3");
  return SG_OK;
}

}  // namespace sg
