// Split-TF32 evaluation of the interpolant contraction on the fifth-generation
// tensor cores (tcgen05, accumulators in tensor memory).
//
// u = Phi W with Phi (queries x nodes) generated on the fly and W (nodes x k)
// the surpluses.  With Phi = Phi_hi + Phi_lo and W = W_hi + W_lo split into
// TF32 parts, u ~ Phi_hi W_hi + Phi_hi W_lo + Phi_lo W_hi (the 3xTF32 scheme):
// an accumulator D (128 rows x 16 columns, FP32) receives
//   Phi_hi x [W_hi | W_lo | 0]  and  Phi_lo x [W_hi | 0 | 0],
// so that u = D[:, 0:k] + D[:, k:2k] (k <= 8 outputs).
//
// The 1-D basis tables are computed in pair-of-floats arithmetic (about 48
// bits) and rounded once to FP32, so Phi carries only the FP32 rounding of its
// factors and products; the nodes are split over kTcAcc accumulators (each a
// 16-column block of tensor memory) that are added in FP64 at the end, so the
// FP32 accumulation runs over at most ceil(M / kTcAcc) nodes.
//
// One CTA per 128 queries, warp-specialised:
//   warps 0..7   producers: threads t and t + 128 own query row t; per chunk
//                of 16 nodes each writes one K-step (8 nodes) of its row of
//                Phi_hi and Phi_lo into a stage of a shared-memory ring, in
//                the no-swizzle K-major core-matrix layout, then arrives on
//                the stage's "full" mbarrier;
//   warp 8       lane 0 waits for a full stage, issues its 2 x 2 MMAs
//                (M = 128, N = 16, K = 8, kind::tf32) and commits them to the
//                stage's "empty" mbarrier, which the producers wait on before
//                refilling the stage.
// No thread waits for another producer; the ring has kTcStages stages.  Every
// wait on an mbarrier has an iteration limit: on timeout the kernel records
// an error flag, writes NaN outputs, releases its tensor memory and returns.
#include "basis.cuh"
#include "common.cuh"
#include "diag.cuh"
#include "interp.cuh"
#include "tcgen05.cuh"

namespace sg {

constexpr int kTcRows = 128;          // queries per CTA (= MMA M)
constexpr int kTcProducers = 256;     // two producer threads per query row
constexpr int kTcThreads = kTcProducers + 32;   // + the MMA warp
constexpr int kTcN = 16;              // MMA N (2k <= 16)
constexpr int kTcChunk = 16;          // nodes per stage (2 MMA K-steps of 8, one per producer of a row)
constexpr int kTcStages = 3;          // ring depth
constexpr int kTcAcc = 8;             // accumulators (16 tensor-memory columns each)
constexpr int kTcAStep = kTcRows * 32;          // bytes of one K-step of A (128 rows x 8 tf32)
constexpr int kTcABytes = 2 * kTcAStep;         // one chunk of Phi_hi or Phi_lo: 8 KB
constexpr int kTcBStep = kTcN * 32;             // bytes of one K-step of B (16 rows x 8 tf32)
constexpr int kTcBBytes = 2 * kTcBStep;         // one chunk of one B matrix: 1 KB
constexpr int kTcBPack = 2 * kTcBBytes / 4;     // floats per chunk of [B1 | B2]
constexpr int kTcStageBytes = 2 * kTcABytes + 2 * kTcBBytes;   // Phi_hi | Phi_lo | B1 | B2

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

struct TcArgs {
  EvalArgs e;
  int d;
  const float* bpack;      // nchunks x kTcBPack
  const uint16_t* tcoff;   // M x 8: table offsets (ops x kTcRows); padded slots point at tab[0] = 1
  int nchunks;
  int* err;
};

// One K-step (8 nodes) of Phi_hi and Phi_lo for query row `row`: node j of
// the step has its table offsets at offs[8 j ..] and is the product of its A
// basis values; nodes j >= nvalid (past the last node) are zero.
template <int A, bool kFull>
__device__ __forceinline__ void tc_produce_kstep(const uint16_t* __restrict__ offs, int nvalid,
                                                 const float* __restrict__ tabrow, unsigned char* ahi,
                                                 unsigned char* alo, int off) {
#pragma unroll
  for (int c2 = 0; c2 < 2; ++c2) {
    float hv[4], lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int jj = c2 * 4 + j;
      float phi = 0.0f;
      if (kFull || jj < nvalid) {
        const uint4 ov = reinterpret_cast<const uint4*>(offs)[jj];
        const uint32_t w[4] = {ov.x, ov.y, ov.z, ov.w};
        phi = tabrow[w[0] & 0xFFFFu];
#pragma unroll
        for (int a = 1; a < A; ++a) phi = __fmul_rn(phi, tabrow[(a & 1) ? (w[a >> 1] >> 16) : (w[a >> 1] & 0xFFFFu)]);
      }
      tf32_split(phi, hv[j], lv[j]);
    }
    *reinterpret_cast<float4*>(ahi + off + c2 * 128) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4*>(alo + off + c2 * 128) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
}

template <int A>
__device__ __forceinline__ void tc_produce(const uint16_t* __restrict__ offs, int nvalid,
                                           const float* __restrict__ tabrow, unsigned char* ahi, unsigned char* alo,
                                           int off) {
  if (nvalid >= 8) tc_produce_kstep<A, true>(offs, 8, tabrow, ahi, alo, off);
  else tc_produce_kstep<A, false>(offs, nvalid, tabrow, ahi, alo, off);
}

__global__ void __launch_bounds__(kTcThreads) k_eval_tf32x3(TcArgs t) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const EvalArgs& e = t.e;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nf = e.nf;
  const int nchunks = t.nchunks;
  // layout: stages (kTcStages x [Phi_hi | Phi_lo | B1 | B2]) | tables | barriers
  unsigned char* ring = smem;
  float* tab = reinterpret_cast<float*>(ring + kTcStages * kTcStageBytes);     // d * nf * kTcRows
  uint64_t* bars = reinterpret_cast<uint64_t*>(tab + size_t(t.d) * nf * kTcRows);
  uint64_t* full = bars;                    // kTcStages, count kTcProducers
  uint64_t* empty = bars + kTcStages;       // kTcStages, count 1 (tcgen05.commit)
  uint64_t* done = bars + 2 * kTcStages;    // 1: every MMA has completed
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 1);
  int* flag = reinterpret_cast<int*>(tmem_holder + 1);   // 0 = all waits succeeded

  const int row = tid & (kTcRows - 1), half = (tid >> 7) & 1;
  const int64_t q = blockIdx.x * int64_t(kTcRows) + row;
  const bool producer = tid < kTcProducers;
  const bool live = producer && q < e.Q;
  if (producer) {
    // the two threads of a row share its 1-D tables, computed in pairs of
    // floats and rounded once to FP32
    for (int dim = half; dim < t.d; dim += 2) {
      const double u = live ? (e.xq[q * t.d + dim] - e.lo[dim]) / e.width[dim] : 0.5;
      basis_row_df_hi(u, e.level, e.xfdf, tab + (dim * nf) * kTcRows + row, kTcRows);
    }
  } else if (warp == kTcProducers / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(16 * kTcAcc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    if (lane == 0) {
      for (int s = 0; s < kTcStages; ++s) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(kTcProducers));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
      }
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
      *flag = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_holder;
  bool ok = true;

  if (producer) {
    for (int c = 0; c < nchunks && ok; ++c) {
      const int st = c % kTcStages;
      if (c >= kTcStages) ok = mbar_wait(smem_u32(&empty[st]), ((c / kTcStages) - 1) & 1);
      if (!ok) break;
      unsigned char* stage = ring + st * kTcStageBytes;
      unsigned char* ahi = stage;
      unsigned char* alo = stage + kTcABytes;
      // the chunk's nodes are sorted by active count: its last node has the most
      const int64_t m0 = int64_t(c) * kTcChunk;
      const int64_t mlast = (m0 + kTcChunk < e.M ? m0 + kTcChunk : e.M) - 1;
      const int A = e.nact[mlast];
      // element (r, k) of K-step s at
      //   s * kTcAStep + ((r / 8) * 2 + (k % 8) / 4) * 128 + (r % 8) * 16 + (k % 4) * 4
      const int off = half * kTcAStep + ((row / 8) * 2) * 128 + (row % 8) * 16;
      const float* tabrow = tab + row;
      const int64_t mk = m0 + half * 8;
      const int nvalid = static_cast<int>(e.M - mk < 8 ? e.M - mk : 8);
      const uint16_t* offs = t.tcoff + mk * kMaxDim;
      switch (A) {
        case 0:
        case 1: tc_produce<1>(offs, nvalid, tabrow, ahi, alo, off); break;
        case 2: tc_produce<2>(offs, nvalid, tabrow, ahi, alo, off); break;
        case 3: tc_produce<3>(offs, nvalid, tabrow, ahi, alo, off); break;
        case 4: tc_produce<4>(offs, nvalid, tabrow, ahi, alo, off); break;
        case 5: tc_produce<5>(offs, nvalid, tabrow, ahi, alo, off); break;
        case 6: tc_produce<6>(offs, nvalid, tabrow, ahi, alo, off); break;
        case 7: tc_produce<7>(offs, nvalid, tabrow, ahi, alo, off); break;
        default: tc_produce<8>(offs, nvalid, tabrow, ahi, alo, off); break;
      }
      // the chunk of [B1 | B2], pre-packed in the same layout: the first
      // kTcBPack / 4 producers copy one 16-byte word each
      if (tid < kTcBPack / 4) {
        const float4* src = reinterpret_cast<const float4*>(t.bpack + size_t(c) * kTcBPack);
        reinterpret_cast<float4*>(stage + 2 * kTcABytes)[tid] = src[tid];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full[st]));
    }
  } else if (lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32();
    const int per_acc = (nchunks + kTcAcc - 1) / kTcAcc;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int st = c % kTcStages;
      ok = mbar_wait(smem_u32(&full[st]), (c / kTcStages) & 1);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned char* stage = ring + st * kTcStageBytes;
      const uint32_t a_hi = smem_u32(stage), a_lo = a_hi + kTcABytes;
      const uint32_t b1 = a_hi + 2 * kTcABytes, b2 = b1 + kTcBBytes;
      const uint32_t acc_col = tmem + static_cast<uint32_t>((c / per_acc) * kTcN);
      const bool first = (c % per_acc) == 0;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint64_t da_hi = smem_desc(a_hi + s * kTcAStep, 128, 256);
        const uint64_t da_lo = smem_desc(a_lo + s * kTcAStep, 128, 256);
        const uint64_t db1 = smem_desc(b1 + s * kTcBStep, 128, 256);
        const uint64_t db2 = smem_desc(b2 + s * kTcBStep, 128, 256);
        const uint32_t acc = (first && s == 0) ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_col),
            "l"(da_hi), "l"(db1), "r"(idesc), "r"(acc));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_col),
            "l"(da_lo), "l"(db2), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty[st])));
    }
    // completes when every MMA issued above has finished
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(done)));
  }
  if (!ok) atomicExch(flag, 1);
  // epilogue: warps 0..3 read tensor-memory lanes 32w .. 32w + 31 (accumulator rows)
  double epi_sum[kTcN / 2];
  bool epi_fin = false;
  if (warp < 4) {
    bool fin = mbar_wait(smem_u32(done), 0);
    if (!fin) atomicExch(flag, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    double sum[kTcN / 2];
#pragma unroll
    for (int j = 0; j < kTcN / 2; ++j) sum[j] = 0.0;
    const int per_acc = (nchunks + kTcAcc - 1) / kTcAcc;
    const int nacc = nchunks > 0 ? (nchunks + per_acc - 1) / per_acc : 0;
    for (int a = 0; a < nacc && fin; ++a) {
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(a * kTcN);
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      for (int cix = 0; cix < e.k; ++cix) {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (j == cix) hi = __uint_as_float(r[j]);
          if (j == e.k + cix) lo = __uint_as_float(r[j]);
        }
#pragma unroll
        for (int j = 0; j < kTcN / 2; ++j)
          if (j == cix) sum[j] += static_cast<double>(hi) + static_cast<double>(lo);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncwarp();
    epi_fin = fin;
#pragma unroll
    for (int j = 0; j < kTcN / 2; ++j) epi_sum[j] = sum[j];
  }
  __syncwarp();
  __syncthreads();   // every wait of every thread is over: the flag is final
  const bool good = *reinterpret_cast<volatile int*>(flag) == 0;
  if (warp < 4 && q < e.Q) {
    for (int cix = 0; cix < e.k; ++cix) {
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < kTcN / 2; ++j)
        if (j == cix) v = epi_sum[j];
      e.out[q * e.k + cix] = good && epi_fin ? v : NAN;
    }
  }
  if (tid == 0 && !good) atomicExch(t.err, 1);
  if (warp == kTcProducers / 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(16 * kTcAcc));
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

// s->bpack (tf32_pack_floats(M, k) floats) and s->tc_err (zeroed) come with the
// surplus's allocation.
int pack_tf32(sg_surplus* s, cudaStream_t st) {
  if (s->k > kTcN / 2 || !s->bpack) return SG_OK;   // k <= 8, and only where the pack was allocated
  const int nchunks = static_cast<int>(ceil_div(s->M, kTcChunk));
  s->tc_chunks = nchunks;
  const int64_t total = int64_t(nchunks) * kTcChunk * kTcN;
  SG_TIMED("k_pack_tf32", st,
           (k_pack_tf32<<<static_cast<unsigned>(ceil_div(total, 256)), 256, 0, st>>>(s->M, s->k, nchunks, s->Ws,
                                                                                   s->bpack)));
  SG_LAUNCH_CHECK("k_pack_tf32");
  return SG_OK;
}

int eval_tf32x3(const EvalArgs& e, const sg_surplus* s, cudaStream_t st) {
  if (!s->bpack) return fail(SG_EUNSUPPORTED, "sg_eval_feedback: SG_EVAL_TF32X3 needs k <= 8");
  if (!s->tcoff) return fail(SG_EUNSUPPORTED, "sg_eval_feedback: grid level too high for TF32X3");
  TcArgs t{};
  t.e = e;
  t.d = s->d;
  t.bpack = s->bpack;
  t.tcoff = s->tcoff;
  t.nchunks = s->tc_chunks;
  t.err = s->tc_err;
  const size_t smem = size_t(kTcStages) * kTcStageBytes + sizeof(float) * s->d * s->nf * kTcRows + 128;
  if (smem > 227 * 1024) return fail(SG_EUNSUPPORTED, "sg_eval_feedback: grid level too high for TF32X3");
  SG_CUDA_TRY(ensure_dynamic_smem(k_eval_tf32x3, static_cast<int>(smem)));
  const unsigned blocks = static_cast<unsigned>(ceil_div(e.Q, kTcRows));
  SG_TIMED("k_eval_tf32x3", st, (k_eval_tf32x3<<<blocks, kTcThreads, smem, st>>>(t)));
  SG_LAUNCH_CHECK("k_eval_tf32x3");
  return SG_OK;
}

}  // namespace sg
