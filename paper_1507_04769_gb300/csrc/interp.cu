// Step III and the on-line phase: hierarchical surpluses and evaluation of the
// sparse-grid interpolant (Section 3.3, Eq. interpo).
//
// The 1-D hierarchical basis a^i_j is the Lagrange polynomial on the CGL set
// X^i that is 1 at its point of dX^i.  It is evaluated in barycentric form
// with the Chebyshev-Lobatto weights w_m = (-1)^m delta_m (delta = 1/2 at the
// two ends), which needs the reciprocals 1/(x - x_m) of the finest set only:
// every coarser X^i is a subset of it.
//
// Distinct 1-D functions are numbered per dimension: id 0 = a^1 (constant),
// then level 2 (points 0 and 1), level 3 (2 points), level 4 (4), ..., so a
// node is a tuple of d ids and its basis function is the product of d table
// entries.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "diag.cuh"
#include "grid.cuh"
#include "basis.cuh"
#include "interp.cuh"

namespace sg {

// Number of 1-D functions for levels 1..L+1.
int n_functions(int level) {
  int nf = 0;
  for (int l = 1; l <= level + 1; ++l) nf += delta_count(l);
  return nf;
}

int function_id(int l, int kidx) {
  int off = 0;
  for (int m = 1; m < l; ++m) off += delta_count(m);
  const int j = l == 1 ? 0 : (l == 2 ? kidx / 2 : (kidx - 1) / 2);
  return off + j;
}

// The grid's box (lo, then hi - lo), passed by value so that no host copy
// waits for the stream.
struct SurplusBox {
  double v[2 * kMaxDim];
};

// Points of the finest set X^{L+1} on [0, 1]: x_p = (1 - cos(p pi / 2^L)) / 2
// = sin^2(p pi / 2^(L+1)) (Eq. CGL).  The first 2d threads also store the box.
__global__ void k_fine_coords(int level, double* xf, SurplusBox box, int nbox, double* dbox) {
  const int fine_n = 1 << level;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nbox) dbox[p] = box.v[p];
  if (p > fine_n) return;
  if (level == 0) {
    xf[p] = 0.5;
    return;
  }
  if (p == 0 || p == fine_n || 2 * p == fine_n) {
    xf[p] = p == 0 ? 0.0 : (p == fine_n ? 1.0 : 0.5);   // exact ends and middle
    return;
  }
  const double s = sinpi(static_cast<double>(p) / static_cast<double>(2 * fine_n));
  xf[p] = s * s;
}

// Basis values of every 1-D function at every point of the finest set:
// tab1[id * (fine_n+1) + p].  Used by the surplus build, whose nodes sit on it.
__global__ void k_fine_table(int level, const double* xf, double* tab1) {
  const int fine_n = 1 << level;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > fine_n) return;
  basis_row(level == 0 ? 0.5 : xf[p], level, xf, tab1 + p, fine_n + 1);
}

// One level of Eq. interpo: for the nodes n in [n0, n1) (all with |i| = s),
// w_n = f_n - sum over coarser nodes m < n0 of phi_m(x_n) w_m.  A warp per
// node n: lane l takes the coarser nodes m = l (mod 32), then the 32 partial
// sums are added by a fixed shuffle tree (the result does not depend on the
// launch).
constexpr int kSurpWarps = 4;
template <int KM>   // compile-time bound on the outputs k (so the sums stay in registers)
__global__ void __launch_bounds__(32 * kSurpWarps)
    k_surplus_level(int64_t n0, int64_t n1, int d, int k, int fine_n, const uint16_t* __restrict__ fid,
                    const int16_t* __restrict__ fpt, const double* __restrict__ tab1,
                    const double* __restrict__ f, double* __restrict__ W) {
  const int lane = threadIdx.x & 31;
  const int64_t n = n0 + blockIdx.x * int64_t(kSurpWarps) + (threadIdx.x >> 5);
  if (n >= n1) return;
  double acc[KM];
#pragma unroll
  for (int c = 0; c < KM; ++c) acc[c] = 0.0;
  int pts[kMaxDim];
#pragma unroll
  for (int dim = 0; dim < kMaxDim; ++dim) pts[dim] = dim < d ? fpt[n * d + dim] : 0;
  for (int64_t m = lane; m < n0; m += 32) {
    double phi = 1.0;
#pragma unroll
    for (int dim = 0; dim < kMaxDim; ++dim)
      if (dim < d && phi != 0.0) phi *= tab1[int(fid[m * d + dim]) * (fine_n + 1) + pts[dim]];
    if (phi != 0.0) {
#pragma unroll
      for (int c = 0; c < KM; ++c)
        if (c < k) acc[c] = fma(phi, W[m * k + c], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < KM; ++c) {
    if (c < k) {
      double v = acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) W[n * k + c] = f[n * k + c] - v;
    }
  }
}

// Gather rows of W into the evaluation order.
__global__ void k_gather_rows(int64_t M, int k, const int32_t* __restrict__ order,
                              const double* __restrict__ W, double* __restrict__ Ws) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= M * k) return;
  const int64_t r = e / k, c = e % k;
  Ws[e] = W[int64_t(order[r]) * k + c];
}

// FP64 evaluation: thread per query.  The d x nf basis table of each query
// lives in shared memory (query index fastest, so a warp's accesses are
// consecutive).  The node loop is uniform across the block.  Each node
// carries the table offsets of its active dimensions only (level >= 2; the
// level-1 factor is the constant 1), so its basis product costs
// (active - 1) multiplications, taken by a warp-uniform branch, and the
// contraction costs K fused multiply-adds.
template <int K>
__device__ __forceinline__ void eval_accumulate(const EvalArgs& e, const double* __restrict__ tab,
                                                int tid, double* acc) {
  for (int64_t m = 0; m < e.M; ++m) {
    const int na = e.nact[m];
    const uint16_t* o = e.ops + m * kMaxDim;
    double phi;
    switch (na) {
      case 0: phi = 1.0; break;
      case 1: phi = tab[o[0] * kEvalThreads + tid]; break;
      case 2: phi = tab[o[0] * kEvalThreads + tid] * tab[o[1] * kEvalThreads + tid]; break;
      case 3:
        phi = tab[o[0] * kEvalThreads + tid] * tab[o[1] * kEvalThreads + tid] * tab[o[2] * kEvalThreads + tid];
        break;
      default: {
        phi = tab[o[0] * kEvalThreads + tid] * tab[o[1] * kEvalThreads + tid] *
              tab[o[2] * kEvalThreads + tid] * tab[o[3] * kEvalThreads + tid];
        for (int j = 4; j < na; ++j) phi *= tab[o[j] * kEvalThreads + tid];
      }
    }
    const double* w = e.W + m * K;
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = fma(phi, w[c], acc[c]);
  }
}

template <int D, int K>
__global__ void __launch_bounds__(kEvalThreads) k_eval_fp64(EvalArgs e) {
  extern __shared__ double tabs_s[];
  const int tid = threadIdx.x;
  const int64_t q = blockIdx.x * int64_t(kEvalThreads) + tid;
  const bool live = q < e.Q;
  const int nf = e.nf;
  // tab[(dim * nf + id) * kEvalThreads + tid]
  for (int dim = 0; dim < D; ++dim) {
    const double u = live ? (e.xq[q * D + dim] - e.lo[dim]) / e.width[dim] : 0.5;
    basis_row(u, e.level, e.xf, tabs_s + (dim * nf) * kEvalThreads + tid, kEvalThreads);
  }
  __syncthreads();
  double acc[K];
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = 0.0;
  eval_accumulate<K>(e, tabs_s, tid, acc);
  if (live) {
#pragma unroll
    for (int c = 0; c < K; ++c) e.out[q * K + c] = acc[c];
  }
}

// Any output count: the same loop with a runtime count (rarely used shapes).
template <int D>
__global__ void __launch_bounds__(kEvalThreads) k_eval_fp64_anyk(EvalArgs e) {
  extern __shared__ double tabs_s[];
  const int tid = threadIdx.x;
  const int64_t q = blockIdx.x * int64_t(kEvalThreads) + tid;
  const bool live = q < e.Q;
  const int nf = e.nf;
  for (int dim = 0; dim < D; ++dim) {
    const double u = live ? (e.xq[q * D + dim] - e.lo[dim]) / e.width[dim] : 0.5;
    basis_row(u, e.level, e.xf, tabs_s + (dim * nf) * kEvalThreads + tid, kEvalThreads);
  }
  __syncthreads();
  const int k = e.k;
  for (int c0 = 0; c0 < k; c0 += 4) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t m = 0; m < e.M; ++m) {
      const int na = e.nact[m];
      const uint16_t* o = e.ops + m * kMaxDim;
      double phi = 1.0;
      for (int j = 0; j < na; ++j) phi *= tabs_s[o[j] * kEvalThreads + tid];
      const double* w = e.W + m * k;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c0 + c < k) acc[c] = fma(phi, w[c0 + c], acc[c]);
    }
    if (live)
      for (int c = 0; c < 4 && c0 + c < k; ++c) e.out[q * k + c0 + c] = acc[c];
  }
}

template <int D>
static int launch_eval_fp64(const EvalArgs& e, cudaStream_t st) {
  const size_t smem = sizeof(double) * D * e.nf * kEvalThreads;
  if (smem > 200 * 1024) return fail(SG_EUNSUPPORTED, "sg_eval_feedback: grid level too high for the FP64 kernel");
  const unsigned blocks = static_cast<unsigned>(ceil_div(e.Q, kEvalThreads));
#define SG_EVAL_K(KK)                                                                              \
  case KK:                                                                                         \
    SG_CUDA_TRY(ensure_dynamic_smem(k_eval_fp64<D, KK>, smem));                                  \
    SG_TIMED("k_eval_fp64", st, (k_eval_fp64<D, KK><<<blocks, kEvalThreads, smem, st>>>(e)));      \
    break;
  switch (e.k) {
    SG_EVAL_K(1)
    SG_EVAL_K(2)
    SG_EVAL_K(3)
    SG_EVAL_K(4)
    SG_EVAL_K(6)
    default:
      SG_CUDA_TRY(ensure_dynamic_smem(k_eval_fp64_anyk<D>, static_cast<int>(smem)));
      SG_TIMED("k_eval_fp64", st, (k_eval_fp64_anyk<D><<<blocks, kEvalThreads, smem, st>>>(e)));
  }
#undef SG_EVAL_K
  SG_LAUNCH_CHECK("k_eval_fp64");
  return SG_OK;
}

int eval_fp64(const EvalArgs& e, int d, cudaStream_t st) {
  switch (d) {
    case 1: return launch_eval_fp64<1>(e, st);
    case 2: return launch_eval_fp64<2>(e, st);
    case 3: return launch_eval_fp64<3>(e, st);
    case 4: return launch_eval_fp64<4>(e, st);
    case 5: return launch_eval_fp64<5>(e, st);
    case 6: return launch_eval_fp64<6>(e, st);
    case 7: return launch_eval_fp64<7>(e, st);
    case 8: return launch_eval_fp64<8>(e, st);
    default: return fail(SG_EUNSUPPORTED, "sg_eval_feedback: d must be 1..8");
  }
}

}  // namespace sg

using namespace sg;

namespace sg {
namespace {
// The host-made part of a surplus build: the integer structure of the grid's
// nodes (function ids, fine positions, level ranges, evaluation order, active
// dimensions and table offsets, the sum-factorised plan), the layout of the
// surplus's one device allocation, and the bytes of it that the host fills
// (all but the box).  It depends on the grid's node structure and on k only,
// so builds on grids of the same structure (a grid rebuilt every step) reuse
// it: a small cache keyed by (d, L, k) and checked against the grid's levels
// and indices.
struct SurplusHost {
  int d = 0, L = 0, k = 0, nf = 0, amax = 0;
  int64_t M = 0;
  std::vector<int8_t> lev;      // the key: the grid's integer structure
  std::vector<int16_t> kidx;
  std::vector<int64_t> level_start;
  int64_t grp[kMaxDim + 2] = {};
  bool sf_ok = false, tcoff_ok = false;
  SfPlan sf;                    // scalar fields (its tables are in the staged bytes)
  size_t npack = 0, off = 0, ohost = 0;
  size_t oW = 0, oWs = 0, oWdf = 0, oxf = 0, oxfdf = 0, otab1 = 0, obp = 0, oerr = 0, osfb = 0;
  size_t obox = 0, onact = 0, oops = 0, otcoff = 0, ofid = 0, ofpt = 0, oorder = 0, ometa = 0, obmap = 0;
  std::vector<unsigned char> staging;   // bytes [ohost, off) of the allocation, box zero
  // The same bytes in page-locked memory when it could be had (then
  // `staging` is emptied): a copy from it is queued without waiting for the
  // stream, where a copy from pageable memory first synchronises it.
  unsigned char* pinned = nullptr;
  const unsigned char* bytes() const { return pinned ? pinned : staging.data(); }
  SurplusHost() = default;
  SurplusHost(const SurplusHost&) = delete;
  SurplusHost& operator=(const SurplusHost&) = delete;
  ~SurplusHost() {
    if (pinned) {
      cudaDeviceSynchronize();   // a build may still be copying from it
      cudaFreeHost(pinned);
    }
  }
};

std::shared_ptr<const SurplusHost> make_surplus_host(const sg_grid* g, int k) {
  auto h = std::make_shared<SurplusHost>();
  const int d = g->d, L = g->level, fine_n = 1 << L;
  const int64_t M = g->M;
  h->d = d;
  h->L = L;
  h->k = k;
  h->M = M;
  h->nf = n_functions(L);
  h->lev = g->h_lev;
  h->kidx = g->h_kidx;
  // integer structure (function ids, fine positions, level ranges, order)
  std::vector<uint16_t> fid(M * d);
  std::vector<int16_t> fpt(M * d);
  int prev_sum = -1;
  for (int64_t n = 0; n < M; ++n) {
    int sum = 0;
    for (int dim = 0; dim < d; ++dim) {
      const int l = g->h_lev[n * d + dim], kk = g->h_kidx[n * d + dim];
      sum += l;
      fid[n * d + dim] = static_cast<uint16_t>(function_id(l, kk));
      fpt[n * d + dim] = static_cast<int16_t>(l == 1 ? fine_n / 2 : kk * (fine_n >> (l - 1)));
    }
    if (sum != prev_sum) {
      h->level_start.push_back(n);
      prev_sum = sum;
    }
  }
  h->level_start.push_back(M);
  // evaluation order: by the number of active dimensions (so that a kernel
  // can take each group with a fixed-length basis product), then the
  // function ids lexicographically
  std::vector<int> na_of(M, 0);
  for (int64_t n = 0; n < M; ++n)
    for (int dim = 0; dim < d; ++dim) na_of[n] += fid[n * d + dim] != 0;
  std::vector<int32_t> order(M);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (na_of[a] != na_of[b]) return na_of[a] < na_of[b];
    for (int dim = 0; dim < d; ++dim) {
      if (fid[a * d + dim] != fid[b * d + dim]) return fid[a * d + dim] < fid[b * d + dim];
    }
    return false;
  });
  std::vector<uint8_t> nact(M, 0);
  std::vector<uint16_t> ops(M * kMaxDim, 0);
  for (int a = 0; a <= kMaxDim + 1; ++a) h->grp[a] = M;
  for (int64_t r = M - 1; r >= 0; --r) {
    const int32_t n = order[r];
    int na = 0;
    for (int dim = 0; dim < d; ++dim) {
      const int id = fid[int64_t(n) * d + dim];
      if (id != 0) ops[r * kMaxDim + na++] = static_cast<uint16_t>(dim * h->nf + id);
    }
    nact[r] = static_cast<uint8_t>(na);
    if (na > h->amax) h->amax = na;
    for (int a = 0; a <= na; ++a) h->grp[a] = r < h->grp[a] ? r : h->grp[a];
  }
  // grp[a] = first node with at least a active dimensions (non-decreasing)
  for (int a = kMaxDim; a >= 0; --a) h->grp[a] = h->grp[a] < h->grp[a + 1] ? h->grp[a] : h->grp[a + 1];

  // one device allocation: the surplus's arrays and the build's tables; the
  // device-computed ones first, then the host-made ones (one copy)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  h->oW = take(M * k * sizeof(double));
  h->oWs = take(M * k * sizeof(double));
  h->oWdf = take(M * k * sizeof(float2));
  h->oxf = take((fine_n + 1) * sizeof(double));
  h->oxfdf = take((fine_n + 1) * sizeof(float2));
  h->otab1 = take(size_t(h->nf) * (fine_n + 1) * sizeof(double));
  // the sum-factorised tensor-core plan; the per-node tensor-core pack only
  // where that plan does not fit
  h->sf_ok = sf_plan(d, L, h->nf, k, M, fid, h->sf);
  h->npack = h->sf_ok ? 0 : tf32_pack_floats(M, k);
  h->obp = take(h->npack * sizeof(float));
  h->oerr = take(sizeof(int));
  h->osfb = take(h->sf_ok ? h->sf.bbytes : 0);   // filled on the device (k_pack_sf)
  h->ohost = off;
  h->obox = take(2 * d * sizeof(double));
  h->onact = take(M);
  h->oops = take(M * kMaxDim * sizeof(uint16_t));
  // the tensor-core kernel's table offsets: ops scaled by its 128 table rows
  // (uint16, so the tables must have at most 511 entries per query)
  h->tcoff_ok = h->npack && size_t(d) * h->nf <= 511;
  h->otcoff = take(h->tcoff_ok ? M * kMaxDim * sizeof(uint16_t) : 0);
  h->ofid = take(M * d * sizeof(uint16_t));
  h->ofpt = take(M * d * sizeof(int16_t));
  h->oorder = take(M * sizeof(int32_t));
  h->ometa = take(h->sf_ok ? h->sf.meta.size() : 0);
  h->obmap = take(h->sf_ok ? h->sf.bmap.size() * sizeof(int32_t) : 0);
  h->off = off;
  const size_t oh = h->ohost;
  auto& st = h->staging;
  st.assign(off - oh, 0);
  std::memcpy(st.data() + (h->onact - oh), nact.data(), M);
  std::memcpy(st.data() + (h->oops - oh), ops.data(), M * kMaxDim * sizeof(uint16_t));
  if (h->tcoff_ok) {
    std::vector<uint16_t> tco(M * kMaxDim);
    for (size_t x = 0; x < tco.size(); ++x) tco[x] = static_cast<uint16_t>(ops[x] * 128u);
    std::memcpy(st.data() + (h->otcoff - oh), tco.data(), M * kMaxDim * sizeof(uint16_t));
  }
  std::memcpy(st.data() + (h->ofid - oh), fid.data(), M * d * sizeof(uint16_t));
  std::memcpy(st.data() + (h->ofpt - oh), fpt.data(), M * d * sizeof(int16_t));
  std::memcpy(st.data() + (h->oorder - oh), order.data(), M * sizeof(int32_t));
  if (h->sf_ok) {
    std::memcpy(st.data() + (h->ometa - oh), h->sf.meta.data(), h->sf.meta.size());
    std::memcpy(st.data() + (h->obmap - oh), h->sf.bmap.data(), h->sf.bmap.size() * sizeof(int32_t));
    h->sf.bfloats_ = h->sf.bmap.size();
    h->sf.meta_bytes_ = h->sf.meta.size();
    h->sf.meta.clear();
    h->sf.meta.shrink_to_fit();
    h->sf.bmap.clear();
    h->sf.bmap.shrink_to_fit();
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&h->pinned), st.size(), cudaHostAllocDefault) == cudaSuccess) {
    std::memcpy(h->pinned, st.data(), st.size());
    st.clear();
    st.shrink_to_fit();
  } else {
    h->pinned = nullptr;
    (void)cudaGetLastError();   // pageable staging still works, the copy then waits
  }
  return h;
}

std::shared_ptr<const SurplusHost> surplus_host(const sg_grid* g, int k) {
  static std::mutex mu;
  // most recent last; never destroyed (its entries' page-locked memory is not
  // handed back to a CUDA runtime that may already be shut down at exit)
  static auto* cache = new std::vector<std::shared_ptr<const SurplusHost>>();
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& c : *cache)
      if (c->d == g->d && c->L == g->level && c->k == k && c->M == g->M && c->lev == g->h_lev && c->kidx == g->h_kidx)
        return c;
  }
  auto h = make_surplus_host(g, k);
  std::lock_guard<std::mutex> lk(mu);
  if (cache->size() >= 8) cache->erase(cache->begin());
  cache->push_back(h);
  return h;
}
}  // namespace
}  // namespace sg

extern "C" int sg_build_surpluses(const sg_grid* g, const double* d_values, int k, sg_surplus** out,
                                  void* stream) {
  clear_error();
  if (!g || !d_values || !out) return fail(SG_EINVAL, "sg_build_surpluses: null pointer");
  *out = nullptr;
  if (k < 1 || k > kMaxOut) return fail(SG_EINVAL, "sg_build_surpluses: k must be 1..16");
  if (g->level > kMaxLevel) return fail(SG_EUNSUPPORTED, "sg_build_surpluses: level above 8");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int d = g->d, L = g->level, fine_n = 1 << L;
  const int64_t M = g->M;
  std::shared_ptr<const SurplusHost> hp;
  try {
    hp = surplus_host(g, k);
  } catch (const std::bad_alloc&) {
    return fail(SG_ENOMEM, "sg_build_surpluses: host memory");
  }
  const SurplusHost& h = *hp;
  auto* s = new sg_surplus();
  s->d = d;
  s->level = L;
  s->k = k;
  s->M = M;
  s->nf = h.nf;
  s->amax = h.amax;
  for (int a = 0; a <= kMaxDim + 1; ++a) s->grp[a] = h.grp[a];
  cudaError_t e = block_alloc(&s->block, h.off, st);
  if (e != cudaSuccess) {
    delete s;
    return e == cudaErrorMemoryAllocation ? fail(SG_ENOMEM, "sg_build_surpluses: device allocation") : cuda_fail(e, "sg_build_surpluses: device allocation");
  }
  char* base = static_cast<char*>(s->block);
  s->W = reinterpret_cast<double*>(base + h.oW);
  s->Ws = reinterpret_cast<double*>(base + h.oWs);
  s->Wdf = reinterpret_cast<float2*>(base + h.oWdf);
  s->xf = reinterpret_cast<double*>(base + h.oxf);
  s->xfdf = reinterpret_cast<float2*>(base + h.oxfdf);
  s->bpack = h.npack ? reinterpret_cast<float*>(base + h.obp) : nullptr;
  s->tc_err = reinterpret_cast<int*>(base + h.oerr);
  s->box = reinterpret_cast<double*>(base + h.obox);
  s->nact = reinterpret_cast<uint8_t*>(base + h.onact);
  s->ops = reinterpret_cast<uint16_t*>(base + h.oops);
  s->tcoff = h.tcoff_ok ? reinterpret_cast<uint16_t*>(base + h.otcoff) : nullptr;
  auto* d_fid = reinterpret_cast<uint16_t*>(base + h.ofid);
  auto* d_fpt = reinterpret_cast<int16_t*>(base + h.ofpt);
  auto* d_tab1 = reinterpret_cast<double*>(base + h.otab1);
  auto* d_order = reinterpret_cast<int32_t*>(base + h.oorder);
  if (h.sf_ok) {
    const SfPlan& sf = h.sf;
    s->sf_ok = 1;
    s->sf_side = sf.side;
    s->sf_nks = sf.nks;
    s->sf_ngemv = sf.ngemv;
    for (int i = 0; i < 5; ++i) s->sf_gseg[i] = sf.gseg[i];
    s->sf_kw = sf.kw;
    s->sf_o_gw = sf.o_gw;
    s->sf_o_gops = sf.o_gops;
    s->sf_nepi = sf.nepi;
    s->sf_tmem = sf.tmem_cols;
    s->sf_bbytes = sf.bbytes;
    s->sf_smem = sf.smem;
    s->sf_bfloats = sf.bfloats_;
    s->sf_meta_bytes = sf.meta_bytes_;
    s->sf_o_aops = sf.o_aops;
    s->sf_o_epi = sf.o_epi;
    s->sf_o_prog = sf.o_prog;
    s->sf_o_pstart = sf.o_pstart;
    s->sf_meta = reinterpret_cast<unsigned char*>(base + h.ometa);
    s->sf_bmap = reinterpret_cast<int32_t*>(base + h.obmap);
    s->sf_b = reinterpret_cast<float*>(base + h.osfb);
  }
  auto cleanup = [&](cudaError_t err, const char* what) {
    sg_surplus_free(s);
    return err == cudaErrorMemoryAllocation ? fail(SG_ENOMEM, what) : cuda_fail(err, what);
  };
#define SG_TRY_CLEAN(expr)                                  \
  if ((e = (expr)) != cudaSuccess) return cleanup(e, #expr);
  // the host-made tables (cached), then this grid's box over their zero
  // bytes (written by k_fine_coords from its arguments)
  SurplusBox box{};
  for (int dim = 0; dim < d; ++dim) {
    box.v[dim] = g->h_lo[dim];
    box.v[d + dim] = g->h_hi[dim] - g->h_lo[dim];
  }
  SG_TRY_CLEAN(cudaMemcpyAsync(base + h.ohost, h.bytes(), h.off - h.ohost, cudaMemcpyHostToDevice, st));
  SG_TIMED("k_fine_coords", st,
           (k_fine_coords<<<static_cast<unsigned>(ceil_div(fine_n + 1 > 2 * d ? fine_n + 1 : 2 * d, 64)), 64, 0, st>>>(
               L, s->xf, box, 2 * d, s->box)));
  SG_TIMED("k_fine_table", st, (k_fine_table<<<static_cast<unsigned>(ceil_div(fine_n + 1, 64)), 64, 0, st>>>(L, s->xf, d_tab1)));
  SG_TRY_CLEAN(cudaGetLastError());
  for (size_t lv = 0; lv + 1 < h.level_start.size(); ++lv) {
    const int64_t n0 = h.level_start[lv], n1 = h.level_start[lv + 1];
    auto* kern = k <= 4 ? k_surplus_level<4> : k_surplus_level<kMaxOut>;
    SG_TIMED("k_surplus_level", st,
             (kern<<<static_cast<unsigned>(ceil_div(n1 - n0, kSurpWarps)), 32 * kSurpWarps, 0, st>>>(
                 n0, n1, d, k, fine_n, d_fid, d_fpt, d_tab1, d_values, s->W)));
    SG_TRY_CLEAN(cudaGetLastError());
  }
  SG_TIMED("k_gather_rows", st, (k_gather_rows<<<static_cast<unsigned>(ceil_div(M * k, 256)), 256, 0, st>>>(M, k, d_order, s->W, s->Ws)));
  SG_TRY_CLEAN(cudaGetLastError());
  if (split_df(fine_n + 1, s->xf, s->xfdf, st) != SG_OK || split_df(M * k, s->Ws, s->Wdf, st) != SG_OK)
    return cleanup(cudaGetLastError(), "split_df");
  SG_TRY_CLEAN(cudaMemsetAsync(s->tc_err, 0, sizeof(int), st));
  if (pack_tf32(s, st) != SG_OK) return cleanup(cudaGetLastError(), "pack_tf32");
  if (sf_pack(s, st) != SG_OK) return cleanup(cudaGetLastError(), "sf_pack");
#undef SG_TRY_CLEAN
  *out = s;
  return SG_OK;
}

extern "C" int sg_surplus_info(const sg_surplus* s, int64_t* n_nodes, int* k, const double** d_W) {
  clear_error();
  if (!s) return fail(SG_EINVAL, "sg_surplus_info: null handle");
  if (n_nodes) *n_nodes = s->M;
  if (k) *k = s->k;
  if (d_W) *d_W = s->W;
  return SG_OK;
}

extern "C" void sg_surplus_free(sg_surplus* s) {
  if (!s) return;
  block_free(s->block);
  delete s;
}

extern "C" int sg_eval_feedback(const sg_surplus* s, const double* d_xq, int64_t Q, int mode, double* d_out,
                                void* stream) {
  clear_error();
  if (!s) return fail(SG_EINVAL, "sg_eval_feedback: null handle");
  if (Q < 0) return fail(SG_EINVAL, "sg_eval_feedback: Q < 0");
  if (Q == 0) return SG_OK;
  if (!d_xq || !d_out) return fail(SG_EINVAL, "sg_eval_feedback: null device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  EvalArgs e{};
  e.xq = d_xq;
  e.Q = Q;
  e.M = s->M;
  e.k = s->k;
  e.nf = s->nf;
  e.level = s->level;
  e.amax = s->amax;
  e.nact = s->nact;
  e.ops = s->ops;
  e.W = s->Ws;
  e.lo = s->box;
  e.width = s->box + s->d;
  e.xf = s->xf;
  e.xfdf = s->xfdf;
  e.Wdf = s->Wdf;
  for (int a = 0; a <= kMaxDim + 1; ++a) e.grp[a] = s->grp[a];
  e.out = d_out;
  if (mode == SG_EVAL_FP64) return eval_fp64(e, s->d, st);
  if (mode == SG_EVAL_TF32X3) return s->sf_ok ? eval_sf_tf32x3(e, s, st) : eval_tf32x3(e, s, st);
  if (mode == SG_EVAL_DF32) return eval_df32(e, s->d, st);
  return fail(SG_EINVAL, "sg_eval_feedback: unknown mode");
}
