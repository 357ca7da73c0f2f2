// Step II: the characteristic BVP at every node (Section 3.1, Eq. hamchar).
// Host side of the solver: workspace layout, the Newton loop over the kernels
// of bvp_kernels.cuh, and the C ABI entry points.
#include <cmath>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "bvp_kernels.cuh"
#include "bvp_persistent.cuh"
#include "common.cuh"
#include "diag.cuh"

namespace sg {

static Workspace carve(void* base, int64_t n, int Nmax, size_t tsize) {
  Workspace w{};
  const int64_t P = 3 * int64_t(Nmax) + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return static_cast<char*>(base) + o;
  };
  w.Y = reinterpret_cast<double*>(take(n * P * 12 * sizeof(double)));
  w.D = reinterpret_cast<double*>(take(n * P * 12 * sizeof(double)));
  w.Y2 = tsize == sizeof(float) ? reinterpret_cast<double*>(take(n * P * 12 * sizeof(double))) : nullptr;
  w.Jm = take(n * P * 144 * tsize);
  w.Res = take(n * int64_t(Nmax) * kResRows * tsize);
  w.Cond = take(n * int64_t(Nmax) * kBlk * tsize);
  w.Rec = take(n * int64_t(Nmax) * kRec * tsize);
  w.Abd = take(n * int64_t(Nmax) * kBlk * tsize);
  w.Seg = take(n * int64_t(Nmax) * kSegBlk * tsize);
  w.Red = take(n * int64_t(seg_count(Nmax)) * kBlk * tsize);
  w.part = reinterpret_cast<double*>(take(n * int64_t(Nmax) * 2 * sizeof(double)));
  w.ns = reinterpret_cast<NodeState*>(take(n * sizeof(NodeState)));
  w.counters = reinterpret_cast<int*>(take(256));
  w.bytes = off;
  return w;
}

// ---------------------------------------------------------------- host
static bool invert3(const double* R, double* Ri) {
  const double a = R[0], b = R[1], c = R[2], d = R[3], e = R[4], f = R[5], g = R[6], h = R[7], k = R[8];
  const double det = a * (e * k - f * h) - b * (d * k - f * g) + c * (d * h - e * g);
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
  const double id = 1.0 / det;
  Ri[0] = (e * k - f * h) * id;
  Ri[1] = (c * h - b * k) * id;
  Ri[2] = (b * f - c * e) * id;
  Ri[3] = (f * g - d * k) * id;
  Ri[4] = (a * k - c * g) * id;
  Ri[5] = (c * d - a * f) * id;
  Ri[6] = (d * h - e * g) * id;
  Ri[7] = (b * g - a * h) * id;
  Ri[8] = (a * e - b * d) * id;
  return true;
}

static float2 split_pair(double x) {
  const float hi = static_cast<float>(x);
  return make_float2(hi, static_cast<float>(x - static_cast<double>(hi)));
}

bool make_dev_problem(const sg_problem& in, DevProblem* out) {
  DevProblem p{};
  p.kind = in.kind;
  if (in.kind == SG_PROBLEM_ATTITUDE) {
    if (!(in.r > 0.0)) return false;
    for (int i = 0; i < 3; ++i) {
      if (!(in.J[i] > 0.0)) return false;
      p.Jinv[i] = 1.0 / in.J[i];
      p.hm[i] = in.hmom[i];
    }
    const int m = in.m == 0 ? 3 : in.m;
    if (m != 2 && m != 3) return false;
    p.m = m;
    p.target = in.d_target;
    double Bm[9];   // B with the columns beyond m zeroed
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Bm[3 * i + j] = j < m ? in.B[3 * i + j] : 0.0;
    double JB[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) JB[3 * i + j] = p.Jinv[i] * Bm[3 * i + j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += JB[3 * i + m] * JB[3 * j + m];
        p.Kw[3 * i + j] = s / in.r;
        p.Gw[3 * i + j] = Bm[3 * j + i] * p.Jinv[j] / in.r;
      }
    // plant input matrix J^-1 B in rows 3..5 of a 6 x 3 (rows 0..2 zero)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) p.Bu[3 * (3 + i) + j] = JB[3 * i + j];
    p.wv = in.wv;
    p.ww = in.ww;
    p.r = in.r;
    p.tv = in.tv;
    p.tw = in.tw;
  } else if (in.kind == SG_PROBLEM_LQ) {
    double Ri[9];
    if (!invert3(in.R, Ri)) return false;
    for (int e = 0; e < 36; ++e) {
      p.A[e] = in.A[e];
      p.Q[e] = in.Q[e];
      p.QT[e] = in.QT[e];
    }
    for (int e = 0; e < 9; ++e) p.R[e] = in.R[e];
    for (int e = 0; e < 18; ++e) p.Bu[e] = in.Blq[e];
    // G = R^-1 B' (3 x 6); K = B G (6 x 6)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 6; ++j) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += Ri[3 * i + m] * in.Blq[3 * j + m];
        p.G[6 * i + j] = s;
      }
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += in.Blq[3 * i + m] * p.G[6 * m + j];
        p.K[6 * i + j] = s;
      }
  } else if (in.kind != SG_PROBLEM_EXAMPLE3) {
    return false;
  }
  for (int i = 0; i < 3; ++i) {
    p.Jinv_f[i] = split_pair(p.Jinv[i]);
    p.hm_f[i] = split_pair(p.hm[i]);
  }
  for (int i = 0; i < 9; ++i) p.Kw_f[i] = split_pair(p.Kw[i]);
  p.wv_f = split_pair(p.wv);
  p.ww_f = split_pair(p.ww);
  for (int i = 0; i < 36; ++i) {
    p.A_f[i] = split_pair(p.A[i]);
    p.K_f[i] = split_pair(p.K[i]);
    p.Q_f[i] = split_pair(p.Q[i]);
  }
  *out = p;
  return true;
}

// Interned kernel names (KernelTimer keeps the pointer until collection).
static const char* intern(const std::string& s) {
  static std::mutex mu;
  static std::vector<std::string*> names;
  std::lock_guard<std::mutex> lk(mu);
  for (auto* n : names)
    if (*n == s) return n->c_str();
  names.push_back(new std::string(s));
  return names.back()->c_str();
}

// The forms with an FP32 direction (their workspace holds floats).
static bool fp32_direction(int precision) {
  return precision == SG_PREC_MIXED || precision == SG_PREC_MIXED_PAIR;
}

static size_t ws_bytes(int64_t n, int Nmax, int precision) {
  const size_t tsize = fp32_direction(precision) ? sizeof(float) : sizeof(double);
  return carve(nullptr, n, Nmax, tsize).bytes;
}

template <typename T>
static const char* kname(const char* base) {
  // static names per (kernel, precision) for the launch accounting
  static thread_local std::string buf;
  buf = std::string(base) + (sizeof(T) == sizeof(double) ? "_fp64" : "_fp32");
  return intern(buf);
}

template <typename T>
static int run_solve(const SolveArgs& a, Workspace w, cudaStream_t st, double* lambda0, double* u0,
                     double* V, int32_t* status, int32_t* iters, double* Yout) {
  const int64_t P = npts(a.Nmax);
  const int64_t npoint = a.n * P;
  const int64_t nint = a.n * a.Nmax;
  const unsigned gp = static_cast<unsigned>(ceil_div(npoint, 128));
  const unsigned gupd = static_cast<unsigned>(ceil_div(npoint * kUpdPer, 128));
  const unsigned ginit = static_cast<unsigned>(ceil_div(npoint * kInitPer, 128));
  const unsigned gi = static_cast<unsigned>(a.n * trial_chunks(a.Nmax));
  const unsigned gnode_thr = static_cast<unsigned>(ceil_div(a.n, 128));
  const unsigned gnode_warp = static_cast<unsigned>(ceil_div(a.n * 32, 128));
  const unsigned gwarp_int = static_cast<unsigned>(ceil_div(nint, 4));
  const unsigned gwarp_node = static_cast<unsigned>(ceil_div(a.n, 4));
  const unsigned gwarp_seg = static_cast<unsigned>(ceil_div(a.n * seg_count(a.Nmax), 4));
  const unsigned gseg_blk = static_cast<unsigned>(ceil_div(a.n * seg_count(a.Nmax), seg_warps<T>()));
  const size_t cond_smem = sizeof(double) * kCondWarps * 36 * kCols;
  if constexpr (sizeof(T) == sizeof(double)) {
    SG_CUDA_TRY(ensure_dynamic_smem(k_condense_smem, static_cast<int>(cond_smem)));
  }
  if (a.persistent) {
    // one warp per node, nodes from a device queue, no host round trip
    const int smem = 4 * persist_smem_per_warp<T>();
    SG_CUDA_TRY(ensure_dynamic_smem(k_newton_persistent<T>, smem));
    int dev = 0, sms = 0, per_sm = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    SG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_newton_persistent<T>, 128, smem));
    if (per_sm < 1) per_sm = 1;
    if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
    const int64_t want = ceil_div(a.n, 4);
    const unsigned grid = static_cast<unsigned>(want < int64_t(sms) * per_sm ? want : int64_t(sms) * per_sm);
    SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 4 * sizeof(int), st));
    SG_TIMED("k_init", st, (k_init<<<ginit, 128, 0, st>>>(a, w)));
    SG_TIMED(kname<T>("k_newton_persistent"), st, (k_newton_persistent<T><<<grid, 128, smem, st>>>(a, w)));
    SG_TIMED("k_outputs", st, (k_outputs<<<gnode_warp, 128, 0, st>>>(a, w, lambda0, u0, V, status, iters)));
    if (Yout) SG_TIMED("k_copy_Y", st, (k_copy_Y<<<gp, 128, 0, st>>>(a, w, Yout)));
    SG_LAUNCH_CHECK("persistent solve");
    if (a.sync_at_end) SG_CUDA_TRY(cudaStreamSynchronize(st));
    return SG_OK;
  }
  int h_cnt[2] = {0, 0};
  auto read_counters = [&]() -> int {
    cudaError_t e = cudaMemcpyAsync(h_cnt, w.counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "counter copy");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "solver kernels");
    return SG_OK;
  };
  int rc;
  SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), st));
  SG_TIMED("k_init", st, (k_init<<<ginit, 128, 0, st>>>(a, w)));
  SG_TIMED("k_trial", st, (trial_kernel<T>(a)<<<gi, 128, 0, st>>>(a, w)));
  SG_TIMED("k_ls_reduce", st, (k_ls_reduce<<<gnode_warp, 128, 0, st>>>(a, w, 0)));
  SG_LAUNCH_CHECK("init kernels");
  if ((rc = read_counters()) != SG_OK) return rc;
  int active = h_cnt[1];
  for (int it = 0; it < a.max_iter && active > 0; ++it) {
    SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), st));
    if (!a.jac_in_trial) SG_TIMED(kname<T>("k_point"), st, (k_point<T><<<gp, 128, 0, st>>>(a, w)));   // else stored by the last trial
    if constexpr (sizeof(T) == sizeof(float)) {
      const int cw = condense_reg_warps(a.cond_warps);
      SG_TIMED("k_condense_reg_fp32", st,
               (condense_reg_kernel(cw)<<<static_cast<unsigned>(ceil_div(nint, cw)), 32 * cw, 0, st>>>(a, w)));
    } else {
      SG_TIMED("k_condense_smem_fp64", st,
               (k_condense_smem<<<static_cast<unsigned>(ceil_div(nint, kCondWarps)), 32 * kCondWarps, cond_smem,
                                  st>>>(a, w)));
    }
    SG_TIMED(kname<T>("k_abd_seg"), st, (k_abd_seg<T><<<gseg_blk, 32 * seg_warps<T>(), 0, st>>>(a, w)));
    SG_TIMED(kname<T>("k_abd_red"), st, (k_abd_red<T><<<gwarp_node, 128, 0, st>>>(a, w)));
    SG_TIMED(kname<T>("k_abd_segback"), st, (k_abd_segback<T><<<gwarp_seg, 128, 0, st>>>(a, w)));
    SG_TIMED(kname<T>("k_recover"), st, (k_recover<T><<<gwarp_int, 128, 0, st>>>(a, w)));
    SG_TIMED("k_ls_begin", st, (k_ls_begin<<<gnode_thr, 128, 0, st>>>(a, w)));
    SG_LAUNCH_CHECK("newton kernels");
    for (int trial = 0; trial < 12; ++trial) {
      SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, sizeof(int), st));
      SG_TIMED("k_trial", st, (trial_kernel<T>(a)<<<gi, 128, 0, st>>>(a, w)));
      SG_TIMED("k_ls_reduce", st, (k_ls_reduce<<<gnode_warp, 128, 0, st>>>(a, w, 1)));
      SG_LAUNCH_CHECK("line search kernels");
      if ((rc = read_counters()) != SG_OK) return rc;
      if (h_cnt[0] == 0) break;
    }
    SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), st));
    if (!a.jac_in_trial) SG_TIMED("k_update", st, (k_update<<<gupd, 128, 0, st>>>(a, w)));   // else the accepted trial point
    SG_TIMED("k_after_update", st, (k_after_update<<<gnode_thr, 128, 0, st>>>(a, w)));
    SG_LAUNCH_CHECK("update kernels");
    if ((rc = read_counters()) != SG_OK) return rc;
    active = h_cnt[1];
  }
  SG_TIMED("k_outputs", st, (k_outputs<<<gnode_warp, 128, 0, st>>>(a, w, lambda0, u0, V, status, iters)));
  if (Yout) SG_TIMED("k_copy_Y", st, (k_copy_Y<<<gp, 128, 0, st>>>(a, w, Yout)));
  SG_LAUNCH_CHECK("output kernels");
  SG_CUDA_TRY(cudaStreamSynchronize(st));
  return SG_OK;
}

// ---------------------------------------------------------------- graph form
// The launch-per-phase solve as one CUDA graph: the Newton iteration and the
// line search are WHILE conditional nodes whose conditions are set on the
// device from the active / searching counters, so the data-dependent loop
// trip counts never reach the host.  Executable graphs are cached per
// (sizes, precision, buffers, problem): one per mesh size for a given batch.
__global__ void k_set_cond(cudaGraphConditionalHandle h, const int* cnt) {
  cudaGraphSetConditional(h, cnt[0] > 0 ? 1u : 0u);
}
__global__ void k_set_cond_one(cudaGraphConditionalHandle h) { cudaGraphSetConditional(h, 1u); }

// Counts the nodes that start a line search (replaces the host read).
__global__ void k_count_searching(SolveArgs a, Workspace w) {
  const int64_t node = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (node >= a.n) return;
  if (w.ns[node].searching) atomicAdd(&w.counters[0], 1);
}

struct GraphBuilder {
  cudaGraph_t g;
  std::vector<cudaGraphNode_t> last;   // dependencies for the next node
  cudaError_t err = cudaSuccess;

  template <typename... Args>
  void kernel(void (*f)(Args...), unsigned grid, unsigned block, size_t smem, Args... args) {
    if (err != cudaSuccess) return;
    void* ptrs[] = {static_cast<void*>(&args)...};
    cudaKernelNodeParams p{};
    p.func = reinterpret_cast<void*>(f);
    p.gridDim = dim3(grid);
    p.blockDim = dim3(block);
    p.sharedMemBytes = static_cast<unsigned>(smem);
    p.kernelParams = ptrs;
    cudaGraphNode_t n;
    err = cudaGraphAddKernelNode(&n, g, last.data(), last.size(), &p);
    last.assign(1, n);
  }
  void memset0(void* ptr, size_t bytes) {
    if (err != cudaSuccess) return;
    cudaMemsetParams p{};
    p.dst = ptr;
    p.value = 0;
    p.elementSize = 1;
    p.width = bytes;
    p.height = 1;
    cudaGraphNode_t n;
    err = cudaGraphAddMemsetNode(&n, g, last.data(), last.size(), &p);
    last.assign(1, n);
  }
  // Adds a WHILE node; returns its body graph (empty) through *body.
  void loop(cudaGraphConditionalHandle h, cudaGraph_t* body) {
    if (err != cudaSuccess) return;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t n;
    err = cudaGraphAddNode(&n, g, last.data(), nullptr, last.size(), &p);
    if (err != cudaSuccess) return;   // no body graph was made
    last.assign(1, n);
    *body = p.conditional.phGraph_out[0];
  }
};

template <typename T>
static cudaError_t build_solve_graph(const SolveArgs& a, const Workspace& w, double* lambda0, double* u0,
                                     double* V, int32_t* status, int32_t* iters, double* Yout,
                                     cudaGraph_t* out) {
  const int64_t P = npts(a.Nmax);
  const int64_t nint = a.n * a.Nmax;
  const unsigned gp = static_cast<unsigned>(ceil_div(a.n * P, 128));
  const unsigned gi = static_cast<unsigned>(a.n * trial_chunks(a.Nmax));
  const unsigned gnt = static_cast<unsigned>(ceil_div(a.n, 128));
  const unsigned gnw = static_cast<unsigned>(ceil_div(a.n * 32, 128));
  const unsigned gwi = static_cast<unsigned>(ceil_div(nint, 4));
  const unsigned gwn = static_cast<unsigned>(ceil_div(a.n, 4));
  const unsigned gws = static_cast<unsigned>(ceil_div(a.n * seg_count(a.Nmax), 4));
  const size_t cond_smem = sizeof(double) * kCondWarps * 36 * kCols;
  cudaGraph_t root;
  cudaError_t e = cudaGraphCreate(&root, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle hn, hl;
  if ((e = cudaGraphConditionalHandleCreate(&hn, root, 0, 0)) != cudaSuccess) return e;
  if ((e = cudaGraphConditionalHandleCreate(&hl, root, 0, 0)) != cudaSuccess) return e;
  GraphBuilder rb{root, {}};
  rb.memset0(w.counters, 4 * sizeof(int));
  rb.kernel(k_init, static_cast<unsigned>(ceil_div(a.n * P * kInitPer, 128)), 128, 0, a, w);
  rb.kernel(trial_kernel<T>(a), gi, 128, 0, a, w);
  rb.kernel(k_ls_reduce, gnw, 128, 0, a, w, 0);
  rb.kernel(k_set_cond, 1, 1, 0, hn, static_cast<const int*>(w.counters + 1));
  cudaGraph_t newton_body;
  rb.loop(hn, &newton_body);
  rb.kernel(k_outputs, gnw, 128, 0, a, w, lambda0, u0, V, status, iters);
  if (Yout) rb.kernel(k_copy_Y, gp, 128, 0, a, w, Yout);
  if (rb.err != cudaSuccess) return rb.err;

  GraphBuilder nb{newton_body, {}};
  nb.memset0(w.counters, 2 * sizeof(int));
  if (!a.jac_in_trial) nb.kernel(k_point<T>, gp, 128, 0, a, w);   // else stored by the last trial
  if constexpr (sizeof(T) == sizeof(float)) {
    const int cw = condense_reg_warps(a.cond_warps);
    nb.kernel(condense_reg_kernel(cw), static_cast<unsigned>(ceil_div(nint, cw)), 32 * cw, 0, a, w);
  } else {
    nb.kernel(k_condense_smem, static_cast<unsigned>(ceil_div(nint, kCondWarps)), 32 * kCondWarps, cond_smem, a, w);
  }
  nb.kernel(k_abd_seg<T>, static_cast<unsigned>(ceil_div(a.n * seg_count(a.Nmax), seg_warps<T>())),
            32 * seg_warps<T>(), 0, a, w);
  nb.kernel(k_abd_red<T>, gwn, 128, 0, a, w);
  nb.kernel(k_abd_segback<T>, gws, 128, 0, a, w);
  nb.kernel(k_recover<T>, gwi, 128, 0, a, w);
  nb.kernel(k_ls_begin, gnt, 128, 0, a, w);
  nb.kernel(k_set_cond_one, 1, 1, 0, hl);
  cudaGraph_t ls_body;
  nb.loop(hl, &ls_body);
  nb.memset0(w.counters, 2 * sizeof(int));
  if (!a.jac_in_trial)   // else the accepted trial point is the iterate
    nb.kernel(k_update, static_cast<unsigned>(ceil_div(a.n * npts(a.Nmax) * kUpdPer, 128)), 128, 0, a, w);
  nb.kernel(k_after_update, gnt, 128, 0, a, w);
  nb.kernel(k_set_cond, 1, 1, 0, hn, static_cast<const int*>(w.counters + 1));
  if (nb.err != cudaSuccess) return nb.err;

  GraphBuilder lb{ls_body, {}};
  lb.memset0(w.counters, sizeof(int));
  lb.kernel(trial_kernel<T>(a), gi, 128, 0, a, w);
  lb.kernel(k_ls_reduce, gnw, 128, 0, a, w, 1);
  lb.kernel(k_set_cond, 1, 1, 0, hl, static_cast<const int*>(w.counters));
  if (lb.err != cudaSuccess) return lb.err;
  *out = root;
  return cudaSuccess;
}

// Persistent form as a graph: queue reset, init, persistent kernel, outputs.
template <typename T>
static cudaError_t build_persistent_graph(const SolveArgs& a, const Workspace& w, unsigned grid, int smem,
                                          double* lambda0, double* u0, double* V, int32_t* status,
                                          int32_t* iters, double* Yout, cudaGraph_t* out) {
  const int64_t P = npts(a.Nmax);
  cudaGraph_t root;
  cudaError_t e = cudaGraphCreate(&root, 0);
  if (e != cudaSuccess) return e;
  GraphBuilder rb{root, {}};
  rb.memset0(w.counters, 4 * sizeof(int));
  rb.kernel(k_init, static_cast<unsigned>(ceil_div(a.n * P * kInitPer, 128)), 128, 0, a, w);
  rb.kernel(k_newton_persistent<T>, grid, 128, static_cast<size_t>(smem), a, w);
  rb.kernel(k_outputs, static_cast<unsigned>(ceil_div(a.n * 32, 128)), 128, 0, a, w, lambda0, u0, V, status, iters);
  if (Yout) rb.kernel(k_copy_Y, static_cast<unsigned>(ceil_div(a.n * P, 128)), 128, 0, a, w, Yout);
  if (rb.err != cudaSuccess) return rb.err;
  *out = root;
  return cudaSuccess;
}

struct GraphKey {
  std::string bytes;
  bool operator<(const GraphKey& o) const { return bytes < o.bytes; }
};

// An instantiated solve graph shared between the cache and the callers that
// launch it: the executable is destroyed when the last holder lets go, so an
// entry evicted by one host thread stays valid for another thread that has
// already looked it up and is launching it on its own stream.
// The graph forms return without waiting for their graphs, so an executable
// may still be running when its last reference goes (an entry evicted from
// the cache): the device is synchronised before it is destroyed.
struct GraphExec {
  cudaGraphExec_t exec = nullptr;
  ~GraphExec() {
    if (exec) {
      cudaDeviceSynchronize();
      cudaGraphExecDestroy(exec);
    }
  }
};
using GraphExecPtr = std::shared_ptr<GraphExec>;

static std::mutex g_graph_mu;
static std::map<GraphKey, GraphExecPtr>& graph_cache() {
  static auto* m = new std::map<GraphKey, GraphExecPtr>();
  return *m;
}
static std::vector<GraphKey>& graph_order() {   // insertion order, for eviction
  static auto* v = new std::vector<GraphKey>();
  return *v;
}
constexpr size_t kGraphCacheCap = 32;

// Looks up (or builds and caches) the solve graph of these arguments and
// launches it on `st` without waiting; *held keeps the executable alive until
// the caller has synchronised `st`.
template <typename T>
static int launch_solve_graph(const SolveArgs& a, Workspace w, cudaStream_t st, double* lambda0, double* u0,
                              double* V, int32_t* status, int32_t* iters, double* Yout, GraphExecPtr* held_out) {
  int dev = 0;
  SG_CUDA_TRY(cudaGetDevice(&dev));
  unsigned grid = 0;
  int smem = 0;
  if (a.persistent) {
    smem = 4 * persist_smem_per_warp<T>();
    SG_CUDA_TRY(ensure_dynamic_smem(k_newton_persistent<T>, smem));
    int sms = 0, per_sm = 0;
    SG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_newton_persistent<T>, 128, smem));
    if (per_sm < 1) per_sm = 1;
    if (a.blocks_per_sm > 0 && a.blocks_per_sm < per_sm) per_sm = a.blocks_per_sm;
    const int64_t want = ceil_div(a.n, 4);
    grid = static_cast<unsigned>(want < int64_t(sms) * per_sm ? want : int64_t(sms) * per_sm);
  } else if constexpr (sizeof(T) == sizeof(double)) {
    SG_CUDA_TRY(ensure_dynamic_smem(k_condense_smem, static_cast<int>(sizeof(double) * kCondWarps * 36 * kCols)));
  }
  // key: every byte that is baked into the graph's kernel parameters
  GraphKey key;
  key.bytes.append(reinterpret_cast<const char*>(&a), sizeof(a));
  key.bytes.append(reinterpret_cast<const char*>(&w), sizeof(w));
  const void* outs[6] = {lambda0, u0, V, status, iters, Yout};
  key.bytes.append(reinterpret_cast<const char*>(outs), sizeof(outs));
  key.bytes.append(reinterpret_cast<const char*>(&dev), sizeof(dev));
  key.bytes.append(reinterpret_cast<const char*>(&grid), sizeof(grid));
  const int tsz = sizeof(T);
  key.bytes.append(reinterpret_cast<const char*>(&tsz), sizeof(tsz));
  GraphExecPtr held;   // keeps the executable alive until this solve has synchronised
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = graph_cache().find(key);
    if (it != graph_cache().end()) held = it->second;
  }
  if (!held) {
    cudaGraph_t g = nullptr;
    cudaError_t e = a.persistent
                        ? build_persistent_graph<T>(a, w, grid, smem, lambda0, u0, V, status, iters, Yout, &g)
                        : build_solve_graph<T>(a, w, lambda0, u0, V, status, iters, Yout, &g);
    if (e != cudaSuccess) return cuda_fail(e, "sg_solve_bvps: building the solve graph");
    held = std::make_shared<GraphExec>();
    e = cudaGraphInstantiate(&held->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      held->exec = nullptr;
      return cuda_fail(e, "sg_solve_bvps: instantiating the solve graph");
    }
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = graph_cache().find(key);
    if (it != graph_cache().end()) {
      held = it->second;   // another thread instantiated the same graph first
    } else {
      if (graph_cache().size() >= kGraphCacheCap) {
        // drop the oldest entry; a thread still launching it holds its own reference
        const GraphKey old = graph_order().front();
        graph_order().erase(graph_order().begin());
        graph_cache().erase(old);
      }
      graph_cache()[key] = held;
      graph_order().push_back(key);
    }
  }
  {
    KernelTimer kt(a.persistent ? kname<T>("graph_persistent") : kname<T>("graph_solve"), st);
    SG_CUDA_TRY(cudaGraphLaunch(held->exec, st));
  }
  *held_out = held;
  return SG_OK;
}

template <typename T>
static int run_solve_graph(const SolveArgs& a, Workspace w, cudaStream_t st, double* lambda0, double* u0,
                           double* V, int32_t* status, int32_t* iters, double* Yout) {
  GraphExecPtr held;   // the cache keeps the executable (see GraphExec)
  return launch_solve_graph<T>(a, w, st, lambda0, u0, V, status, iters, Yout, &held);
}

// ---------------------------------------------------------------- a graph per mesh size
// The batch split by mesh size: the nodes of each N are gathered into a
// contiguous sub-batch with its own workspace laid out for that N, solved by
// its own cached graph on its own stream (the sub-batches run concurrently),
// and the outputs are scattered back.  Each node's arithmetic is the same as
// in the one-graph form.
__global__ void k_group_gather(const double* x0, const double* T, const int32_t* N, const int64_t* idx, int64_t m,
                               double* gx0, double* gT, int32_t* gN) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= m) return;
  const int64_t i = idx[j];
  for (int c = 0; c < 6; ++c) gx0[j * 6 + c] = x0[i * 6 + c];
  gT[j] = T[i];
  gN[j] = N[i];
}

__global__ void k_group_scatter(const int64_t* idx, int64_t m, const double* glam, const double* gu,
                                const double* gV, const int32_t* gst, const int32_t* git, double* lambda0,
                                double* u0, double* V, int32_t* status, int32_t* iters) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= m) return;
  const int64_t i = idx[j];
  for (int c = 0; c < 6; ++c) lambda0[i * 6 + c] = glam[j * 6 + c];
  for (int c = 0; c < 3; ++c) u0[i * 3 + c] = gu[j * 3 + c];
  V[i] = gV[j];
  status[i] = gst[j];
  iters[i] = git[j];
}

constexpr int kMaxMeshGroups = 8;

struct MeshStreams {
  cudaStream_t s[kMaxMeshGroups] = {};
  cudaEvent_t fork = nullptr, join[kMaxMeshGroups] = {};
  bool ok = false;
};

// Streams and events of the per-mesh-size form, made once per device and kept.
static MeshStreams* mesh_streams(int dev) {
  static std::mutex mu;
  static MeshStreams* per_dev[64] = {};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!per_dev[dev]) {
    auto* m = new MeshStreams();
    bool ok = cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kMaxMeshGroups && ok; ++k)
      ok = cudaStreamCreateWithFlags(&m->s[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&m->join[k], cudaEventDisableTiming) == cudaSuccess;
    m->ok = ok;
    per_dev[dev] = m;
  }
  return per_dev[dev]->ok ? per_dev[dev] : nullptr;
}

// Returns SG_OK with *ran = false when the split does not apply (one mesh
// size, more than kMaxMeshGroups sizes, a requested iterate, or a workspace
// too small for the groups' layouts); the caller then runs the one-graph form.
template <typename T>
static int run_solve_mesh_groups(const SolveArgs& a, void* work, size_t work_bytes, cudaStream_t st,
                                 double* lambda0, double* u0, double* V, int32_t* status, int32_t* iters,
                                 bool* ran) {
  *ran = false;
  if (a.Yin || a.persistent) return SG_OK;
  std::vector<int32_t> Nh(a.n);
  SG_CUDA_TRY(cudaMemcpyAsync(Nh.data(), a.N, a.n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SG_CUDA_TRY(cudaStreamSynchronize(st));
  // mesh size -> nodes, largest mesh first (the longest solves start first);
  // nodes with an invalid size go with n_max (their solve reports SG_BADINPUT)
  std::map<int32_t, std::vector<int64_t>, std::greater<int32_t>> groups;
  for (int64_t i = 0; i < a.n; ++i) {
    const int32_t Ni = (Nh[i] >= 1 && Nh[i] <= a.Nmax) ? Nh[i] : a.Nmax;
    groups[Ni].push_back(i);
  }
  if (groups.size() < 2 || groups.size() > size_t(kMaxMeshGroups)) return SG_OK;
  // layout: per node the index, the gathered inputs and the group outputs; then each group's workspace
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_idx = take(a.n * sizeof(int64_t)), o_x0 = take(a.n * 6 * sizeof(double)),
               o_T = take(a.n * sizeof(double)), o_N = take(a.n * sizeof(int32_t)),
               o_lam = take(a.n * 6 * sizeof(double)), o_u = take(a.n * 3 * sizeof(double)),
               o_V = take(a.n * sizeof(double)), o_st = take(a.n * sizeof(int32_t)),
               o_it = take(a.n * sizeof(int32_t));
  std::vector<size_t> o_ws;
  for (auto& g : groups) o_ws.push_back(take(carve(nullptr, int64_t(g.second.size()), g.first, sizeof(T)).bytes));
  if (off > work_bytes) return SG_OK;
  int dev = 0;
  SG_CUDA_TRY(cudaGetDevice(&dev));
  MeshStreams* ms = mesh_streams(dev);
  if (!ms) return SG_OK;
  char* base = static_cast<char*>(work);
  auto* idx = reinterpret_cast<int64_t*>(base + o_idx);
  std::vector<int64_t> order;
  order.reserve(a.n);
  for (auto& g : groups) order.insert(order.end(), g.second.begin(), g.second.end());
  SG_CUDA_TRY(cudaMemcpyAsync(idx, order.data(), a.n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  auto* gx0 = reinterpret_cast<double*>(base + o_x0);
  auto* gT = reinterpret_cast<double*>(base + o_T);
  auto* gN = reinterpret_cast<int32_t*>(base + o_N);
  auto* glam = reinterpret_cast<double*>(base + o_lam);
  auto* gu = reinterpret_cast<double*>(base + o_u);
  auto* gV = reinterpret_cast<double*>(base + o_V);
  auto* gst = reinterpret_cast<int32_t*>(base + o_st);
  auto* git = reinterpret_cast<int32_t*>(base + o_it);
  const unsigned gb = static_cast<unsigned>(ceil_div(a.n, 128));
  SG_TIMED("k_group_gather", st, (k_group_gather<<<gb, 128, 0, st>>>(a.x0, a.T, a.N, idx, a.n, gx0, gT, gN)));
  SG_LAUNCH_CHECK("k_group_gather");
  SG_CUDA_TRY(cudaEventRecord(ms->fork, st));
  std::vector<GraphExecPtr> held(groups.size());
  int64_t start = 0;
  int k = 0;
  for (auto& g : groups) {
    const int64_t m = int64_t(g.second.size());
    SolveArgs ag = a;
    ag.x0 = gx0 + start * 6;
    ag.T = gT + start;
    ag.N = gN + start;
    ag.n = m;
    ag.Nmax = g.first;
    Workspace wg = carve(base + o_ws[k], m, g.first, sizeof(T));
    cudaStream_t sk = ms->s[k];
    SG_CUDA_TRY(cudaStreamWaitEvent(sk, ms->fork, 0));
    const int rc = launch_solve_graph<T>(ag, wg, sk, glam + start * 6, gu + start * 3, gV + start, gst + start,
                                         git + start, nullptr, &held[k]);
    if (rc != SG_OK) return rc;
    SG_CUDA_TRY(cudaEventRecord(ms->join[k], sk));
    SG_CUDA_TRY(cudaStreamWaitEvent(st, ms->join[k], 0));
    start += m;
    ++k;
  }
  SG_TIMED("k_group_scatter", st,
           (k_group_scatter<<<gb, 128, 0, st>>>(idx, a.n, glam, gu, gV, gst, git, lambda0, u0, V, status, iters)));
  SG_LAUNCH_CHECK("k_group_scatter");
  *ran = true;   // queued on st (which waits for every sub-batch); not waited for here
  return SG_OK;
}

}  // namespace sg

using namespace sg;

extern "C" size_t sg_solve_workspace_bytes(int64_t n, int n_max_intervals, int precision) {
  if (n < 0 || n_max_intervals < 1) return 0;
  if (precision != SG_PREC_FP64 && !fp32_direction(precision)) return 0;
  return ws_bytes(n, n_max_intervals, precision);
}

extern "C" int sg_solve_bvps(const sg_problem* prob, const double* d_x0, int64_t n, const double* d_T,
                             const int32_t* d_N, int n_max_intervals, const sg_solve_opts* opts,
                             void* d_work, size_t work_bytes, double* d_lambda0, double* d_u0,
                             double* d_V, int32_t* d_status, int32_t* d_iters, double* d_Y,
                             void* stream) {
  clear_error();
  if (!prob) return fail(SG_EINVAL, "sg_solve_bvps: null problem");
  if (n < 0) return fail(SG_EINVAL, "sg_solve_bvps: n < 0");
  if (n == 0) return SG_OK;
  if (n_max_intervals < 1 || n_max_intervals > (1 << 16))
    return fail(SG_EINVAL, "sg_solve_bvps: n_max_intervals must be 1..65536");
  if (!d_x0 || !d_T || !d_N || !d_work || !d_lambda0 || !d_u0 || !d_V || !d_status || !d_iters)
    return fail(SG_EINVAL, "sg_solve_bvps: null device pointer");
  sg_solve_opts o{1e-8, 50, SG_PREC_FP64, 1, 0, 0, 0, 0, 0};
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iter < 0) return fail(SG_EINVAL, "sg_solve_bvps: bad tol or max_iter");
  if (o.warm_start && !d_Y) return fail(SG_EINVAL, "sg_solve_bvps: warm_start needs d_Y");
  if (o.precision != SG_PREC_FP64 && !fp32_direction(o.precision))
    return fail(SG_EINVAL, "sg_solve_bvps: unknown precision");
  if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0)
    return fail(SG_EINVAL, "sg_solve_bvps: workspace must be 256-byte aligned");
  const size_t need = ws_bytes(n, n_max_intervals, o.precision);
  if (work_bytes < need)
    return fail(SG_EINVAL, "sg_solve_bvps: workspace too small (need " + std::to_string(need) + " bytes)");
  SolveArgs a{};
  if (!make_dev_problem(*prob, &a.P)) return fail(SG_EINVAL, "sg_solve_bvps: invalid problem parameters");
  a.x0 = d_x0;
  a.T = d_T;
  a.N = d_N;
  a.n = n;
  a.Nmax = n_max_intervals;
  a.tol = o.tol;
  a.max_iter = o.max_iter;
  a.damping = o.damping;
  a.persistent = o.persistent;
  a.blocks_per_sm = o.blocks_per_sm;
  a.cond_warps = o.cond_warps;
  a.sync_at_end = 1;
  a.Yin = o.warm_start ? d_Y : nullptr;
  a.res_pair = o.precision == SG_PREC_MIXED_PAIR ? 1 : 0;
  // the FP32 Jacobian from the FP64 residual kernel (its FP32 pipe is idle
  // beside the FP64 work) in the launch-per-phase and graph forms
  a.jac_in_trial = fp32_direction(o.precision) && !a.res_pair && !o.persistent ? 1 : 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.graph == 2 && !d_Y) {
    bool ran = false;
    const int rc = fp32_direction(o.precision)
                       ? run_solve_mesh_groups<float>(a, d_work, work_bytes, st, d_lambda0, d_u0, d_V, d_status,
                                                      d_iters, &ran)
                       : run_solve_mesh_groups<double>(a, d_work, work_bytes, st, d_lambda0, d_u0, d_V, d_status,
                                                       d_iters, &ran);
    if (rc != SG_OK || ran) return rc;
  }
  if (fp32_direction(o.precision)) {
    Workspace w = carve(d_work, n, n_max_intervals, sizeof(float));
    if (o.graph) return run_solve_graph<float>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
    return run_solve<float>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
  }
  Workspace w = carve(d_work, n, n_max_intervals, sizeof(double));
  if (o.graph) return run_solve_graph<double>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
  return run_solve<double>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
}

// ---------------------------------------------------------------- no-allocation variant
// sg_solve_bvps_static: the same solve with its workspace in a fixed array
// compiled into this library, for callers that cannot allocate device memory
// when they solve (see include/sg.h).  Nothing here calls cudaMalloc/cudaFree.
namespace sg {

static __device__ __align__(256) unsigned char g_static_scratch[SG_STATIC_SCRATCH_BYTES];

constexpr int kMaxStaticDevices = 64;
static std::mutex g_static_mu;
static void* g_static_ptr[kMaxStaticDevices] = {nullptr};

// Device address of g_static_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.  The cache assumes the
// device's context lives as long as the library: after cudaDeviceReset the
// cached address is stale.
static int static_scratch_address(void** out) {
  int dev = -1;
  SG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxStaticDevices)
    return fail(SG_EUNSUPPORTED, "sg_solve_bvps_static: device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "sg_solve_bvps_static: cudaGetSymbolAddress");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SG_OK;
}

}  // namespace sg

extern "C" int sg_solve_bvps_static(const sg_problem* prob, const double* d_x0, int64_t n, const double* d_T,
                                    const int32_t* d_N, int n_max_intervals, const sg_solve_opts* opts,
                                    double* d_lambda0, double* d_u0, double* d_V, int32_t* d_status,
                                    int32_t* d_iters, double* d_Y, void* stream) {
  clear_error();
  if (!prob) return fail(SG_EINVAL, "sg_solve_bvps_static: null problem");
  if (n < 0) return fail(SG_EINVAL, "sg_solve_bvps_static: n < 0");
  if (n == 0) return SG_OK;
  if (n_max_intervals < 1 || n_max_intervals > (1 << 16))
    return fail(SG_EINVAL, "sg_solve_bvps_static: n_max_intervals must be 1..65536");
  if (!d_x0 || !d_T || !d_N || !d_lambda0 || !d_u0 || !d_V || !d_status || !d_iters)
    return fail(SG_EINVAL, "sg_solve_bvps_static: null device pointer");
  sg_solve_opts o{1e-8, 50, SG_PREC_FP64, 1, 0, 0, 0, 0, 0};
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iter < 0) return fail(SG_EINVAL, "sg_solve_bvps_static: bad tol or max_iter");
  if (o.warm_start && !d_Y) return fail(SG_EINVAL, "sg_solve_bvps_static: warm_start needs d_Y");
  if (o.precision != SG_PREC_FP64 && !fp32_direction(o.precision))
    return fail(SG_EINVAL, "sg_solve_bvps_static: unknown precision");
  if (o.graph)
    return fail(SG_EINVAL,
                "sg_solve_bvps_static: opts->graph must be 0 (the graph form instantiates CUDA graphs, "
                "which allocate memory)");
  const size_t need = ws_bytes(n, n_max_intervals, o.precision);
  if (need > SG_STATIC_SCRATCH_BYTES)
    return fail(SG_EINVAL, "sg_solve_bvps_static: this batch needs " + std::to_string(need) +
                               " bytes of scratch but the static array holds " +
                               std::to_string(size_t(SG_STATIC_SCRATCH_BYTES)) +
                               "; solve fewer nodes per call, or use sg_solve_bvps with a caller workspace");
  SolveArgs a{};
  if (!make_dev_problem(*prob, &a.P)) return fail(SG_EINVAL, "sg_solve_bvps_static: invalid problem parameters");
  void* scratch = nullptr;
  int rc = static_scratch_address(&scratch);
  if (rc != SG_OK) return rc;
  a.x0 = d_x0;
  a.T = d_T;
  a.N = d_N;
  a.n = n;
  a.Nmax = n_max_intervals;
  a.tol = o.tol;
  a.max_iter = o.max_iter;
  a.damping = o.damping;
  a.persistent = o.persistent;
  a.blocks_per_sm = o.blocks_per_sm;
  a.cond_warps = o.cond_warps;
  a.sync_at_end = 1;
  a.Yin = o.warm_start ? d_Y : nullptr;
  a.res_pair = o.precision == SG_PREC_MIXED_PAIR ? 1 : 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Every region the solver reads is written first in this call (k_init sets the
  // iterate, the corrections and the per-node state; the counters are zeroed
  // before each use), so the previous call's contents need no clearing here.
  if (fp32_direction(o.precision)) {
    Workspace w = carve(scratch, n, n_max_intervals, sizeof(float));
    return run_solve<float>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
  }
  Workspace w = carve(scratch, n, n_max_intervals, sizeof(double));
  return run_solve<double>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
}

// ---------------------------------------------------------------- resident solver pool
// sg_pool_*: a fixed set of node slots whose Newton state stays on the device.
// Solves are admitted into free slots between iterations and leave when they
// end, so work that arrives while others are iterating joins the batch at the
// next iteration (continuous batching at Newton-iteration granularity).  One
// iteration of the pool is one CUDA graph replay: the initial residual of the
// slots admitted since the last iteration, then one damped Newton step of
// every slot in progress, with the line search as a device-side WHILE loop.
// Every kernel works per node and skips slots that are free or finished, so a
// slot's arithmetic is that of the same node in sg_solve_bvps.
namespace sg {

enum : uint8_t { kSlotFree = 0, kSlotBusy = 1, kSlotDone = 2 };

struct sg_pool_impl {
  SolveArgs a{};
  Workspace w{};
  bool fp32 = false;
  int64_t slots = 0;
  // iteration graphs per tier: tier k covers slots [0, tier_size[k]) (64, 128,
  // ..., doubling, then all slots), built when first needed, so that an
  // iteration's grids span the occupied slots rather than the whole pool
  std::vector<int64_t> tier_size;
  std::vector<cudaGraphExec_t> tier_exec;
  int64_t* d_list = nullptr;           // slot list of an admit / collect (slots entries)
  uint8_t* d_flags = nullptr;          // per-slot "still iterating" (written after an iteration)
  int64_t* h_list = nullptr;           // pinned staging of d_list
  uint8_t* h_flags = nullptr;          // pinned copy of d_flags
  std::vector<uint8_t> state;          // host: free / in progress / ended, not collected
  std::set<int64_t> free_set;          // free slots; admission takes the lowest
  int64_t n_busy = 0;
  std::mutex mu;
};

// The pool's inputs (x0, T, N per slot) and its list and flag arrays sit in
// front of the solver workspace.
struct PoolLayout {
  size_t x0, T, N, list, flags, ws, total;
};
static PoolLayout pool_layout(int64_t slots, int Nmax, int precision) {
  PoolLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.x0 = take(slots * 6 * sizeof(double));
  L.T = take(slots * sizeof(double));
  L.N = take(slots * sizeof(int32_t));
  L.list = take(slots * sizeof(int64_t));
  L.flags = take(slots);
  L.ws = off;
  L.total = off + ws_bytes(slots, Nmax, precision);
  return L;
}

// Copies entry j of the caller's inputs into slot list[j].
__global__ void k_pool_put(SolveArgs a, const int64_t* list, int64_t count, const double* x0, const double* T,
                           const int32_t* N) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= count) return;
  const int64_t s = list[j];
  double* px0 = const_cast<double*>(a.x0) + s * 6;
  for (int c = 0; c < 6; ++c) px0[c] = x0[j * 6 + c];
  const_cast<double*>(a.T)[s] = T[j];
  const_cast<int32_t*>(a.N)[s] = N[j];
}

// k_init for the slots of `list` (zero-control guess, fresh node state).
__global__ void k_pool_init(SolveArgs a, Workspace w, const int64_t* list, int64_t count) {
  const int64_t P = npts(a.Nmax);
  const int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (u >= count * P * kInitPer) return;
  const int64_t t = u / kInitPer;
  const int64_t node = list[t / P];
  const int64_t p = t % P;
  const int q = static_cast<int>(u % kInitPer);
  init_pair(a, w, node, p, q, (node * P + p) * kInitPer + q);
}

__global__ void k_pool_flags(SolveArgs a, Workspace w, uint8_t* flags) {
  const int64_t node = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (node >= a.n) return;
  flags[node] = w.ns[node].active ? 1 : 0;
}

__global__ void k_pool_outputs(SolveArgs a, Workspace w, const int64_t* list, int64_t count, double* lambda0,
                               double* u0, double* V, int32_t* status, int32_t* iters) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (j >= count) return;
  node_outputs(a, w, list[j], j, lane, lambda0, u0, V, status, iters);
}

// Marks the slots of `list` free for the solver kernels (inactive, not searching).
__global__ void k_pool_release(Workspace w, const int64_t* list, int64_t count) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= count) return;
  NodeState s{};
  s.status = SG_BADINPUT;
  w.ns[list[j]] = s;
}

// One pool iteration as a graph: the initial residual of new slots, then one
// Newton step of every active slot (the body of the Newton loop of
// build_solve_graph, run once).
template <typename T>
static cudaError_t build_pool_graph(const SolveArgs& a, const Workspace& w, uint8_t* flags, cudaGraph_t* out) {
  const int64_t P = npts(a.Nmax);
  const int64_t nint = a.n * a.Nmax;
  const unsigned gp = static_cast<unsigned>(ceil_div(a.n * P, 128));
  const unsigned gi = static_cast<unsigned>(a.n * trial_chunks(a.Nmax));
  const unsigned gnt = static_cast<unsigned>(ceil_div(a.n, 128));
  const unsigned gnw = static_cast<unsigned>(ceil_div(a.n * 32, 128));
  const unsigned gwi = static_cast<unsigned>(ceil_div(nint, 4));
  const unsigned gwn = static_cast<unsigned>(ceil_div(a.n, 4));
  const unsigned gws = static_cast<unsigned>(ceil_div(a.n * seg_count(a.Nmax), 4));
  const size_t cond_smem = sizeof(double) * kCondWarps * 36 * kCols;
  cudaGraph_t root;
  cudaError_t e = cudaGraphCreate(&root, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle hl;
  if ((e = cudaGraphConditionalHandleCreate(&hl, root, 0, 0)) != cudaSuccess) return e;
  GraphBuilder rb{root, {}};
  rb.memset0(w.counters, 4 * sizeof(int));
  rb.kernel(trial_kernel<T>(a), gi, 128, 0, a, w);     // new slots only (searching at alpha = 0)
  rb.kernel(k_ls_reduce, gnw, 128, 0, a, w, 0);
  rb.memset0(w.counters, 2 * sizeof(int));
  rb.kernel(k_point<T>, gp, 128, 0, a, w);
  if constexpr (sizeof(T) == sizeof(float)) {
    const int cw = condense_reg_warps(a.cond_warps);
    rb.kernel(condense_reg_kernel(cw), static_cast<unsigned>(ceil_div(nint, cw)), 32 * cw, 0, a, w);
  } else {
    rb.kernel(k_condense_smem, static_cast<unsigned>(ceil_div(nint, kCondWarps)), 32 * kCondWarps, cond_smem, a, w);
  }
  rb.kernel(k_abd_seg<T>, static_cast<unsigned>(ceil_div(a.n * seg_count(a.Nmax), seg_warps<T>())),
            32 * seg_warps<T>(), 0, a, w);
  rb.kernel(k_abd_red<T>, gwn, 128, 0, a, w);
  rb.kernel(k_abd_segback<T>, gws, 128, 0, a, w);
  rb.kernel(k_recover<T>, gwi, 128, 0, a, w);
  rb.kernel(k_ls_begin, gnt, 128, 0, a, w);
  rb.kernel(k_set_cond_one, 1, 1, 0, hl);
  cudaGraph_t ls_body;
  rb.loop(hl, &ls_body);
  rb.memset0(w.counters, 2 * sizeof(int));
  rb.kernel(k_update, static_cast<unsigned>(ceil_div(a.n * P * kUpdPer, 128)), 128, 0, a, w);
  rb.kernel(k_after_update, gnt, 128, 0, a, w);
  rb.kernel(k_pool_flags, gnt, 128, 0, a, w, flags);
  if (rb.err != cudaSuccess) return rb.err;
  GraphBuilder lb{ls_body, {}};
  lb.memset0(w.counters, sizeof(int));
  lb.kernel(trial_kernel<T>(a), gi, 128, 0, a, w);
  lb.kernel(k_ls_reduce, gnw, 128, 0, a, w, 1);
  lb.kernel(k_set_cond, 1, 1, 0, hl, static_cast<const int*>(w.counters));
  if (lb.err != cudaSuccess) return lb.err;
  *out = root;
  return cudaSuccess;
}

static void pool_release_host(sg_pool_impl* p) {
  for (auto e : p->tier_exec)
    if (e) cudaGraphExecDestroy(e);
  if (p->h_list) cudaFreeHost(p->h_list);
  if (p->h_flags) cudaFreeHost(p->h_flags);
  delete p;
}

}  // namespace sg

struct sg_pool {
  sg::sg_pool_impl* impl;
};

extern "C" size_t sg_pool_workspace_bytes(int64_t slots, int n_max_intervals, int precision) {
  if (slots < 1 || n_max_intervals < 1) return 0;
  if (precision != SG_PREC_FP64 && !fp32_direction(precision)) return 0;
  return pool_layout(slots, n_max_intervals, precision).total;
}

extern "C" int sg_pool_create(const sg_problem* prob, int64_t slots, int n_max_intervals, const sg_solve_opts* opts,
                              void* d_work, size_t work_bytes, sg_pool** out, void* stream) {
  clear_error();
  if (!prob || !out || !d_work) return fail(SG_EINVAL, "sg_pool_create: null argument");
  *out = nullptr;
  if (slots < 1 || slots > (int64_t(1) << 26)) return fail(SG_EINVAL, "sg_pool_create: slots must be 1..2^26");
  if (n_max_intervals < 1 || n_max_intervals > (1 << 16))
    return fail(SG_EINVAL, "sg_pool_create: n_max_intervals must be 1..65536");
  sg_solve_opts o{1e-8, 50, SG_PREC_FP64, 1, 0, 0, 0, 0, 0};
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iter < 0) return fail(SG_EINVAL, "sg_pool_create: bad tol or max_iter");
  if (o.precision != SG_PREC_FP64 && !fp32_direction(o.precision))
    return fail(SG_EINVAL, "sg_pool_create: unknown precision");
  if (o.warm_start) return fail(SG_EINVAL, "sg_pool_create: warm_start is not available in a pool");
  if (prob->kind == SG_PROBLEM_ATTITUDE && prob->d_target)
    return fail(SG_EINVAL, "sg_pool_create: per-node target attitudes are not supported in a pool");
  if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0)
    return fail(SG_EINVAL, "sg_pool_create: workspace must be 256-byte aligned");
  const PoolLayout L = pool_layout(slots, n_max_intervals, o.precision);
  if (work_bytes < L.total)
    return fail(SG_EINVAL, "sg_pool_create: workspace too small (need " + std::to_string(L.total) + " bytes)");
  auto* p = new sg_pool_impl();
  char* base = static_cast<char*>(d_work);
  if (!make_dev_problem(*prob, &p->a.P)) {
    delete p;
    return fail(SG_EINVAL, "sg_pool_create: invalid problem parameters");
  }
  p->a.x0 = reinterpret_cast<const double*>(base + L.x0);
  p->a.T = reinterpret_cast<const double*>(base + L.T);
  p->a.N = reinterpret_cast<const int32_t*>(base + L.N);
  p->a.n = slots;
  p->a.Nmax = n_max_intervals;
  p->a.tol = o.tol;
  p->a.max_iter = o.max_iter;
  p->a.damping = o.damping;
  p->a.cond_warps = o.cond_warps;
  p->a.sync_at_end = 1;
  p->a.res_pair = o.precision == SG_PREC_MIXED_PAIR ? 1 : 0;
  p->fp32 = fp32_direction(o.precision);
  p->w = carve(base + L.ws, slots, n_max_intervals, p->fp32 ? sizeof(float) : sizeof(double));
  p->d_list = reinterpret_cast<int64_t*>(base + L.list);
  p->d_flags = reinterpret_cast<uint8_t*>(base + L.flags);
  p->slots = slots;
  p->state.assign(slots, kSlotFree);
  for (int64_t s = 0; s < slots; ++s) p->free_set.insert(p->free_set.end(), s);
  for (int64_t t = 64; t < slots; t *= 2) p->tier_size.push_back(t);
  p->tier_size.push_back(slots);
  p->tier_exec.assign(p->tier_size.size(), nullptr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto bail = [&](cudaError_t e, const char* where) {
    pool_release_host(p);
    return cuda_fail(e, where);
  };
  cudaError_t e;
  if ((e = cudaHostAlloc(reinterpret_cast<void**>(&p->h_list), slots * sizeof(int64_t), cudaHostAllocDefault)) !=
      cudaSuccess)
    return bail(e, "sg_pool_create: pinned list");
  if ((e = cudaHostAlloc(reinterpret_cast<void**>(&p->h_flags), slots, cudaHostAllocDefault)) != cudaSuccess)
    return bail(e, "sg_pool_create: pinned flags");
  // every slot starts free: node state zero (inactive, not searching), inputs
  // of a valid empty node so that no kernel reads garbage
  if ((e = cudaMemsetAsync(p->w.ns, 0, slots * sizeof(NodeState), st)) != cudaSuccess)
    return bail(e, "sg_pool_create: clearing the node states");
  if ((e = cudaMemsetAsync(base + L.x0, 0, L.ws - L.x0, st)) != cudaSuccess)
    return bail(e, "sg_pool_create: clearing the inputs");
  if (!p->fp32) {
    if ((e = ensure_dynamic_smem(k_condense_smem, static_cast<int>(sizeof(double) * kCondWarps * 36 * kCols))) != cudaSuccess)
      return bail(e, "sg_pool_create: condensation shared memory");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "sg_pool_create");
  *out = new sg_pool{p};
  return SG_OK;
}

extern "C" void sg_pool_free(sg_pool* pool) {
  if (!pool) return;
  pool_release_host(pool->impl);
  delete pool;
}

extern "C" int sg_pool_info(const sg_pool* pool, int64_t* n_free, int64_t* n_busy) {
  clear_error();
  if (!pool) return fail(SG_EINVAL, "sg_pool_info: null pool");
  sg_pool_impl* p = pool->impl;
  std::lock_guard<std::mutex> lk(p->mu);
  if (n_free) *n_free = static_cast<int64_t>(p->free_set.size());
  if (n_busy) *n_busy = p->n_busy;
  return SG_OK;
}

extern "C" int sg_pool_admit(sg_pool* pool, const double* d_x0, const double* d_T, const int32_t* d_N, int64_t count,
                             int64_t* slots_out, void* stream) {
  clear_error();
  if (!pool || !slots_out) return fail(SG_EINVAL, "sg_pool_admit: null argument");
  if (count < 0) return fail(SG_EINVAL, "sg_pool_admit: count < 0");
  if (count == 0) return SG_OK;
  if (!d_x0 || !d_T || !d_N) return fail(SG_EINVAL, "sg_pool_admit: null device pointer");
  sg_pool_impl* p = pool->impl;
  std::lock_guard<std::mutex> lk(p->mu);
  if (count > static_cast<int64_t>(p->free_set.size()))
    return fail(SG_EFULL, "sg_pool_admit: " + std::to_string(count) + " slots asked, " +
                              std::to_string(p->free_set.size()) + " free");
  for (int64_t j = 0; j < count; ++j) {
    const int64_t s = *p->free_set.begin();
    p->free_set.erase(p->free_set.begin());
    p->state[s] = kSlotBusy;
    p->h_list[j] = s;
    slots_out[j] = s;
  }
  p->n_busy += count;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t P = npts(p->a.Nmax);
  SG_CUDA_TRY(cudaMemcpyAsync(p->d_list, p->h_list, count * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SG_TIMED("k_pool_put", st,
           (k_pool_put<<<static_cast<unsigned>(ceil_div(count, 128)), 128, 0, st>>>(p->a, p->d_list, count, d_x0,
                                                                                     d_T, d_N)));
  SG_TIMED("k_pool_init", st,
           (k_pool_init<<<static_cast<unsigned>(ceil_div(count * P * kInitPer, 128)), 128, 0, st>>>(
               p->a, p->w, p->d_list, count)));
  SG_LAUNCH_CHECK("sg_pool_admit");
  // the pinned list is reused by the next call: let this copy finish first
  SG_CUDA_TRY(cudaStreamSynchronize(st));
  return SG_OK;
}

extern "C" int sg_pool_iterate(sg_pool* pool, int64_t* n_active, void* stream) {
  clear_error();
  if (!pool) return fail(SG_EINVAL, "sg_pool_iterate: null pool");
  sg_pool_impl* p = pool->impl;
  std::lock_guard<std::mutex> lk(p->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p->n_busy > 0) {
    // the smallest tier that holds every slot in progress
    int64_t top = p->slots;
    while (top > 0 && p->state[top - 1] != kSlotBusy) --top;
    size_t k = 0;
    while (p->tier_size[k] < top) ++k;
    if (!p->tier_exec[k]) {
      SolveArgs at = p->a;
      at.n = p->tier_size[k];
      cudaGraph_t g = nullptr;
      cudaError_t e = p->fp32 ? build_pool_graph<float>(at, p->w, p->d_flags, &g)
                              : build_pool_graph<double>(at, p->w, p->d_flags, &g);
      if (e != cudaSuccess) return cuda_fail(e, "sg_pool_iterate: building the iteration graph");
      e = cudaGraphInstantiate(&p->tier_exec[k], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        p->tier_exec[k] = nullptr;
        return cuda_fail(e, "sg_pool_iterate: instantiating the iteration graph");
      }
    }
    const int64_t span = p->tier_size[k];
    {
      KernelTimer kt(p->fp32 ? "graph_pool_iteration_fp32" : "graph_pool_iteration_fp64", st);
      SG_CUDA_TRY(cudaGraphLaunch(p->tier_exec[k], st));
    }
    SG_CUDA_TRY(cudaMemcpyAsync(p->h_flags, p->d_flags, span, cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t s = 0; s < span; ++s)
      if (p->state[s] == kSlotBusy && !p->h_flags[s]) {
        p->state[s] = kSlotDone;
        --p->n_busy;
      }
  }
  if (n_active) *n_active = p->n_busy;
  return SG_OK;
}

extern "C" int sg_pool_finished(sg_pool* pool, int64_t* slots_out, int64_t max_count, int64_t* count) {
  clear_error();
  if (!pool || !count || (max_count > 0 && !slots_out)) return fail(SG_EINVAL, "sg_pool_finished: null argument");
  sg_pool_impl* p = pool->impl;
  std::lock_guard<std::mutex> lk(p->mu);
  int64_t c = 0;
  for (int64_t s = 0; s < p->slots && c < max_count; ++s)
    if (p->state[s] == kSlotDone) slots_out[c++] = s;
  *count = c;
  return SG_OK;
}

extern "C" int sg_pool_collect(sg_pool* pool, const int64_t* slots, int64_t count, double* d_lambda0, double* d_u0,
                               double* d_V, int32_t* d_status, int32_t* d_iters, void* stream) {
  clear_error();
  if (!pool || (count > 0 && !slots)) return fail(SG_EINVAL, "sg_pool_collect: null argument");
  if (count < 0) return fail(SG_EINVAL, "sg_pool_collect: count < 0");
  if (count == 0) return SG_OK;
  if (!d_lambda0 || !d_u0 || !d_V || !d_status || !d_iters)
    return fail(SG_EINVAL, "sg_pool_collect: null device pointer");
  sg_pool_impl* p = pool->impl;
  std::lock_guard<std::mutex> lk(p->mu);
  if (count > p->slots) return fail(SG_EINVAL, "sg_pool_collect: more slots than the pool holds");
  for (int64_t j = 0; j < count; ++j) {
    const int64_t s = slots[j];
    if (s < 0 || s >= p->slots || p->state[s] != kSlotDone)
      return fail(SG_EINVAL, "sg_pool_collect: slot " + std::to_string(s) + " has no finished solve");
    for (int64_t k = 0; k < j; ++k)
      if (slots[k] == s) return fail(SG_EINVAL, "sg_pool_collect: slot listed twice");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int64_t j = 0; j < count; ++j) p->h_list[j] = slots[j];
  SG_CUDA_TRY(cudaMemcpyAsync(p->d_list, p->h_list, count * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SG_TIMED("k_pool_outputs", st,
           (k_pool_outputs<<<static_cast<unsigned>(ceil_div(count * 32, 128)), 128, 0, st>>>(
               p->a, p->w, p->d_list, count, d_lambda0, d_u0, d_V, d_status, d_iters)));
  SG_TIMED("k_pool_release", st,
           (k_pool_release<<<static_cast<unsigned>(ceil_div(count, 128)), 128, 0, st>>>(p->w, p->d_list, count)));
  SG_LAUNCH_CHECK("sg_pool_collect");
  SG_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t j = 0; j < count; ++j) {
    p->state[slots[j]] = kSlotFree;
    p->free_set.insert(slots[j]);
  }
  return SG_OK;
}
