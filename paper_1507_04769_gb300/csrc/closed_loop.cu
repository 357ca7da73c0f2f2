// Closed-loop simulation with the interpolated feedback (the on-line phase of
// Section 3.3, as simulated with zero-order hold in Section 5): at every
// sampling instant u_k = I^q(u*)(x_k) from the sparse-grid interpolant, held
// over [t_k, t_k + dt] while one classical RK4 step advances the plant and
// the running cost z' = L(x, u_k).
//
// One warp per trajectory.  Per step the warp builds the d 1-D basis tables
// (lane k < d takes dimension k), splits the nodes over its lanes for the
// contraction (FP64, or pairs of floats with a compensated sum), reduces the
// partial controls in a fixed order, and advances the state; all lanes carry
// the same state, so no broadcast is needed.
#include "basis.cuh"
#include "common.cuh"
#include "diag.cuh"
#include "interp.cuh"
#include "problems.cuh"

namespace sg {

constexpr int kClWarps = 4;

struct ClArgs {
  DevProblem P;
  EvalArgs e;         // interpolant data (xq/out/Q unused)
  int d;
  const double* x0;   // ntraj x 6
  int64_t ntraj;
  int nsteps;
  double dt;
  double* xT;         // ntraj x 6
  double* cost;       // ntraj
  double* traj;       // ntraj x (nsteps + 1) x 6, or null
  double* ctrl;       // ntraj x nsteps x 3, or null
};

template <int MODE>
__device__ __forceinline__ void feedback(const ClArgs& c, const double* x, unsigned char* tabraw, int lane,
                                         double* u) {
  const EvalArgs& e = c.e;
  const int nf = e.nf;
  if (lane < c.d) {
    const double uu = (x[lane] - e.lo[lane]) / e.width[lane];
    if constexpr (MODE == SG_EVAL_DF32)
      basis_row_df(uu, e.level, e.xfdf, reinterpret_cast<float2*>(tabraw) + lane * nf, 1);
    else
      basis_row(uu, e.level, e.xf, reinterpret_cast<double*>(tabraw) + lane * nf, 1);
  }
  __syncwarp();
  double part[3] = {0.0, 0.0, 0.0};
  if constexpr (MODE == SG_EVAL_DF32) {
    const float2* tab = reinterpret_cast<const float2*>(tabraw);
    float ah[3] = {0.f, 0.f, 0.f}, al[3] = {0.f, 0.f, 0.f};
    for (int64_t m = lane; m < e.M; m += 32) {
      const uint16_t* o = e.ops + m * kMaxDim;
      df phi = {tab[o[0]].x, tab[o[0]].y};
      for (int j = 1; j < e.amax; ++j) phi = df_mul(phi, {tab[o[j]].x, tab[o[j]].y});
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float2 wc = e.Wdf[m * 3 + q];
        const float p = __fmul_rn(phi.hi, wc.x);
        const float pe = __fmaf_rn(phi.hi, wc.x, -p);
        const float t = __fadd_rn(__fmaf_rn(phi.hi, wc.y, __fmul_rn(phi.lo, wc.x)), pe);
        const float s = __fadd_rn(ah[q], p);
        const float bb = __fsub_rn(s, ah[q]);
        const float se = __fadd_rn(__fsub_rn(ah[q], __fsub_rn(s, bb)), __fsub_rn(p, bb));
        ah[q] = s;
        al[q] = __fadd_rn(al[q], __fadd_rn(se, t));
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) part[q] = static_cast<double>(ah[q]) + static_cast<double>(al[q]);
  } else {
    const double* tab = reinterpret_cast<const double*>(tabraw);
    for (int64_t m = lane; m < e.M; m += 32) {
      const uint16_t* o = e.ops + m * kMaxDim;
      double phi = tab[o[0]];
      for (int j = 1; j < e.amax; ++j) phi *= tab[o[j]];
#pragma unroll
      for (int q = 0; q < 3; ++q) part[q] = fma(phi, e.W[m * 3 + q], part[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double v = part[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    u[q] = v;
  }
  __syncwarp();
}

template <int MODE>
__global__ void __launch_bounds__(32 * kClWarps) k_closed_loop(ClArgs c) {
  extern __shared__ __align__(16) unsigned char cl_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tr = blockIdx.x * int64_t(kClWarps) + warp;
  if (tr >= c.ntraj) return;
  unsigned char* tab = cl_smem + size_t(warp) * c.d * c.e.nf * 8;
  double x[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) x[i] = c.x0[tr * 6 + i];
  double z = 0.0;
  const double dt = c.dt;
  if (c.traj && lane < 6) c.traj[tr * int64_t(c.nsteps + 1) * 6 + lane] = c.x0[tr * 6 + lane];
  for (int k = 0; k < c.nsteps; ++k) {
    double u[3];
    feedback<MODE>(c, x, tab, lane, u);
    // the FP64 plant step runs on lane 0 only (the FP64 pipe is narrow on
    // this part) and the new state is broadcast to the warp
    if (lane == 0) {
      double k1[6], k2[6], k3[6], k4[6], xs[6];
      plant_rhs(c.P, x, u, k1);
      const double l1 = running_cost_xu(c.P, x, u);
#pragma unroll
      for (int i = 0; i < 6; ++i) xs[i] = x[i] + 0.5 * dt * k1[i];
      plant_rhs(c.P, xs, u, k2);
      const double l2 = running_cost_xu(c.P, xs, u);
#pragma unroll
      for (int i = 0; i < 6; ++i) xs[i] = x[i] + 0.5 * dt * k2[i];
      plant_rhs(c.P, xs, u, k3);
      const double l3 = running_cost_xu(c.P, xs, u);
#pragma unroll
      for (int i = 0; i < 6; ++i) xs[i] = x[i] + dt * k3[i];
      plant_rhs(c.P, xs, u, k4);
      const double l4 = running_cost_xu(c.P, xs, u);
#pragma unroll
      for (int i = 0; i < 6; ++i) x[i] = x[i] + (dt / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
      z = z + (dt / 6.0) * (l1 + 2.0 * l2 + 2.0 * l3 + l4);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = __shfl_sync(0xffffffffu, x[i], 0);
    if (c.ctrl && lane < 3) {
      double mine = lane == 0 ? u[0] : (lane == 1 ? u[1] : u[2]);
      c.ctrl[(tr * int64_t(c.nsteps) + k) * 3 + lane] = mine;
    }
    if (c.traj && lane < 6) {
      double mine = 0.0;
#pragma unroll
      for (int i = 0; i < 6; ++i)
        if (i == lane) mine = x[i];
      c.traj[(tr * int64_t(c.nsteps + 1) + k + 1) * 6 + lane] = mine;
    }
  }
  if (lane < 6) {
    double mine = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i == lane) mine = x[i];
    c.xT[tr * 6 + lane] = mine;
  }
  if (lane == 0) c.cost[tr] = z;   // z lives on lane 0
}

}  // namespace sg

using namespace sg;

extern "C" int sg_simulate_closed_loop(const sg_problem* prob, const sg_surplus* s, const double* d_x0,
                                       int64_t ntraj, int nsteps, double dt, int mode, double* d_xT,
                                       double* d_cost, double* d_traj, double* d_ctrl, void* stream) {
  clear_error();
  if (!prob || !s) return fail(SG_EINVAL, "sg_simulate_closed_loop: null problem or surplus");
  if (ntraj < 0 || nsteps < 0 || !(dt > 0.0)) return fail(SG_EINVAL, "sg_simulate_closed_loop: bad sizes or dt");
  if (ntraj == 0) return SG_OK;
  if (!d_x0 || !d_xT || !d_cost) return fail(SG_EINVAL, "sg_simulate_closed_loop: null device pointer");
  if (s->d != 6 || s->k != 3)
    return fail(SG_EINVAL, "sg_simulate_closed_loop: the surplus must interpolate u* (d = 6 states, k = 3 controls)");
  if (mode != SG_EVAL_FP64 && mode != SG_EVAL_DF32)
    return fail(SG_EINVAL, "sg_simulate_closed_loop: mode must be SG_EVAL_FP64 or SG_EVAL_DF32");
  if (prob->kind == SG_PROBLEM_ATTITUDE && prob->d_target)
    return fail(SG_EINVAL, "sg_simulate_closed_loop: per-node target attitudes are not supported");
  ClArgs c{};
  if (!make_dev_problem(*prob, &c.P)) return fail(SG_EINVAL, "sg_simulate_closed_loop: invalid problem");
  c.e.M = s->M;
  c.e.k = s->k;
  c.e.nf = s->nf;
  c.e.level = s->level;
  c.e.amax = s->amax < 1 ? 1 : s->amax;
  c.e.ops = s->ops;
  c.e.W = s->Ws;
  c.e.Wdf = s->Wdf;
  c.e.lo = s->box;
  c.e.width = s->box + s->d;
  c.e.xf = s->xf;
  c.e.xfdf = s->xfdf;
  c.d = s->d;
  c.x0 = d_x0;
  c.ntraj = ntraj;
  c.nsteps = nsteps;
  c.dt = dt;
  c.xT = d_xT;
  c.cost = d_cost;
  c.traj = d_traj;
  c.ctrl = d_ctrl;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = size_t(kClWarps) * c.d * c.e.nf * 8;
  const unsigned grid = static_cast<unsigned>(ceil_div(ntraj, kClWarps));
  if (mode == SG_EVAL_DF32) {
    SG_CUDA_TRY(ensure_dynamic_smem(k_closed_loop<SG_EVAL_DF32>, static_cast<int>(smem)));
    SG_TIMED("k_closed_loop_df32", st, (k_closed_loop<SG_EVAL_DF32><<<grid, 32 * kClWarps, smem, st>>>(c)));
  } else {
    SG_CUDA_TRY(ensure_dynamic_smem(k_closed_loop<SG_EVAL_FP64>, static_cast<int>(smem)));
    SG_TIMED("k_closed_loop_fp64", st, (k_closed_loop<SG_EVAL_FP64><<<grid, 32 * kClWarps, smem, st>>>(c)));
  }
  SG_LAUNCH_CHECK("k_closed_loop");
  return SG_OK;
}
