// Persistent batched form of the Newton solve: one warp per node, nodes pulled
// from a device work queue.  A warp runs the whole damped Newton iteration of
// its node (residual, Jacobian, condensation, staircase elimination, stage
// recovery, line search, update) and, when the node has converged, failed or
// used its iteration budget, takes the next node from the queue.  Nodes that
// need more iterations (uneven convergence) or more intervals simply keep
// their warp longer; no host round trip or grid-wide barrier is involved.
//
// The arithmetic is the same as the one-launch-per-phase form: the same
// kernels' per-warp device functions, the same residual and Armijo rule.
#pragma once

#include "bvp_kernels.cuh"

namespace sg {

// Shared-memory scratch per warp: the FP64 condensation system (36 x 49
// doubles), or the FP32 condensation's tables.
template <typename T>
__host__ __device__ constexpr int persist_smem_per_warp() {
  return sizeof(T) == sizeof(double) ? 36 * kCols * 8 : kCondSmemFloats * 4;
}

// Residual at Y + alpha D for the whole node, by one warp.  The
// right-hand side F at every point goes to `Fs` (the node's Jacobian slot,
// free during the line search); each lane then forms the stage rows of the
// intervals lane, lane+32, ..., stores them (precision T) for the next
// condensation, and the warp reduces |.|_2^2 and |.|_inf in a fixed order.
template <typename T, bool kPair>
__device__ __forceinline__ void residual_node_t(const SolveArgs& a, const Workspace& w, int64_t node, int N,
                                                double alpha, int lane, double* ss_out, double* mx_out) {
  const int64_t pb = node * npts(a.Nmax);
  const double* Y = w.Y + pb * 12;
  const double* D = w.D + pb * 12;
  // F at every point (the node's Jacobian slot is free during the line
  // search); with kPair F and the stage rows are pairs of floats, as in the
  // launch-per-phase residual
  double* Fs = reinterpret_cast<double*>(static_cast<T*>(w.Jm) + pb * 144);
  for (int p = lane; p <= 3 * N; p += 32) {
    if constexpr (kPair) {
      dfnum y[12], F[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) y[c] = dfnum(__fma_rn(alpha, D[12 * p + c], Y[12 * p + c]));
      char_rhs_t<dfnum>(a.P, y, F, node_target(a.P, node));
      dfnum* fp = reinterpret_cast<dfnum*>(Fs + 12 * p);
#pragma unroll
      for (int c = 0; c < 12; ++c) fp[c] = F[c];
    } else {
      double y[12], F[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) y[c] = __fma_rn(alpha, D[12 * p + c], Y[12 * p + c]);
      char_rhs(a.P, y, F, node_target(a.P, node));
#pragma unroll
      for (int c = 0; c < 12; ++c) Fs[12 * p + c] = F[c];
    }
  }
  __syncwarp();
  const double h = a.T[node] / N;
  double ss = 0.0, mx = 0.0;
  bool bad = false;
  for (int i = lane; i < N; i += 32) {
    T* res = static_cast<T*>(w.Res) + (node * a.Nmax + i) * kResRows;
    const int p0 = 3 * i;
    if constexpr (kPair) {
      const dfnum* Fd = reinterpret_cast<const dfnum*>(Fs);
#pragma unroll
      for (int k = 1; k < 4; ++k) {
        const dfnum c0(h * kLobA[k][0]), c1(h * kLobA[k][1]), c2(h * kLobA[k][2]), c3(h * kLobA[k][3]);
        dfnum ssd(0.0);
        float mxf = 0.0f;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          const dfnum y0(__fma_rn(alpha, D[12 * p0 + c], Y[12 * p0 + c]));
          const dfnum yk(__fma_rn(alpha, D[12 * (p0 + k) + c], Y[12 * (p0 + k) + c]));
          const dfnum r = (yk - y0) - (((c0 * Fd[12 * p0 + c] + c1 * Fd[12 * (p0 + 1) + c]) +
                                        c2 * Fd[12 * (p0 + 2) + c]) + c3 * Fd[12 * (p0 + 3) + c]);
          res[12 * (k - 1) + c] = r.hi;
          bad = bad || !isfinite(r.hi);
          ssd = ssd + r * r;
          mxf = fmaxf(mxf, fabsf(r.hi));
        }
        ss += ssd.to_double();
        mx = fmax(mx, double(mxf));
      }
    } else {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const double y0 = __fma_rn(alpha, D[12 * p0 + c], Y[12 * p0 + c]);
        const double f0 = Fs[12 * p0 + c], f1 = Fs[12 * (p0 + 1) + c], f2 = Fs[12 * (p0 + 2) + c],
                     f3 = Fs[12 * (p0 + 3) + c];
#pragma unroll
        for (int k = 1; k < 4; ++k) {
          const double yk = __fma_rn(alpha, D[12 * (p0 + k) + c], Y[12 * (p0 + k) + c]);
          const double r = yk - y0 - h * (kLobA[k][0] * f0 + kLobA[k][1] * f1 + kLobA[k][2] * f2 + kLobA[k][3] * f3);
          res[12 * (k - 1) + c] = static_cast<T>(r);
          bad = bad || !isfinite(r);
          ss += r * r;
          mx = fmax(mx, fabs(r));
        }
      }
    }
    if (i == 0) {
      const double* x0 = a.x0 + node * 6;
      for (int c = 0; c < 6; ++c) {
        const double r = __fma_rn(alpha, D[c], Y[c]) - x0[c];
        bad = bad || !isfinite(r);
        ss += r * r;
        mx = fmax(mx, fabs(r));
      }
    }
    if (i == N - 1) {
      double yN[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) yN[c] = __fma_rn(alpha, D[12 * 3 * N + c], Y[12 * 3 * N + c]);
      for (int c = 0; c < 6; ++c) {
        const double r = yN[6 + c] - terminal_grad(a.P, yN, c);
        bad = bad || !isfinite(r);
        ss += r * r;
        mx = fmax(mx, fabs(r));
      }
    }
  }
  ss = warp_sum(ss);
  mx = warp_max(mx);
  const bool anybad = __any_sync(0xffffffffu, bad);
  *ss_out = anybad ? INFINITY : ss;
  *mx_out = anybad ? INFINITY : mx;
  __syncwarp();
}

template <typename T>
__device__ __forceinline__ void residual_node(const SolveArgs& a, const Workspace& w, int64_t node, int N,
                                              double alpha, int lane, double* ss_out, double* mx_out) {
  if constexpr (sizeof(T) == sizeof(float)) {
    if (a.res_pair) return residual_node_t<T, true>(a, w, node, N, alpha, lane, ss_out, mx_out);
  }
  residual_node_t<T, false>(a, w, node, N, alpha, lane, ss_out, mx_out);
}

template <typename T>
__device__ void solve_node_persistent(const SolveArgs& a, const Workspace& w, int64_t node, int lane,
                                      unsigned char* scratch) {
  NodeState s = w.ns[node];
  if (!s.active) return;   // bad input: outputs are written by k_outputs
  const int N = a.N[node];
  const int64_t pb = node * npts(a.Nmax);
  double fn2, fmx;
  residual_node<T>(a, w, node, N, 0.0, lane, &fn2, &fmx);
  int iters = 0;
  int status = SG_MAXITER;
  if (!(fmx < INFINITY)) {
    status = SG_NONFINITE;
  } else if (fmx <= a.tol) {
    status = SG_CONVERGED;
  } else {
    while (iters < a.max_iter) {
      // Jacobian at every point
      for (int p = lane; p <= 3 * N; p += 32) {
        double y[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) y[c] = w.Y[(pb + p) * 12 + c];
        char_jacobian<T>(a.P, y, static_cast<T*>(w.Jm) + (pb + p) * 144, nullptr);
      }
      __syncwarp();
      // condensation of every interval
      bool ok = true;
      for (int i = 0; i < N; ++i) {
        if constexpr (sizeof(T) == sizeof(float)) {
          condense_interval_reg(a, w, node, i, N, lane, reinterpret_cast<float*>(scratch));
        } else {
          condense_interval_smem(a, w, node, i, N, lane, reinterpret_cast<double*>(scratch));
        }
      }
      __syncwarp();
      ok = abd_node_reg<T>(a, w, node, N, lane) && ok;
      __syncwarp();
      for (int i = 0; i < N; ++i) recover_interval<T>(a, w, node, i, lane);
      __syncwarp();
      // the condensation reports zero pivots through the node state
      const bool sing = !__all_sync(0xffffffffu, ok) || w.ns[node].singular;
      if (sing) {
        status = SG_SINGULAR;
        break;
      }
      // damped step (Armijo backtracking, same rule as the launch-per-phase form)
      double alpha = 1.0, tn2 = 0.0, tmx = 0.0;
      while (true) {
        residual_node<T>(a, w, node, N, alpha, lane, &tn2, &tmx);
        const bool finite = tn2 < INFINITY;
        if (!a.damping || (finite && tn2 <= (1.0 - 2e-4 * alpha) * fn2) || alpha <= 0x1p-10) break;
        alpha *= 0.5;
      }
      for (int p = lane; p <= 3 * N; p += 32) {
#pragma unroll
        for (int c = 0; c < 12; ++c)
          w.Y[(pb + p) * 12 + c] = __fma_rn(alpha, w.D[(pb + p) * 12 + c], w.Y[(pb + p) * 12 + c]);
      }
      __syncwarp();
      fn2 = tn2;
      fmx = tmx;
      ++iters;
      if (!(fmx < INFINITY)) {
        status = SG_NONFINITE;
        break;
      }
      if (fmx <= a.tol) {
        status = SG_CONVERGED;
        break;
      }
    }
  }
  if (lane == 0) {
    s.fnorm2 = fn2;
    s.fmax = fmx;
    s.iters = iters;
    s.status = status;
    s.active = 0;
    w.ns[node] = s;
  }
  __syncwarp();
}

// counters[2] is the queue head (zeroed before the launch).
template <typename T>
__global__ void __launch_bounds__(128) k_newton_persistent(SolveArgs a, Workspace w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* scratch = smem_raw + warp * persist_smem_per_warp<T>();
  while (true) {
    long long node = 0;
    if (lane == 0) node = atomicAdd(reinterpret_cast<unsigned long long*>(w.counters + 2), 1ull);
    node = __shfl_sync(0xffffffffu, node, 0);
    if (node >= a.n) break;
    solve_node_persistent<T>(a, w, node, lane, scratch);
  }
}

}  // namespace sg
