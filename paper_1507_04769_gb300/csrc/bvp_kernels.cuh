// Kernels of the characteristic BVP solver (Section 3.1, Eq. hamchar):
// four-stage Lobatto IIIA collocation on N equal intervals, damped Newton.
//
// One Newton iteration:
//   k_point     Jacobian dF/dy (precision T) at every collocation point (in
//               the mixed form with the FP64 residual, k_trial stores it
//               instead: the last trial of a line search is the next
//               iterate)
//   k_condense  the 36 linearised stage equations of one interval; Gaussian
//               elimination of the two interior stages (24 columns, partial
//               pivoting over the 24 interior rows) leaves the 12 x 25 block
//               row [S | T | rhs] that couples y_i and y_{i+1}
//   k_abd_*     staircase elimination with partial pivoting over
//               [x(0) rows; block rows; lambda(T) rows] and back substitution
//               for the mesh-point corrections, segmented so that the serial
//               chain per node is short (parallel over nodes and segments)
//   k_recover   interior-stage corrections from the stored pivot rows
//   k_trial     residual at Y + alpha D, per interval; it also stores the
//               stage residual rows (the right-hand side of the next
//               condensation); k_ls_reduce takes the Armijo decision per node
//               in a fixed reduction order
// T = double gives the FP64 form, T = float the mixed forms (FP32 Jacobian,
// elimination and direction; FP64 line search and update; the residual in
// FP64, or in pairs of floats in the mixed-pair form).
#pragma once

#include <cmath>

#include "common.cuh"
#include "linalg.cuh"
#include "problems.cuh"

namespace sg {

// ---------------------------------------------------------------- tableau
// Four-stage Lobatto IIIA (Hairer & Wanner, Solving ODEs II, Sec. IV.5):
// c = 0, (5 - sqrt5)/10, (5 + sqrt5)/10, 1; b = (1, 5, 5, 1)/12.
#define SG_S5 2.2360679774997896964091736687312762
#define SG_LOB_A                                                                                    \
  {{0.0, 0.0, 0.0, 0.0},                                                                            \
   {(11.0 + SG_S5) / 120.0, (25.0 - SG_S5) / 120.0, (25.0 - 13.0 * SG_S5) / 120.0,                  \
    (-1.0 + SG_S5) / 120.0},                                                                        \
   {(11.0 - SG_S5) / 120.0, (25.0 + 13.0 * SG_S5) / 120.0, (25.0 + SG_S5) / 120.0,                  \
    (-1.0 - SG_S5) / 120.0},                                                                        \
   {1.0 / 12.0, 5.0 / 12.0, 5.0 / 12.0, 1.0 / 12.0}}
__constant__ double kLobA[4][4] = SG_LOB_A;
__constant__ float kLobAf[4][4] = SG_LOB_A;
__constant__ double kLobB[4] = {1.0 / 12.0, 5.0 / 12.0, 5.0 / 12.0, 1.0 / 12.0};

struct NodeState {
  double fnorm2;   // |F|_2^2 at the current iterate
  double fmax;     // |F|_inf at the current iterate
  double alpha;    // current step length
  int active;      // still iterating
  int searching;   // in the line search
  int singular;    // a zero pivot was met this iteration
  int iters;
  int status;
  int ybuf;        // 1: the current iterate is in Y2 (see Workspace)
};

constexpr int kCols = 49;        // 24 interior + 12 (y_i) + 12 (y_{i+1}) + rhs
constexpr int kRecLd = 52;       // row stride of a stored interior pivot row (16-byte multiple)
constexpr int kRecInv = 49;      // column of a stored pivot row holding 1/pivot
constexpr int kRec = 24 * kRecLd;
// FP32 recovery rows are stored chunk-major: the 16-byte chunk q (columns
// 4q..4q+3) of rows 0..23 lie side by side, so a warp reading chunk q of its
// 24 rows reads 384 contiguous bytes.  Float offset of (row r, column c):
__host__ __device__ __forceinline__ int rec_at(int r, int c) { return ((c >> 2) * 24 + r) * 4 + (c & 3); }
constexpr int kBlkLd = 28;       // row stride of a 12-row block of 25 columns
constexpr int kBlk = 12 * kBlkLd;
constexpr int kResRows = 36;     // stage residual rows per interval
constexpr int kSegLen = 16;      // intervals per segment of the segmented staircase
constexpr int kSegLd = 40;       // row stride of a segment pivot row: F | U | V | rhs (37) + pad
constexpr int kSegBlk = 12 * kSegLd;

__host__ __device__ __forceinline__ int seg_count(int N) { return (N + kSegLen - 1) / kSegLen; }

struct Workspace {
  double* Y;       // n x P x 12, current iterate
  double* D;       // n x P x 12, Newton direction
  double* Y2;      // n x P x 12 (FP32-direction forms): with the Jacobian from the residual
                   // kernel, each trial point goes here (or to Y), and an accepted step only
                   // flips the node's ybuf: no update pass
  void* Jm;        // n x P x 144 (T), Jacobians
  void* Res;       // n x Nmax x 36 (T), stage residuals at the iterate
  void* Cond;      // n x Nmax x kBlk (T), condensed block rows
  void* Rec;       // n x Nmax x kRec (T), interior pivot rows (FP32: chunk-major, rec_at)
  void* Abd;       // n x Nmax x kBlk (T), staircase pivot rows
  void* Seg;       // n x Nmax x kSegBlk (T), pivot rows of the segment eliminations
  void* Red;       // n x seg_count(Nmax) x kBlk (T), reduced block rows of the segments
  double* part;    // n x Nmax x 2, partial |F|^2 and |F|_inf
  NodeState* ns;   // n
  int* counters;   // 2
  size_t bytes;
};

struct SolveArgs {
  DevProblem P;
  const double* x0;
  const double* T;
  const int32_t* N;
  int64_t n;
  int Nmax;
  double tol;
  int max_iter;
  int damping;
  int persistent;      // one warp per node from a device queue (bvp_persistent.cuh)
  int blocks_per_sm;   // cap on resident 4-warp blocks per SM for the persistent form (0 = occupancy)
  int cond_warps;      // intervals (warps) per block of the FP32 condensation: 2, 4 or 8
  int sync_at_end;
  const double* Yin;   // initial iterate (n x P x 12), or null for the zero-control guess
  int res_pair;        // FP32-direction form: 1 = residual in pairs of floats, 0 = in FP64
  int jac_in_trial;    // FP32-direction form with the FP64 residual: the residual kernel also stores the Jacobian
};

__host__ __device__ __forceinline__ int64_t npts(int Nmax) { return 3 * int64_t(Nmax) + 1; }

// ---------------------------------------------------------------- setup
// A thread per pair of components of a collocation point (consecutive
// threads write consecutive 16-byte words); the node's first thread also
// sets up its state.
constexpr int kInitPer = 6;   // threads per collocation point

// Components 2q, 2q + 1 of point p of `node` (u = its global pair index);
// the point-0, q-0 thread also sets up the node's state.
__device__ __forceinline__ void init_pair(const SolveArgs& a, const Workspace& w, int64_t node, int64_t p, int q,
                                          int64_t u) {
  const double* x0 = a.x0 + node * 6;
  double2 y;
  if (a.Yin) {
    // warm start (the caller's array may be only 8-byte aligned)
    y = (reinterpret_cast<uintptr_t>(a.Yin) & 15u) ? make_double2(a.Yin[2 * u], a.Yin[2 * u + 1])
                                                   : reinterpret_cast<const double2*>(a.Yin)[u];
  } else {
    // x held at x0, lambda = 0 (zero control)
    y = q < 3 ? make_double2(x0[2 * q], x0[2 * q + 1]) : make_double2(0.0, 0.0);
  }
  reinterpret_cast<double2*>(w.Y)[u] = y;
  reinterpret_cast<double2*>(w.D)[u] = make_double2(0.0, 0.0);
  if (p == 0 && q == 0) {
    NodeState s{};
    const int N = a.N[node];
    const double T = a.T[node];
    bool ok = N >= 1 && N <= a.Nmax && T >= 0.0 && T < INFINITY;
    for (int c = 0; c < 6; ++c) ok = ok && isfinite(x0[c]);
    s.alpha = 0.0;   // the first residual evaluation is at Y itself
    s.active = ok ? 1 : 0;
    s.searching = ok ? 1 : 0;
    s.status = ok ? SG_MAXITER : SG_BADINPUT;
    w.ns[node] = s;
  }
}

__global__ void k_init(SolveArgs a, Workspace w) {
  const int64_t P = npts(a.Nmax);
  const int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (u >= a.n * P * kInitPer) return;
  const int64_t t = u / kInitPer;
  init_pair(a, w, t / P, t % P, static_cast<int>(u % kInitPer), u);
}

// ---------------------------------------------------------------- residual
// Residual at Y + alpha D.  A block takes kTrialIv consecutive intervals
// of one node: first every thread evaluates F at one collocation point of the
// chunk (3 kTrialIv + 1 <= 128 points, so the shared end points are evaluated
// once), then the stage rows 2..4 of each interval are formed from the
// points in shared memory (the first interval adds the x(0) rows, the last
// the lambda(T) rows).  Writes the partial |.|_2^2 and |.|_inf per interval
// and the 36 stage rows (precision T) for the next condensation.
constexpr int kTrialIv = 42;                     // intervals per block
constexpr int kTrialPts = 3 * kTrialIv + 1;      // 127 points

__host__ __device__ __forceinline__ int trial_chunks(int Nmax) { return (Nmax + kTrialIv - 1) / kTrialIv; }

// A residual row entry in the precision of the Newton direction.  For FP32
// the double is truncated to 24 significant bits from its bit pattern (the
// integer pipe; the rounding of the FP32 direction's input does not matter,
// and the conversion instruction would run on the FP64 pipe, which the FP64
// residual saturates).  Below the FP32 normal range it becomes a signed zero;
// above it, infinity; a NaN stays a NaN.
template <typename T>
__device__ __forceinline__ T narrow_row(double x) {
  if constexpr (sizeof(T) == sizeof(double)) {
    return x;
  } else {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
    const unsigned e = (hi >> 20) & 0x7FFu, sign = hi & 0x80000000u;
    if (e >= 897u && e <= 1150u)
      return __uint_as_float(sign | (((hi & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lo >> 29));
    if (e < 897u) return __uint_as_float(sign);
    if (e == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u) return __uint_as_float(0x7FC00000u);
    return __uint_as_float(sign | 0x7F800000u);
  }
}

// Round to the nearest FP32 value from the bit pattern (integer pipe), the
// same value as the conversion instruction, which runs on the FP64 pipe.
__device__ __forceinline__ float f32_rn_bits(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e < 897u || e > 1150u) return __double2float_rn(x);   // zero, subnormal, huge, non-finite
  const unsigned sign = hi & 0x80000000u;
  unsigned f = (((hi & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lo >> 29);   // exponent and 23 bits
  const unsigned rest = lo & 0x1FFFFFFFu;
  if (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ++f;   // ties to even; a carry bumps the exponent
  return __uint_as_float(sign | f);
}

constexpr int kTrialJLd = 40;   // staged rows of one point in the fused Jacobian: three rows (36) + 4

// (kJac: five blocks per SM, 96 registers with a few spilled dual values,
// against 126 registers and four blocks; 2 % faster)
template <typename T, bool kPair, bool kJac>
__global__ void __launch_bounds__(128, 5) k_trial(SolveArgs a, Workspace w) {
  // kPair = false: points and rows in FP64 (the FP64 and mixed forms).
  // kPair = true (the mixed-pair form): the right-hand side and the stage rows
  // in pair-of-floats arithmetic (about 48 bits, on the FP32 pipe); the
  // boundary rows and the iterate Y + alpha D stay FP64.
  // kJac (mixed form): the FP32 Jacobian at the trial point as well, on the
  // FP32 pipe beside the FP64 residual; the last trial of a line search is
  // the accepted iterate, so its Jacobian is the next iteration's.
  __shared__ __align__(16) double yfs[2][kTrialPts][12];   // points and F (dfnum in the mixed-pair form)
  auto& ys = yfs[0];
  auto& fs = yfs[1];
  __shared__ double part_s[3 * kTrialIv][2];
  __shared__ double cA_s[3][4];          // h a_kj: a pair (pair residual) or FP64, k = 1..3
  const int tid = threadIdx.x;
  const int nchunk = trial_chunks(a.Nmax);
  const int64_t node = blockIdx.x / nchunk;
  const int i0 = static_cast<int>(blockIdx.x % nchunk) * kTrialIv;
  if (node >= a.n) return;
  const NodeState& s = w.ns[node];
  if (!s.searching) return;
  const int N = a.N[node];
  if (i0 >= N) return;
  const int niv = N - i0 < kTrialIv ? N - i0 : kTrialIv;
  const double alpha = s.alpha;
  const int64_t base = node * npts(a.Nmax) + 3 * int64_t(i0);
  float yf[12];   // kJac: the point rounded to FP32
#pragma unroll
  for (int c = 0; c < 12; ++c) yf[c] = 0.0f;
  const double* Ycur = s.ybuf ? w.Y2 : w.Y;
  auto ypoint = [&](int64_t pt, int c) { return __fma_rn(alpha, w.D[pt * 12 + c], Ycur[pt * 12 + c]); };
  // the stage coefficients h a_kj once per block (the last 12 threads)
  if (tid >= 128 - 12) {
    const int e = tid - (128 - 12), k = e / 4 + 1, jj = e % 4;
    const double h = a.T[node] / N;
    if constexpr (kPair) {
      *reinterpret_cast<dfnum*>(&cA_s[k - 1][jj]) = dfnum(h * kLobA[k][jj]);
    } else {
      cA_s[k - 1][jj] = h * kLobA[k][jj];
    }
  }
  if (tid <= 3 * niv) {
    if constexpr (kPair) {
      dfnum y[12], F[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) y[c] = dfnum(ypoint(base + tid, c));
      char_rhs_t<dfnum>(a.P, y, F, node_target(a.P, node));
      dfnum* yp = reinterpret_cast<dfnum*>(ys[tid]);
      dfnum* fp = reinterpret_cast<dfnum*>(fs[tid]);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        yp[c] = y[c];
        fp[c] = F[c];
      }
    } else {
      double y[12], F[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) y[c] = ypoint(base + tid, c);
      char_rhs(a.P, y, F, node_target(a.P, node));
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        ys[tid][c] = y[c];
        fs[tid][c] = F[c];
      }
      if constexpr (kJac) {
#pragma unroll
        for (int c = 0; c < 12; ++c) yf[c] = f32_rn_bits(y[c]);
        // the trial point to the other iterate buffer: if the step is
        // accepted it becomes the iterate (the same fma as an update pass)
        double2* alt = reinterpret_cast<double2*>((s.ybuf ? w.Y : w.Y2) + (base + tid) * 12);
#pragma unroll
        for (int c = 0; c < 6; ++c) alt[c] = make_double2(y[2 * c], y[2 * c + 1]);
      }
    }
  }
  __syncthreads();
  if (tid < 3 * niv) {
    // interval j = tid / 3 of the chunk, stage row block k = tid % 3 + 1
    const int j = tid / 3, k = tid % 3 + 1;
    const int p0 = 3 * j;
    T* res = static_cast<T*>(w.Res) + (node * a.Nmax + i0 + j) * kResRows + 12 * (k - 1);
    double ss = 0.0, mx = 0.0;
    bool bad = false;
    if constexpr (kPair) {
      const dfnum* cA = reinterpret_cast<const dfnum*>(&cA_s[k - 1][0]);
      const dfnum c0 = cA[0], c1 = cA[1], c2 = cA[2], c3 = cA[3];
      const dfnum* y0 = reinterpret_cast<const dfnum*>(ys[p0]);
      const dfnum* yk = reinterpret_cast<const dfnum*>(ys[p0 + k]);
      const dfnum* f0 = reinterpret_cast<const dfnum*>(fs[p0]);
      const dfnum* f1 = reinterpret_cast<const dfnum*>(fs[p0 + 1]);
      const dfnum* f2 = reinterpret_cast<const dfnum*>(fs[p0 + 2]);
      const dfnum* f3 = reinterpret_cast<const dfnum*>(fs[p0 + 3]);
      dfnum ssd(0.0);
      float mxf = 0.0f;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const dfnum r = (yk[c] - y0[c]) - (((c0 * f0[c] + c1 * f1[c]) + c2 * f2[c]) + c3 * f3[c]);
        res[c] = r.hi;
        bad = bad || !isfinite(r.hi);
        ssd = ssd + r * r;
        mxf = fmaxf(mxf, fabsf(r.hi));
      }
      ss = ssd.to_double();
      mx = mxf;
    } else {
      const double* cA = cA_s[k - 1];
      const double c0 = cA[0], c1 = cA[1], c2 = cA[2], c3 = cA[3];
      // |r|_inf and finiteness from the bit patterns (integer pipe): for
      // non-negative doubles the bit patterns order like the values, and a
      // non-finite value has all exponent bits set
      unsigned long long mxb = 0ull;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        double r = ys[p0 + k][c] - ys[p0][c];
        r = fma(-c0, fs[p0][c], r);
        r = fma(-c1, fs[p0 + 1][c], r);
        r = fma(-c2, fs[p0 + 2][c], r);
        r = fma(-c3, fs[p0 + 3][c], r);
        res[c] = narrow_row<T>(r);
        const unsigned long long ab = static_cast<unsigned long long>(__double_as_longlong(r)) & 0x7FFFFFFFFFFFFFFFull;
        mxb = ab > mxb ? ab : mxb;
        ss = fma(r, r, ss);
      }
      bad = bad || mxb >= 0x7FF0000000000000ull;
      mx = __longlong_as_double(static_cast<long long>(mxb));
    }
    // boundary rows in FP64 from the iterate itself
    if (k == 1 && i0 + j == 0) {
      const double* x0 = a.x0 + node * 6;
      for (int c = 0; c < 6; ++c) {
        const double r = ypoint(base, c) - x0[c];
        bad = bad || !isfinite(r);
        ss += r * r;
        mx = fmax(mx, fabs(r));
      }
    }
    if (k == 3 && i0 + j == N - 1) {
      double yN[12];
      for (int c = 0; c < 12; ++c) yN[c] = ypoint(base + p0 + 3, c);
      for (int c = 0; c < 6; ++c) {
        const double r = yN[6 + c] - terminal_grad(a.P, yN, c);
        bad = bad || !isfinite(r);
        ss += r * r;
        mx = fmax(mx, fabs(r));
      }
    }
    if (bad) {
      ss = INFINITY;
      mx = INFINITY;
    }
    part_s[tid][0] = ss;
    part_s[tid][1] = mx;
  }
  __syncthreads();
  if (tid < niv) {
    const double ss = part_s[3 * tid][0] + part_s[3 * tid + 1][0] + part_s[3 * tid + 2][0];
    const double mx = fmax(fmax(part_s[3 * tid][1], part_s[3 * tid + 1][1]), part_s[3 * tid + 2][1]);
    const int64_t t = node * a.Nmax + i0 + tid;
    w.part[2 * t] = ss;
    w.part[2 * t + 1] = mx;
  }
  if constexpr (kJac) {
    // The Jacobian of this thread's point.  The points of a warp are
    // consecutive in Jm; rows are staged three at a time in the point tables
    // (free now) and the warp writes them as contiguous 144-byte runs.
    const int lane = tid & 31, warp = tid >> 5;
    const bool valid = tid <= 3 * niv;
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    if (vmask != 0u) {
      float* stage = reinterpret_cast<float*>(&yfs[0][0][0]) + warp * 32 * kTrialJLd;
      float* mine = stage + lane * kTrialJLd;
      float* Jw = static_cast<float*>(w.Jm) + (base + 32 * warp) * 144;
      char_jacobian_rows<float>(
          a.P, yf,
          [&](int r, const float (&row)[12]) {
            float4* dst = reinterpret_cast<float4*>(mine + 12 * (r % 3));
#pragma unroll
            for (int q4 = 0; q4 < 3; ++q4)
              dst[q4] = make_float4(row[4 * q4], row[4 * q4 + 1], row[4 * q4 + 2], row[4 * q4 + 3]);
            if (r % 3 == 2) {
              __syncwarp();
              const int h = r / 3;
              for (int e = lane; e < 32 * 9; e += 32) {
                const int pt = e / 9, q = e % 9;
                if ((vmask >> pt) & 1u)
                  reinterpret_cast<float4*>(Jw + pt * 144 + 36 * h)[q] =
                      reinterpret_cast<const float4*>(stage + pt * kTrialJLd)[q];
              }
              __syncwarp();
            }
          },
          nullptr);
    }
  }
}

// The residual kernel of a solve: FP64, or pairs of floats in the
// FP32-direction form when asked for.
template <typename T>
inline void (*trial_kernel(const SolveArgs& a))(SolveArgs, Workspace) {
  if constexpr (sizeof(T) == sizeof(float)) {
    if (a.res_pair) return k_trial<float, true, false>;
    return a.jac_in_trial ? k_trial<float, false, true> : k_trial<float, false, false>;
  } else {
    return k_trial<double, false, false>;
  }
}

// Warp per node: reduce the partial norms in a fixed order and decide.
// mode 0: initial residual (convergence test at iteration 0);
// mode 1: Armijo test for the current alpha.
__global__ void k_ls_reduce(SolveArgs a, Workspace w, int mode) {
  const int lane = threadIdx.x & 31;
  const int64_t node = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (node >= a.n) return;
  NodeState s = w.ns[node];
  if (!s.searching) return;
  const int N = a.N[node];
  double ss = 0.0, mx = 0.0;
  for (int i = lane; i < N; i += 32) {
    ss += w.part[2 * (node * a.Nmax + i)];
    mx = fmax(mx, w.part[2 * (node * a.Nmax + i) + 1]);
  }
  ss = warp_sum(ss);
  mx = warp_max(mx);
  if (lane != 0) return;
  if (mode == 0) {
    s.fnorm2 = ss;
    s.fmax = mx;
    s.searching = 0;
    if (!(mx < INFINITY)) {
      s.status = SG_NONFINITE;
      s.active = 0;
    } else if (mx <= a.tol) {
      s.status = SG_CONVERGED;
      s.active = 0;
    } else {
      atomicAdd(&w.counters[1], 1);
    }
  } else {
    const bool finite = ss < INFINITY;
    const bool accept = !a.damping || (finite && ss <= (1.0 - 2e-4 * s.alpha) * s.fnorm2) ||
                        s.alpha <= 0x1p-10;
    if (accept) {
      s.fnorm2 = ss;
      s.fmax = mx;
      s.searching = 0;
      if (a.jac_in_trial) s.ybuf ^= 1;   // the trial point is the iterate
    } else {
      s.alpha *= 0.5;
      atomicAdd(&w.counters[0], 1);
    }
  }
  w.ns[node] = s;
}

// ---------------------------------------------------------------- Jacobian
constexpr int kPtWarps = 4;    // warps per block of k_point
constexpr int kPtLd = 76;      // staged row stride of a point: six rows (72) + 4, 16-byte aligned

template <typename T>
__global__ void __launch_bounds__(32 * kPtWarps) k_point(SolveArgs a, Workspace w) {
  const int64_t P = npts(a.Nmax);
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  bool valid = t < a.n * P;
  if (valid) {
    const int64_t node = t / P, p = t % P;
    valid = w.ns[node].active && p <= 3 * int64_t(a.N[node]);
  }
  double y[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) y[c] = valid ? w.Y[t * 12 + c] : 0.0;
  if constexpr (sizeof(T) == 8) {
    if (valid) char_jacobian<T>(a.P, y, static_cast<T*>(w.Jm) + t * 144, nullptr);
  } else {
    // The 32 points of a warp are consecutive in Jm.  Rows are staged in
    // shared memory six at a time and the warp writes them as contiguous
    // 288-byte runs (one per point) instead of 48-byte rows 576 bytes apart.
    __shared__ __align__(16) float stage[kPtWarps][32 * kPtLd];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    if (vmask == 0u) return;   // the whole warp
    float* mine = stage[warp] + lane * kPtLd;
    float* Jw = static_cast<float*>(w.Jm) + (t - lane) * 144;   // the warp's first point
    char_jacobian_rows<float>(
        a.P, y,
        [&](int r, const float (&row)[12]) {
          float4* dst = reinterpret_cast<float4*>(mine + 12 * (r % 6));
#pragma unroll
          for (int q4 = 0; q4 < 3; ++q4)
            dst[q4] = make_float4(row[4 * q4], row[4 * q4 + 1], row[4 * q4 + 2], row[4 * q4 + 3]);
          if (r % 6 == 5) {
            __syncwarp();
            const int h = r / 6;
            for (int e = lane; e < 32 * 18; e += 32) {
              const int pt = e / 18, q = e % 18;
              if ((vmask >> pt) & 1u)
                reinterpret_cast<float4*>(Jw + pt * 144 + 72 * h)[q] =
                    reinterpret_cast<const float4*>(stage[warp] + pt * kPtLd)[q];
            }
            __syncwarp();
          }
        },
        nullptr);
  }
}

// ---------------------------------------------------------------- helpers
// Pivot search of the register-resident kernels: the largest |v| over the
// candidate lanes, ties to the lower lane (magnitude bits with the 5 low bits
// replaced by 31 - lane, reduced by one warp max).
template <typename T>
__device__ __forceinline__ int warp_pivot_lane(T v, bool cand, int lane) {
  const float m = fabsf(static_cast<float>(v));
  const unsigned key = cand ? ((__float_as_uint(m) & ~31u) | unsigned(31 - lane)) : 0u;
  const unsigned best = __reduce_max_sync(0xffffffffu, key);
  return 31 - int(best & 31u);
}

template <typename T>
__device__ __forceinline__ void load_row25(const T* __restrict__ src, T (&r)[25]) {
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float4 v = s4[q];
      r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const double2 v = s2[q];
      r[2 * q] = v.x; r[2 * q + 1] = v.y;
    }
  }
  r[24] = src[24];
}

// A 25-entry row into a kBlkLd (28) slot, the 3 pad entries zeroed: whole
// 32-byte sectors are written, so the memory system need not read the slot
// first.
template <typename T>
__device__ __forceinline__ void store_row25(T* __restrict__ dst, const T (&r)[25]) {
  if constexpr (sizeof(T) == 4) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < 6; ++q) d4[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    d4[6] = make_float4(r[24], 0.0f, 0.0f, 0.0f);
  } else {
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int q = 0; q < 12; ++q) d2[q] = make_double2(r[2 * q], r[2 * q + 1]);
    d2[12] = make_double2(r[24], 0.0);
    d2[13] = make_double2(0.0, 0.0);
  }
}

// Pivot-search key: the magnitude bits (sign shifted out; for doubles the
// upper word) in the top 31 bits, ordered like |x|.
__device__ __forceinline__ unsigned mag_key(float x) { return __float_as_uint(x) << 1; }
__device__ __forceinline__ unsigned mag_key(double x) {
  return static_cast<unsigned>(static_cast<unsigned long long>(__double_as_longlong(x)) >> 32) << 1;
}

// 16-byte asynchronous global -> shared copies (cp.async, completion by
// cp.async.wait_all; other lanes see the data after a __syncwarp).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Correctly rounded reciprocal (the same value as 1 / x, without the
// division's slow-path branch).
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return __drcp_rn(x); }

// 1/pivot in the condensation and segment eliminations.  FP32: the
// approximate reciprocal instruction (rcp.approx.ftz, within about one unit
// in the last place; a subnormal pivot flushes to zero): the FP32
// eliminations only give a Newton direction whose residual is evaluated in
// FP64, so the last bit of 1/pivot carries no weight.  FP64: correctly
// rounded.  `good` is false for a zero, subnormal (FP32) or non-finite pivot,
// whose reciprocal is then 0.
__device__ __forceinline__ float pivot_recip(float p, bool& good) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
  good = fabsf(r) < INFINITY && r != 0.0f;
  return good ? r : 0.0f;
}
__device__ __forceinline__ double pivot_recip(double p, bool& good) {
  good = p != 0.0 && isfinite(p);
  return good ? __drcp_rn(p) : 0.0;
}

// 40-entry rows (F | Y | Z | rhs and padding) loaded as 16-byte vectors.
template <typename T>
__device__ __forceinline__ void load_row40(const T* __restrict__ src, T (&r)[40]) {
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const float4 v = s4[q];
      r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int q = 0; q < 20; ++q) {
      const double2 v = s2[q];
      r[2 * q] = v.x; r[2 * q + 1] = v.y;
    }
  }
}

// Twelve pivot steps with partial pivoting on 25-column rows held one per
// lane.  cand: this lane's row takes part.  The pivot row of step k keeps
// 1/pivot at column k; plane[k] is the lane that held it.
template <typename T>
__device__ __forceinline__ void panel_eliminate12(T (&r)[25], bool cand, bool& done, int& my_step,
                                                  int (&plane)[12], bool& ok, int lane) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int p = warp_pivot_lane<T>(r[k], cand && !done, lane);
    plane[k] = p;
    const T piv = __shfl_sync(0xffffffffu, r[k], p);
    // (the correctly rounded reciprocal: on this serial chain the approximate
    // instruction measured 19 % slower)
    const bool good = piv != T(0) && isfinite(piv);
    ok = ok && good;
    const T inv = good ? recip_rn(piv) : T(0);
    const bool is_p = lane == p;
    const T l = (cand && !done && !is_p) ? r[k] * inv : T(0);
#pragma unroll
    for (int c = k + 1; c < 25; ++c) {
      const T pc = __shfl_sync(0xffffffffu, r[c], p);
      r[c] = fma(-l, pc, r[c]);
    }
    if (is_p) {
      done = true;
      my_step = k;
      r[k] = inv;
    }
  }
}

// ---------------------------------------------------------------- condensation
// Register-resident FP32 form, warp per interval, in two phases.
//
// The 36 x 49 system splits into the 24 interior columns (stages 2 and 3,
// eliminated) and the 25 passive columns [y_i | y_{i+1} | rhs].
//   Phase A (rows on lanes): lane r holds interior row r (r < 24) or stage-4
//   row r (24..31); stage-4 rows 32..35 are spread over the warp for the first
//   four pivot steps and then move into the lanes of the first four pivot
//   rows, which are free by then.  Only the 24 interior columns live in
//   registers.  Partial pivoting over the interior
//   rows; at step k the pivot lane publishes its row in the
//   shared-memory table U (16-byte broadcast reads), every lane forms
//   1/pivot from it, and every row records its multiplier l(r, k) in L.
//   Phase B (columns on lanes): lane c < 25 owns passive column c.  With the
//   pivot order p_k, the passive part of pivot row k is
//       Q_k = P(p_k) - sum_{j<k} l(p_k, j) Q_j
//   and the condensed stage-4 rows are P(r) - sum_k l(r, k) Q_k, where P is
//   the original passive block (built into shared memory).
// Rows never move.  The stored recovery rows are [U_k | Q_k] in pivot order
// (raw pivot on the diagonal), the condensed block row is [S | T | rhs].
constexpr int kCondLd = 28;                          // row stride of P, L and U (floats)
constexpr int kSpreadSteps = 4;                      // pivot steps before rows 32..35 move into lanes
constexpr int kCondSmemFloats = 36 * kCondLd * 2 + 8 * kCondLd + 32 + 24;   // P, L, U (ring of 8 rows), pivot order, 1/pivot

// (sm is not __restrict__: lanes exchange pivot rows through it across
// __syncwarp, and a no-alias promise would let the compiler read it before
// the barrier.)
__device__ __forceinline__ void condense_interval_reg(const SolveArgs& a, const Workspace& w, int64_t node,
                                                      int i, int N, int lane, float* sm) {
  const int64_t wid = node * a.Nmax + i;
  const float hf = static_cast<float>(a.T[node]) / static_cast<float>(N);
  const int64_t pbase = node * npts(a.Nmax) + 3 * int64_t(i);
  const float* J = static_cast<const float*>(w.Jm) + pbase * 144;
  const float* res = static_cast<const float*>(w.Res) + wid * kResRows;
  float* P_s = sm;                         // [36][kCondLd] passive columns, original
  float* L_s = sm + 36 * kCondLd;          // [36][kCondLd] multipliers l(r, k)
  float* U_s = sm + 72 * kCondLd;          // [8][kCondLd] pivot row of step k at k % 8, 1/pivot at 24
  int* perm_s = reinterpret_cast<int*>(sm + 80 * kCondLd);   // [24] pivot row of step k
  float* inv_s = sm + 80 * kCondLd + 32;   // [24] 1/pivot of step k (for the stored rows)
  const int64_t blk = node * a.Nmax + i;
  float* rec = static_cast<float*>(w.Rec) + blk * kRec;

  // row r = 12 (k - 1) + comp for stage k = 1, 2, 3 (Lobatto stages 2, 3, 4):
  // passive part to P_s[r], interior part through L_s[r] (free until the end
  // of phase A) to act[24]; the identity terms are added in shared memory
  auto build = [&](int r, float (&act)[24]) {
    const int k = r / 12 + 1, comp = r % 12;
    float4* dP = reinterpret_cast<float4*>(P_s + r * kCondLd);
    float4* dA = reinterpret_cast<float4*>(L_s + r * kCondLd);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float cf = -hf * kLobAf[k][j];
      const float4* src = reinterpret_cast<const float4*>(J + j * 144 + comp * 12);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float4 x = src[q];
        const float4 v = make_float4(cf * x.x, cf * x.y, cf * x.z, cf * x.w);
        if (j == 0) dP[q] = v;            // y_i
        if (j == 1) dA[q] = v;            // stage 2
        if (j == 2) dA[3 + q] = v;        // stage 3
        if (j == 3) dP[3 + q] = v;        // y_{i+1}
      }
    }
    P_s[r * kCondLd + 24] = -res[r];
    P_s[r * kCondLd + comp] -= 1.0f;                     // -I on y_i
    if (k == 3) P_s[r * kCondLd + 12 + comp] += 1.0f;    // +I on the stage's own point
    else L_s[r * kCondLd + r] += 1.0f;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float4 v = dA[q];
      act[4 * q] = v.x; act[4 * q + 1] = v.y; act[4 * q + 2] = v.z; act[4 * q + 3] = v.w;
    }
  };

  float ra[24];
  build(lane, ra);
  // rows 32..35 (stage 4, components 8..11) start spread over the warp: lane
  // group g = lane / 8 holds row 32 + g, lane sub = lane % 8 holds columns
  // sub, sub + 8 and sub + 16 of its interior part and of its passive part
  // (the passive part stays there: it goes to P)
  const int g = lane >> 3, sub = lane & 7;
  const int r2 = 32 + g, comp2 = 8 + g;
  float rb[3];
  {
    const float cf0 = -hf * kLobAf[3][0], cf1 = -hf * kLobAf[3][1];
    const float cf2 = -hf * kLobAf[3][2], cf3 = -hf * kLobAf[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int c = sub + 8 * m;
      const int j = c < 12 ? 1 : 2;                 // interior column c: point j, component c % 12
      rb[m] = (j == 1 ? cf1 : cf2) * J[j * 144 + comp2 * 12 + (c < 12 ? c : c - 12)];
      // passive column c: y_i (point 0) below 12, y_{i+1} (point 3) from 12
      float pv = c < 12 ? cf0 * J[comp2 * 12 + c] : cf3 * J[3 * 144 + comp2 * 12 + c - 12];
      if (c == comp2) pv -= 1.0f;
      if (c - 12 == comp2) pv += 1.0f;
      P_s[r2 * kCondLd + c] = pv;
    }
    if (sub == 0) P_s[r2 * kCondLd + 24] = -res[r2];
  }

  // ---- phase A: interior columns
  // pivot key: |a| (sign shifted out) with the low 5 bits replaced by
  // 31 - lane, so one warp max finds the largest magnitude, ties to the lower
  // lane; a lane that is no candidate (stage-4 row, or already a pivot row)
  // has an all-zero mask and tag
  const unsigned itag = 31u - unsigned(lane);
  unsigned kmask = lane < 24 ? ~31u : 0u;
  unsigned ktag = lane < 24 ? itag : 0u;
  float live = 1.0f;                        // 0 once the row is a pivot row
  bool bad = false;                         // a zero or non-finite pivot (the same in every lane)
  float inv_keep = 0.0f;                    // lane j < 8: 1/pivot of the last step k with k % 8 == j
  float lbk = 0.f;                          // multiplier of row r2 at column sub (steps 0..3)
  int myrow = lane;                         // the row this lane holds (32..35 once moved in)
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    const int q0 = k / 4;
    const unsigned key = ((__float_as_uint(ra[k]) << 1) & kmask) | ktag;
    const unsigned best = __reduce_max_sync(0xffffffffu, key);
    if (key == best) {   // candidates' keys are nonzero and differ in the tag; the others are 0
      float4* dst = reinterpret_cast<float4*>(U_s + (k & 7) * kCondLd);
#pragma unroll
      for (int q = q0; q < 6; ++q) dst[q] = make_float4(ra[4 * q], ra[4 * q + 1], ra[4 * q + 2], ra[4 * q + 3]);
      perm_s[k] = lane;
      kmask = 0u;
      ktag = 0u;
      live = 0.0f;
    }
    __syncwarp();
    const float4* src = reinterpret_cast<const float4*>(U_s + (k & 7) * kCondLd);
    // every lane forms 1/pivot from the published row (the same value in
    // every lane; zero for an unusable pivot)
    bool good;
    const float inv = pivot_recip(U_s[(k & 7) * kCondLd + k], good);
    if (lane == (k & 7)) inv_keep = inv;
    bad = bad || !good;
    const float la = ra[k] * (inv * live);
#pragma unroll
    for (int q = q0; q < 6; ++q) {
      const float4 u4 = src[q];
      const float u[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = 4 * q + t;
        if (c > k) ra[c] = fmaf(-la, u[t], ra[c]);
      }
    }
    // column k is done: row `lane` keeps its multiplier there
    ra[k] = la;
    if (k < kSpreadSteps) {
      // rows 32..35: column k sits on lane k % 8 of each group, register k / 8
      const float lb = __shfl_sync(0xffffffffu, rb[k >> 3], k & 7, 8) * inv;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (8 * m + 7 > k) {
          const int c = sub + 8 * m;
          if (c > k) rb[m] = fmaf(-lb, U_s[(k & 7) * kCondLd + c], rb[m]);
        }
      }
      if (k == sub) lbk = lb;   // row r2's multiplier of column k, kept by lane sub
    }
    if (k == kSpreadSteps - 1) {
      // The lanes of the first pivot rows are free now: rows 32..35 move into
      // them (the row's remaining columns from its group's registers, its
      // multipliers so far from lbk) and take part in the row updates from
      // here on.  The pivot rows' own multipliers go to L first (phase B
      // reads them).
      int gm = -1;
#pragma unroll
      for (int j = 0; j < kSpreadSteps; ++j)
        if (perm_s[j] == lane) gm = j;
      if (gm >= 0) {
        float4* d4 = reinterpret_cast<float4*>(L_s + lane * kCondLd);
#pragma unroll
        for (int q = 0; q < 6; ++q) d4[q] = make_float4(ra[4 * q], ra[4 * q + 1], ra[4 * q + 2], ra[4 * q + 3]);
      }
      const int src = (gm >= 0 ? gm : 0) * 8;
#pragma unroll
      for (int c = 0; c < 24; ++c) {
        const float v = c < kSpreadSteps ? __shfl_sync(0xffffffffu, lbk, src + c)
                                         : __shfl_sync(0xffffffffu, rb[c >> 3], src + (c & 7));
        if (gm >= 0) ra[c] = v;
      }
      if (gm >= 0) {
        live = 1.0f;
        myrow = 32 + gm;
      }
    }
    if ((k & 7) == 7) {
      // the ring is full: rows k - 7 .. k to the recovery rows (at and right
      // of the diagonal chunk) with 1/pivot
      const int k0 = k - 7;
      for (int e = lane; e < 48; e += 32) {   // eight consecutive lanes: one chunk of the eight rows
        const int q = e >> 3, kk = k0 + (e & 7);
        if (q >= kk / 4)
          reinterpret_cast<float4*>(rec)[q * 24 + kk] = reinterpret_cast<const float4*>(U_s + (kk & 7) * kCondLd)[q];
      }
      if (lane < 8) inv_s[k0 + lane] = inv_keep;
      __syncwarp();
    }
  }
  if (bad && lane == 0) w.ns[node].singular = 1;
  // multipliers to L (a pivot row's entries from its own step on are never
  // read; the first pivot rows were stored when rows 32..35 moved in)
  {
    float4* d4 = reinterpret_cast<float4*>(L_s + myrow * kCondLd);
#pragma unroll
    for (int q = 0; q < 6; ++q) d4[q] = make_float4(ra[4 * q], ra[4 * q + 1], ra[4 * q + 2], ra[4 * q + 3]);
  }
  __syncwarp();

  // ---- phase B: passive columns
  float* cond = static_cast<float*>(w.Cond) + blk * kBlk;
  const bool col = lane < 25;
  const int cl = col ? lane : 0;
  float Q[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    const int pk = perm_s[k];
    // two partial sums (even and odd j) to halve the dependent chain
    float x = P_s[pk * kCondLd + cl], y = 0.0f;
    const float4* l4 = reinterpret_cast<const float4*>(L_s + pk * kCondLd);
#pragma unroll
    for (int q = 0; q < (k + 3) / 4; ++q) {
      const float4 lv = l4[q];
      const float l[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (4 * q + t < k) {
          if (t & 1) y = fmaf(-l[t], Q[4 * q + t], y);
          else x = fmaf(-l[t], Q[4 * q + t], x);
        }
      }
    }
    x += y;
    Q[k] = x;
  }
#pragma unroll 4
  for (int r = 24; r < 36; ++r) {
    float f = P_s[r * kCondLd + cl];
    const float4* l4 = reinterpret_cast<const float4*>(L_s + r * kCondLd);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float4 lv = l4[q];
      f = fmaf(-lv.x, Q[4 * q], f);
      f = fmaf(-lv.y, Q[4 * q + 1], f);
      f = fmaf(-lv.z, Q[4 * q + 2], f);
      f = fmaf(-lv.w, Q[4 * q + 3], f);
    }
    if (lane < kBlkLd) cond[(r - 24) * kBlkLd + lane] = col ? f : 0.0f;   // pad zeroed: whole sectors
  }
  // the passive parts Q_k and 1/pivot to the stored rows: through P's rows
  // 0..23 (read for the last time in the Q loop) so that the stores of each
  // chunk are contiguous (rec_at)
  float* T_s = P_s;   // [24][kCondLd]: row k = Q_k (columns 24..48 of the stored row)
  __syncwarp();
  if (col) {
#pragma unroll
    for (int k = 0; k < 24; ++k) T_s[k * kCondLd + lane] = Q[k];
  }
  __syncwarp();
  float4* rec4 = reinterpret_cast<float4*>(rec);
  for (int e = lane; e < 24 * 6; e += 32) {   // chunks 6..11 (columns 24..47), 24 rows each
    const int q = e / 24, k = e - 24 * q;
    rec4[(6 + q) * 24 + k] = *reinterpret_cast<const float4*>(T_s + k * kCondLd + 4 * q);
  }
  if (lane < 24)   // chunk 12: column 48 (rhs) and 49 (1/pivot)
    rec4[12 * 24 + lane] = make_float4(T_s[lane * kCondLd + 24], inv_s[lane], 0.0f, 0.0f);
  __syncwarp();   // the tables are reused by the warp's next interval
}

// W warps (intervals) per block, a shape the autotuner picks among 2, 4, 8;
// 24 / W blocks per SM keep 24 warps resident at 80 registers whatever W.
template <int W>
__global__ void __launch_bounds__(32 * W, 24 / W) k_condense_reg(SolveArgs a, Workspace w) {
  __shared__ __align__(16) float sm[W][kCondSmemFloats];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t wid = blockIdx.x * int64_t(W) + warp;
  if (wid >= a.n * a.Nmax) return;
  const int64_t node = wid / a.Nmax;
  const int i = static_cast<int>(wid % a.Nmax);
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  if (i >= N) return;
  condense_interval_reg(a, w, node, i, N, lane, sm[warp]);
}

// The FP32 condensation kernel and its block size for a given shape.
inline void (*condense_reg_kernel(int cond_warps))(SolveArgs, Workspace) {
  return cond_warps == 2 ? k_condense_reg<2> : (cond_warps == 8 ? k_condense_reg<8> : k_condense_reg<4>);
}
inline int condense_reg_warps(int cond_warps) { return cond_warps == 2 || cond_warps == 8 ? cond_warps : 4; }

// Shared-memory FP64 form (used by the FP64 solve): the 36 x 49 system of one
// interval in shared memory, one warp per interval, elimination of the first
// 24 columns with partial pivoting over all 36 rows (warp_eliminate).
constexpr int kCondWarps = 4;
__device__ __forceinline__ void condense_interval_smem(const SolveArgs& a, const Workspace& w, int64_t node,
                                                       int i, int N, int lane, double* M) {
  const int64_t wid = node * a.Nmax + i;
  const double h = a.T[node] / N;
  const int64_t pbase = node * npts(a.Nmax) + 3 * int64_t(i);
  const double* J = static_cast<const double*>(w.Jm) + pbase * 144;
  const double* res = static_cast<const double*>(w.Res) + wid * kResRows;
  double cf[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) cf[k][j] = -h * kLobA[k][j];
  for (int e = lane; e < 36 * 48; e += 32) {
    const int r = e / 48, c = e % 48;
    const int k = r / 12 + 1, comp = r % 12;
    int j, cc;
    if (c < 24) {
      j = c / 12 + 1;
      cc = c % 12;
    } else if (c < 36) {
      j = 0;
      cc = c - 24;
    } else {
      j = 3;
      cc = c - 36;
    }
    double v = cf[k][j] * J[j * 144 + comp * 12 + cc];
    if (comp == cc) {
      if (j == k) v += 1.0;
      if (j == 0) v -= 1.0;
    }
    M[r * kCols + c] = v;
  }
  for (int r = lane; r < 36; r += 32) M[r * kCols + 48] = -res[r];
  __syncwarp();
  const bool ok = warp_eliminate<double, 36, kCols, 24>(M, lane);
  if (!ok && lane == 0) w.ns[node].singular = 1;
  const int64_t blk = node * a.Nmax + i;
  double* rec = static_cast<double*>(w.Rec) + blk * kRec;
  for (int e = lane; e < 24 * kCols; e += 32) rec[(e / kCols) * kRecLd + e % kCols] = M[e];
  if (lane < 24) {
    const double pv = M[lane * kCols + lane];
    rec[lane * kRecLd + kRecInv] = (pv != 0.0 && isfinite(pv)) ? recip_rn(pv) : 0.0;
  }
  double* cond = static_cast<double*>(w.Cond) + blk * kBlk;
  for (int e = lane; e < 12 * 25; e += 32) {
    const int r = e / 25, c = e % 25;
    cond[r * kBlkLd + c] = M[(24 + r) * kCols + 24 + c];
  }
  __syncwarp();
}

__global__ void __launch_bounds__(32 * kCondWarps) k_condense_smem(SolveArgs a, Workspace w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wid = blockIdx.x * int64_t(kCondWarps) + warp;
  if (wid >= a.n * a.Nmax) return;
  const int64_t node = wid / a.Nmax;
  const int i = static_cast<int>(wid % a.Nmax);
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  if (i >= N) return;
  condense_interval_smem(a, w, node, i, N, lane, reinterpret_cast<double*>(smem_raw) + warp * (36 * kCols));
}

// ---------------------------------------------------------------- staircase
// Register-resident staircase elimination: warp per node, lanes 0..17 hold the
// 18 rows of the current panel [carry (6) ; block row i (12)] over the 25
// columns [y_i (12) | y_{i+1} (12) | rhs].  Twelve pivot steps leave 12 pivot
// rows (stored in pivot order, 1/pivot on the diagonal) and 6 rows that carry
// y_{i+1} into the next panel.  The next block row is prefetched into lanes
// 0..11 while the current panel is eliminated.  The lambda(T) rows close the
// system; back substitution then runs from the last mesh point to the first.
//
// The blocks may be the N interval block rows of the node (pt_stride = 3:
// block i couples mesh points 3i and 3i + 3) or the reduced block rows of the
// segmented form (block s couples the segment ends, pt_stride = 3 x segment
// length); the last block always ends at mesh point 3N.
template <typename T>
__device__ __forceinline__ bool abd_staircase(const SolveArgs& a, const Workspace& w, int64_t node, int N,
                                              const T* __restrict__ cond, int nblk, int pt_stride,
                                              T* __restrict__ abd, int lane) {
  const int64_t pb = node * npts(a.Nmax);
  const double* Y = (w.ns[node].ybuf ? w.Y2 : w.Y) + pb * 12;
  const double* x0 = a.x0 + node * 6;
  double* D = w.D + pb * 12;
  const bool rowlane = lane < 18;
  const unsigned lt_mask = (1u << lane) - 1u;
  T r[25], nx[25];
#pragma unroll
  for (int c = 0; c < 25; ++c) {
    r[c] = T(0);
    nx[c] = T(0);
  }
  if (lane < 6) {
    // x(0) - x0 = 0 linearised: [I 0] dy_0 = -(x(0) - x0)
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (c == lane) r[c] = T(1);
    r[24] = T(-(Y[lane] - x0[lane]));
  } else if (rowlane) {
    load_row25<T>(cond + (lane - 6) * kBlkLd, r);
  }
  bool ok = true;
  bool done = false;
  int rank = 0;
  int plane[12];
  for (int i = 0; i < nblk; ++i) {
    if (i + 1 < nblk && lane < 12) load_row25<T>(cond + int64_t(i + 1) * kBlk + lane * kBlkLd, nx);
    done = false;
    int my_step = -1;
    panel_eliminate12<T>(r, rowlane, done, my_step, plane, ok, lane);
    if (done) store_row25<T>(abd + int64_t(i) * kBlk + my_step * kBlkLd, r);
    rank = __popc(__ballot_sync(0xffffffffu, done) & lt_mask);
    // next panel: carry rows shift y_{i+1} into the first block; the pivot
    // lanes take the prefetched block row i+1, in lane order
#pragma unroll
    for (int c = 0; c < 25; ++c) {
      const T v = __shfl_sync(0xffffffffu, nx[c], rank & 15);
      if (done) {
        r[c] = v;
      } else if (c < 12) {
        r[c] = r[c < 12 ? c + 12 : c];
      } else if (c < 24) {
        r[c] = T(0);
      }
    }
  }
  // closing rows: lambda(T) - grad h(x(T)) = 0, taken by pivot lanes of rank
  // 0..5 (the other pivot lanes sit out); the carry lanes hold the rest
  const double* yN = Y + 3 * int64_t(N) * 12;
  if (done) {
#pragma unroll
    for (int c = 0; c < 25; ++c) r[c] = T(0);
    if (rank < 6) {
#pragma unroll
      for (int c = 0; c < 6; ++c) r[c] = T(-terminal_hess(a.P, rank, c));
#pragma unroll
      for (int c = 0; c < 6; ++c)
        if (c == rank) r[6 + c] = T(1);
      r[24] = T(-(yN[6 + rank] - terminal_grad(a.P, yN, rank)));
    }
  }
  {
    const bool cand = rowlane && (!done || rank < 6);
    bool done2 = false;
    int my2 = -1;
    panel_eliminate12<T>(r, cand, done2, my2, plane, ok, lane);
  }
  // back substitution of the closing system: dy_N (uniform across lanes)
  T dy[12];
  {
    T t = r[24];
#pragma unroll
    for (int k = 11; k >= 0; --k) {
      const T dk = __shfl_sync(0xffffffffu, t * r[k], plane[k]);
      dy[k] = dk;
      t = fma(-r[k], dk, t);
    }
  }
  if (lane < 12) {
    T mine = T(0);
#pragma unroll
    for (int c = 0; c < 12; ++c)
      if (c == lane) mine = dy[c];
    D[3 * int64_t(N) * 12 + lane] = double(mine);
  }
  // backward sweep: lane k holds the stored pivot row of step k of interval ii:
  // U (cols k..11, 1/pivot at k), V (cols 12..23), rhs (24)
  T row[25], pre[25];
#pragma unroll
  for (int c = 0; c < 25; ++c) {
    row[c] = T(0);
    pre[c] = T(0);
  }
  if (lane < 12) load_row25<T>(abd + int64_t(nblk - 1) * kBlk + lane * kBlkLd, row);
  for (int ii = nblk - 1; ii >= 0; --ii) {
    if (ii > 0 && lane < 12) load_row25<T>(abd + int64_t(ii - 1) * kBlk + lane * kBlkLd, pre);
    T tt = row[24];
#pragma unroll
    for (int c = 0; c < 12; ++c) tt = fma(-row[12 + c], dy[c], tt);
#pragma unroll
    for (int k = 11; k >= 0; --k) {
      const T dk = __shfl_sync(0xffffffffu, tt * row[k], k);
      dy[k] = dk;
      tt = (lane < k) ? fma(-row[k], dk, tt) : tt;
    }
    if (lane < 12) {
      T mine = T(0);
#pragma unroll
      for (int c = 0; c < 12; ++c)
        if (c == lane) mine = dy[c];
      D[int64_t(ii) * pt_stride * 12 + lane] = double(mine);
    }
#pragma unroll
    for (int c = 0; c < 25; ++c) row[c] = pre[c];
  }
  return ok;
}

// The whole staircase of one node over its N interval block rows.
template <typename T>
__device__ __forceinline__ bool abd_node_reg(const SolveArgs& a, const Workspace& w, int64_t node, int N,
                                             int lane) {
  const T* cond = static_cast<const T*>(w.Cond) + node * a.Nmax * int64_t(kBlk);
  T* abd = static_cast<T*>(w.Abd) + node * a.Nmax * int64_t(kBlk);
  return abd_staircase<T>(a, w, node, N, cond, N, 3, abd, lane);
}

// ---------------------------------------------------------------- segmented staircase
// The serial chain of the staircase is N panels long.  The segmented form
// cuts the mesh of a node into segments of kSegLen intervals and runs three
// kernels:
//   k_abd_seg      warp per (node, segment): eliminates the segment's interior
//                  mesh points.  A panel holds the 12 carry rows [F | G | r]
//                  (coupling the segment's first point y_a with y_i) and the
//                  block row i [0 | S_i | T_i | r_i]; twelve pivot steps with
//                  partial pivoting over all 24 rows remove y_i, leave 12
//                  pivot rows [F | U | V | r] (1/pivot on U's diagonal) and 12
//                  new carry rows on (y_a, y_{i+1}).  After the last panel the
//                  carry rows are the segment's reduced block row on
//                  (y_a, y_b), in the same 12 x 25 format as a block row.
//   k_abd_red      warp per node: the staircase over the reduced block rows
//                  and the boundary rows gives the segment ends.
//   k_abd_segback  warp per (node, segment): back substitution through the
//                  stored pivot rows for the interior mesh points.
// This is Gaussian elimination with partial pivoting restricted to the block
// rows of a segment, the structured pairwise reduction of block rows of
// Wright (SIAM J. Sci. Stat. Comput. 13, 1992) taken sequentially inside a
// segment; the chain becomes kSegLen + N / kSegLen panels.
//
// Each panel runs in two phases, like the condensation:
//   phase A (rows on lanes): lane r < 24 holds the 12 y_i entries of panel
//   row r in registers.  Partial pivoting over the 24 rows; at step k the
//   pivot lane writes its row (1/pivot on the diagonal) to the table U and
//   every row keeps its multiplier l(r, k) in the eliminated column, stored
//   to L at the end.
//   phase B (columns on lanes): lane c < 25 owns passive column c of
//   [F | Z | rhs].  With the pivot order p_k the passive part of pivot row k
//   is Q_k = P(p_k) - sum_{j<k} l(p_k, j) Q_j, and a carry row r leaves as
//   P(r) - sum_k l(r, k) Q_k.
// The panel rows live in shared memory between panels: their passive parts
// in P and their y_i parts in Y.  Carry rows move Z into Y; the slots of the
// pivot rows take block row i + 1.
template <typename T>
__host__ __device__ constexpr int seg_warps() { return sizeof(T) == 4 ? 4 : 2; }   // warps per block
constexpr int kSegP = 25;   // row stride of the passive table P
// P, Y, L, U and the staged block row (elements), then 32 ints (pivot slots, carry slots)
constexpr int kSegSmem = 24 * kSegP + 24 * 12 + 24 * 12 + 12 * 12 + 12 * kBlkLd;
template <typename T>
__host__ __device__ constexpr int seg_smem_elems() { return kSegSmem + 32 * 4 / int(sizeof(T)); }

template <typename T>
__device__ __forceinline__ void load_row12(const T* __restrict__ src, T (&r)[12]) {
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 v = s4[q];
      r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double2 v = s2[q];
      r[2 * q] = v.x; r[2 * q + 1] = v.y;
    }
  }
}

// 16-byte vectors q < nq of a 12-entry row (the rest left unset)
template <typename T>
__device__ __forceinline__ void load_row12_upto(const T* __restrict__ src, T (&r)[12], int nq) {
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q < nq) {
        const float4 v = s4[q];
        r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
      }
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (q < nq) {
        const double2 v = s2[q];
        r[2 * q] = v.x; r[2 * q + 1] = v.y;
      }
    }
  }
}

// 16-byte vectors q >= q0 of a 12-entry row
template <typename T>
__device__ __forceinline__ void store_row12_from(T* __restrict__ dst, const T (&r)[12], int q0) {
  if constexpr (sizeof(T) == 4) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (q >= q0) d4[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
  } else {
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (q >= q0) d2[q] = make_double2(r[2 * q], r[2 * q + 1]);
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * seg_warps<T>()) k_abd_seg(SolveArgs a, Workspace w) {
  constexpr int W = seg_warps<T>();
  constexpr int V = 16 / int(sizeof(T));   // entries per 16-byte vector
  __shared__ __align__(16) T sm[W][seg_smem_elems<T>()];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int smax = seg_count(a.Nmax);
  const int64_t wid = blockIdx.x * int64_t(W) + warp;
  const int64_t node = wid / smax;
  const int s = static_cast<int>(wid % smax);
  if (node >= a.n) return;
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  if (s >= seg_count(N)) return;
  const int i0 = s * kSegLen;
  const int i1 = i0 + kSegLen < N ? i0 + kSegLen : N;
  T* P_s = sm[warp];                  // [24][kSegP] passive parts [F | Z | rhs] of the panel rows
  T* Y_s = P_s + 24 * kSegP;          // [24][12] y_i parts
  T* L_s = Y_s + 24 * 12;             // [24][12] multipliers l(r, k)
  T* U_s = L_s + 24 * 12;             // [12][12] pivot rows (y_i part), 1/pivot on the diagonal
  T* stage = U_s + 12 * 12;           // [12][kBlkLd] block row i + 1
  int* perm_s = reinterpret_cast<int*>(stage + 12 * kBlkLd);   // [12] slot of the pivot row of step k
  int* cslot_s = perm_s + 16;                                   // [12] carry slots in lane order
  const T* cond = static_cast<const T*>(w.Cond) + node * a.Nmax * int64_t(kBlk);
  T* seg = static_cast<T*>(w.Seg) + node * a.Nmax * int64_t(kSegBlk);
  T* red = static_cast<T*>(w.Red) + (node * smax + s) * int64_t(kBlk);
  const unsigned lt_mask = (1u << lane) - 1u;
  const bool col = lane < 25;               // phase B: passive column c = F (0..11), Z (12..23), rhs (24)
  const int c = col ? lane : 0;
  const int segc = c < 12 ? c : c + 12;     // its column in a stored pivot row [F | U | V | rhs]

  const T* b0 = cond + int64_t(i0) * kBlk;
  if (i0 + 1 >= i1) {   // a one-interval segment: its block row is the reduced row
    for (int e = lane; e < kBlk; e += 32) red[e] = b0[e];
    return;
  }
  // panel rows: slots 0..11 = block row i0 = [F = S | Y = T | Z = 0 | r],
  // slots 12..23 = block row i0 + 1 = [F = 0 | Y = S | Z = T | r]
  const T* b1 = b0 + kBlk;
  if (col) {
#pragma unroll 4
    for (int r = 0; r < 12; ++r) {
      P_s[r * kSegP + c] = c < 12 ? b0[r * kBlkLd + c] : (c < 24 ? T(0) : b0[r * kBlkLd + 24]);
      P_s[(12 + r) * kSegP + c] = c < 12 ? T(0) : b1[r * kBlkLd + c];
    }
  }
  if (lane < 24) {
    T y[12];
    load_row12<T>(lane < 12 ? b0 + lane * kBlkLd + 12 : b1 + (lane - 12) * kBlkLd, y);
    store_row12_from<T>(Y_s + lane * 12, y, 0);
  }
  __syncwarp();

  const unsigned itag = 31u - unsigned(lane);
  bool bad = false;
  for (int i = i0 + 1; i < i1; ++i) {
    const bool more = i + 1 < i1;
    if (more) {   // block row i + 1 to the stage (asynchronous copy)
      const char* src = reinterpret_cast<const char*>(cond + int64_t(i + 1) * kBlk);
      for (int e = lane; e < 12 * kBlkLd * int(sizeof(T)) / 16; e += 32)
        cp_async16(reinterpret_cast<char*>(stage) + 16 * e, src + 16 * e);
      cp_async_commit();
    }
    // ---- phase A
    T ya[12];
    if (lane < 24) {
      load_row12<T>(Y_s + lane * 12, ya);
    } else {
#pragma unroll
      for (int t = 0; t < 12; ++t) ya[t] = T(0);
    }
    // pivot key: magnitude with the low 5 bits replaced by a lane tag (ties
    // to the lower lane); rows that are no candidates have zero mask and tag
    unsigned kmask = lane < 24 ? ~31u : 0u;
    unsigned ktag = lane < 24 ? itag : 0u;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int q0 = k / V;
      const unsigned key = (mag_key(ya[k]) & kmask) | ktag;
      const unsigned best = __reduce_max_sync(0xffffffffu, key);
      if (key == best) {   // candidates' keys are nonzero and differ in the tag; the others are 0
        if constexpr (sizeof(T) == sizeof(double)) {   // FP64: the pivot lane publishes 1/pivot
          const T piv = ya[k];
          const bool good = piv != T(0) && isfinite(piv);
          bad = bad || !good;
          ya[k] = good ? recip_rn(piv) : T(0);
        }
        store_row12_from<T>(U_s + k * 12, ya, q0);
        perm_s[k] = lane;
        kmask = 0u;
        ktag = 0u;
      }
      __syncwarp();
      const T* u = U_s + k * 12;
      T inv = u[k];
      if constexpr (sizeof(T) == sizeof(float)) {
        // FP32: the row is published with its raw pivot and every lane forms
        // the same 1/pivot (off the pivot lane's path)
        bool good;
        inv = pivot_recip(inv, good);
        bad = bad || !good;
      }
      // (lanes that are no candidate update rows whose entries from here on
      // are never read)
      const T la = ya[k] * inv;
#pragma unroll
      for (int q = q0; q < 12 / V; ++q) {
        T uv[V];
        if constexpr (sizeof(T) == 4) {
          const float4 v4 = reinterpret_cast<const float4*>(u)[q];
          uv[0] = v4.x; uv[1] = v4.y; uv[2] = v4.z; uv[3] = v4.w;
        } else {
          const double2 v2 = reinterpret_cast<const double2*>(u)[q];
          uv[0] = v2.x; uv[1] = v2.y;
        }
#pragma unroll
        for (int t = 0; t < V; ++t) {
          const int cc = V * q + t;
          if (cc > k) ya[cc] = fma(-la, uv[t], ya[cc]);
        }
      }
      ya[k] = la;   // column k is done: the row keeps its multiplier there
    }
    if (lane < 24) store_row12_from<T>(L_s + lane * 12, ya, 0);   // a pivot row's entries from its step on are never read
    if constexpr (sizeof(T) == sizeof(float)) {
      if (lane < 12) {   // 1/pivot on the diagonal of the stored rows (formed again: the same value)
        bool gd;
        U_s[lane * 12 + lane] = pivot_recip(U_s[lane * 12 + lane], gd);
      }
    }
    const unsigned cmask = __ballot_sync(0xffffffffu, ktag != 0u);   // the 12 rows that were no pivot
    if (ktag != 0u) cslot_s[__popc(cmask & lt_mask)] = lane;
    __syncwarp();

    // ---- phase B
    T* segp = seg + int64_t(i) * 12 * kSegLd;
    T Q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int pk = perm_s[k];
      T x = P_s[pk * kSegP + c], y = T(0);
      T l[12];
      load_row12_upto<T>(L_s + pk * 12, l, (k + V - 1) / V);
#pragma unroll
      for (int j = 0; j < k; ++j) {
        if (j & 1) y = fma(-l[j], Q[j], y);
        else x = fma(-l[j], Q[j], x);
      }
      x += y;
      Q[k] = x;
      if (col) segp[k * kSegLd + segc] = x;
    }
    // y_i part of the pivot rows (1/pivot on the diagonal; left of it unread)
    for (int e = lane; e < 12 * (12 / V); e += 32) {
      const int k = e / (12 / V), q = e % (12 / V);
      if (q >= k / V)
        reinterpret_cast<float4*>(segp + k * kSegLd + 12)[q] = reinterpret_cast<const float4*>(U_s + k * 12)[q];
    }
    const bool zcol = c >= 12 && c < 24;
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      const int r = cslot_s[m];
      T f = P_s[r * kSegP + c], g = T(0);
      T l[12];
      load_row12<T>(L_s + r * 12, l);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        if (k & 1) g = fma(-l[k], Q[k], g);
        else f = fma(-l[k], Q[k], f);
      }
      f += g;
      if (more) {
        // Z moves into the y_i slot
        if (col) P_s[r * kSegP + c] = zcol ? T(0) : f;
        if (zcol) Y_s[r * 12 + c - 12] = f;
      } else if (col) {
        red[m * kBlkLd + c] = f;   // last panel: the carry rows are the reduced row [F | Y | rhs]
      }
    }
    if (more) {   // the pivot slots take block row i + 1 = [0 | S | T | r]
      cp_async_wait_all();   // this lane's part of the stage has landed
      __syncwarp();          // ... and every lane's
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int slot = perm_s[k];
        if (col) P_s[slot * kSegP + c] = c < 12 ? T(0) : stage[k * kBlkLd + c];
        if (lane < 12) Y_s[slot * 12 + lane] = stage[k * kBlkLd + lane];
      }
    }
    __syncwarp();   // tables written before the next panel reads them
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) w.ns[node].singular = 1;
}

template <typename T>
__global__ void __launch_bounds__(128) k_abd_red(SolveArgs a, Workspace w) {
  const int lane = threadIdx.x & 31;
  const int64_t node = blockIdx.x * int64_t(4) + (threadIdx.x >> 5);
  if (node >= a.n) return;
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  const int smax = seg_count(a.Nmax);
  const T* red = static_cast<const T*>(w.Red) + node * smax * int64_t(kBlk);
  T* abd = static_cast<T*>(w.Abd) + node * a.Nmax * int64_t(kBlk);
  const bool ok = abd_staircase<T>(a, w, node, N, red, seg_count(N), 3 * kSegLen, abd, lane);
  if (!ok && lane == 0) w.ns[node].singular = 1;
}

template <typename T>
__global__ void __launch_bounds__(128) k_abd_segback(SolveArgs a, Workspace w) {
  // the pivot rows of panel i - 1 are copied to shared memory (asynchronously)
  // while panel i is substituted
  __shared__ __align__(16) T buf_s[4][2][12 * kSegLd];
  const int lane = threadIdx.x & 31;
  const int smax = seg_count(a.Nmax);
  const int64_t wid = blockIdx.x * int64_t(4) + (threadIdx.x >> 5);
  const int64_t node = wid / smax;
  const int s = static_cast<int>(wid % smax);
  if (node >= a.n) return;
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  if (s >= seg_count(N)) return;
  const int i0 = s * kSegLen;
  const int i1 = i0 + kSegLen < N ? i0 + kSegLen : N;
  if (i1 - i0 < 2) return;
  double* D = w.D + node * npts(a.Nmax) * 12;
  const T* seg = static_cast<const T*>(w.Seg) + node * a.Nmax * int64_t(kSegBlk);
  T dya[12], dyn[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    dya[c] = T(D[3 * int64_t(i0) * 12 + c]);
    dyn[c] = T(D[3 * int64_t(i1) * 12 + c]);
  }
  T (*buf)[12 * kSegLd] = buf_s[threadIdx.x >> 5];
  auto fetch = [&](int i, int b) {   // panel i's 12 pivot rows to buf[b]
    const char* src = reinterpret_cast<const char*>(seg + int64_t(i) * 12 * kSegLd);
    for (int e = lane; e < 12 * kSegLd * int(sizeof(T)) / 16; e += 32)
      cp_async16(reinterpret_cast<char*>(buf[b]) + 16 * e, src + 16 * e);
    cp_async_commit();
  };
  fetch(i1 - 1, 0);
  for (int i = i1 - 1, b = 0; i > i0; --i, b ^= 1) {
    cp_async_wait_all();   // panel i has landed (this lane's part) ...
    __syncwarp();          // ... and every lane's; buf[b ^ 1] was read in the last pass
    if (i - 1 > i0) fetch(i - 1, b ^ 1);
    // lane k holds pivot row k of panel i: [F | U (1/pivot at k) | V | rhs]
    T r[37];
#pragma unroll
    for (int c = 0; c < 37; ++c) r[c] = T(0);
    if (lane < 12) {
      T row[40];
      load_row40<T>(buf[b] + lane * kSegLd, row);
#pragma unroll
      for (int c = 0; c < 37; ++c) r[c] = row[c];
    }
    T tt = r[36];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      tt = fma(-r[c], dya[c], tt);
      tt = fma(-r[24 + c], dyn[c], tt);
    }
#pragma unroll
    for (int k = 11; k >= 0; --k) {
      const T dk = __shfl_sync(0xffffffffu, tt * r[12 + k], k);
      dyn[k] = dk;
      tt = (lane < k) ? fma(-r[12 + k], dk, tt) : tt;
    }
    if (lane < 12) {
      T mine = T(0);
#pragma unroll
      for (int c = 0; c < 12; ++c)
        if (c == lane) mine = dyn[c];
      D[3 * int64_t(i) * 12 + lane] = double(mine);
    }
  }
}

// Interior-stage corrections from the stored condensation pivot rows: lane
// k < 24 holds pivot row k = [U_k (interior, pivot at k) | Q_k (y_i, y_{i+1},
// rhs) | 1/pivot at column 49] in registers.  acc_k = rhs_k - Q_k [dy_i;
// dy_{i+1}], then back substitution through U by shuffles.
template <typename T>
__device__ __forceinline__ void recover_interval(const SolveArgs& a, const Workspace& w, int64_t node, int i,
                                                 int lane) {
  const int64_t wid = node * a.Nmax + i;
  const T* rec = static_cast<const T*>(w.Rec) + wid * kRec;
  double* D = w.D + (node * npts(a.Nmax) + 3 * int64_t(i)) * 12;
  const T dyl = lane < 12 ? T(D[lane]) : T(0);
  const T dyr = lane < 12 ? T(D[36 + lane]) : T(0);
  // the part of row k left of its diagonal is never read (the FP32
  // condensation does not store it)
  T row[kRecLd];
#pragma unroll
  for (int c = 0; c < kRecLd; ++c) row[c] = T(0);
  if (lane < 24) {
    if constexpr (sizeof(T) == 4) {
      const float4* s4 = reinterpret_cast<const float4*>(rec) + lane;   // chunk-major (rec_at)
#pragma unroll
      for (int q = 0; q < kRecLd / 4; ++q) {
        if (4 * q + 3 < lane) continue;
        const float4 v = s4[q * 24];
        row[4 * q] = v.x; row[4 * q + 1] = v.y; row[4 * q + 2] = v.z; row[4 * q + 3] = v.w;
      }
    } else {
      const double2* s2 = reinterpret_cast<const double2*>(rec + lane * kRecLd);
#pragma unroll
      for (int q = 0; q < kRecLd / 2; ++q) {
        if (2 * q + 1 < lane) continue;
        const double2 v = s2[q];
        row[2 * q] = v.x; row[2 * q + 1] = v.y;
      }
    }
  }
  T acc = row[48];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const T l = __shfl_sync(0xffffffffu, dyl, c);
    const T r = __shfl_sync(0xffffffffu, dyr, c);
    acc = fma(-row[24 + c], l, acc);
    acc = fma(-row[36 + c], r, acc);
  }
  T x = T(0);
#pragma unroll
  for (int c = 23; c >= 0; --c) {
    const T xc = __shfl_sync(0xffffffffu, acc * row[kRecInv], c);
    if (lane == c) x = xc;
    acc = lane < c ? fma(-row[c], xc, acc) : acc;
  }
  if (lane < 24) D[12 + lane] = double(x);   // points 3i+1 and 3i+2 are contiguous
}

template <typename T>
__global__ void k_recover(SolveArgs a, Workspace w) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wid = blockIdx.x * int64_t(4) + warp;
  if (wid >= a.n * a.Nmax) return;
  const int64_t node = wid / a.Nmax;
  const int i = static_cast<int>(wid % a.Nmax);
  if (!w.ns[node].active) return;
  if (i >= a.N[node]) return;
  recover_interval<T>(a, w, node, i, lane);
}

// ---------------------------------------------------------------- update
__global__ void k_ls_begin(SolveArgs a, Workspace w) {
  const int64_t node = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (node >= a.n) return;
  NodeState s = w.ns[node];
  if (!s.active) return;
  if (s.singular) {
    s.status = SG_SINGULAR;
    s.active = 0;
  } else {
    s.searching = 1;
    s.alpha = 1.0;
  }
  w.ns[node] = s;
}

// Y += alpha D, a thread per pair of components (consecutive threads touch
// consecutive 16-byte words).
constexpr int kUpdPer = 6;   // threads per collocation point
__global__ void k_update(SolveArgs a, Workspace w) {
  const int64_t P = npts(a.Nmax);
  const int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (u >= a.n * P * kUpdPer) return;
  const int64_t t = u / kUpdPer;
  const int64_t node = t / P;
  if (!w.ns[node].active) return;
  if (t % P > 3 * int64_t(a.N[node])) return;
  const double alpha = w.ns[node].alpha;
  double2* y2 = reinterpret_cast<double2*>(w.Y) + u;
  const double2 d = reinterpret_cast<const double2*>(w.D)[u];
  const double2 y = *y2;
  *y2 = make_double2(__fma_rn(alpha, d.x, y.x), __fma_rn(alpha, d.y, y.y));
}

__global__ void k_after_update(SolveArgs a, Workspace w) {
  const int64_t node = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (node >= a.n) return;
  NodeState s = w.ns[node];
  if (!s.active) return;
  s.iters += 1;
  if (!(s.fmax < INFINITY)) {
    s.status = SG_NONFINITE;
    s.active = 0;
  } else if (s.fmax <= a.tol) {
    s.status = SG_CONVERGED;
    s.active = 0;
  } else if (s.iters >= a.max_iter) {
    s.status = SG_MAXITER;
    s.active = 0;
  } else {
    atomicAdd(&w.counters[1], 1);
  }
  w.ns[node] = s;
}

// Outputs (Eq. optuv): lambda(0), u*(x0, lambda(0)), V = z(T) + h(x(T)) with
// z(T) = h sum_i sum_j b_j L(Y_ij) (the Lobatto IIIA step of z' = L).  One
// warp per node; the results go to output row `row`.
__device__ __forceinline__ void node_outputs(const SolveArgs& a, const Workspace& w, int64_t node, int64_t row,
                                             int lane, double* lambda0, double* u0, double* V, int32_t* status,
                                             int32_t* iters) {
  const NodeState s = w.ns[node];
  const double* Y = (s.ybuf ? w.Y2 : w.Y) + node * npts(a.Nmax) * 12;
  if (s.status == SG_BADINPUT) {
    if (lane == 0) {
      for (int c = 0; c < 6; ++c) lambda0[row * 6 + c] = NAN;
      for (int c = 0; c < 3; ++c) u0[row * 3 + c] = NAN;
      V[row] = NAN;
      status[row] = s.status;
      iters[row] = 0;
    }
    return;
  }
  const int N = a.N[node];
  const double h = a.T[node] / N;
  double z = 0.0;
  for (int i = lane; i < N; i += 32) {
    const double* yi = Y + 3 * int64_t(i) * 12;
    const double* ve = node_target(a.P, node);
    z += h * (kLobB[0] * running_cost(a.P, yi, ve) + kLobB[1] * running_cost(a.P, yi + 12, ve) +
              kLobB[2] * running_cost(a.P, yi + 24, ve) + kLobB[3] * running_cost(a.P, yi + 36, ve));
  }
  z = warp_sum(z);
  if (lane == 0) {
    const double* yN = Y + 3 * int64_t(N) * 12;
    V[row] = z + terminal_cost(a.P, yN);
    double u[3];
    optimal_control(a.P, Y, Y + 6, u);
    for (int c = 0; c < 6; ++c) lambda0[row * 6 + c] = Y[6 + c];
    for (int c = 0; c < 3; ++c) u0[row * 3 + c] = u[c];
    status[row] = s.status;
    iters[row] = s.iters;
  }
}

__global__ void k_outputs(SolveArgs a, Workspace w, double* lambda0, double* u0, double* V,
                          int32_t* status, int32_t* iters) {
  const int lane = threadIdx.x & 31;
  const int64_t node = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (node >= a.n) return;
  node_outputs(a, w, node, node, lane, lambda0, u0, V, status, iters);
}

__global__ void k_copy_Y(SolveArgs a, Workspace w, double* out) {
  const int64_t P = npts(a.Nmax);
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= a.n * P) return;
  const int64_t node = t / P;
  if (t % P > 3 * int64_t(a.N[node])) return;
  const double* Yb = w.ns[node].ybuf ? w.Y2 : w.Y;
#pragma unroll
  for (int c = 0; c < 12; ++c) out[t * 12 + c] = Yb[t * 12 + c];
}

}  // namespace sg
