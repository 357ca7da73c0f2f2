// Step II: the characteristic BVP at every node (Section 3.1, Eq. hamchar),
// four-stage Lobatto IIIA collocation on N equal intervals and damped Newton.
//
// One Newton iteration is five kernels:
//   k_point     F (FP64) and the 12x12 Jacobian dF/dy (precision T) at every
//               collocation point                       thread per (node, point)
//   k_condense  the 36 linearised stage equations of one interval; Gaussian
//               elimination of its two interior stages (24 columns, partial
//               pivoting over all 36 rows) leaves a 12 x 25 block row
//               [S | T | rhs] coupling y_i and y_{i+1}     warp per (node, interval)
//   k_abd       staircase elimination with partial pivoting over
//               [x(0) rows; block rows; lambda(T) rows], then back substitution
//               for the mesh-point corrections               warp per node
//   k_recover   interior-stage corrections from the stored pivot rows
//                                                          warp per (node, interval)
//   k_trial     FP64 residual at Y + alpha D, per interval; k_ls_reduce makes
//               the Armijo decision per node in a fixed reduction order
// T = double gives the FP64 form; T = float the mixed form (FP32 Jacobian,
// elimination and search direction; FP64 residual, line search and update).
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "diag.cuh"
#include "linalg.cuh"
#include "problems.cuh"

namespace sg {

// ---------------------------------------------------------------- tableau
// Four-stage Lobatto IIIA (Hairer & Wanner, Solving ODEs II, Sec. IV.5):
// c = 0, (5 - sqrt5)/10, (5 + sqrt5)/10, 1; b = (1, 5, 5, 1)/12.
#define SG_S5 2.2360679774997896964091736687312762
__constant__ double kLobA[4][4] = {
    {0.0, 0.0, 0.0, 0.0},
    {(11.0 + SG_S5) / 120.0, (25.0 - SG_S5) / 120.0, (25.0 - 13.0 * SG_S5) / 120.0, (-1.0 + SG_S5) / 120.0},
    {(11.0 - SG_S5) / 120.0, (25.0 + 13.0 * SG_S5) / 120.0, (25.0 + SG_S5) / 120.0, (-1.0 - SG_S5) / 120.0},
    {1.0 / 12.0, 5.0 / 12.0, 5.0 / 12.0, 1.0 / 12.0}};
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
  int _pad;
};

constexpr int kCondLd = 49;                 // 24 + 12 + 12 columns + rhs
constexpr int kCondRows = 36;
constexpr int kBlk = 12 * 25;               // condensed / ABD pivot block
constexpr int kRec = 24 * kCondLd;          // stored interior pivot rows
constexpr int kCondWarps = 4;

struct Workspace {
  double* Y;
  double* D;
  double* Fv;
  void* Jm;
  void* Cond;
  void* Rec;
  void* Abd;
  double* part;
  NodeState* ns;
  int* counters;
  size_t bytes;
};

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
  w.Fv = reinterpret_cast<double*>(take(n * P * 12 * sizeof(double)));
  w.Jm = take(n * P * 144 * tsize);
  w.Cond = take(n * int64_t(Nmax) * kBlk * tsize);
  w.Rec = take(n * int64_t(Nmax) * kRec * tsize);
  w.Abd = take(n * int64_t(Nmax) * kBlk * tsize);
  w.part = reinterpret_cast<double*>(take(n * int64_t(Nmax) * 2 * sizeof(double)));
  w.ns = reinterpret_cast<NodeState*>(take(n * sizeof(NodeState)));
  w.counters = reinterpret_cast<int*>(take(256));
  w.bytes = off;
  return w;
}

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
};

__host__ __device__ __forceinline__ int64_t npts(int Nmax) { return 3 * int64_t(Nmax) + 1; }

// ---------------------------------------------------------------- kernels
__global__ void k_init(SolveArgs a, Workspace w) {
  const int64_t P = npts(a.Nmax);
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= a.n * P) return;
  const int64_t node = t / P;
  const int64_t p = t % P;
  const double* x0 = a.x0 + node * 6;
  double* y = w.Y + t * 12;
  double* d = w.D + t * 12;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    y[c] = x0[c];   // x held at x0, lambda = 0 (zero control)
    y[6 + c] = 0.0;
    d[c] = 0.0;
    d[6 + c] = 0.0;
  }
  if (p == 0) {
    NodeState s{};
    const int N = a.N[node];
    const double T = a.T[node];
    bool ok = N >= 1 && N <= a.Nmax && T > 0.0 && T < INFINITY;
    for (int c = 0; c < 6; ++c) ok = ok && isfinite(x0[c]);
    s.fnorm2 = 0.0;
    s.fmax = 0.0;
    s.alpha = 0.0;   // the first residual evaluation is at Y itself
    s.active = ok ? 1 : 0;
    s.searching = ok ? 1 : 0;
    s.singular = 0;
    s.iters = 0;
    s.status = ok ? SG_MAXITER : SG_BADINPUT;
    w.ns[node] = s;
  }
}

// FP64 residual at Y + alpha D for one interval (stage rows 2..4; the first
// interval adds the x(0) rows, the last the lambda(T) rows); writes its
// partial |.|_2^2 and |.|_inf.
__global__ void k_trial(SolveArgs a, Workspace w) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= a.n * a.Nmax) return;
  const int64_t node = t / a.Nmax;
  const int i = static_cast<int>(t % a.Nmax);
  const NodeState& s = w.ns[node];
  if (!s.searching) return;
  const int N = a.N[node];
  if (i >= N) return;
  const double h = a.T[node] / N;
  const double alpha = s.alpha;
  const int64_t base = (node * npts(a.Nmax) + 3 * int64_t(i)) * 12;
  double y[4][12], F[4][12];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int c = 0; c < 12; ++c) y[j][c] = __fma_rn(alpha, w.D[base + 12 * j + c], w.Y[base + 12 * j + c]);
    char_rhs(a.P, y[j], F[j]);
  }
  double ss = 0.0, mx = 0.0;
  bool bad = false;
  auto acc = [&](double r) {
    bad = bad || !isfinite(r);
    ss += r * r;
    mx = fmax(mx, fabs(r));
  };
#pragma unroll
  for (int k = 1; k < 4; ++k) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double r = y[k][c] - y[0][c] -
                 h * (kLobA[k][0] * F[0][c] + kLobA[k][1] * F[1][c] + kLobA[k][2] * F[2][c] +
                      kLobA[k][3] * F[3][c]);
      acc(r);
    }
  }
  if (i == 0) {
    const double* x0 = a.x0 + node * 6;
    for (int c = 0; c < 6; ++c) acc(y[0][c] - x0[c]);
  }
  if (i == N - 1) {
    for (int c = 0; c < 6; ++c) acc(y[3][6 + c] - terminal_grad(a.P, y[3], c));
  }
  if (bad) {
    ss = INFINITY;
    mx = INFINITY;
  }
  w.part[2 * t] = ss;
  w.part[2 * t + 1] = mx;
}

// Warp per node: reduce the partial norms in a fixed order and make the
// decision.  mode 0: initial residual (convergence test at iteration 0);
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
    } else {
      s.alpha *= 0.5;
      atomicAdd(&w.counters[0], 1);
    }
  }
  w.ns[node] = s;
}

// F (FP64) and the Jacobian (precision T) at every collocation point.
template <typename T>
__global__ void k_point(SolveArgs a, Workspace w) {
  const int64_t P = npts(a.Nmax);
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= a.n * P) return;
  const int64_t node = t / P;
  const int64_t p = t % P;
  if (!w.ns[node].active) return;
  if (p > 3 * int64_t(a.N[node])) return;
  double y[12], F[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) y[c] = w.Y[t * 12 + c];
  T* J = static_cast<T*>(w.Jm) + t * 144;
  if constexpr (sizeof(T) == sizeof(double)) {
    char_jacobian<T>(a.P, y, J, F);
  } else {
    char_jacobian<T>(a.P, y, J, nullptr);
    char_rhs(a.P, y, F);
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) w.Fv[t * 12 + c] = F[c];
}

// Stage condensation of one interval.  Columns: [Y_{i,2} (12), Y_{i,3} (12) |
// y_i (12) | y_{i+1} (12) | rhs]; rows: stage equations k = 2, 3, 4.
template <typename T>
__global__ void __launch_bounds__(32 * kCondWarps) k_condense(SolveArgs a, Workspace w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wid = blockIdx.x * int64_t(kCondWarps) + warp;
  if (wid >= a.n * a.Nmax) return;
  const int64_t node = wid / a.Nmax;
  const int i = static_cast<int>(wid % a.Nmax);
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  if (i >= N) return;
  const double h = a.T[node] / N;
  T* M = reinterpret_cast<T*>(smem_raw) + warp * (kCondRows * kCondLd);
  const int64_t pbase = node * npts(a.Nmax) + 3 * int64_t(i);
  const T* J = static_cast<const T*>(w.Jm) + pbase * 144;
  const double* Y = w.Y + pbase * 12;
  const double* F = w.Fv + pbase * 12;
  for (int e = lane; e < kCondRows * 48; e += 32) {
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
    T v = T(-h * kLobA[k][j]) * J[j * 144 + comp * 12 + cc];
    if (comp == cc) {
      if (j == k) v += T(1);
      if (j == 0) v -= T(1);
    }
    M[r * kCondLd + c] = v;
  }
  for (int r = lane; r < kCondRows; r += 32) {
    const int k = r / 12 + 1, comp = r % 12;
    double res = Y[12 * k + comp] - Y[comp] -
                 h * (kLobA[k][0] * F[comp] + kLobA[k][1] * F[12 + comp] + kLobA[k][2] * F[24 + comp] +
                      kLobA[k][3] * F[36 + comp]);
    M[r * kCondLd + 48] = T(-res);
  }
  __syncwarp();
  const bool ok = warp_eliminate<T, kCondRows, kCondLd, 24>(M, lane);
  if (!ok && lane == 0) w.ns[node].singular = 1;
  const int64_t blk = node * a.Nmax + i;
  T* rec = static_cast<T*>(w.Rec) + blk * kRec;
  for (int e = lane; e < kRec; e += 32) rec[e] = M[e];
  T* cond = static_cast<T*>(w.Cond) + blk * kBlk;
  for (int e = lane; e < kBlk; e += 32) {
    const int r = e / 25, c = e % 25;
    cond[e] = M[(24 + r) * kCondLd + 24 + c];
  }
}

// Stage condensation, register-resident FP32 form: warp per interval.  Lane
// r < 24 holds interior equation row r (stage 2 or 3); lanes 24..31 hold the
// stage-4 rows 24..31 and lanes 0..3 also hold stage-4 rows 32..35.  Partial
// pivoting over the 24 interior rows: the pivot is the largest |a_rk| among
// the rows not yet pivoted, found by one warp max-reduction of
// (|a_rk| bits with the 5 low bits replaced by 31 - lane), so ties go to the
// lower row.  Rows never move: the pivot row is broadcast by shuffles and
// every other row updates itself in registers.  At the end the pivot rows
// (in pivot order) are the stored interior rows and the stage-4 rows hold the
// condensed block row in columns 24..48.
__global__ void __launch_bounds__(128) k_condense_reg(SolveArgs a, Workspace w) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = blockIdx.x * int64_t(4) + (threadIdx.x >> 5);
  if (wid >= a.n * a.Nmax) return;
  const int64_t node = wid / a.Nmax;
  const int i = static_cast<int>(wid % a.Nmax);
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  if (i >= N) return;
  const double h = a.T[node] / N;
  const int64_t pbase = node * npts(a.Nmax) + 3 * int64_t(i);
  const float* J = static_cast<const float*>(w.Jm) + pbase * 144;
  const double* Y = w.Y + pbase * 12;
  const double* F = w.Fv + pbase * 12;

  // row r = 12 (k - 1) + comp, k = stage 2, 3, 4 (1-based 2..4 -> k = 1..3)
  auto build = [&](int r, float* row) {
    const int k = r / 12 + 1, comp = r % 12;
    float cf[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cf[j] = static_cast<float>(-h * kLobA[k][j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4* src = reinterpret_cast<const float4*>(J + j * 144 + comp * 12);
      const int c0 = j == 0 ? 24 : (j == 3 ? 36 : 12 * (j - 1));
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float4 v = src[q];
        row[c0 + 4 * q + 0] = cf[j] * v.x;
        row[c0 + 4 * q + 1] = cf[j] * v.y;
        row[c0 + 4 * q + 2] = cf[j] * v.z;
        row[c0 + 4 * q + 3] = cf[j] * v.w;
      }
    }
    // identity terms: +I on the stage's own point, -I on y_i (static
    // register indices: compare against every column)
    const int plus = k < 3 ? 12 * (k - 1) + comp : 36 + comp;
    const int minus = 24 + comp;
#pragma unroll
    for (int c = 0; c < 48; ++c) {
      if (c == plus) row[c] += 1.0f;
      if (c == minus) row[c] -= 1.0f;
    }
    const double res = Y[12 * k + comp] - Y[comp] -
                       h * (kLobA[k][0] * F[comp] + kLobA[k][1] * F[12 + comp] + kLobA[k][2] * F[24 + comp] +
                            kLobA[k][3] * F[36 + comp]);
    row[48] = static_cast<float>(-res);
  };

  float ra[kCondLd], rb[kCondLd];
  build(lane, ra);
  const bool has_b = lane < 4;
  if (has_b) build(32 + lane, rb);
  const bool interior = lane < 24;
  bool done = false;
  int my_step = -1;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    const bool cand = interior && !done;
    const unsigned key = cand ? ((__float_as_uint(fabsf(ra[k])) & ~31u) | unsigned(31 - lane)) : 0u;
    const unsigned best = __reduce_max_sync(0xffffffffu, key);
    const int p = 31 - int(best & 31u);
    const float piv = __shfl_sync(0xffffffffu, ra[k], p);
    const bool good = piv != 0.0f && isfinite(piv);
    ok = ok && good;
    const float inv = good ? 1.0f / piv : 0.0f;
    if (lane == p) {
      done = true;
      my_step = k;
    }
    const bool upd = !(interior && done);
    const float la = upd ? ra[k] * inv : 0.0f;
    const float lb = has_b ? rb[k] * inv : 0.0f;
#pragma unroll
    for (int c = k + 1; c < kCondLd; ++c) {
      const float pc = __shfl_sync(0xffffffffu, ra[c], p);
      if (upd) ra[c] = fmaf(-la, pc, ra[c]);
      rb[c] = fmaf(-lb, pc, rb[c]);
    }
  }
  if (!ok && lane == 0) w.ns[node].singular = 1;
  const int64_t blk = node * a.Nmax + i;
  float* rec = static_cast<float*>(w.Rec) + blk * kRec;
  float* cond = static_cast<float*>(w.Cond) + blk * kBlk;
  if (interior) {
    float* dst = rec + my_step * kCondLd;
#pragma unroll
    for (int c = 0; c < kCondLd; ++c) dst[c] = ra[c];
  } else {
    float* dst = cond + (lane - 24) * 25;
#pragma unroll
    for (int c = 0; c < 25; ++c) dst[c] = ra[24 + c];
  }
  if (has_b) {
    float* dst = cond + (8 + lane) * 25;
#pragma unroll
    for (int c = 0; c < 25; ++c) dst[c] = rb[24 + c];
  }
}

// Staircase elimination over the block rows of one node, then back substitution.
template <typename T>
__global__ void k_abd(SolveArgs a, Workspace w) {
  __shared__ T panel_s[4][18 * 25];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t node = blockIdx.x * int64_t(4) + warp;
  if (node >= a.n) return;
  if (!w.ns[node].active) return;
  T* pan = panel_s[warp];
  const int N = a.N[node];
  const int64_t pb = node * npts(a.Nmax);
  const double* Y = w.Y + pb * 12;
  const double* x0 = a.x0 + node * 6;
  const T* cond = static_cast<const T*>(w.Cond) + node * a.Nmax * int64_t(kBlk);
  T* abd = static_cast<T*>(w.Abd) + node * a.Nmax * int64_t(kBlk);
  bool ok = true;
  // carry rows: x(0) - x0 = 0 linearised, [I 0] dy_0 = -(x(0) - x0)
  for (int e = lane; e < 6 * 25; e += 32) {
    const int r = e / 25, c = e % 25;
    T v = T(0);
    if (c == r) v = T(1);
    if (c == 24) v = T(-(Y[r] - x0[r]));
    pan[r * 25 + c] = v;
  }
  __syncwarp();
  for (int i = 0; i < N; ++i) {
    const T* ci = cond + int64_t(i) * kBlk;
    for (int e = lane; e < kBlk; e += 32) pan[6 * 25 + e] = ci[e];
    __syncwarp();
    ok = warp_eliminate<T, 18, 25, 12>(pan, lane) && ok;
    T* ai = abd + int64_t(i) * kBlk;
    for (int e = lane; e < kBlk; e += 32) ai[e] = pan[e];
    __syncwarp();
    for (int e = lane; e < 6 * 25; e += 32) {
      const int r = e / 25, c = e % 25;
      T v = T(0);
      if (c < 12) v = pan[(12 + r) * 25 + 12 + c];
      if (c == 24) v = pan[(12 + r) * 25 + 24];
      pan[r * 25 + c] = v;
    }
    __syncwarp();
  }
  // terminal rows: lambda(T) - grad h(x(T)) = 0 linearised
  const double* yN = Y + 3 * int64_t(N) * 12;
  T* sys = pan + 6 * 25;   // 12 x 13 system after the carry rows are moved in
  __syncwarp();
  // move the 6 carry rows into a 12 x 13 layout: [carry (cols 0..11, rhs 24)]
  for (int e = lane; e < 12 * 13; e += 32) {
    const int r = e / 13, c = e % 13;
    T v;
    if (r < 6) {
      v = pan[r * 25 + (c < 12 ? c : 24)];
    } else {
      const int rr = r - 6;
      if (c < 6) v = T(-terminal_hess(a.P, rr, c));
      else if (c < 12) v = (c - 6 == rr) ? T(1) : T(0);
      else v = T(-(yN[6 + rr] - terminal_grad(a.P, yN, rr)));
    }
    sys[e] = v;
  }
  __syncwarp();
  ok = warp_eliminate<T, 12, 13, 12>(sys, lane) && ok;
  T t = lane < 12 ? sys[lane * 13 + 12] : T(0);
  T dy = warp_backsolve<T, 12>(sys, 13, t, lane);
  double* D = w.D + pb * 12;
  if (lane < 12) D[3 * int64_t(N) * 12 + lane] = double(dy);
  // back substitution: U_i dy_i = rhs_i - V_i dy_{i+1}
  for (int i = N - 1; i >= 0; --i) {
    const T* ai = abd + int64_t(i) * kBlk;
    __syncwarp();
    for (int e = lane; e < kBlk; e += 32) pan[e] = ai[e];
    __syncwarp();
    T acc = T(0);
    if (lane < 12) {
      acc = pan[lane * 25 + 24];
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      T dyc = __shfl_sync(0xffffffffu, dy, c);
      if (lane < 12) acc -= pan[lane * 25 + 12 + c] * dyc;
    }
    dy = warp_backsolve<T, 12>(pan, 25, acc, lane);
    if (lane < 12) D[3 * int64_t(i) * 12 + lane] = double(dy);
  }
  if (!ok && lane == 0) w.ns[node].singular = 1;
}

// Pivot search shared by the register-resident kernels: the largest |v| over
// the candidate lanes, ties to the lower lane (magnitude bits with the 5 low
// bits replaced by 31 - lane, reduced by one warp max).
template <typename T>
__device__ __forceinline__ int warp_pivot_lane(T v, bool cand, int lane) {
  const float m = fabsf(static_cast<float>(v));
  const unsigned key = cand ? ((__float_as_uint(m) & ~31u) | unsigned(31 - lane)) : 0u;
  const unsigned best = __reduce_max_sync(0xffffffffu, key);
  return 31 - int(best & 31u);
}

// Staircase elimination, register-resident: warp per node, lanes 0..17 hold
// the 18 rows of the current panel [carry (6) ; block row i (12)] over the
// 25 columns [y_i (12) | y_{i+1} (12) | rhs].  Twelve pivot steps with partial
// pivoting leave 12 pivot rows (stored in pivot order, with the reciprocal of
// the pivot in place of the pivot) and 6 rows that carry y_{i+1} into the next
// panel.  The next block row is prefetched into lanes 0..11 while the current
// panel is eliminated.  After the lambda(T) rows close the system, back
// substitution runs from the last mesh point to the first.
template <typename T>
__global__ void __launch_bounds__(128) k_abd_reg(SolveArgs a, Workspace w) {
  const int lane = threadIdx.x & 31;
  const int64_t node = blockIdx.x * int64_t(4) + (threadIdx.x >> 5);
  if (node >= a.n) return;
  if (!w.ns[node].active) return;
  const int N = a.N[node];
  const int64_t pb = node * npts(a.Nmax);
  const double* Y = w.Y + pb * 12;
  const double* x0 = a.x0 + node * 6;
  const T* cond = static_cast<const T*>(w.Cond) + node * a.Nmax * int64_t(kBlk);
  T* abd = static_cast<T*>(w.Abd) + node * a.Nmax * int64_t(kBlk);
  double* D = w.D + pb * 12;
  const bool rowlane = lane < 18;
  T r[25], nx[25];
  // carry rows: [I 0] dy_0 = -(x(0) - x0); lanes 6..17: block row 0
#pragma unroll
  for (int c = 0; c < 25; ++c) r[c] = T(0);
  if (lane < 6) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (c == lane) r[c] = T(1);
    r[24] = T(-(Y[lane] - x0[lane]));
  } else if (rowlane) {
#pragma unroll
    for (int c = 0; c < 25; ++c) r[c] = cond[(lane - 6) * 25 + c];
  }
  bool ok = true;
  for (int i = 0; i < N; ++i) {
    // prefetch block row i+1 into lanes 0..11
    if (i + 1 < N && lane < 12) {
      const T* src = cond + int64_t(i + 1) * kBlk + lane * 25;
#pragma unroll
      for (int c = 0; c < 25; ++c) nx[c] = src[c];
    }
    bool done = false;
    int my_step = -1;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int p = warp_pivot_lane<T>(r[k], rowlane && !done, lane);
      const T piv = __shfl_sync(0xffffffffu, r[k], p);
      const bool good = piv != T(0) && isfinite(piv);
      ok = ok && good;
      const T inv = good ? T(1) / piv : T(0);
      if (lane == p) {
        done = true;
        my_step = k;
        r[k] = inv;   // stored pivot row keeps 1/pivot on the diagonal
      }
      const bool upd = rowlane && !done;
      const T l = upd ? r[k] * inv : T(0);
#pragma unroll
      for (int c = k + 1; c < 25; ++c) {
        const T pc = __shfl_sync(0xffffffffu, r[c], p);
        if (upd) r[c] -= l * pc;
      }
    }
    if (done) {
      T* dst = abd + int64_t(i) * kBlk + my_step * 25;
#pragma unroll
      for (int c = 0; c < 25; ++c) dst[c] = r[c];
    }
    // next panel: carry rows shift y_{i+1} into the first block; pivot lanes
    // take the prefetched block row i+1 (in lane order)
    const unsigned dmask = __ballot_sync(0xffffffffu, done);
    const int rank = __popc(dmask & ((1u << lane) - 1u));
    const bool last = i + 1 == N;
#pragma unroll
    for (int c = 0; c < 25; ++c) {
      const T v = __shfl_sync(0xffffffffu, nx[c], rank & 15);
      if (rowlane && !done) {
        if (c < 12) r[c] = r[c + 12];
        else if (c < 24) r[c] = T(0);
      } else if (done && !last) {
        r[c] = v;
      }
    }
    if (last && done) {
      // closing rows: lambda(T) - grad h(x(T)) = 0 for ranks 0..5, empty rows above
      const double* yN = Y + 3 * int64_t(N) * 12;
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
    if (last) {
      // the closing 12 x 12 system: carry lanes and the 6 terminal rows
      const bool active_row = rowlane && (!done || rank < 6);
      bool done2 = false;
      int my2 = -1;
      int plane[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int p = warp_pivot_lane<T>(r[k], active_row && !done2, lane);
        plane[k] = p;
        const T piv = __shfl_sync(0xffffffffu, r[k], p);
        const bool good = piv != T(0) && isfinite(piv);
        ok = ok && good;
        const T inv = good ? T(1) / piv : T(0);
        if (lane == p) {
          done2 = true;
          my2 = k;
          r[k] = inv;
        }
        const bool upd = active_row && !done2;
        const T l = upd ? r[k] * inv : T(0);
#pragma unroll
        for (int c = k + 1; c < 12; ++c) {
          const T pc = __shfl_sync(0xffffffffu, r[c], p);
          if (upd) r[c] -= l * pc;
        }
        const T pr = __shfl_sync(0xffffffffu, r[24], p);
        if (upd) r[24] -= l * pr;
      }
      (void)my2;
      // back substitution of the closing system: dy_N
      T dy[12];
      T t = r[24];
#pragma unroll
      for (int k = 11; k >= 0; --k) {
        const int p = plane[k];
        const T dk = __shfl_sync(0xffffffffu, t * r[k], p);
        dy[k] = dk;
        // every row pivoted before step k subtracts its column-k term
        t -= r[k] * dk;
      }
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 12; ++c) D[3 * int64_t(N) * 12 + c] = double(dy[c]);
      }
      // backward sweep over the stored pivot rows
      T row[25];
      if (lane < 12) {
        const T* src = abd + int64_t(N - 1) * kBlk + lane * 25;
#pragma unroll
        for (int c = 0; c < 25; ++c) row[c] = src[c];
      }
      for (int ii = N - 1; ii >= 0; --ii) {
        T pre[25];
        if (ii > 0 && lane < 12) {
          const T* src = abd + int64_t(ii - 1) * kBlk + lane * 25;
#pragma unroll
          for (int c = 0; c < 25; ++c) pre[c] = src[c];
        }
        // lane k holds the pivot row of step k: U (cols k..11, 1/pivot at k),
        // V (cols 12..23), rhs (24)
        T tt = row[24];
#pragma unroll
        for (int c = 0; c < 12; ++c) tt -= row[12 + c] * dy[c];
        T nd[12];
#pragma unroll
        for (int k = 11; k >= 0; --k) {
          const T dk = __shfl_sync(0xffffffffu, tt * row[k], k);
          nd[k] = dk;
          if (lane < k) tt -= row[k] * dk;
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) dy[c] = nd[c];
        if (lane < 12) {
          T mine = T(0);
#pragma unroll
          for (int c = 0; c < 12; ++c)
            if (c == lane) mine = dy[c];
          D[3 * int64_t(ii) * 12 + lane] = double(mine);
        }
        if (ii > 0) {
#pragma unroll
          for (int c = 0; c < 25; ++c) row[c] = pre[c];
        }
      }
    }
  }
  if (!ok && lane == 0) w.ns[node].singular = 1;
}

// Interior-stage corrections from the stored condensation pivot rows.
template <typename T>
__global__ void k_recover(SolveArgs a, Workspace w) {
  __shared__ T rows_s[4][kRec];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wid = blockIdx.x * int64_t(4) + warp;
  if (wid >= a.n * a.Nmax) return;
  const int64_t node = wid / a.Nmax;
  const int i = static_cast<int>(wid % a.Nmax);
  if (!w.ns[node].active) return;
  if (i >= a.N[node]) return;
  T* U = rows_s[warp];
  const T* rec = static_cast<const T*>(w.Rec) + wid * kRec;
  for (int e = lane; e < kRec; e += 32) U[e] = rec[e];
  double* D = w.D + (node * npts(a.Nmax) + 3 * int64_t(i)) * 12;
  const T dyl = lane < 12 ? T(D[lane]) : T(0);
  const T dyr = lane < 12 ? T(D[36 + lane]) : T(0);
  __syncwarp();
  T acc = lane < 24 ? U[lane * kCondLd + 48] : T(0);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const T l = __shfl_sync(0xffffffffu, dyl, c);
    const T r = __shfl_sync(0xffffffffu, dyr, c);
    if (lane < 24) acc -= U[lane * kCondLd + 24 + c] * l + U[lane * kCondLd + 36 + c] * r;
  }
  const T x = warp_backsolve<T, 24>(U, kCondLd, acc, lane);
  if (lane < 24) D[12 + lane] = double(x);   // points 3i+1 and 3i+2 are contiguous
}

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
    atomicAdd(&w.counters[0], 1);
  }
  w.ns[node] = s;
}

__global__ void k_update(SolveArgs a, Workspace w) {
  const int64_t P = npts(a.Nmax);
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= a.n * P) return;
  const int64_t node = t / P;
  if (!w.ns[node].active) return;
  if (t % P > 3 * int64_t(a.N[node])) return;
  const double alpha = w.ns[node].alpha;
#pragma unroll
  for (int c = 0; c < 12; ++c) w.Y[t * 12 + c] = __fma_rn(alpha, w.D[t * 12 + c], w.Y[t * 12 + c]);
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
// z(T) = h sum_i sum_j b_j L(Y_ij) (the Lobatto IIIA step of z' = L).
__global__ void k_outputs(SolveArgs a, Workspace w, double* lambda0, double* u0, double* V,
                          int32_t* status, int32_t* iters) {
  const int lane = threadIdx.x & 31;
  const int64_t node = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (node >= a.n) return;
  const NodeState s = w.ns[node];
  const double* Y = w.Y + node * npts(a.Nmax) * 12;
  if (s.status == SG_BADINPUT) {
    if (lane == 0) {
      for (int c = 0; c < 6; ++c) lambda0[node * 6 + c] = NAN;
      for (int c = 0; c < 3; ++c) u0[node * 3 + c] = NAN;
      V[node] = NAN;
      status[node] = s.status;
      iters[node] = 0;
    }
    return;
  }
  const int N = a.N[node];
  const double h = a.T[node] / N;
  double z = 0.0;
  for (int i = lane; i < N; i += 32) {
    const double* yi = Y + 3 * int64_t(i) * 12;
    z += h * (kLobB[0] * running_cost(a.P, yi) + kLobB[1] * running_cost(a.P, yi + 12) +
              kLobB[2] * running_cost(a.P, yi + 24) + kLobB[3] * running_cost(a.P, yi + 36));
  }
  z = warp_sum(z);
  if (lane == 0) {
    const double* yN = Y + 3 * int64_t(N) * 12;
    V[node] = z + terminal_cost(a.P, yN);
    double u[3];
    optimal_control(a.P, Y + 6, u);
    for (int c = 0; c < 6; ++c) lambda0[node * 6 + c] = Y[6 + c];
    for (int c = 0; c < 3; ++c) u0[node * 3 + c] = u[c];
    status[node] = s.status;
    iters[node] = s.iters;
  }
}

__global__ void k_copy_Y(SolveArgs a, Workspace w, double* out) {
  const int64_t P = npts(a.Nmax);
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= a.n * P) return;
  const int64_t node = t / P;
  if (t % P > 3 * int64_t(a.N[node])) return;
#pragma unroll
  for (int c = 0; c < 12; ++c) out[t * 12 + c] = w.Y[t * 12 + c];
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
    double JB[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) JB[3 * i + j] = p.Jinv[i] * in.B[3 * i + j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += JB[3 * i + m] * JB[3 * j + m];
        p.Kw[3 * i + j] = s / in.r;
        p.Gw[3 * i + j] = in.B[3 * j + i] * p.Jinv[j] / in.r;
      }
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
  } else {
    return false;
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

static size_t ws_bytes(int64_t n, int Nmax, int precision) {
  const size_t tsize = precision == SG_PREC_MIXED ? sizeof(float) : sizeof(double);
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
  const unsigned gi = static_cast<unsigned>(ceil_div(nint, 128));
  const unsigned gnode_thr = static_cast<unsigned>(ceil_div(a.n, 128));
  const unsigned gnode_warp = static_cast<unsigned>(ceil_div(a.n * 32, 128));
  const unsigned gcond = static_cast<unsigned>(ceil_div(nint, kCondWarps));
  const unsigned grec = static_cast<unsigned>(ceil_div(nint, 4));
  const unsigned gabd = static_cast<unsigned>(ceil_div(a.n, 4));
  const size_t cond_smem = sizeof(T) * kCondWarps * kCondRows * kCondLd;
  SG_CUDA_TRY(cudaFuncSetAttribute(k_condense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(cond_smem)));
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
  SG_TIMED("k_init", st, (k_init<<<gp, 128, 0, st>>>(a, w)));
  SG_TIMED("k_trial", st, (k_trial<<<gi, 128, 0, st>>>(a, w)));
  SG_TIMED("k_ls_reduce", st, (k_ls_reduce<<<gnode_warp, 128, 0, st>>>(a, w, 0)));
  SG_LAUNCH_CHECK("init kernels");
  if ((rc = read_counters()) != SG_OK) return rc;
  int active = h_cnt[1];
  for (int it = 0; it < a.max_iter && active > 0; ++it) {
    SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), st));
    SG_TIMED(kname<T>("k_point"), st, (k_point<T><<<gp, 128, 0, st>>>(a, w)));
    if constexpr (sizeof(T) == sizeof(float)) {
      SG_TIMED("k_condense_reg_fp32", st, (k_condense_reg<<<grec, 128, 0, st>>>(a, w)));
    } else {
      SG_TIMED(kname<T>("k_condense"), st, (k_condense<T><<<gcond, 32 * kCondWarps, cond_smem, st>>>(a, w)));
    }
    SG_TIMED(kname<T>("k_abd_reg"), st, (k_abd_reg<T><<<gabd, 128, 0, st>>>(a, w)));
    SG_TIMED(kname<T>("k_recover"), st, (k_recover<T><<<grec, 128, 0, st>>>(a, w)));
    SG_TIMED("k_ls_begin", st, (k_ls_begin<<<gnode_thr, 128, 0, st>>>(a, w)));
    SG_LAUNCH_CHECK("newton kernels");
    for (int trial = 0; trial < 12; ++trial) {
      SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, sizeof(int), st));
      SG_TIMED("k_trial", st, (k_trial<<<gi, 128, 0, st>>>(a, w)));
      SG_TIMED("k_ls_reduce", st, (k_ls_reduce<<<gnode_warp, 128, 0, st>>>(a, w, 1)));
      SG_LAUNCH_CHECK("line search kernels");
      if ((rc = read_counters()) != SG_OK) return rc;
      if (h_cnt[0] == 0) break;
    }
    SG_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), st));
    SG_TIMED("k_update", st, (k_update<<<gp, 128, 0, st>>>(a, w)));
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

}  // namespace sg

using namespace sg;

extern "C" size_t sg_solve_workspace_bytes(int64_t n, int n_max_intervals, int precision) {
  if (n < 0 || n_max_intervals < 1) return 0;
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
  sg_solve_opts o{1e-8, 50, SG_PREC_FP64, 1, 0};
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iter < 0) return fail(SG_EINVAL, "sg_solve_bvps: bad tol or max_iter");
  if (o.precision != SG_PREC_FP64 && o.precision != SG_PREC_MIXED)
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
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.precision == SG_PREC_MIXED) {
    Workspace w = carve(d_work, n, n_max_intervals, sizeof(float));
    return run_solve<float>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
  }
  Workspace w = carve(d_work, n, n_max_intervals, sizeof(double));
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
// device (with that device current) and cached.
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
  sg_solve_opts o{1e-8, 50, SG_PREC_FP64, 1, 0};
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iter < 0) return fail(SG_EINVAL, "sg_solve_bvps_static: bad tol or max_iter");
  if (o.precision != SG_PREC_FP64 && o.precision != SG_PREC_MIXED)
    return fail(SG_EINVAL, "sg_solve_bvps_static: unknown precision");
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
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Every region the solver reads is written first in this call (k_init sets the
  // iterate, the corrections and the per-node state; the counters are zeroed
  // before each use), so the previous call's contents need no clearing here.
  if (o.precision == SG_PREC_MIXED) {
    Workspace w = carve(scratch, n, n_max_intervals, sizeof(float));
    return run_solve<float>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
  }
  Workspace w = carve(scratch, n, n_max_intervals, sizeof(double));
  return run_solve<double>(a, w, st, d_lambda0, d_u0, d_V, d_status, d_iters, d_Y);
}
