// Example II (Section 5, Eq. optim_attitude): the target attitude reachable
// from an initial state of the rigid body with two pairs of momentum wheels.
//
// With C' B = 0 the component C'(J w - R(v) H) of the angular momentum cannot
// be changed by the wheels, so the attitudes reachable from (v0, w0) at rest
// satisfy -C' R(vt) H = C'(J w0 - R(v0) H).  The target is the one closest to
// the identity, i.e. the maximiser of tr R(vt) on that surface.
//
// One thread per initial state: Newton's method on the optimality conditions
// grad tr R + mu grad c = 0, c = 0 (c the constraint), with the gradients from
// forward-mode duals and the Hessians by central differences of those
// gradients; a backtracking search on the norm of the conditions.  The point
// found must be a maximum on the surface (negative projected Hessian);
// otherwise the iteration restarts from vt = 0.
#include <cmath>

#include "common.cuh"
#include "diag.cuh"
#include "problems.cuh"

namespace sg {
namespace {

struct TargetArgs {
  double C[3];     // unit normal of the two wheel axes
  double J[3];
  double H[3];
  const double* x0;
  int64_t n;
  double* target;
  int32_t* status;
};

// tr R(v) and c(v) = -C' R(v) H - b for R = Rx(phi) Ry(theta) Rz(psi).
template <typename S>
__device__ __forceinline__ void trace_and_constraint(const TargetArgs& a, const S* v, double b, S* f, S* c) {
  S sp, cp, st, ct, ss, cs;
  dsincos(v[0], &sp, &cp);
  dsincos(v[1], &st, &ct);
  dsincos(v[2], &ss, &cs);
  *f = ct * cs + cp * cs + sp * st * ss + cp * ct;
  const double h0 = a.H[0], h1 = a.H[1], h2 = a.H[2];
  const S az0 = cs * h0 + ss * h1;
  const S az1 = cs * h1 - ss * h0;
  const S ay0 = ct * az0 - st * h2;
  const S ay2 = st * az0 + ct * h2;
  const S g1 = cp * az1 + sp * ay2;
  const S g2 = cp * ay2 - sp * az1;
  *c = -(ay0 * a.C[0] + g1 * a.C[1] + g2 * a.C[2]) + (-b);
}

// value and gradient of f and c at v
__device__ void grads(const TargetArgs& a, const double* v, double b, double* f, double* gf, double* c,
                      double* gc) {
  using D = Dual<double, 3>;
  D vd[3], fd, cd;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vd[i] = dconst<double, 3>(v[i]);
    vd[i].d[i] = 1.0;
  }
  trace_and_constraint<D>(a, vd, b, &fd, &cd);
  *f = fd.v;
  *c = cd.v;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gf[i] = fd.d[i];
    gc[i] = cd.d[i];
  }
}

// Solves the 4 x 4 system M z = r by Gaussian elimination with partial pivoting.
__device__ bool solve4(double (&M)[4][4], double (&r)[4]) {
  for (int k = 0; k < 4; ++k) {
    int p = k;
    for (int i = k + 1; i < 4; ++i)
      if (fabs(M[i][k]) > fabs(M[p][k])) p = i;
    if (!(fabs(M[p][k]) > 0.0)) return false;
    if (p != k) {
      for (int j = 0; j < 4; ++j) {
        const double t = M[k][j];
        M[k][j] = M[p][j];
        M[p][j] = t;
      }
      const double t = r[k];
      r[k] = r[p];
      r[p] = t;
    }
    for (int i = k + 1; i < 4; ++i) {
      const double l = M[i][k] / M[k][k];
      for (int j = k; j < 4; ++j) M[i][j] -= l * M[k][j];
      r[i] -= l * r[k];
    }
  }
  for (int k = 3; k >= 0; --k) {
    double s = r[k];
    for (int j = k + 1; j < 4; ++j) s -= M[k][j] * r[j];
    r[k] = s / M[k][k];
  }
  return true;
}

// Norm of the optimality conditions at (v, mu); res receives them.
__device__ double kkt(const TargetArgs& a, const double* v, double mu, double b, double* res) {
  double f, c, gf[3], gc[3];
  grads(a, v, b, &f, gf, &c, gc);
  for (int i = 0; i < 3; ++i) res[i] = gf[i] + mu * gc[i];
  res[3] = c;
  return sqrt(res[0] * res[0] + res[1] * res[1] + res[2] * res[2] + res[3] * res[3]);
}

// Newton from v (overwritten); true if it reached a maximum on the surface.
__device__ bool newton_target(const TargetArgs& a, double b, double (&v)[3]) {
  constexpr double kStep = 1e-6;   // central differences of the gradients
  double mu = 0.0;
  {
    double f, c, gf[3], gc[3];
    grads(a, v, b, &f, gf, &c, gc);
    const double g2 = gc[0] * gc[0] + gc[1] * gc[1] + gc[2] * gc[2];
    if (g2 > 0.0) mu = -(gf[0] * gc[0] + gf[1] * gc[1] + gf[2] * gc[2]) / g2;   // least-squares multiplier
  }
  for (int it = 0; it < 60; ++it) {
    double res[4];
    const double nr = kkt(a, v, mu, b, res);
    if (!(nr < INFINITY)) return false;
    if (nr < 1e-13) break;
    double f, c, gf[3], gc[3];
    grads(a, v, b, &f, gf, &c, gc);
    double M[4][4], rhs[4];
    for (int j = 0; j < 3; ++j) {   // Hessian of the Lagrangian, column j
      double vp[3] = {v[0], v[1], v[2]}, vm[3] = {v[0], v[1], v[2]};
      vp[j] += kStep;
      vm[j] -= kStep;
      double fp, cp, gfp[3], gcp[3], fm, cm, gfm[3], gcm[3];
      grads(a, vp, b, &fp, gfp, &cp, gcp);
      grads(a, vm, b, &fm, gfm, &cm, gcm);
      for (int i = 0; i < 3; ++i) M[i][j] = ((gfp[i] - gfm[i]) + mu * (gcp[i] - gcm[i])) / (2.0 * kStep);
    }
    for (int i = 0; i < 3; ++i) {
      M[i][3] = gc[i];
      M[3][i] = gc[i];
    }
    M[3][3] = 0.0;
    for (int i = 0; i < 4; ++i) rhs[i] = -res[i];
    if (!solve4(M, rhs)) return false;
    double alpha = 1.0;
    for (int k = 0; k < 30; ++k, alpha *= 0.5) {
      const double vt[3] = {v[0] + alpha * rhs[0], v[1] + alpha * rhs[1], v[2] + alpha * rhs[2]};
      double rt[4];
      if (kkt(a, vt, mu + alpha * rhs[3], b, rt) < (1.0 - 1e-4 * alpha) * nr || k == 29) {
        for (int i = 0; i < 3; ++i) v[i] = vt[i];
        mu += alpha * rhs[3];
        break;
      }
    }
  }
  double res[4];
  if (!(kkt(a, v, mu, b, res) < 1e-10)) return false;
  // a maximum on the surface: the Lagrangian's second derivative is negative
  // on the tangent plane of the constraint (two directions orthogonal to grad c)
  double f, c, gf[3], gc[3];
  grads(a, v, b, &f, gf, &c, gc);
  const double ngc = sqrt(gc[0] * gc[0] + gc[1] * gc[1] + gc[2] * gc[2]);
  const double e[3] = {fabs(gc[0]) < 0.9 * ngc ? 1.0 : 0.0, fabs(gc[0]) < 0.9 * ngc ? 0.0 : 1.0, 0.0};
  double t1[3], t2[3];
  t1[0] = gc[1] * e[2] - gc[2] * e[1];
  t1[1] = gc[2] * e[0] - gc[0] * e[2];
  t1[2] = gc[0] * e[1] - gc[1] * e[0];
  t2[0] = gc[1] * t1[2] - gc[2] * t1[1];
  t2[1] = gc[2] * t1[0] - gc[0] * t1[2];
  t2[2] = gc[0] * t1[1] - gc[1] * t1[0];
  auto dir2 = [&](const double* t) {   // second derivative of the Lagrangian along t
    double vp[3], vm[3];
    for (int i = 0; i < 3; ++i) {
      vp[i] = v[i] + 1e-4 * t[i];
      vm[i] = v[i] - 1e-4 * t[i];
    }
    double fp, cp, fm, cm, g[3], h[3];
    grads(a, vp, b, &fp, g, &cp, h);
    grads(a, vm, b, &fm, g, &cm, h);
    return ((fp + mu * cp) - 2.0 * (f + mu * c) + (fm + mu * cm)) / 1e-8;
  };
  const double h11 = dir2(t1), h22 = dir2(t2);
  double t12[3];
  for (int i = 0; i < 3; ++i) t12[i] = t1[i] + t2[i];
  const double h12 = 0.5 * (dir2(t12) - h11 - h22);
  return h11 < 0.0 && h11 * h22 - h12 * h12 > 0.0;
}

__global__ void k_attitude_targets(TargetArgs a) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= a.n) return;
  const double* x = a.x0 + i * 6;
  // b = C' (J w0 - R(v0) H)
  double f, c;
  trace_and_constraint<double>(a, x, 0.0, &f, &c);   // c = -C' R(v0) H
  const double b = a.C[0] * a.J[0] * x[3] + a.C[1] * a.J[1] * x[4] + a.C[2] * a.J[2] * x[5] + c;
  double v[3] = {x[0], x[1], x[2]};
  bool ok = newton_target(a, b, v);
  if (!ok) {
    v[0] = v[1] = v[2] = 0.0;
    ok = newton_target(a, b, v);
  }
  for (int k = 0; k < 3; ++k) a.target[i * 3 + k] = ok ? v[k] : NAN;
  if (a.status) a.status[i] = ok ? 0 : 1;
}

}  // namespace
}  // namespace sg

extern "C" int sg_attitude_targets(const sg_problem* prob, const double* d_x0, int64_t n, double* d_target,
                                   int32_t* d_status, void* stream) {
  sg::clear_error();
  if (!prob || prob->kind != SG_PROBLEM_ATTITUDE || prob->m != 2)
    return sg::fail(SG_EINVAL, "sg_attitude_targets: needs an attitude problem with m = 2");
  if (n < 0) return sg::fail(SG_EINVAL, "sg_attitude_targets: n < 0");
  if (n == 0) return SG_OK;
  if (!d_x0 || !d_target) return sg::fail(SG_EINVAL, "sg_attitude_targets: null device pointer");
  sg::TargetArgs a{};
  const double* B = prob->B;   // row-major 3 x 3; columns 0 and 1 are the wheel axes
  const double c[3] = {B[3] * B[7] - B[6] * B[4], B[6] * B[1] - B[0] * B[7], B[0] * B[4] - B[3] * B[1]};
  const double nc = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  if (!(nc > 0.0)) return sg::fail(SG_EINVAL, "sg_attitude_targets: the columns of B are parallel");
  for (int i = 0; i < 3; ++i) {
    a.C[i] = c[i] / nc;
    a.J[i] = prob->J[i];
    a.H[i] = prob->hmom[i];
  }
  a.x0 = d_x0;
  a.n = n;
  a.target = d_target;
  a.status = d_status;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SG_TIMED("k_attitude_targets", st,
           (sg::k_attitude_targets<<<static_cast<unsigned>(sg::ceil_div(n, 64)), 64, 0, st>>>(a)));
  SG_LAUNCH_CHECK("k_attitude_targets");
  return SG_OK;
}
