// Device-side optimal control problems and their characteristic equations.
//
// Section 2: H = L + lambda' f, u* = argmin_u H.  Eq. hamchar: x' = H_lambda',
// lambda' = -H_x'.  Both families are control-affine with cost 0.5 u'Ru, so
//   u*      = -G lambda                 (G = R^-1 Bf')
//   x'      = f0(x) - K lambda          (K = Bf R^-1 Bf')
//   lambda' = -grad l(x) - f0_x(x)' lambda
// The Jacobian dF/dy of the 12-dimensional right-hand side is the Hamiltonian
// matrix [[f0_x, -K], [-(l_xx + d2(lambda' f0)/dx2), -f0_x']]; f0_x and the
// second derivative come from one forward-mode pass with dual numbers carrying
// the six state directions.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "dfnum.cuh"

namespace sg {

// Problem data with the derived matrices precomputed on the host.
struct DevProblem {
  int kind;
  int m;                 // attitude: number of controls (2 or 3)
  const double* target;  // attitude: per-node target attitudes v_e (n x 3) or null
  // attitude (Section 5, Eq. sat_model)
  double Jinv[3];
  double hm[3];
  double Kw[9];   // (J^-1 B)(J^-1 B)' / r : K restricted to the w block
  double Gw[9];   // B' J^-1 / r : u* = -Gw lambda_w
  double wv, ww, r, tv, tw;
  // LQ
  double A[36];
  double K[36];   // B R^-1 B'
  double Q[36];
  double QT[36];
  double G[18];   // R^-1 B' (3 x 6)
  double R[9];
  double Bu[18];  // plant input matrix: attitude J^-1 B (rows 3..5 of a 6 x 3), LQ B (6 x 3)
  // the constants of the right-hand side as (hi, lo) float pairs, for the
  // pair-of-floats residual of the mixed-pair form (filled on the host)
  float2 Jinv_f[3], hm_f[3], Kw_f[9], wv_f, ww_f;
  float2 A_f[36], K_f[36], Q_f[36];
};

// A problem constant in the number type S of templated code: the double, its
// float pair, or its float rounding (FP32 Jacobian).
template <typename S>
__device__ __forceinline__ S pconst(double d, float2 f);
template <>
__device__ __forceinline__ double pconst<double>(double d, float2) { return d; }
template <>
__device__ __forceinline__ float pconst<float>(double, float2 f) { return f.x; }   // the nearest float, stored
template <>
__device__ __forceinline__ dfnum pconst<dfnum>(double, float2 f) { return dfnum(f.x, f.y, 0); }

// ------------------------------------------------------------------ duals
// FP64 sine and cosine.  On |a| <= pi/4 (where the Euler angles of the
// attitude problem stay), with z = a^2,
//   sin a = a + a z P(z),  cos a = 1 + z (-1/2 + z Q(z)),
// P and Q of degree 5 being the weighted minimax polynomials for the relative
// error of sin and cos on that interval (the Remez exchange algorithm; the
// derivation, and its check of these literals, are in sincos_coeffs.py beside
// this package's sources).  The rounded polynomials are within 1.3e-17
// (sin) and 6e-19 (cos) of the functions; with the fused Horner evaluation
// the results are within about one unit in the last place.  Larger arguments
// take the CUDA library sincos.
__device__ __forceinline__ void dsincos(double a, double* s, double* c) {
  if (fabs(a) <= 0.78539816339744831) {
    const double z = a * a;
    double ps = 0x1.5d8773e0ff40dp-33;
    ps = fma(ps, z, -0x1.ae5e4c58b3d0ap-26);
    ps = fma(ps, z, 0x1.71de356f7490ap-19);
    ps = fma(ps, z, -0x1.a01a019c30bb6p-13);
    ps = fma(ps, z, 0x1.111111110fb50p-7);
    ps = fma(ps, z, -0x1.555555555554dp-3);
    *s = fma(a * z, ps, a);
    double pc = -0x1.8ff9dcba514eep-37;
    pc = fma(pc, z, 0x1.1eea895d2f6e9p-29);
    pc = fma(pc, z, -0x1.27e4f9040bb84p-22);
    pc = fma(pc, z, 0x1.a01a019e24efcp-16);
    pc = fma(pc, z, -0x1.6c16c16c16134p-10);
    pc = fma(pc, z, 0x1.5555555555553p-5);
    pc = fma(pc, z, -0.5);
    *c = fma(z, pc, 1.0);
  } else {
    sincos(a, s, c);
  }
}
__device__ __forceinline__ void dsincos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ double recip(double a) { return __drcp_rn(a); }   // = 1.0 / a, without the division path
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }

template <typename T, int N>
struct Dual {
  T v;
  T d[N];
};

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> dconst(T a) {
  Dual<T, N> r;
  r.v = a;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = T(0);
  return r;
}

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, T s) {
  Dual<T, N> r;
  r.v = a.v * s;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator*(T s, const Dual<T, N>& a) { return a * s; }
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, T s) {
  Dual<T, N> r = a;
  r.v += s;
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> recip(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = T(1) / a.v;
  T m = -r.v * r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * m;
  return r;
}
template <typename T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, T s) {
  Dual<T, N> r = a;
  r.v = a.v - s;
  return r;
}

// Scalar type of a plain or dual number (for constants in templated code).
template <typename S>
struct ScalarOf {
  using type = S;
};
template <typename T, int N>
struct ScalarOf<Dual<T, N>> {
  using type = T;
};

template <typename T, int N>
__device__ __forceinline__ void dsincos(const Dual<T, N>& a, Dual<T, N>* s, Dual<T, N>* c) {
  T sv, cv;
  dsincos(a.v, &sv, &cv);
  s->v = sv;
  c->v = cv;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    s->d[i] = cv * a.d[i];
    c->d[i] = -sv * a.d[i];
  }
}


// ------------------------------------------------------------------ attitude
// f0(x) and g = grad_x(lambda' f0(x)) for x of scalar type S (plain or dual)
// and lambda of plain type T.
//   v' = E(v) w with 3-2-1 Euler angles,
//   w' = J^-1 (g x w), g = R(v) h, R = Rx(phi) Ry(theta) Rz(psi).
//   lambda' f0 = lv' E(v) w + p . (g x w), p = J^-1 lw:
//     d/dw   = E(v)' lv + p x g
//     d/dv_k = lv' (dE/dv_k) w + (dg/dv_k) . (w x p)
template <typename S, typename T>
__device__ __forceinline__ void attitude_f0_grad(const DevProblem& P, const S* x, const T* lam,
                                                 S* f0, S* g) {
  const S& ph = x[0];
  const S& th = x[1];
  const S& ps = x[2];
  const S& w1 = x[3];
  const S& w2 = x[4];
  const S& w3 = x[5];
  S sp, cp, st, ct, ss, cs;
  dsincos(ph, &sp, &cp);
  dsincos(th, &st, &ct);
  dsincos(ps, &ss, &cs);
  S sec = recip(ct);
  S tt = st * sec;
  S a = sp * w2 + cp * w3;          // sp w2 + cp w3
  S b = cp * w2 - sp * w3;          // cp w2 - sp w3
  // E(v) w
  f0[0] = w1 + tt * a;
  f0[1] = b;
  f0[2] = sec * a;
  // g = Rx Ry Rz h
  const T h0 = pconst<T>(P.hm[0], P.hm_f[0]), h1 = pconst<T>(P.hm[1], P.hm_f[1]), h2 = pconst<T>(P.hm[2], P.hm_f[2]);
  S az0 = cs * h0 + ss * h1;
  S az1 = cs * h1 - ss * h0;
  // Ry applied to (az0, az1, h2)
  S ay0 = ct * az0 - st * h2;
  S ay2 = st * az0 + ct * h2;
  // Rx applied to (ay0, az1, ay2)
  S g0 = ay0;
  S g1 = cp * az1 + sp * ay2;
  S g2 = cp * ay2 - sp * az1;
  const T j0 = pconst<T>(P.Jinv[0], P.Jinv_f[0]), j1 = pconst<T>(P.Jinv[1], P.Jinv_f[1]),
          j2 = pconst<T>(P.Jinv[2], P.Jinv_f[2]);
  // g x w
  f0[3] = (g1 * w3 - g2 * w2) * j0;
  f0[4] = (g2 * w1 - g0 * w3) * j1;
  f0[5] = (g0 * w2 - g1 * w1) * j2;

  // ---- gradient of lambda' f0
  const T lv0 = lam[0], lv1 = lam[1], lv2 = lam[2];
  const T p0 = lam[3] * j0, p1 = lam[4] * j1, p2 = lam[5] * j2;
  // w x p
  S q0 = w2 * p2 - w3 * p1;
  S q1 = w3 * p0 - w1 * p2;
  S q2 = w1 * p1 - w2 * p0;
  // dg/dphi = dRx (ay0, az1, ay2) = (0, -sp az1 + cp ay2, -cp az1 - sp ay2)
  S dphi1 = cp * ay2 - sp * az1;
  S dphi2 = -(cp * az1 + sp * ay2);
  // dg/dtheta = Rx dRy (az0, az1, h2); dRy a = (-st a0 - ct a2, 0, ct a0 - st a2)
  S e0 = -(st * az0 + ct * h2);
  S e2 = ct * az0 - st * h2;
  S dth0 = e0;
  S dth1 = sp * e2;
  S dth2 = cp * e2;
  // dg/dpsi = Rx Ry dRz h; dRz h = (-ss h0 + cs h1, -cs h0 - ss h1, 0) = (az1, -az0, 0)
  S f0y = ct * az1;           // Ry (az1, -az0, 0): (ct az1, -az0, st az1)
  S f2y = st * az1;
  S dps0 = f0y;
  S dps1 = sp * f2y - cp * az0;
  S dps2 = cp * f2y + sp * az0;
  // dE/dphi w = (tt b', -a, sec b')  with b' = cp w2 - sp w3 = b, a as above
  // dE/dtheta w = (sec^2 a, 0, sec^2 st a)
  S sec2a = sec * sec * a;
  g[0] = (tt * b) * lv0 - a * lv1 + (sec * b) * lv2 + dphi1 * q1 + dphi2 * q2;
  g[1] = sec2a * lv0 + (st * sec2a) * lv2 + dth0 * q0 + dth1 * q1 + dth2 * q2;
  g[2] = dps0 * q0 + dps1 * q1 + dps2 * q2;
  // E' lv + p x g
  g[3] = (g2 * p1 - g1 * p2) + lv0;
  g[4] = (sp * tt) * lv0 + cp * lv1 + (sp * sec) * lv2 + (p2 * g0 - p0 * g2);
  g[5] = (cp * tt) * lv0 - sp * lv1 + (cp * sec) * lv2 + (p0 * g1 - p1 * g0);
}


// ------------------------------------------------------------------ Example III
// Section 5, Example III: x1' = -x1 + x2, x2' = -x2 + x3 / g,
// x3' = (-2 x1^2 + 2 x1 x2 - 2 x2^2 + 2 x2 x3 / g) x3 / g + g u with
// g = 1 + x1^2 + x2^2, running cost 0.5 (x3^2 / g^2 + u^2), no terminal cost.
// The three states sit in components 0..2 of the six-state layout; the
// others have zero dynamics and cost (they stay 0 from x0 = 0).  With
// B(x) = g e3: u* = -g lambda3 and H* = l + lambda' f0 - 0.5 g^2 lambda3^2, so
//   x'      = f0 - g^2 lambda3 e3
//   lambda' = -(grad l + f0_x' lambda - g lambda3^2 grad g).
// Templated on the number type so that one source gives the FP64 right-hand
// side and, with duals over (x1, x2, x3, lambda1..3), the Jacobian.
template <typename S>
__device__ __forceinline__ void ex3_char(const S* x, const S* lam, S* dx, S* dl) {
  using R = typename ScalarOf<S>::type;
  const S& x1 = x[0];
  const S& x2 = x[1];
  const S& x3 = x[2];
  const S& l1 = lam[0];
  const S& l2 = lam[1];
  const S& l3 = lam[2];
  const S g = x1 * x1 + x2 * x2 + R(1);
  const S gi = recip(g);
  const S gi2 = gi * gi;
  const S x3gi = x3 * gi;
  const S q = R(2) * (x1 * x2 - x1 * x1 - x2 * x2 + x2 * x3gi);
  dx[0] = x2 - x1;
  dx[1] = x3gi - x2;
  dx[2] = q * x3gi - g * g * l3;
  // partial derivatives of f0_2, q, f0_3
  const S x3gi2 = x3 * gi2;
  const S f2_1 = R(-2) * x1 * x3gi2;
  const S f2_2 = R(-2) * x2 * x3gi2 - R(1);
  const S q_1 = R(2) * (x2 - R(2) * x1) - R(4) * x1 * x2 * x3gi2;
  const S q_2 = R(2) * (x1 - R(2) * x2) + R(2) * x3gi - R(4) * x2 * x2 * x3gi2;
  const S q_3 = R(2) * x2 * gi;
  const S f3_1 = x3gi * (q_1 - R(2) * x1 * q * gi);
  const S f3_2 = x3gi * (q_2 - R(2) * x2 * q * gi);
  const S f3_3 = q * gi + x3gi * q_3;
  // grad l, l = 0.5 x3^2 / g^2
  const S lx3 = x3 * gi2;
  const S lx1 = R(-2) * x1 * x3gi * lx3;
  const S lx2 = R(-2) * x2 * x3gi * lx3;
  const S gl32 = g * l3 * l3;
  dl[0] = -(lx1 - l1 + l2 * f2_1 + l3 * f3_1 - R(2) * x1 * gl32);
  dl[1] = -(lx2 + l1 + l2 * f2_2 + l3 * f3_2 - R(2) * x2 * gl32);
  dl[2] = -(lx3 + l2 * gi + l3 * f3_3);
}

// ------------------------------------------------------------------ RHS and Jacobian
// F(y) for y = (x, lambda) in the number type S: double (FP64) or dfnum
// (pair of floats, the residual of the mixed-pair form).
template <typename S>
__device__ __forceinline__ void char_rhs_t(const DevProblem& P, const S* y, S* F, const double* ve = nullptr) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) {
    S dx[3], dl[3];
    ex3_char<S>(y, y + 6, dx, dl);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      F[i] = dx[i];
      F[3 + i] = S(0.0);
      F[6 + i] = dl[i];
      F[9 + i] = S(0.0);
    }
    return;
  }
  if (P.kind == SG_PROBLEM_ATTITUDE) {
    S f0[6], g[6];
    attitude_f0_grad<S, S>(P, y, y + 6, f0, g);
#pragma unroll
    for (int i = 0; i < 3; ++i) F[i] = f0[i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      F[3 + i] = f0[3 + i] - (pconst<S>(P.Kw[3 * i], P.Kw_f[3 * i]) * y[9] +
                              pconst<S>(P.Kw[3 * i + 1], P.Kw_f[3 * i + 1]) * y[10] +
                              pconst<S>(P.Kw[3 * i + 2], P.Kw_f[3 * i + 2]) * y[11]);
    const S wv = pconst<S>(P.wv, P.wv_f), ww = pconst<S>(P.ww, P.ww_f);
    if (ve) {   // running cost on v - v_e
#pragma unroll
      for (int i = 0; i < 3; ++i) F[6 + i] = -(wv * (y[i] - S(ve[i]))) - g[i];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) F[6 + i] = -(wv * y[i]) - g[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) F[9 + i] = -(ww * y[3 + i]) - g[3 + i];
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      S ax(0.0), kl(0.0), qx(0.0), atl(0.0);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        ax = ax + pconst<S>(P.A[6 * i + j], P.A_f[6 * i + j]) * y[j];
        kl = kl + pconst<S>(P.K[6 * i + j], P.K_f[6 * i + j]) * y[6 + j];
        qx = qx + pconst<S>(P.Q[6 * i + j], P.Q_f[6 * i + j]) * y[j];
        atl = atl + pconst<S>(P.A[6 * j + i], P.A_f[6 * j + i]) * y[6 + j];
      }
      F[i] = ax - kl;
      F[6 + i] = -qx - atl;
    }
  }
}

__device__ __forceinline__ void char_rhs(const DevProblem& P, const double* y, double* F,
                                         const double* ve = nullptr) {
  char_rhs_t<double>(P, y, F, ve);
}

// The target attitude row of a node (attitude family), or null.
__device__ __forceinline__ const double* node_target(const DevProblem& P, int64_t node) {
  return (P.kind == SG_PROBLEM_ATTITUDE && P.target) ? P.target + node * 3 : nullptr;
}

// Jacobian dF/dy (12 x 12) in precision T, from one dual pass over the six
// state directions, at y of type Y (double, or float already rounded).  Row r
// goes to put_row(r, row[12]), in the order r = 0..11 (every thread of a warp
// makes the same calls, so the sink may work across the warp).  If Fout is
// non-null and y is double, the FP64 right-hand side from the value parts is
// written there as well.
template <typename T, typename Y, typename Sink>
__device__ __forceinline__ void char_jacobian_rows(const DevProblem& P, const Y* y, Sink&& put_row,
                                                   double* Fout) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) {
    using D = Dual<T, 6>;
    D x[3], lam[3], dx[3], dl[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x[i] = dconst<T, 6>(T(y[i]));
      x[i].d[i] = T(1);
      lam[i] = dconst<T, 6>(T(y[6 + i]));
      lam[i].d[3 + i] = T(1);
    }
    ex3_char<D>(x, lam, dx, dl);
    // rows 0..2 (x') and 6..8 (lambda'); columns 0..2 (x) and 6..8 (lambda)
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      T row[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) row[c] = T(0);
      if (r < 3 || (r >= 6 && r < 9)) {
        const D& f = r < 3 ? dx[r] : dl[r - 6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          row[c] = f.d[c];
          row[6 + c] = f.d[3 + c];
        }
      }
      put_row(r, row);
    }
    if constexpr (sizeof(Y) == sizeof(double)) {
      if (Fout) char_rhs(P, y, Fout);
    }
    return;
  }
  if (P.kind == SG_PROBLEM_ATTITUDE) {
    using D = Dual<T, 6>;
    D x[6], f0[6], g[6];
    T lam[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      x[i] = dconst<T, 6>(T(y[i]));
      x[i].d[i] = T(1);
      lam[i] = T(y[6 + i]);
    }
    attitude_f0_grad<D, T>(P, x, lam, f0, g);
    const T wv = pconst<T>(P.wv, P.wv_f), ww = pconst<T>(P.ww, P.ww_f);
    const T wdiag[6] = {wv, wv, wv, ww, ww, ww};
    // rows are assembled in registers and written as 16-byte vectors
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      T row[12];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (r < 6) {
          row[c] = f0[r].d[c];                                             // f0_x
          T k = T(0);
          if (r >= 3 && c >= 3) k = pconst<T>(P.Kw[3 * (r - 3) + (c - 3)], P.Kw_f[3 * (r - 3) + (c - 3)]);
          row[6 + c] = -k;                                                 // -K
        } else {
          row[c] = -g[r - 6].d[c] - (r - 6 == c ? wdiag[r - 6] : T(0));    // -(l_xx + phi_xx)
          row[6 + c] = -f0[c].d[r - 6];                                    // -f0_x'
        }
      }
      put_row(r, row);
    }
    if (sizeof(Y) == sizeof(double) && Fout) {
#pragma unroll
      for (int i = 0; i < 3; ++i) Fout[i] = double(f0[i].v);
#pragma unroll
      for (int i = 0; i < 3; ++i)
        Fout[3 + i] = double(f0[3 + i].v) -
                      (P.Kw[3 * i] * y[9] + P.Kw[3 * i + 1] * y[10] + P.Kw[3 * i + 2] * y[11]);
#pragma unroll
      for (int i = 0; i < 3; ++i) Fout[6 + i] = -P.wv * y[i] - double(g[i].v);
#pragma unroll
      for (int i = 0; i < 3; ++i) Fout[9 + i] = -P.ww * y[3 + i] - double(g[3 + i].v);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      T row[12];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (r < 6) {
          row[c] = T(P.A[6 * r + c]);
          row[6 + c] = T(-P.K[6 * r + c]);
        } else {
          row[c] = T(-P.Q[6 * (r - 6) + c]);
          row[6 + c] = T(-P.A[6 * c + (r - 6)]);
        }
      }
      put_row(r, row);
    }
    if constexpr (sizeof(Y) == sizeof(double)) {
      if (Fout) char_rhs(P, y, Fout);
    }
  }
}

// The same Jacobian stored row-major at Jm (16-byte rows).
template <typename T>
__device__ __forceinline__ void char_jacobian(const DevProblem& P, const double* y, T* Jm, double* Fout) {
  char_jacobian_rows<T>(
      P, y,
      [&](int r, const T (&row)[12]) {
        if constexpr (sizeof(T) == 4) {
          float4* dst = reinterpret_cast<float4*>(Jm + 12 * r);
#pragma unroll
          for (int q4 = 0; q4 < 3; ++q4)
            dst[q4] = make_float4(row[4 * q4], row[4 * q4 + 1], row[4 * q4 + 2], row[4 * q4 + 3]);
        } else {
          double2* dst = reinterpret_cast<double2*>(Jm + 12 * r);
#pragma unroll
          for (int q2 = 0; q2 < 6; ++q2) dst[q2] = make_double2(row[2 * q2], row[2 * q2 + 1]);
        }
      },
      Fout);
}

// Running cost L(x, u*(x, lambda)) (Section 2) at y = (x, lambda).
__device__ __forceinline__ double running_cost(const DevProblem& P, const double* y, const double* ve = nullptr) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) {
    const double g = 1.0 + y[0] * y[0] + y[1] * y[1];
    const double u = -g * y[8];
    return 0.5 * (y[2] * y[2] / (g * g) + u * u);
  }
  if (P.kind == SG_PROBLEM_ATTITUDE) {
    double u[3], su = 0.0, sv = 0.0, sw = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      u[i] = -(P.Gw[3 * i] * y[9] + P.Gw[3 * i + 1] * y[10] + P.Gw[3 * i + 2] * y[11]);
      su += u[i] * u[i];
      const double dv = ve ? y[i] - ve[i] : y[i];
      sv += dv * dv;
      sw += y[3 + i] * y[3 + i];
    }
    return 0.5 * (P.wv * sv + P.ww * sw + P.r * su);
  }
  double u[3], xqx = 0.0, uru = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) s += P.G[6 * i + j] * y[6 + j];
    u[i] = -s;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) s += P.Q[6 * i + j] * y[j];
    xqx += y[i] * s;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) s += P.R[3 * i + j] * u[j];
    uru += u[i] * s;
  }
  return 0.5 * (xqx + uru);
}

// Terminal cost h(x(T)), its gradient and Hessian.
__device__ __forceinline__ double terminal_cost(const DevProblem& P, const double* x) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) return 0.0;
  if (P.kind == SG_PROBLEM_ATTITUDE)
    return 0.5 * (P.tv * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) +
                  P.tw * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]));
  double v = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) s += P.QT[6 * i + j] * x[j];
    v += x[i] * s;
  }
  return 0.5 * v;
}

__device__ __forceinline__ double terminal_grad(const DevProblem& P, const double* x, int i) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) return 0.0;
  if (P.kind == SG_PROBLEM_ATTITUDE) return (i < 3 ? P.tv : P.tw) * x[i];
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) s += P.QT[6 * i + j] * x[j];
  return s;
}

__device__ __forceinline__ double terminal_hess(const DevProblem& P, int i, int j) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) return 0.0;
  if (P.kind == SG_PROBLEM_ATTITUDE) return i == j ? (i < 3 ? P.tv : P.tw) : 0.0;
  return P.QT[6 * i + j];
}

// u*(x, lambda) = -R^-1 B(x)' lambda.
__device__ __forceinline__ void optimal_control(const DevProblem& P, const double* x, const double* lam,
                                                double* u) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) {
    u[0] = -(1.0 + x[0] * x[0] + x[1] * x[1]) * lam[2];
    u[1] = 0.0;
    u[2] = 0.0;
  } else if (P.kind == SG_PROBLEM_ATTITUDE) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
      u[i] = -(P.Gw[3 * i] * lam[3] + P.Gw[3 * i + 1] * lam[4] + P.Gw[3 * i + 2] * lam[5]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < 6; ++j) s += P.G[6 * i + j] * lam[j];
      u[i] = -s;
    }
  }
}

// ------------------------------------------------------------------ plant
// Closed-loop plant x' = f(x, u) = f0(x) + Bu u for a given control u
// (attitude: v' = E(v) w, w' = J^-1 (R(v) h x w) + J^-1 B u; LQ: A x + B u).
__device__ __forceinline__ void plant_rhs(const DevProblem& P, const double* x, const double* u, double* f) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) {
    const double lam0[3] = {0.0, 0.0, 0.0};
    double dx[3], dl[3];
    ex3_char<double>(x, lam0, dx, dl);
    f[0] = dx[0];
    f[1] = dx[1];
    f[2] = dx[2] + (1.0 + x[0] * x[0] + x[1] * x[1]) * u[0];
    f[3] = f[4] = f[5] = 0.0;
  } else if (P.kind == SG_PROBLEM_ATTITUDE) {
    double f0[6], g[6];
    const double lam0[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    attitude_f0_grad<double, double>(P, x, lam0, f0, g);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      f[i] = f0[i] + P.Bu[3 * i] * u[0] + P.Bu[3 * i + 1] * u[1] + P.Bu[3 * i + 2] * u[2];
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double s = P.Bu[3 * i] * u[0] + P.Bu[3 * i + 1] * u[1] + P.Bu[3 * i + 2] * u[2];
#pragma unroll
      for (int j = 0; j < 6; ++j) s += P.A[6 * i + j] * x[j];
      f[i] = s;
    }
  }
}

// Running cost L(x, u) (Section 2) for a given control.
__device__ __forceinline__ double running_cost_xu(const DevProblem& P, const double* x, const double* u) {
  if (P.kind == SG_PROBLEM_EXAMPLE3) {
    const double g = 1.0 + x[0] * x[0] + x[1] * x[1];
    return 0.5 * (x[2] * x[2] / (g * g) + u[0] * u[0]);
  }
  if (P.kind == SG_PROBLEM_ATTITUDE) {
    double sv = 0.0, sw = 0.0, su = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sv += x[i] * x[i];
      sw += x[3 + i] * x[3 + i];
      su += u[i] * u[i];
    }
    return 0.5 * (P.wv * sv + P.ww * sw + P.r * su);
  }
  double xqx = 0.0, uru = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) s += P.Q[6 * i + j] * x[j];
    xqx += x[i] * s;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) s += P.R[3 * i + j] * u[j];
    uru += u[i] * s;
  }
  return 0.5 * (xqx + uru);
}

// Host: derive the device problem from the ABI struct.  Returns false if R is singular.
bool make_dev_problem(const sg_problem& in, DevProblem* out);

}  // namespace sg
