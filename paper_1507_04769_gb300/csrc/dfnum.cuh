// Pair-of-floats number type for templated device code (about 48
// significant bits on the FP32 pipe).  A value is hi + lo with |lo| <= ulp(hi)/2
// after every operation.  Sums use Knuth's two_sum, products the FMA-based
// exact product; every step is an explicitly rounded intrinsic, so the
// compiler cannot contract them.  Sine and cosine on |x| <= pi/4 are the
// Taylor polynomials through x^17 / x^18 evaluated in this arithmetic; larger
// arguments go through the FP64 function.
#pragma once

#include <cuda_runtime.h>

namespace sg {

struct dfnum {
  float hi, lo;
  __device__ __forceinline__ dfnum() = default;
  __device__ __forceinline__ constexpr dfnum(float h, float l, int) : hi(h), lo(l) {}
  // nearest pair to x (plain conversions, so constant arguments fold at compile time)
  __device__ __forceinline__ constexpr dfnum(double x)
      : hi(static_cast<float>(x)), lo(static_cast<float>(x - static_cast<double>(static_cast<float>(x)))) {}
  __device__ __forceinline__ double to_double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

__device__ __forceinline__ dfnum df_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfnum(h, __fsub_rn(e, __fsub_rn(h, s)), 0);
}

__device__ __forceinline__ dfnum operator+(dfnum a, dfnum b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_renorm(s, e);
}
__device__ __forceinline__ dfnum operator-(dfnum a) { return dfnum(-a.hi, -a.lo, 0); }
__device__ __forceinline__ dfnum operator-(dfnum a, dfnum b) { return a + (-b); }
__device__ __forceinline__ dfnum operator*(dfnum a, dfnum b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_renorm(p, e);
}
__device__ __forceinline__ dfnum operator+(dfnum a, double b) { return a + dfnum(b); }
__device__ __forceinline__ dfnum operator+(double a, dfnum b) { return dfnum(a) + b; }
__device__ __forceinline__ dfnum operator-(dfnum a, double b) { return a - dfnum(b); }
__device__ __forceinline__ dfnum operator-(double a, dfnum b) { return dfnum(a) - b; }
__device__ __forceinline__ dfnum operator*(dfnum a, double b) { return a * dfnum(b); }
__device__ __forceinline__ dfnum operator*(double a, dfnum b) { return dfnum(a) * b; }

// 1 / a: FP32 reciprocal corrected by one Newton step on the pair.
__device__ __forceinline__ dfnum recip(dfnum a) {
  const float q = __frcp_rn(a.hi);
  float r = __fmaf_rn(-a.hi, q, 1.0f);
  r = __fmaf_rn(-a.lo, q, r);
  return df_renorm(q, __fmul_rn(q, r));
}

__device__ __forceinline__ void dsincos(dfnum a, dfnum* s, dfnum* c) {
  const double ad = a.to_double();
  if (fabs(ad) > 0.78539816339744831) {
    double sd, cd;
    sincos(ad, &sd, &cd);
    *s = dfnum(sd);
    *c = dfnum(cd);
    return;
  }
  const dfnum z = a * a;
  // sin a = a (1 - z/3! + ... + z^8/17!), cos a = 1 - z (1/2! - z/4! + ... + z^8/18!)
  dfnum ps(1.0 / 355687428096000.0);
  ps = ps * z + dfnum(-1.0 / 1307674368000.0);
  ps = ps * z + dfnum(1.0 / 6227020800.0);
  ps = ps * z + dfnum(-1.0 / 39916800.0);
  ps = ps * z + dfnum(1.0 / 362880.0);
  ps = ps * z + dfnum(-1.0 / 5040.0);
  ps = ps * z + dfnum(1.0 / 120.0);
  ps = ps * z + dfnum(-1.0 / 6.0);
  *s = a + (a * z) * ps;
  dfnum pc(1.0 / 6402373705728000.0);
  pc = pc * z + dfnum(-1.0 / 20922789888000.0);
  pc = pc * z + dfnum(1.0 / 87178291200.0);
  pc = pc * z + dfnum(-1.0 / 479001600.0);
  pc = pc * z + dfnum(1.0 / 3628800.0);
  pc = pc * z + dfnum(-1.0 / 40320.0);
  pc = pc * z + dfnum(1.0 / 720.0);
  pc = pc * z + dfnum(-1.0 / 24.0);
  pc = pc * z + dfnum(0.5);
  *c = dfnum(1.0) - z * pc;
}

}  // namespace sg
