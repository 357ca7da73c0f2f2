// One-dimensional hierarchical basis on nested Chebyshev-Gauss-Lobatto sets
// (Section 3.3): a^i_j is the Lagrange polynomial on X^i that is 1 at its
// point of dX^i, evaluated in barycentric form with the Chebyshev-Lobatto
// weights w_m = (-1)^m delta_m (delta = 1/2 at the ends) from the reciprocals
// 1/(u - x_p) of the finest set (every coarser set is a subset of it).
// FP64 form and pair-of-floats form (about 48 significant bits on the FP32
// pipe: exact products by FMA, Knuth's two_sum, corrected reciprocal).
#pragma once

#include "common.cuh"
#include "interp.cuh"

namespace sg {

// All 1-D basis values at one coordinate u in [0, 1] for levels 1..L+1,
// written to tab[id * stride].  xf holds the fine_n + 1 = 2^L + 1 points of
// the finest set X^{L+1}.  Exact Kronecker values when u coincides with a
// point of the level's set.
__device__ inline void basis_row(double u, int level, const double* __restrict__ xf, double* tab, int stride) {
  tab[0] = 1.0;   // a^1 = 1
  if (level == 0) return;
  const int fine_n = 1 << level;
  double rinv[kMaxFine + 1];
  int hit = -1;
  for (int p = 0; p <= fine_n; ++p) {
    const double diff = u - xf[p];
    if (diff == 0.0) hit = p;
    rinv[p] = diff == 0.0 ? 0.0 : 1.0 / diff;
  }
  int id = 1;
  for (int l = 2; l <= level + 1; ++l) {
    const int n = 1 << (l - 1);            // X^l has n + 1 points
    const int sf = fine_n / n;             // point m of X^l is fine point m * sf
    const bool exact = hit >= 0 && (hit % sf) == 0;
    double denom = 0.0;
    if (!exact) {
      for (int m = 0; m <= n; ++m) {
        double wm = (m & 1) ? -1.0 : 1.0;
        if (m == 0 || m == n) wm *= 0.5;
        denom += wm * rinv[m * sf];
      }
    }
    const double inv_denom = exact ? 0.0 : 1.0 / denom;
    // increment points of X^l: level 2 -> m = 0, n; level >= 3 -> odd m
    const int cnt = l == 2 ? 2 : (n >> 1);
    for (int j = 0; j < cnt; ++j) {
      const int m = l == 2 ? j * n : 2 * j + 1;
      double v;
      if (exact) {
        v = (m * sf == hit) ? 1.0 : 0.0;
      } else {
        double wm = (m & 1) ? -1.0 : 1.0;
        if (m == 0 || m == n) wm *= 0.5;
        v = wm * rinv[m * sf] * inv_denom;
      }
      tab[(id + j) * stride] = v;
    }
    id += cnt;
  }
}


struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_from(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - static_cast<double>(hi))};
}

__device__ __forceinline__ df df_norm(float s, float e) {
  const float hi = __fadd_rn(s, e);
  return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}

__device__ __forceinline__ df df_scale(df a, float s) {   // s exact power-of-two multiple of +-1
  return {__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)};
}

__device__ __forceinline__ df df_recip(df a) {
  // the hardware's approximate reciprocal (a few ulp); the Newton correction
  // below takes the pair to the same accuracy as from a rounded one
  float q;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(a.hi));
  // residual 1 - a q, with a = hi + lo
  float r = __fmaf_rn(-a.hi, q, 1.0f);
  r = __fmaf_rn(-a.lo, q, r);
  return df_norm(q, __fmul_rn(q, r));
}

// All 1-D basis values at u (FP64 in [0,1]) for levels 1..L+1, as pairs, in
// barycentric form on the finest set (see basis_row in interp.cu).
// The same for a level fixed at compile time: every loop unrolls, so the
// reciprocals stay in registers (the general form indexes them at run time,
// which puts them in local memory).
template <int L, typename Out>
__device__ __forceinline__ void basis_row_df_t(double u, const float2* __restrict__ xf, Out out) {
  constexpr int fine_n = 1 << L;
  out(0, df{1.0f, 0.0f});
  const df uu = df_from(u);
  df rinv[fine_n + 1];
  int hit = -1;
#pragma unroll
  for (int p = 0; p <= fine_n; ++p) {
    const df d = df_sub(uu, {xf[p].x, xf[p].y});
    if (d.hi == 0.0f && d.lo == 0.0f) {
      hit = p;
      rinv[p] = {0.0f, 0.0f};
    } else {
      rinv[p] = df_recip(d);
    }
  }
  int id = 1;
#pragma unroll
  for (int l = 2; l <= L + 1; ++l) {
    const int n = 1 << (l - 1);
    const int sf = fine_n / n;
    const bool exact = hit >= 0 && (hit % sf) == 0;
    df inv_denom = {0.0f, 0.0f};
    if (!exact) {
      df den = {0.0f, 0.0f};
#pragma unroll
      for (int m = 0; m <= n; ++m) {
        float wm = (m & 1) ? -1.0f : 1.0f;
        if (m == 0 || m == n) wm *= 0.5f;
        den = df_add(den, df_scale(rinv[m * sf], wm));
      }
      inv_denom = df_recip(den);
    }
    const int cnt = l == 2 ? 2 : (n >> 1);
#pragma unroll
    for (int j = 0; j < cnt; ++j) {
      const int m = l == 2 ? j * n : 2 * j + 1;
      df v;
      if (exact) {
        v = {(m * sf == hit) ? 1.0f : 0.0f, 0.0f};
      } else {
        float wm = (m & 1) ? -1.0f : 1.0f;
        if (m == 0 || m == n) wm *= 0.5f;
        v = df_mul(df_scale(rinv[m * sf], wm), inv_denom);
      }
      out(id + j, v);
    }
    id += cnt;
  }
}

template <typename Out>
__device__ inline void basis_row_df_out(double u, int level, const float2* __restrict__ xf, Out out) {
  switch (level) {
    case 1: return basis_row_df_t<1>(u, xf, out);
    case 2: return basis_row_df_t<2>(u, xf, out);
    case 3: return basis_row_df_t<3>(u, xf, out);
    case 4: return basis_row_df_t<4>(u, xf, out);
    case 5: return basis_row_df_t<5>(u, xf, out);
    default: break;
  }
  out(0, df{1.0f, 0.0f});
  if (level == 0) return;
  const int fine_n = 1 << level;
  const df uu = df_from(u);
  df rinv[kMaxFine + 1];
  int hit = -1;
  for (int p = 0; p <= fine_n; ++p) {
    const df d = df_sub(uu, {xf[p].x, xf[p].y});
    if (d.hi == 0.0f && d.lo == 0.0f) {
      hit = p;
      rinv[p] = {0.0f, 0.0f};
    } else {
      rinv[p] = df_recip(d);
    }
  }
  int id = 1;
  for (int l = 2; l <= level + 1; ++l) {
    const int n = 1 << (l - 1);
    const int sf = fine_n / n;
    const bool exact = hit >= 0 && (hit % sf) == 0;
    df inv_denom = {0.0f, 0.0f};
    if (!exact) {
      df den = {0.0f, 0.0f};
      for (int m = 0; m <= n; ++m) {
        float wm = (m & 1) ? -1.0f : 1.0f;
        if (m == 0 || m == n) wm *= 0.5f;
        den = df_add(den, df_scale(rinv[m * sf], wm));
      }
      inv_denom = df_recip(den);
    }
    const int cnt = l == 2 ? 2 : (n >> 1);
    for (int j = 0; j < cnt; ++j) {
      const int m = l == 2 ? j * n : 2 * j + 1;
      df v;
      if (exact) {
        v = {(m * sf == hit) ? 1.0f : 0.0f, 0.0f};
      } else {
        float wm = (m & 1) ? -1.0f : 1.0f;
        if (m == 0 || m == n) wm *= 0.5f;
        v = df_mul(df_scale(rinv[m * sf], wm), inv_denom);
      }
      out(id + j, v);
    }
    id += cnt;
  }
}

// Writers of basis_row_df_out: the pairs, or their leading floats (the
// values rounded once to FP32).
struct DfPairOut {
  float2* tab;
  int stride;
  __device__ __forceinline__ void operator()(int id, df v) const { tab[id * stride] = make_float2(v.hi, v.lo); }
};
struct DfHiOut {
  float* tab;
  int stride;
  __device__ __forceinline__ void operator()(int id, df v) const { tab[id * stride] = v.hi; }
};

__device__ inline void basis_row_df(double u, int level, const float2* __restrict__ xf, float2* tab, int stride) {
  basis_row_df_out(u, level, xf, DfPairOut{tab, stride});
}

__device__ inline void basis_row_df_hi(double u, int level, const float2* __restrict__ xf, float* tab,
                                       int stride) {
  basis_row_df_out(u, level, xf, DfHiOut{tab, stride});
}

}  // namespace sg
