// Error amplification of the sparse-grid interpolant (Section 4.2).
//
// Theorem 1 (i): if every nodal value carries an error below eps, the
// interpolant's error is below eps * sum_{l=q-d+1}^{q} C(d-1, q-l) S_l with
// S_l = sum over |i| = l of Lambda_{i_1} ... Lambda_{i_d}.  Lambda_i is taken
// from the bound on the Lebesgue constant of Chebyshev-Gauss-Lobatto
// interpolation (Eq. lebesgue) at N = 2^(i-1) intervals, and Lambda_1 = 1 (the
// one-point set).  Host arithmetic only.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace sg {
static double lebesgue_bound(int i) {
  if (i == 1) return 1.0;
  const double kPi = 3.14159265358979323846;
  const double kEulerGamma = 0.57721566490153286061;
  const double n = std::ldexp(1.0, i - 1);
  return (2.0 / kPi) * (std::log(n) + kEulerGamma + std::log(4.0 / kPi) + std::log(2.0));
}

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int j = 1; j <= k; ++j) r = r * (n - k + j) / j;
  return r;
}
}  // namespace sg

extern "C" int sg_theorem1_bound(int d, int q, double* bound) {
  sg::clear_error();
  if (!bound) return sg::fail(SG_EINVAL, "sg_theorem1_bound: null output");
  if (d < 1 || d > 64 || q < d || q > d + 60) return sg::fail(SG_EINVAL, "sg_theorem1_bound: need 1 <= d <= 64, d <= q <= d + 60");
  // S[l] over dimensions by repeated convolution: S_1(l) = Lambda_l,
  // S_m(l) = sum_{i >= 1} Lambda_i S_{m-1}(l - i)
  std::vector<double> lam(q + 1, 0.0), S(q + 1, 0.0), T(q + 1, 0.0);
  for (int i = 1; i <= q; ++i) lam[i] = sg::lebesgue_bound(i);
  for (int l = 1; l <= q; ++l) S[l] = lam[l];
  for (int m = 2; m <= d; ++m) {
    std::fill(T.begin(), T.end(), 0.0);
    for (int l = m; l <= q; ++l)
      for (int i = 1; i <= l - (m - 1); ++i) T[l] += lam[i] * S[l - i];
    S.swap(T);
  }
  double total = 0.0;
  for (int l = q - d + 1; l <= q; ++l)
    if (l >= d) total += sg::binom(d - 1, q - l) * S[l];
  *bound = total;
  return SG_OK;
}
