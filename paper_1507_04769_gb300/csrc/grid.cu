// Step I: Smolyak sparse grid on nested Chebyshev-Gauss-Lobatto sets
// (Section 3.2, Eq. CGL).  The multi-index enumeration is integer work done
// once on the host; node coordinates are computed on the device.
#include <cstring>
#include <vector>

#include "common.cuh"
#include "diag.cuh"
#include "grid.cuh"

namespace sg {

int delta_count(int i) { return i == 1 ? 1 : (i == 2 ? 2 : (1 << (i - 2))); }

// 0-based index in X^i of the j-th point of the increment set dX^i.
// dX^1 = {1/2} (k = 0 of X^1); dX^2 = {0, 1} (k = 0, 2 of X^2 = {0, 1/2, 1});
// dX^i, i >= 3: the points of X^i not in X^{i-1}, which sits at the even k,
// so dX^i is k = 1, 3, 5, ...
int delta_index(int i, int j) {
  if (i == 1) return 0;
  if (i == 2) return 2 * j;
  return 2 * j + 1;
}

// Appends every multi-index i (i_k >= 1) with |i| == s, in lexicographic
// order, to `out` as d consecutive ints.
static void enumerate_level(int d, int pos, int rem, int* cur, std::vector<int>& out) {
  if (pos == d - 1) {
    if (rem >= 1) {
      cur[pos] = rem;
      for (int k = 0; k < d; ++k) out.push_back(cur[k]);
    }
    return;
  }
  for (int v = 1; v <= rem - (d - 1 - pos); ++v) {
    cur[pos] = v;
    enumerate_level(d, pos + 1, rem - v, cur, out);
  }
}

void enumerate_nodes(int d, int level, std::vector<int8_t>& lev, std::vector<int16_t>& kidx) {
  const int q = d + level;
  lev.clear();
  kidx.clear();
  for (int s = d; s <= q; ++s) {
    std::vector<int> mis;
    int cur[kMaxDim] = {0};
    enumerate_level(d, 0, s, cur, mis);
    for (size_t b = 0; b < mis.size(); b += d) {
      const int* mi = mis.data() + b;
      // all j with j_k < dN_{i_k}, lexicographic (last dimension fastest)
      int j[kMaxDim] = {0};
      while (true) {
        for (int k = 0; k < d; ++k) {
          lev.push_back(static_cast<int8_t>(mi[k]));
          kidx.push_back(static_cast<int16_t>(delta_index(mi[k], j[k])));
        }
        int k = d - 1;
        while (k >= 0) {
          if (++j[k] < delta_count(mi[k])) break;
          j[k] = 0;
          --k;
        }
        if (k < 0) break;
      }
    }
  }
}

// x^i_k = (1 - cos(k pi / 2^(i-1))) / 2 = sin^2(k pi / 2^i); the two ends and
// the middle are set exactly (0, 1, 1/2), so nested points coincide exactly.
__device__ __forceinline__ double cgl_coord(int i, int k) {
  if (i == 1) return 0.5;
  const int n = 1 << (i - 1);
  if (k == 0) return 0.0;
  if (k == n) return 1.0;
  if (2 * k == n) return 0.5;
  double s = sinpi(static_cast<double>(k) / static_cast<double>(1 << i));
  return s * s;
}

__global__ void grid_coords_kernel(int64_t total, int d, const int8_t* __restrict__ lev,
                                   const int16_t* __restrict__ kidx, const double* __restrict__ lo,
                                   const double* __restrict__ hi, double* __restrict__ coords) {
  int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= total) return;
  int k = static_cast<int>(e % d);
  double u = cgl_coord(lev[e], kidx[e]);
  coords[e] = lo[k] + (hi[k] - lo[k]) * u;
}

}  // namespace sg

using namespace sg;

extern "C" int sg_build_grid(int d, int level, const double* h_lo, const double* h_hi, sg_grid** out) {
  clear_error();
  if (!out || !h_lo || !h_hi) return fail(SG_EINVAL, "sg_build_grid: null pointer");
  *out = nullptr;
  if (d < 1 || d > kMaxDim) return fail(SG_EUNSUPPORTED, "sg_build_grid: d must be 1..8");
  if (level < 0 || level > 10) return fail(SG_EUNSUPPORTED, "sg_build_grid: level must be 0..10");
  for (int k = 0; k < d; ++k)
    if (!(h_lo[k] < h_hi[k])) return fail(SG_EINVAL, "sg_build_grid: need lo < hi in every dimension");

  auto* g = new sg_grid();
  g->d = d;
  g->level = level;
  enumerate_nodes(d, level, g->h_lev, g->h_kidx);
  g->M = static_cast<int64_t>(g->h_lev.size()) / d;
  g->h_lo.assign(h_lo, h_lo + d);
  g->h_hi.assign(h_hi, h_hi + d);
  const int64_t total = g->M * d;

  // one device allocation (coordinates, levels, indices, box); the host-made
  // parts go in with one copy
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t ocoords = take(total * sizeof(double));
  const size_t ohost = off;
  const size_t obox = take(2 * d * sizeof(double)), olev = take(total * sizeof(int8_t));
  const size_t okidx = take(total * sizeof(int16_t));
  auto cleanup = [&](int code, const char* what, cudaError_t e) {
    sg_grid_free(g);
    return e == cudaSuccess ? fail(code, what) : cuda_fail(e, what);
  };
  cudaError_t e;
  if ((e = block_alloc(&g->block, off, nullptr)) != cudaSuccess) return cleanup(SG_ENOMEM, "device allocation of the grid", e);
  char* base = static_cast<char*>(g->block);
  g->coords = reinterpret_cast<double*>(base + ocoords);
  g->lev = reinterpret_cast<int8_t*>(base + olev);
  g->kidx = reinterpret_cast<int16_t*>(base + okidx);
  double* d_box = reinterpret_cast<double*>(base + obox);
  {
    std::vector<unsigned char> h(off - ohost);
    std::memcpy(h.data() + (obox - ohost), h_lo, d * sizeof(double));
    std::memcpy(h.data() + (obox - ohost) + d * sizeof(double), h_hi, d * sizeof(double));
    std::memcpy(h.data() + (olev - ohost), g->h_lev.data(), total * sizeof(int8_t));
    std::memcpy(h.data() + (okidx - ohost), g->h_kidx.data(), total * sizeof(int16_t));
    // (a copy from pageable memory is staged before the call returns, so h
    // may go; the kernel follows it on the same stream, and one wait covers both)
    if ((e = cudaMemcpyAsync(base + ohost, h.data(), off - ohost, cudaMemcpyHostToDevice, nullptr)) != cudaSuccess)
      return cleanup(SG_ECUDA, "copy grid tables", e);
  }
  SG_TIMED("grid_coords_kernel", nullptr, (grid_coords_kernel<<<static_cast<unsigned>(ceil_div(total, 256)), 256>>>(total, d, g->lev, g->kidx, d_box, d_box + d, g->coords)));
  if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(SG_ECUDA, "grid_coords_kernel launch", e);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup(SG_ECUDA, "grid_coords_kernel", e);
  *out = g;
  return SG_OK;
}

extern "C" int sg_grid_info(const sg_grid* g, int64_t* n_nodes, int* d, int* level,
                            const double** d_coords, const int8_t** d_levels, const int16_t** d_index) {
  clear_error();
  if (!g) return fail(SG_EINVAL, "sg_grid_info: null grid");
  if (n_nodes) *n_nodes = g->M;
  if (d) *d = g->d;
  if (level) *level = g->level;
  if (d_coords) *d_coords = g->coords;
  if (d_levels) *d_levels = g->lev;
  if (d_index) *d_index = g->kidx;
  return SG_OK;
}

extern "C" void sg_grid_free(sg_grid* g) {
  if (!g) return;
  block_free(g->block);
  delete g;
}
