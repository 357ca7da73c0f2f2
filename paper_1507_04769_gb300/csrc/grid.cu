// Step I: Smolyak sparse grid on nested Chebyshev-Gauss-Lobatto sets
// (Section 3.2, Eq. CGL).  The multi-index enumeration is integer work done
// on the host once per (d, level); node coordinates are computed on the device
// at every build.
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <utility>
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

// The box, passed by value (no host copy to wait for).
struct GridBox {
  double lo[kMaxDim], hi[kMaxDim];
};

__global__ void grid_coords_kernel(int64_t total, int d, const int8_t* __restrict__ lev,
                                   const int16_t* __restrict__ kidx, GridBox box, double* __restrict__ coords) {
  int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= total) return;
  int k = static_cast<int>(e % d);
  double u = cgl_coord(lev[e], kidx[e]);
  coords[e] = box.lo[k] + (box.hi[k] - box.lo[k]) * u;
}

// The host-made part of a grid, a function of (d, level) only: the nodes'
// levels and 1-D indices, and the same bytes in the device layout (levels,
// then indices at a 256-byte boundary) for the copy, in page-locked memory
// when it could be had (a copy from it needs no staging).  Kept for the life
// of the process, for at most 8 (d, level).
struct GridHost {
  std::vector<int8_t> lev;
  std::vector<int16_t> kidx;
  size_t okidx = 0, bytes = 0;   // offsets from the start of the levels
  std::vector<unsigned char> staging;
  unsigned char* pinned = nullptr;
  const unsigned char* data() const { return pinned ? pinned : staging.data(); }
  GridHost() = default;
  GridHost(const GridHost&) = delete;
  GridHost& operator=(const GridHost&) = delete;
  // (a build holds its entry until it has waited for its copy, so the last
  // reference goes with no copy from these bytes in flight)
  ~GridHost() {
    if (pinned) cudaFreeHost(pinned);
  }
};

static std::shared_ptr<const GridHost> grid_host(int d, int level) {
  static std::mutex mu;
  static auto* cache = new std::vector<std::pair<std::pair<int, int>, std::shared_ptr<const GridHost>>>();
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& e : *cache)
      if (e.first == std::make_pair(d, level)) return e.second;
  }
  auto h = std::make_shared<GridHost>();
  enumerate_nodes(d, level, h->lev, h->kidx);
  const size_t nl = h->lev.size();
  h->okidx = (nl + 255) & ~size_t(255);
  h->bytes = h->okidx + h->kidx.size() * sizeof(int16_t);
  h->staging.assign(h->bytes, 0);
  std::memcpy(h->staging.data(), h->lev.data(), nl);
  std::memcpy(h->staging.data() + h->okidx, h->kidx.data(), h->kidx.size() * sizeof(int16_t));
  if (cudaHostAlloc(reinterpret_cast<void**>(&h->pinned), h->bytes, cudaHostAllocDefault) == cudaSuccess) {
    std::memcpy(h->pinned, h->staging.data(), h->bytes);
    h->staging.clear();
    h->staging.shrink_to_fit();
  } else {
    h->pinned = nullptr;
    (void)cudaGetLastError();
  }
  std::lock_guard<std::mutex> lk(mu);
  for (auto& e : *cache)   // another thread made it meanwhile
    if (e.first == std::make_pair(d, level)) return e.second;
  if (cache->size() >= 8) cache->erase(cache->begin());
  cache->emplace_back(std::make_pair(d, level), h);
  return h;
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

  std::shared_ptr<const GridHost> hp;
  try {
    hp = grid_host(d, level);
  } catch (const std::bad_alloc&) {
    return fail(SG_ENOMEM, "sg_build_grid: host memory");
  }
  auto* g = new sg_grid();
  g->d = d;
  g->level = level;
  g->h_lev = hp->lev;
  g->h_kidx = hp->kidx;
  g->M = static_cast<int64_t>(g->h_lev.size()) / d;
  g->h_lo.assign(h_lo, h_lo + d);
  g->h_hi.assign(h_hi, h_hi + d);
  const int64_t total = g->M * d;

  // one device allocation: coordinates, then the levels and indices in the
  // layout of the host-made bytes, which go in with one copy
  const size_t olev = (total * sizeof(double) + 255) & ~size_t(255);
  const size_t off = olev + hp->bytes;
  auto cleanup = [&](int code, const char* what, cudaError_t e) {
    sg_grid_free(g);
    return e == cudaSuccess ? fail(code, what) : cuda_fail(e, what);
  };
  cudaError_t e;
  if ((e = block_alloc(&g->block, off, nullptr)) != cudaSuccess) return cleanup(SG_ENOMEM, "device allocation of the grid", e);
  char* base = static_cast<char*>(g->block);
  g->coords = reinterpret_cast<double*>(base);
  g->lev = reinterpret_cast<int8_t*>(base + olev);
  g->kidx = reinterpret_cast<int16_t*>(base + olev + hp->okidx);
  if ((e = cudaMemcpyAsync(base + olev, hp->data(), hp->bytes, cudaMemcpyHostToDevice, nullptr)) != cudaSuccess)
    return cleanup(SG_ECUDA, "copy grid tables", e);
  GridBox box{};
  for (int k = 0; k < d; ++k) {
    box.lo[k] = h_lo[k];
    box.hi[k] = h_hi[k];
  }
  SG_TIMED("grid_coords_kernel", nullptr, (grid_coords_kernel<<<static_cast<unsigned>(ceil_div(total, 256)), 256>>>(total, d, g->lev, g->kidx, box, g->coords)));
  if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(SG_ECUDA, "grid_coords_kernel launch", e);
  // (the copy and the kernel are on the default stream; one wait covers both,
  // and the host-made bytes are kept, so nothing on the host is freed early)
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
