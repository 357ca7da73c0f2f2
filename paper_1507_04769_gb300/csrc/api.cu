// Error reporting of the C ABI, and the pool the handles' device blocks come
// from.
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"

namespace sg {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t device_pool(int dev, cudaMemPool_t* out) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  cudaError_t e = cudaMemPoolCreate(&pool, &props);
  if (e != cudaSuccess) return e;
  uint64_t keep = uint64_t(1) << 30;   // freed blocks kept for reuse
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) return e;
  g_pools[dev] = pool;
  *out = pool;
  return cudaSuccess;
}
}  // namespace

cudaError_t block_alloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (e == cudaSuccess) e = device_pool(dev, &pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, st);
  return e;
}

void block_free(void* p) {
  if (!p) return;
  int cur = 0, dev = 0;
  cudaPointerAttributes at{};
  if (cudaGetDevice(&cur) != cudaSuccess) return;
  if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeDevice) dev = at.device;
  else dev = cur;
  if (dev != cur) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  cudaFreeAsync(p, nullptr);
  if (dev != cur) cudaSetDevice(cur);
}
}  // namespace sg

extern "C" const char* sg_last_error(void) { return sg::g_last_error.c_str(); }
