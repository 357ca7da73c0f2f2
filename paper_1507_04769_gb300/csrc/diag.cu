// Diagnostics: a count of every kernel the library launches, optional
// per-kernel CUDA-event timing on the launching stream, and an FMA-chain
// throughput probe used to state the FP64 / FP32 pipe peaks.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "diag.cuh"

namespace sg {

namespace {
struct Pending {
  const char* name;
  cudaEvent_t a, b;
};
struct TimerState {
  std::mutex mu;
  bool enabled = false;
  uint64_t launches = 0;
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  std::map<std::string, std::pair<double, int64_t>> totals;
};
TimerState& state() {
  static TimerState* s = new TimerState();   // never destroyed: safe at exit
  return *s;
}
cudaEvent_t take_event(TimerState& s) {
  if (!s.pool.empty()) {
    cudaEvent_t e = s.pool.back();
    s.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

KernelTimer::KernelTimer(const char* name, cudaStream_t st) : name_(name), st_(st) {
  TimerState& s = state();
  std::lock_guard<std::mutex> lk(s.mu);
  ++s.launches;
  if (!s.enabled) return;
  a_ = take_event(s);
  b_ = take_event(s);
  if (a_ && b_) cudaEventRecord(a_, st_);
}

KernelTimer::~KernelTimer() {
  if (!a_ || !b_) return;
  TimerState& s = state();
  cudaEventRecord(b_, st_);
  std::lock_guard<std::mutex> lk(s.mu);
  s.pending.push_back({name_, a_, b_});
}

}  // namespace sg

using namespace sg;

extern "C" uint64_t sg_kernel_launches(void) {
  TimerState& s = state();
  std::lock_guard<std::mutex> lk(s.mu);
  return s.launches;
}

extern "C" void sg_timing_enable(int on) {
  TimerState& s = state();
  std::lock_guard<std::mutex> lk(s.mu);
  s.enabled = on != 0;
}

extern "C" int sg_timing_collect(int max_kernels, char* names, int name_len, double* total_ms,
                                 int64_t* launches, int* n_kernels) {
  clear_error();
  TimerState& s = state();
  std::lock_guard<std::mutex> lk(s.mu);
  for (const Pending& p : s.pending) {
    if (cudaEventSynchronize(p.b) != cudaSuccess) return fail(SG_ECUDA, "sg_timing_collect: event sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& t = s.totals[p.name];
    t.first += ms;
    t.second += 1;
    s.pool.push_back(p.a);
    s.pool.push_back(p.b);
  }
  s.pending.clear();
  int i = 0;
  for (const auto& kv : s.totals) {
    if (i >= max_kernels) break;
    if (names && name_len > 0) {
      std::strncpy(names + size_t(i) * name_len, kv.first.c_str(), name_len - 1);
      names[size_t(i) * name_len + name_len - 1] = '\0';
    }
    if (total_ms) total_ms[i] = kv.second.first;
    if (launches) launches[i] = kv.second.second;
    ++i;
  }
  if (n_kernels) *n_kernels = i;
  s.totals.clear();
  return SG_OK;
}

// ---------------------------------------------------------------- FMA probe
// Independent FMA chains per thread (8 of them, to cover the pipe latency);
// the result is stored so nothing is optimised away.
template <typename T>
__global__ void k_fma_probe(T* out, int iters, T seed) {
  T a0 = seed + T(threadIdx.x) * T(1e-7), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  const T m = T(0.999999), c = T(1e-6);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
      a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

extern "C" int sg_fma_probe(int precision, void* d_scratch, size_t scratch_bytes, int blocks, int threads,
                            int iters, double* flops_per_launch, void* stream) {
  clear_error();
  const size_t tsize = precision == SG_PREC_FP64 ? sizeof(double) : sizeof(float);
  if (!d_scratch || blocks < 1 || threads < 32 || threads > 1024 || iters < 1)
    return fail(SG_EINVAL, "sg_fma_probe: bad arguments");
  if (scratch_bytes < size_t(blocks) * threads * tsize) return fail(SG_EINVAL, "sg_fma_probe: scratch too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    KernelTimer kt(precision == SG_PREC_FP64 ? "k_fma_probe_fp64" : "k_fma_probe_fp32", st);
    if (precision == SG_PREC_FP64)
      k_fma_probe<double><<<blocks, threads, 0, st>>>(static_cast<double*>(d_scratch), iters, 1.0);
    else
      k_fma_probe<float><<<blocks, threads, 0, st>>>(static_cast<float*>(d_scratch), iters, 1.0f);
  }
  SG_LAUNCH_CHECK("k_fma_probe");
  if (flops_per_launch) *flops_per_launch = 2.0 * 8 * 16 * double(iters) * blocks * threads;
  return SG_OK;
}

// ---------------------------------------------------------------- sincos probe
#include "problems.cuh"

namespace sg {
__global__ void k_sincos_probe(int64_t n, const double* __restrict__ x, double* __restrict__ s,
                               double* __restrict__ c) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  double sv, cv;
  dsincos(x[t], &sv, &cv);
  s[t] = sv;
  c[t] = cv;
}
}  // namespace sg

extern "C" int sg_sincos_probe(const double* d_x, int64_t n, double* d_s, double* d_c, void* stream) {
  sg::clear_error();
  if (n < 0) return sg::fail(SG_EINVAL, "sg_sincos_probe: n < 0");
  if (n == 0) return SG_OK;
  if (!d_x || !d_s || !d_c) return sg::fail(SG_EINVAL, "sg_sincos_probe: null device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SG_TIMED("k_sincos_probe", st,
           (sg::k_sincos_probe<<<static_cast<unsigned>(sg::ceil_div(n, 256)), 256, 0, st>>>(n, d_x, d_s, d_c)));
  SG_LAUNCH_CHECK("k_sincos_probe");
  return SG_OK;
}
