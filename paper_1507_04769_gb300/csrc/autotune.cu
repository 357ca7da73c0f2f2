// Autotuner for the batched solve: times the execution forms of
// sg_solve_bvps on the caller's batch and keeps the fastest per shape.
//
// Candidates (in this order; report_ms follows it):
//   0  launch per phase, host-driven loop
//   1  launch per phase as a cached CUDA graph (device-side WHILE loops)
//   2  one such graph per mesh size, the sizes' sub-batches on concurrent streams
//   3  as 2, condensation blocks of 2 intervals (warps)
//   4  as 2, condensation blocks of 8 intervals (warps)
//   5  persistent warp-per-node kernel as a graph, as many blocks per SM as fit
//   6  persistent warp-per-node kernel as a graph, 1 block (4 warps) per SM
// Each candidate runs once to warm up (and build its graph) and once timed
// with CUDA events on `stream`.  The choice is cached per (precision, n,
// n_max_intervals, tolerance, iteration cap, damping).
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace sg {
namespace {
using TuneKey = std::tuple<int, int64_t, int, double, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, sg_solve_opts>& tune_cache() {
  static auto* m = new std::map<TuneKey, sg_solve_opts>();
  return *m;
}
}  // namespace
}  // namespace sg

using namespace sg;

extern "C" int sg_autotune_solve(const sg_problem* prob, const double* d_x0, int64_t n, const double* d_T,
                                 const int32_t* d_N, int n_max_intervals, const sg_solve_opts* base,
                                 void* d_work, size_t work_bytes, double* d_lambda0, double* d_u0,
                                 double* d_V, int32_t* d_status, int32_t* d_iters, sg_solve_opts* best,
                                 double* report_ms, int force, void* stream) {
  clear_error();
  if (!best) return fail(SG_EINVAL, "sg_autotune_solve: null output");
  sg_solve_opts b{1e-8, 50, SG_PREC_FP64, 1, 0, 0, 0, 0, 0};
  if (base) b = *base;
  b.warm_start = 0;   // the forms are timed on the zero-control solve
  const TuneKey key{b.precision, n, n_max_intervals, b.tol, b.max_iter, b.damping};
  if (!force) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      *best = it->second;
      return SG_OK;
    }
  }
  constexpr int kCand = SG_AUTOTUNE_CANDIDATES;
  sg_solve_opts cand[kCand];
  for (int c = 0; c < kCand; ++c) {
    cand[c] = b;
    cand[c].blocks_per_sm = 0;
    cand[c].cond_warps = 4;
  }
  cand[0].persistent = 0; cand[0].graph = 0;
  cand[1].persistent = 0; cand[1].graph = 1;
  cand[2].persistent = 0; cand[2].graph = 2;
  cand[3].persistent = 0; cand[3].graph = 2; cand[3].cond_warps = 2;
  cand[4].persistent = 0; cand[4].graph = 2; cand[4].cond_warps = 8;
  cand[5].persistent = 1; cand[5].graph = 1;
  cand[6].persistent = 1; cand[6].graph = 1; cand[6].blocks_per_sm = 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  SG_CUDA_TRY(cudaEventCreate(&e0));
  SG_CUDA_TRY(cudaEventCreate(&e1));
  double best_ms = 1e300;
  int best_i = -1;
  int rc = SG_OK;
  for (int c = 0; c < kCand && rc == SG_OK; ++c) {
    rc = sg_solve_bvps(prob, d_x0, n, d_T, d_N, n_max_intervals, &cand[c], d_work, work_bytes, d_lambda0, d_u0,
                       d_V, d_status, d_iters, nullptr, stream);
    if (rc != SG_OK) break;
    cudaEventRecord(e0, st);
    rc = sg_solve_bvps(prob, d_x0, n, d_T, d_N, n_max_intervals, &cand[c], d_work, work_bytes, d_lambda0, d_u0,
                       d_V, d_status, d_iters, nullptr, stream);
    cudaEventRecord(e1, st);
    if (rc != SG_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (report_ms) report_ms[c] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best_i = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SG_OK) return rc;
  *best = cand[best_i];
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_cache()[key] = *best;
  return SG_OK;
}
