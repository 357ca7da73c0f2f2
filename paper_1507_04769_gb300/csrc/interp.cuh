// Surplus handle and evaluation arguments shared by the interpolant kernels.
#pragma once

#include "common.cuh"

namespace sg {
constexpr int kMaxLevel = 8;                 // finest 1-D set has 2^8 + 1 points
constexpr int kMaxFine = 1 << kMaxLevel;
constexpr int kMaxOut = 16;
constexpr int kEvalThreads = 128;

struct EvalArgs {
  const double* xq;
  int64_t Q;
  int64_t M;
  int k;
  int nf;
  int level;
  int amax;               // largest number of active dimensions over the nodes
  const uint8_t* nact;    // M: number of active (level >= 2) dimensions
  const uint16_t* ops;    // M x kMaxDim: table offsets dim * nf + id of the active dimensions
  const double* W;        // M x k, evaluation order
  const double* lo;       // d
  const double* width;    // d: hi - lo (divided, so that nodes map exactly)
  const double* xf;       // 2^L + 1 points of the finest 1-D set
  const float2* xfdf;     // the same points as (hi, lo) float pairs
  const float2* Wdf;      // M x k surpluses as (hi, lo) pairs, evaluation order
  int64_t grp[kMaxDim + 2];  // grp[a]: first node (evaluation order) with >= a active dimensions
  double* out;            // Q x k
};

int n_functions(int level);
int function_id(int l, int kidx);
}  // namespace sg

struct sg_surplus {
  int d = 0;
  int level = 0;
  int k = 0;
  int nf = 0;
  int amax = 0;
  int64_t M = 0;
  double* W = nullptr;            // M x k, grid order
  double* Ws = nullptr;           // M x k, evaluation order
  uint8_t* nact = nullptr;        // M, evaluation order (sorted by this count)
  int64_t grp[sg::kMaxDim + 2] = {};  // first node with >= a active dimensions
  uint16_t* ops = nullptr;        // M x kMaxDim
  double* box = nullptr;          // lo[d], (hi-lo)[d]
  double* xf = nullptr;           // finest 1-D set, 2^L + 1 points
  float2* xfdf = nullptr;         // finest 1-D set as (hi, lo) pairs
  float2* Wdf = nullptr;          // Ws as (hi, lo) pairs
  float* bpack = nullptr;         // split-TF32 [W_hi|W_lo], [W_hi|0] per 16-node chunk (k <= 8)
  uint16_t* tcoff = nullptr;      // M x 8: ops * 128, the tensor-core kernel's table offsets (0 if unused)
  int tc_chunks = 0;
  int* tc_err = nullptr;          // set by the tensor-core kernel if a wait timed out
  void* block = nullptr;          // the one device allocation all the arrays above live in
};

namespace sg {
int eval_tf32x3(const EvalArgs& e, const sg_surplus* s, cudaStream_t st);
int eval_df32(const EvalArgs& e, int d, cudaStream_t st);
int split_df(int64_t n, const double* src, float2* dst, cudaStream_t st);
size_t tf32_pack_floats(int64_t M, int k);   // floats of the split-TF32 pack (0 for k > 8)
int pack_tf32(sg_surplus* s, cudaStream_t st);
}
