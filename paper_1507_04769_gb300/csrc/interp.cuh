// Surplus handle and evaluation arguments shared by the interpolant kernels.
#pragma once

#include <vector>

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

// Sum-factorised tensor-core evaluation (interp_sf.cu): one product of the
// program (accumulator column, N, byte offset of the W tile in shared memory,
// accumulate flag) and one 16-column chunk of the epilogue (accumulator
// column, first column within its group, first a-tuple entry of the group).
struct SfMma {
  uint32_t col, n, boff, accum;
};
struct SfEpi {
  uint16_t col, c0, abase, pad;
};
struct SfPlan {
  int side = 0, nks = 0, nepi = 0, tmem_cols = 0, ngemv = 0, kw = 4;
  int gseg[5] = {0, 0, 0, 0, 0};     // CUDA-core column segments by factor count 1 .. 4
  size_t bbytes = 0, smem = 0, o_gw = 0;
  std::vector<unsigned char> meta;   // sops | gops | aops | epi | prog | pstart (copied to shared memory)
  size_t o_gops = 0, o_aops = 0, o_epi = 0, o_prog = 0, o_pstart = 0;
  std::vector<int32_t> bmap;         // per float of the W pack: (W index << 2) | part, or -1
  size_t bfloats_ = 0, meta_bytes_ = 0;   // their sizes, kept when the tables are moved to a staging copy
};
bool sf_plan(int d, int level, int nf, int k, int64_t M, const std::vector<uint16_t>& fid, SfPlan& p);
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
  // sum-factorised tensor-core evaluation (sf_ok: its plan fits the device)
  int sf_ok = 0, sf_side = 0, sf_nks = 0, sf_nepi = 0, sf_tmem = 0, sf_ngemv = 0, sf_kw = 4;
  int sf_gseg[5] = {0, 0, 0, 0, 0};
  size_t sf_bbytes = 0, sf_smem = 0, sf_bfloats = 0, sf_o_gw = 0;
  size_t sf_meta_bytes = 0, sf_o_gops = 0, sf_o_aops = 0, sf_o_epi = 0, sf_o_prog = 0, sf_o_pstart = 0;
  unsigned char* sf_meta = nullptr;   // the plan's small tables
  float* sf_b = nullptr;              // the W pack (TF32 hi and lo tiles)
  int32_t* sf_bmap = nullptr;
  void* block = nullptr;          // the one device allocation all the arrays above live in
};

namespace sg {
int eval_tf32x3(const EvalArgs& e, const sg_surplus* s, cudaStream_t st);
int eval_df32(const EvalArgs& e, int d, cudaStream_t st);
int split_df(int64_t n, const double* src, float2* dst, cudaStream_t st);
size_t tf32_pack_floats(int64_t M, int k);   // floats of the split-TF32 pack (0 for k > 8)
int pack_tf32(sg_surplus* s, cudaStream_t st);
int sf_pack(sg_surplus* s, cudaStream_t st);
int eval_sf_tf32x3(const EvalArgs& e, const sg_surplus* s, cudaStream_t st);
}
