// Sum-factorised 3xTF32 evaluation of the interpolant (Eq. interpo) on the
// fifth-generation tensor cores.
//
// Every node m of the sparse grid carries one 1-D function per dimension, so
// its basis function is a product over the d dimensions.  Split the
// dimensions into a first part (0 .. d1-1) and a second part (d1 .. d-1):
// node m is a pair (a, b) of a first-part tuple a and a second-part tuple b,
// and its basis function is Phi_a(x) Psi_b(x), the products over each part.
// The interpolant's sum, taken in another order, reads
//     u_c(x) = sum_a Phi_a(x) G_{a,c}(x),    G_{a,c}(x) = sum_b Psi_b(x) w_{(a,b),c}.
// On a Smolyak grid the tuples b paired with a given a are those whose level
// sum is at most L minus the level sum of a: with the b's sorted by level sum,
// a prefix whose length depends on the level sum of a only.  With the a's
// grouped by that prefix, each group's G is one dense product
//     G_g = Psi[:, 0:K_g] x W_g     (queries x K_g, K_g x (a, c)),
// a GEMM whose operand A (Psi, one row per query) is built once per query:
// 177 products per query instead of 1457 on the level-4 grid in d = 6.
//
// Which products go where.  A K-step (8 columns of Psi) that several groups
// share is one wide tensor-core product (the groups' accumulator columns
// are consecutive, so N = 256, 112, 48 at level 4).  The K-steps that only
// the constant tuple a0 uses, and the a's paired with the constant tuple b0
// only (the finest first-part levels), are sums over single nodes with k
// outputs: a tf32 MMA costs about as much for N = 16 as for N = 64, so these
// columns run on the CUDA cores (FP32 products times FP32 surpluses, summed
// eight at a time and then compensated).
//
// The host builds the plan once per grid structure (sf_plan): the operand-A
// columns as table offsets, the CUDA-core columns by factor count, the W
// tiles of every K-step's product in the tensor cores' K-major core-matrix
// layout followed by the CUDA-core columns' FP32 rows, the products of every
// K-step, and the 16-column chunks of the epilogue.
//
// The kernel: one persistent CTA per SM over tiles of 128 queries,
// warp-specialised.
//   warps 0..11  producers, three per query row (part p = tid / 128):
//                each computes the 1-D tables of dimensions p, p + 3, ...
//                (compensated FP32 inside the box, pairs of floats outside),
//                then, per ring stage of three K-steps, the K-step p of the
//                row's operand A split into TF32 hi and lo parts, arriving on
//                the stage's "full" mbarrier; then a third of the CUDA-core
//                columns while the products run; then the epilogue: a third
//                of the accumulator chunks read from tensor memory and
//                sum_a Phi_a G_{a,c} formed;
//   warp 12      lane 0 issues, per K-step, the three products
//                A_hi W_hi, A_hi W_lo, A_lo W_hi (M = 128, kind::tf32),
//                commits each stage to its "empty" mbarrier and the whole
//                tile to "done".
// The next tile's coordinates are loaded and converted while a tile computes;
// there is no FP64 arithmetic on the path but the output.  Every mbarrier
// wait is bounded; a timeout sets an error flag, the CTA stops and writes NaN
// for its remaining queries.
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <vector>

#include "basis.cuh"
#include "common.cuh"
#include "diag.cuh"
#include "grid.cuh"
#include "interp.cuh"
#include "tcgen05.cuh"

namespace sg {

constexpr int kSfRows = 128;                         // queries per tile (= MMA M)
constexpr int kSfParts = 3;                          // producer threads per row
constexpr int kSfProducers = kSfRows * kSfParts;
constexpr int kSfThreads = kSfProducers + 32;        // + the MMA warp
constexpr int kSfKsteps = kSfParts;                  // K-steps per ring stage, one per part
constexpr int kSfStages = 3;
constexpr int kSfKstepBytes = kSfRows * 32;          // 128 rows x 8 TF32
constexpr int kSfStageBytes = 2 * kSfKsteps * kSfKstepBytes;   // hi K-steps | lo K-steps
constexpr int kSfMaxTmem = 512;
constexpr size_t kSfMaxSmem = 227 * 1024;

// ------------------------------------------------------------------ host plan
namespace {
using Tuple = std::array<uint16_t, 4>;

inline int pad16(int x) { return (x + 15) & ~15; }

// element (n, k) of an N x 8 K-major tile: core matrix (n / 8, k / 4), row n % 8
inline int tile_float(int n, int k) { return ((n / 8) * 2 + k / 4) * 32 + (n % 8) * 4 + k % 4; }
}  // namespace

bool sf_plan(int d, int level, int nf, int k, int64_t M, const std::vector<uint16_t>& fid, SfPlan& p) {
  p = SfPlan{};
  if (d < 2 || d > 8 || k < 1 || k > 8 || M < 1 || size_t(d) * nf + 1 > 511) return false;
  const int d1 = d / 2, d2 = d - d1;
  p.side = std::max(d1, d2);
  std::vector<int> hlev(nf, 0);   // hierarchical level of each 1-D function id
  {
    int id = 0;
    for (int l = 1; l <= level + 1 && id < nf; ++l)
      for (int j = 0; j < delta_count(l) && id < nf; ++j) hlev[id++] = l - 1;
  }
  auto tuple_of = [&](int64_t n, int first, int cnt) {
    Tuple t{0, 0, 0, 0};
    for (int j = 0; j < cnt; ++j) t[j] = fid[n * d + first + j];
    return t;
  };
  auto lsum = [&](const Tuple& t, int cnt) {
    int s = 0;
    for (int j = 0; j < cnt; ++j) s += hlev[t[j]];
    return s;
  };
  // distinct tuples of each part, sorted by level sum, then by ids
  auto index_tuples = [&](int first, int cnt, std::vector<Tuple>& list, std::vector<int32_t>& of_node) {
    std::map<Tuple, int32_t> seen;
    for (int64_t n = 0; n < M; ++n) seen.emplace(tuple_of(n, first, cnt), 0);
    for (auto& kv : seen) list.push_back(kv.first);
    std::stable_sort(list.begin(), list.end(), [&](const Tuple& x, const Tuple& y) {
      const int lx = lsum(x, cnt), ly = lsum(y, cnt);
      return lx != ly ? lx < ly : x < y;
    });
    for (size_t i = 0; i < list.size(); ++i) seen[list[i]] = static_cast<int32_t>(i);
    of_node.resize(M);
    for (int64_t n = 0; n < M; ++n) of_node[n] = seen[tuple_of(n, first, cnt)];
  };
  std::vector<Tuple> alist, blist;
  std::vector<int32_t> a_of, b_of;
  index_tuples(0, d1, alist, a_of);
  index_tuples(d1, d2, blist, b_of);
  const int nA = static_cast<int>(alist.size()), nB = static_cast<int>(blist.size());
  if (int64_t(nA) * nB > (int64_t(1) << 24)) return false;
  const Tuple zero{0, 0, 0, 0};
  if (blist[0] != zero) return false;   // the constant tuple b0 (every Smolyak grid has it)
  std::vector<int64_t> node_of(size_t(nA) * nB, -1);
  std::vector<int> kmax(nA, 0);
  for (int64_t n = 0; n < M; ++n) {
    node_of[size_t(a_of[n]) * nB + b_of[n]] = n;
    kmax[a_of[n]] = std::max(kmax[a_of[n]], b_of[n] + 1);
  }
  // groups: a's with more than b0 by their number of K-steps (descending),
  // at most 256 accumulator columns each; the direct a's (b0 only) apart
  std::vector<int> f1, f2;
  for (int a = 0; a < nA; ++a) (kmax[a] == 1 ? f2 : f1).push_back(a);
  std::stable_sort(f1.begin(), f1.end(), [&](int x, int y) { return (kmax[x] + 7) / 8 > (kmax[y] + 7) / 8; });
  struct Group {
    int ks, n, N, base, abase;
    std::vector<int> as;
  };
  std::vector<Group> groups;
  const int gmax = 256 / k;
  for (size_t i = 0; i < f1.size();) {
    const int ks = (kmax[f1[i]] + 7) / 8;
    Group g{ks, 0, 0, 0, 0, {}};
    while (i < f1.size() && (kmax[f1[i]] + 7) / 8 == ks && g.n < gmax) {
      g.as.push_back(f1[i++]);
      ++g.n;
    }
    groups.push_back(g);
  }
  // K-steps used by the constant tuple a0 alone (its group has one a and the
  // most K-steps) are per-node sums with k outputs: too narrow for the tensor
  // cores, they go to the CUDA cores with the direct a's.  The tensor cores
  // take the K-steps that some other group shares.
  const int a0 = alist[0] == zero ? 0 : -1;
  const bool a0_tail = !groups.empty() && a0 >= 0 && groups[0].n == 1 && groups[0].as[0] == a0;
  int ks_tc = 0;
  for (size_t gi = a0_tail ? 1 : 0; gi < groups.size(); ++gi) ks_tc = std::max(ks_tc, groups[gi].ks);
  if (!groups.empty() && ks_tc < groups[0].ks) groups[0].ks = ks_tc;
  while (!groups.empty() && groups.back().ks == 0) groups.pop_back();   // a0 with no shared K-step
  p.nks = ks_tc;
  // the CUDA-core columns: nodes (a0, b) with b past the tensor cores' K-steps,
  // then the nodes (a, b0) of the direct a's; each is one product and k outputs
  struct GemvCol {
    const Tuple* t;
    int first, cnt;
    int64_t node;
  };
  std::vector<GemvCol> gcols;
  if (a0_tail)
    for (int b = 8 * ks_tc; b < nB; ++b) {
      const int64_t n = node_of[size_t(a0) * nB + b];
      if (n >= 0) gcols.push_back(GemvCol{&blist[b], d1, d2, n});
    }
  for (int a : f2) gcols.push_back(GemvCol{&alist[a], 0, d1, node_of[size_t(a) * nB]});
  // by the number of non-constant factors (1 .. 4; a product of constants
  // counts as 1), each segment padded to whole rounds of 8 columns per part
  {
    auto nact = [](const GemvCol& g) {
      int n = 0;
      for (int j = 0; j < g.cnt; ++j) n += (*g.t)[j] != 0;
      return std::max(n, 1);
    };
    std::vector<GemvCol> sorted;
    p.gseg[0] = 0;
    for (int S = 1; S <= 4; ++S) {
      for (const GemvCol& g : gcols)
        if (nact(g) == S) sorted.push_back(g);
      while (sorted.size() % (8 * kSfParts)) sorted.push_back(GemvCol{nullptr, 0, 0, -1});
      p.gseg[S] = static_cast<int>(sorted.size());
    }
    gcols.swap(sorted);
  }
  p.ngemv = static_cast<int>(gcols.size());
  p.kw = k <= 4 ? 4 : 8;
  // accumulator columns ([a][c] within a group) and epilogue entries
  int col = 0, aent = 0;
  for (auto& g : groups) {
    g.N = pad16(g.n * k);
    g.base = col;
    col += g.N;
    g.abase = aent;
    aent += (g.N - 1) / k + 1;
  }
  if (col > kSfMaxTmem || aent > 65535) return false;
  p.tmem_cols = 32;
  while (p.tmem_cols < col) p.tmem_cols *= 2;
  // products of each K-step: its active groups (a prefix of the groups)
  // merged over consecutive accumulator columns into products of at most 256
  // columns, each with its own W tile
  struct Piece {
    int s, col, N;
    size_t boff;
  };
  std::vector<Piece> pieces;
  std::vector<SfMma> prog;
  std::vector<int32_t> pstart;
  size_t boff = 0;
  for (int s = 0; s < p.nks; ++s) {
    pstart.push_back(static_cast<int32_t>(prog.size()));
    Piece cur{s, -1, 0, 0};
    auto flush = [&]() {
      if (cur.N == 0) return;
      cur.boff = boff;
      boff += size_t(cur.N) * 32 * 2;   // hi tile, lo tile
      pieces.push_back(cur);
      prog.push_back(SfMma{static_cast<uint32_t>(cur.col), static_cast<uint32_t>(cur.N),
                           static_cast<uint32_t>(cur.boff), s > 0 ? 1u : 0u});
      cur = Piece{s, -1, 0, 0};
    };
    for (auto& g : groups) {
      if (s >= g.ks) continue;
      if (cur.N > 0 && (g.base != cur.col + cur.N || cur.N + g.N > 256)) flush();
      if (cur.N == 0) cur.col = g.base;
      cur.N += g.N;
    }
    flush();
  }
  pstart.push_back(static_cast<int32_t>(prog.size()));
  p.o_gw = boff;                                     // the CUDA-core columns' W rows follow the tiles
  p.bbytes = boff + size_t(p.ngemv) * p.kw * sizeof(float);
  p.bbytes = (p.bbytes + 15) & ~size_t(15);
  const uint16_t ONE = 0;                                         // id 0 of dimension 0: the constant 1
  const uint16_t ZERO = static_cast<uint16_t>(d * nf * kSfRows);  // the zero entry after the tables
  auto offset = [&](int dim, int id) { return static_cast<uint16_t>((dim * nf + id) * kSfRows); };
  auto put_tuple = [&](std::vector<uint16_t>& v, const Tuple* t, int first, int cnt) {
    for (int j = 0; j < 4; ++j) {
      if (!t) v.push_back(j == 0 ? ZERO : ONE);
      else v.push_back(j < cnt ? offset(first + j, (*t)[j]) : ONE);
    }
  };
  // the same with the non-constant factors first (a product over the first
  // S entries, S the count of non-constant factors, is the whole product)
  auto put_active = [&](std::vector<uint16_t>& v, const Tuple* t, int first, int cnt) {
    if (!t) return put_tuple(v, t, first, cnt);
    int n = 0;
    for (int j = 0; j < cnt; ++j)
      if ((*t)[j] != 0) {
        v.push_back(offset(first + j, (*t)[j]));
        ++n;
      }
    for (; n < 4; ++n) v.push_back(ONE);
  };
  // operand-A columns (the b's of the tensor cores' K-steps), the CUDA-core
  // columns, and the epilogue a-tuples (zero past each group's end)
  std::vector<uint16_t> sops, gops, aops;
  for (int c = 0; c < 8 * p.nks; ++c) put_tuple(sops, c < nB ? &blist[c] : nullptr, d1, d2);
  for (const GemvCol& gc : gcols) put_active(gops, gc.t, gc.first, gc.cnt);
  std::vector<SfEpi> epi;
  for (auto& g : groups) {
    const int cnt = (g.N - 1) / k + 1;
    for (int i = 0; i < cnt; ++i) put_active(aops, i < g.n ? &alist[g.as[i]] : nullptr, 0, d1);
    for (int c0 = 0; c0 < g.N; c0 += 16)
      epi.push_back(SfEpi{static_cast<uint16_t>(g.base + c0), static_cast<uint16_t>(c0),
                          static_cast<uint16_t>(g.abase), 0});
  }
  p.nepi = static_cast<int>(epi.size());
  // the kernel's small tables, one blob copied to shared memory:
  // sops | gops | aops | epi | prog | pstart (16-byte aligned parts)
  auto append = [&](const void* src, size_t bytes) {
    const size_t o = p.meta.size();
    p.meta.resize(o + ((bytes + 15) & ~size_t(15)), 0);
    if (bytes) std::memcpy(p.meta.data() + o, src, bytes);
    return o;
  };
  append(sops.data(), sops.size() * sizeof(uint16_t));
  p.o_gops = append(gops.data(), gops.size() * sizeof(uint16_t));
  p.o_aops = append(aops.data(), aops.size() * sizeof(uint16_t));
  p.o_epi = append(epi.data(), epi.size() * sizeof(SfEpi));
  p.o_prog = append(prog.data(), prog.size() * sizeof(SfMma));
  p.o_pstart = append(pstart.data(), pstart.size() * sizeof(int32_t));
  const size_t tab_bytes = (size_t(d) * nf + 1) * kSfRows * sizeof(float);
  p.smem = size_t(kSfStages) * kSfStageBytes + p.bbytes + p.meta.size() + tab_bytes + 128;
  if (p.smem > kSfMaxSmem) return false;
  // pack map, per float: (W index << 2) | part (0: TF32 hi, 1: TF32 lo, 2: FP32)
  p.bmap.assign(p.bbytes / 4, -1);
  auto put = [&](size_t pos, int64_t widx, int part) {
    p.bmap[pos] = static_cast<int32_t>((widx << 2) | part);
  };
  for (const Piece& pc : pieces) {
    const size_t t0 = pc.boff / 4;
    for (int n = 0; n < pc.N; ++n) {
      const int c = pc.col + n;
      const Group* g = nullptr;
      for (auto& gg : groups)
        if (c >= gg.base && c < gg.base + gg.N) g = &gg;
      const int ng = c - g->base, al = ng / k;
      for (int kk = 0; kk < 8; ++kk) {
        const int b = 8 * pc.s + kk;
        if (al >= g->n || b >= nB) continue;
        const int64_t node = node_of[size_t(g->as[al]) * nB + b];
        if (node < 0) continue;
        const size_t pos = t0 + tile_float(n, kk);
        put(pos, node * k + ng % k, 0);
        put(pos + size_t(pc.N) * 8, node * k + ng % k, 1);
      }
    }
  }
  for (int j = 0; j < p.ngemv; ++j)
    for (int c = 0; c < k && gcols[j].node >= 0; ++c) put(p.o_gw / 4 + size_t(j) * p.kw + c, gcols[j].node * k + c, 2);
  if (int64_t(M) * k >= (int64_t(1) << 29)) return false;
  return true;
}

// ------------------------------------------------------------------ W pack
// The surpluses at their places in the pack: TF32 hi and lo parts in the
// tensor cores' tiles, FP32 values in the CUDA-core columns' rows.
__global__ void k_pack_sf(int64_t nfl, const int32_t* __restrict__ map, const double* __restrict__ W,
                          float* __restrict__ bp) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= nfl) return;
  const int32_t m = map[i];
  float v = 0.0f;
  if (m >= 0) {
    const double w = W[m >> 2];
    const int part = m & 3;
    const float hi = tf32_round(static_cast<float>(w));
    v = part == 2 ? static_cast<float>(w) : (part == 1 ? tf32_round(static_cast<float>(w - static_cast<double>(hi))) : hi);
  }
  bp[i] = v;
}

int sf_pack(sg_surplus* s, cudaStream_t st) {
  if (!s->sf_ok) return SG_OK;
  const int64_t n = static_cast<int64_t>(s->sf_bfloats);
  SG_TIMED("k_pack_sf", st,
           (k_pack_sf<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(n, s->sf_bmap, s->W, s->sf_b)));
  SG_LAUNCH_CHECK("k_pack_sf");
  return SG_OK;
}

// ------------------------------------------------------------------ kernel
struct SfArgs {
  const double* xq;
  int64_t Q;
  int d, nf, level, k, side, nks, nepi, tmem_cols;
  int bbytes, meta_bytes, o_gops, o_aops, o_epi, o_prog, o_pstart;
  int ngemv, kw, o_gw;
  int gseg[5];   // CUDA-core column segments by factor count
  const double* lo;
  const double* width;
  const float2* xfdf;
  const unsigned char* meta;   // sops | gops | aops | epi | prog | pstart
  const float* bpack;
  double* out;
  int* err;
};

// s + e = x + y exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float x, float y, float& s, float& e) {
  s = __fadd_rn(x, y);
  const float bb = __fsub_rn(s, x);
  e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(y, bb));
}

// (hi, lo) + (hi, lo), renormalised
__device__ __forceinline__ void pair_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// 1 / (h + l) in FP32: the hardware approximation corrected by one Newton
// step on the residual of the pair
__device__ __forceinline__ float recip_pair(float h, float l) {
  float q;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(h));
  const float r = __fmaf_rn(-l, q, __fmaf_rn(-h, q, 1.0f));
  return __fmaf_rn(q, r, q);
}

// All 1-D basis values at u = uh + ul (a pair of floats) for levels
// 1 .. L + 1, rounded to FP32, in barycentric form on the finest set (the
// same formula as the pair-of-floats tables).  The differences u - x_p are
// formed in pairs of floats and rounded once, so they keep their relative
// accuracy next to a node; the reciprocals are FP32 with one Newton step;
// the denominators are compensated sums over the nested sets: with P_l the
// unsigned weighted sum over X^l and N_{l+1} the sum over the points new in
// X^{l+1} (its odd positions, weight -1),
//     D_{l+1} = P_l - N_{l+1},    P_{l+1} = P_l + N_{l+1}.
// Each value is within a few units in the last place of FP32.
template <int L>
__device__ __forceinline__ void basis_row_f32c(float uh, float ul, const float2* __restrict__ xf, float* tab,
                                               int stride) {
  constexpr int fine_n = 1 << L;
  tab[0] = 1.0f;
  float r[fine_n + 1];
  int hit = -1;
#pragma unroll
  for (int p = 0; p <= fine_n; ++p) {
    const float2 x = xf[p];
    float s, e;
    two_sum(uh, -x.x, s, e);
    const float dd = __fadd_rn(s, __fadd_rn(e, __fsub_rn(ul, x.y)));
    // a difference below 1e-30 is a node hit (and keeps the reciprocal finite)
    const bool at = fabsf(dd) < 1e-30f;
    if (at) hit = p;
    r[p] = at ? 0.0f : recip_pair(dd, 0.0f);
  }
  // level 2: X^2 = {0, 1/2, 1} with weights 1/2, -1, 1/2
  float ph, pl, dh, dl;
  {
    const float a = 0.5f * r[0], c = 0.5f * r[fine_n], m = r[fine_n / 2];
    float s, e;
    two_sum(a, c, s, e);
    pair_add(s, e, m, 0.0f, ph, pl);
    pair_add(s, e, -m, 0.0f, dh, dl);
  }
  int id = 1;
#pragma unroll
  for (int l = 2; l <= L + 1; ++l) {
    const int n = 1 << (l - 1), sf = fine_n / n;
    if (l > 2) {
      float nh = 0.0f, nl = 0.0f;
#pragma unroll
      for (int m = 1; m < n; m += 2) pair_add(nh, nl, r[m * sf], 0.0f, nh, nl);
      pair_add(ph, pl, -nh, -nl, dh, dl);
      pair_add(ph, pl, nh, nl, ph, pl);
    }
    const bool exact = hit >= 0 && (hit % sf) == 0;
    const float inv = exact ? 0.0f : recip_pair(dh, dl);
    const int cnt = l == 2 ? 2 : (n >> 1);
#pragma unroll
    for (int j = 0; j < cnt; ++j) {
      const int m = l == 2 ? j * n : 2 * j + 1;
      float wm = (m & 1) ? -1.0f : 1.0f;
      if (m == 0 || m == n) wm *= 0.5f;
      const float v = exact ? ((m * sf == hit) ? 1.0f : 0.0f) : __fmul_rn(wm * r[m * sf], inv);
      tab[(id + j) * stride] = v;
    }
    id += cnt;
  }
}

// x as a pair of floats h + l without FP64 arithmetic: h keeps the top 24
// bits of the significand (truncated), l the remaining 29 bits (rounded to
// FP32), both from the bit pattern.  Values outside 2^-74 <= |x| < 2^127
// (and zero) take the FP64 conversion.
__device__ __forceinline__ void split_double(double x, float& h, float& l) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
  const int e = static_cast<int>((hi >> 20) & 0x7FFu);
  if (e < 949 || e > 1150) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - static_cast<double>(h));
    return;
  }
  const unsigned sign = hi & 0x80000000u;
  h = __uint_as_float(sign | (static_cast<unsigned>(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
  const float scale = __uint_as_float(static_cast<unsigned>(e - 948) << 23);   // 2^(e - 1075)
  l = __uint_as_float(__float_as_uint(__uint2float_rn(lo & 0x1FFFFFFFu) * scale) | sign);
}

// (ah + al) (bh + bl) as a pair
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  h = __fadd_rn(p, e);
  l = __fsub_rn(e, __fsub_rn(h, p));
}

// The tables of one coordinate for any level: the compensated FP32 form for
// levels up to 5 inside the box, else the pair-of-floats form.  (Outside
// [0, 1] the barycentric sums cancel by the Lebesgue function of the point,
// which grows fast with the distance to the box; there the reciprocals need
// the pairs' precision.)
__device__ __forceinline__ void sf_basis_row(float uh, float ul, int level, const float2* __restrict__ xf,
                                             float* tab, int stride) {
  if (!(uh >= 0.0f && uh <= 1.0f)) level = -level - 1;
  switch (level) {
    case 0: tab[0] = 1.0f; return;
    case 1: return basis_row_f32c<1>(uh, ul, xf, tab, stride);
    case 2: return basis_row_f32c<2>(uh, ul, xf, tab, stride);
    case 3: return basis_row_f32c<3>(uh, ul, xf, tab, stride);
    case 4: return basis_row_f32c<4>(uh, ul, xf, tab, stride);
    case 5: return basis_row_f32c<5>(uh, ul, xf, tab, stride);
    default:
      basis_row_df_hi(static_cast<double>(uh) + static_cast<double>(ul), level < 0 ? -level - 1 : level, xf, tab,
                      stride);
  }
}

// Product of the table entries at four offsets (unused ones point at the
// constant 1, so S of them are read).
template <int S>
__device__ __forceinline__ float sf_prod(uint2 o, const float* __restrict__ tabrow) {
  float v = tabrow[o.x & 0xFFFFu];
  if (S > 1) v = __fmul_rn(v, tabrow[o.x >> 16]);
  if (S > 2) v = __fmul_rn(v, tabrow[o.y & 0xFFFFu]);
  if (S > 3) v = __fmul_rn(v, tabrow[o.y >> 16]);
  return v;
}

// One K-step (8 operand columns) of A_hi and A_lo for one query row, in the
// K-major core-matrix layout (`off`: the row's place in the K-step).
template <int S>
__device__ __forceinline__ void sf_produce(const uint2* __restrict__ ops, const float* __restrict__ tabrow,
                                           unsigned char* ahi, unsigned char* alo, int off) {
#pragma unroll
  for (int c2 = 0; c2 < 2; ++c2) {
    float hv[4], lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tf32_split(sf_prod<S>(ops[c2 * 4 + j], tabrow), hv[j], lv[j]);
    *reinterpret_cast<float4*>(ahi + off + c2 * 128) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4*>(alo + off + c2 * 128) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
}

// Waits for this thread's tensor-memory loads; r is an operand, so no use of
// the loaded registers moves above the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Epilogue of one 16-column accumulator chunk whose first column has index
// c0 within its group ([a][c] order, K = k columns per a, c0 % K = P):
// uf[c] += Phi_a G_{a,c} over the chunk's columns.
// (the chunk's tensor-memory load is in flight on entry: the a-tuple
// products are formed before waiting for it)
template <int K, int P, int S>
__device__ __forceinline__ void sf_epi_body(uint32_t (&r)[16], const uint2* __restrict__ ap,
                                            const float* __restrict__ tabrow, float (&uf)[8]) {
  constexpr int NA = (P + 15) / K + 1;
  float phi[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) phi[i] = sf_prod<S>(ap[i], tabrow);
  tmem_wait_ld(r);
#pragma unroll
  for (int j = 0; j < 16; ++j) uf[(P + j) % K] = fmaf(phi[(P + j) / K], __uint_as_float(r[j]), uf[(P + j) % K]);
}

template <int K, int S>
__device__ __forceinline__ void sf_epi_chunk(uint32_t (&r)[16], int c0, const uint2* __restrict__ ag,
                                             const float* __restrict__ tabrow, float (&sh)[8], float (&sl)[8]) {
  float uf[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const uint2* ap = ag + c0 / K;
  switch (c0 % K) {
    case 0: sf_epi_body<K, 0, S>(r, ap, tabrow, uf); break;
    case 1: if constexpr (K > 1) sf_epi_body<K, 1 % K, S>(r, ap, tabrow, uf); break;
    case 2: if constexpr (K > 2) sf_epi_body<K, 2 % K, S>(r, ap, tabrow, uf); break;
    case 3: if constexpr (K > 3) sf_epi_body<K, 3 % K, S>(r, ap, tabrow, uf); break;
    case 4: if constexpr (K > 4) sf_epi_body<K, 4 % K, S>(r, ap, tabrow, uf); break;
    case 5: if constexpr (K > 5) sf_epi_body<K, 5 % K, S>(r, ap, tabrow, uf); break;
    case 6: if constexpr (K > 6) sf_epi_body<K, 6 % K, S>(r, ap, tabrow, uf); break;
    default: if constexpr (K > 7) sf_epi_body<K, 7 % K, S>(r, ap, tabrow, uf); break;
  }
  // the chunk's sums enter a compensated (hi, lo) accumulator per output
#pragma unroll
  for (int c = 0; c < K; ++c) {
    float e;
    two_sum(sh[c], uf[c], sh[c], e);
    sl[c] = __fadd_rn(sl[c], e);
  }
}

// The CUDA-core columns [j0, j1) of this part (j = j0 + part, + 3, ...; the
// segment is whole rounds of 8 columns per part): product of the column's S
// table entries times its row of FP32 surpluses, summed in FP32 over eight
// columns at a time, then into the compensated accumulators.
template <int S>
__device__ __forceinline__ void sf_gemv(const uint2* __restrict__ gops, const float4* __restrict__ gw, int j0,
                                        int j1, int kw, int K, int part, const float* __restrict__ tabrow,
                                        float (&sh)[8], float (&sl)[8]) {
  const int stride4 = kw / 4;
  for (int jb = j0 + part; jb < j1; jb += 8 * kSfParts) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = jb + i * kSfParts;
      const float v = sf_prod<S>(gops[j], tabrow);
      const float4 w0 = gw[j * stride4];
      acc[0] = fmaf(v, w0.x, acc[0]);
      acc[1] = fmaf(v, w0.y, acc[1]);
      acc[2] = fmaf(v, w0.z, acc[2]);
      acc[3] = fmaf(v, w0.w, acc[3]);
      if (K > 4) {
        const float4 w1 = gw[j * stride4 + 1];
        acc[4] = fmaf(v, w1.x, acc[4]);
        acc[5] = fmaf(v, w1.y, acc[5]);
        acc[6] = fmaf(v, w1.z, acc[6]);
        acc[7] = fmaf(v, w1.w, acc[7]);
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < K) {
        float e;
        two_sum(sh[c], acc[c], sh[c], e);
        sl[c] = __fadd_rn(sl[c], e);
      }
    }
  }
}

template <int S>
__device__ __forceinline__ void sf_epi_k(int K, uint32_t (&r)[16], int c0, const uint2* __restrict__ ag,
                                         const float* __restrict__ tabrow, float (&sh)[8], float (&sl)[8]) {
  switch (K) {
    case 1: sf_epi_chunk<1, S>(r, c0, ag, tabrow, sh, sl); break;
    case 2: sf_epi_chunk<2, S>(r, c0, ag, tabrow, sh, sl); break;
    case 3: sf_epi_chunk<3, S>(r, c0, ag, tabrow, sh, sl); break;
    case 4: sf_epi_chunk<4, S>(r, c0, ag, tabrow, sh, sl); break;
    case 5: sf_epi_chunk<5, S>(r, c0, ag, tabrow, sh, sl); break;
    case 6: sf_epi_chunk<6, S>(r, c0, ag, tabrow, sh, sl); break;
    case 7: sf_epi_chunk<7, S>(r, c0, ag, tabrow, sh, sl); break;
    default: sf_epi_chunk<8, S>(r, c0, ag, tabrow, sh, sl); break;
  }
}

__device__ __forceinline__ void sf_mma(uint32_t dcol, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__global__ void __launch_bounds__(kSfThreads, 1) k_eval_sf_tf32x3(SfArgs t) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kSfRows - 1), part = tid >> 7;
  const bool producer = tid < kSfProducers;
  const int K = t.k;
  // layout: ring | W tiles | plan tables | 1-D tables (+ the zero entry) | barriers
  unsigned char* ring = smem;
  unsigned char* bsm = ring + kSfStages * kSfStageBytes;
  unsigned char* meta = bsm + t.bbytes;
  float* tab = reinterpret_cast<float*>(meta + t.meta_bytes);
  const int ntab = t.d * t.nf + 1;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tab + size_t(ntab) * kSfRows);
  uint64_t* full = bars;
  uint64_t* empty = bars + kSfStages;
  uint64_t* done = bars + 2 * kSfStages;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kSfStages + 1);
  const uint2* sops = reinterpret_cast<const uint2*>(meta);
  const uint2* gops = reinterpret_cast<const uint2*>(meta + t.o_gops);
  const uint2* aops = reinterpret_cast<const uint2*>(meta + t.o_aops);
  const float4* gw = reinterpret_cast<const float4*>(bsm + t.o_gw);
  const SfEpi* epi = reinterpret_cast<const SfEpi*>(meta + t.o_epi);
  const SfMma* prog = reinterpret_cast<const SfMma*>(meta + t.o_prog);
  const int32_t* pstart = reinterpret_cast<const int32_t*>(meta + t.o_pstart);

  for (int i = tid; i < t.bbytes / 16; i += kSfThreads)
    reinterpret_cast<float4*>(bsm)[i] = reinterpret_cast<const float4*>(t.bpack)[i];
  for (int i = tid; i < t.meta_bytes / 16; i += kSfThreads)
    reinterpret_cast<float4*>(meta)[i] = reinterpret_cast<const float4*>(t.meta)[i];
  if (producer && part == 0) tab[size_t(ntab - 1) * kSfRows + row] = 0.0f;
  if (warp == kSfProducers / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(t.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    if (lane == 0) {
      for (int s = 0; s < kSfStages; ++s) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(kSfProducers));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
      }
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the W tiles, for the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_holder;
  const int nchunks = (t.nks + kSfKsteps - 1) / kSfKsteps;
  const int64_t ntiles = (t.Q + kSfRows - 1) / kSfRows;
  // this row's place in a K-step: element (r, k) at ((r/8)*2 + k/4)*128 + (r%8)*16 + (k%4)*4
  const int aoff = ((row / 8) * 2) * 128 + (row % 8) * 16;
  const float* tabrow = tab + row;
  float2* partial = reinterpret_cast<float2*>(ring);   // [part][row][8] pairs, after the tile's products
  // the dimensions whose 1-D tables this thread computes (at most 3 for d <= 8),
  // their reciprocal box widths, and their coordinates for the coming tile
  constexpr int kDims = (kMaxDim + kSfParts - 1) / kSfParts;
  double xn[kDims];
  float loh[kDims], lol[kDims], rwh[kDims], rwl[kDims];   // box corner and 1 / width as pairs
  float uh[kDims], ul[kDims];   // the coming tile's unit coordinates as pairs of floats
  // unit coordinate (x - lo) / width of the loaded x as a pair, in pair-of-floats
  // arithmetic (0.5 for rows past the end)
  auto to_pair = [&](int j, bool live, float& h, float& l) {
    if (!live) {
      h = 0.5f;
      l = 0.0f;
      return;
    }
    float xh, xl, dh, dl;
    split_double(xn[j], xh, xl);
    pair_add(xh, xl, -loh[j], -lol[j], dh, dl);
    pair_mul(dh, dl, rwh[j], rwl[j], h, l);
  };
#pragma unroll
  for (int j = 0; j < kDims; ++j) {
    const int dim = part + j * kSfParts;
    const bool mine = producer && dim < t.d;
    const double rw = mine ? 1.0 / t.width[dim] : 0.0;
    rwh[j] = __double2float_rn(rw);
    rwl[j] = __double2float_rn(rw - static_cast<double>(rwh[j]));
    const double lo = mine ? t.lo[dim] : 0.0;
    loh[j] = __double2float_rn(lo);
    lol[j] = __double2float_rn(lo - static_cast<double>(loh[j]));
    const int64_t q = int64_t(blockIdx.x) * kSfRows + row;
    xn[j] = mine && q < t.Q ? t.xq[q * t.d + dim] : 0.0;
    if (mine) to_pair(j, q < t.Q, uh[j], ul[j]);
  }
  int64_t tile = blockIdx.x;
  int it = 0;
  int failed = 0;   // this thread saw a wait time out
  for (; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t q = tile * kSfRows + row;
    const int64_t qn = q + int64_t(gridDim.x) * kSfRows;   // this row in the next tile
    if (producer) {
#pragma unroll
      for (int j = 0; j < kDims; ++j) {
        const int dim = part + j * kSfParts;
        if (dim < t.d) sf_basis_row(uh[j], ul[j], t.level, t.xfdf, tab + (dim * t.nf) * kSfRows + row, kSfRows);
      }
      // the next tile's coordinates, loaded while this tile computes
#pragma unroll
      for (int j = 0; j < kDims; ++j) {
        const int dim = part + j * kSfParts;
        if (dim < t.d && qn < t.Q) xn[j] = t.xq[qn * t.d + dim];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    // tables complete; the previous tile's epilogue is over; any thread's
    // failed wait stops the CTA (the same decision in every thread)
    const int stop = __syncthreads_or(failed);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (stop) break;
    bool ok = true;
    float sh[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, sl[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (producer) {
      for (int c = 0; c < nchunks && ok; ++c) {
        const int g = it * nchunks + c, st = g % kSfStages;
        if (g >= kSfStages) ok = mbar_wait(smem_u32(&empty[st]), ((g / kSfStages) - 1) & 1);
        if (!ok) break;
        const int ks = c * kSfKsteps + part;
        if (ks < t.nks) {
          unsigned char* ahi = ring + st * kSfStageBytes + part * kSfKstepBytes;
          unsigned char* alo = ahi + kSfKsteps * kSfKstepBytes;
          const uint2* ops = sops + size_t(ks) * 8;
          switch (t.side) {
            case 1: sf_produce<1>(ops, tabrow, ahi, alo, aoff); break;
            case 2: sf_produce<2>(ops, tabrow, ahi, alo, aoff); break;
            case 3: sf_produce<3>(ops, tabrow, ahi, alo, aoff); break;
            default: sf_produce<4>(ops, tabrow, ahi, alo, aoff); break;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full[st]));
      }
      // the next tile's unit coordinates
#pragma unroll
      for (int j = 0; j < kDims; ++j)
        if (part + j * kSfParts < t.d) to_pair(j, qn < t.Q, uh[j], ul[j]);
      // the CUDA-core columns (one node each), while the products run
      sf_gemv<1>(gops, gw, t.gseg[0], t.gseg[1], t.kw, K, part, tabrow, sh, sl);
      sf_gemv<2>(gops, gw, t.gseg[1], t.gseg[2], t.kw, K, part, tabrow, sh, sl);
      sf_gemv<3>(gops, gw, t.gseg[2], t.gseg[3], t.kw, K, part, tabrow, sh, sl);
      sf_gemv<4>(gops, gw, t.gseg[3], t.gseg[4], t.kw, K, part, tabrow, sh, sl);
    } else if (lane == 0) {
      const uint32_t bbase = smem_u32(bsm);
      for (int c = 0; c < nchunks && ok; ++c) {
        const int g = it * nchunks + c, st = g % kSfStages;
        ok = mbar_wait(smem_u32(&full[st]), (g / kSfStages) & 1);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sbase = smem_u32(ring + st * kSfStageBytes);
        for (int j = 0; j < kSfKsteps; ++j) {
          const int ks = c * kSfKsteps + j;
          if (ks >= t.nks) break;
          const uint64_t dhi = smem_desc(sbase + j * kSfKstepBytes, 128, 256);
          const uint64_t dlo = smem_desc(sbase + (kSfKsteps + j) * kSfKstepBytes, 128, 256);
          for (int e = pstart[ks]; e < pstart[ks + 1]; ++e) {
            const SfMma m = prog[e];
            const uint32_t idesc = idesc_tf32_mn(kSfRows, static_cast<int>(m.n));
            const uint64_t bhi = smem_desc(bbase + m.boff, 128, 256);
            const uint64_t blo = smem_desc(bbase + m.boff + m.n * 32, 128, 256);
            sf_mma(tmem + m.col, dhi, bhi, idesc, m.accum);
            sf_mma(tmem + m.col, dhi, blo, idesc, 1u);
            sf_mma(tmem + m.col, dlo, bhi, idesc, 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&empty[st])));
      }
      // arrives when every product of the tile has completed
      if (t.nks > 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(done)));
    }
    __syncwarp();
    if (!ok) failed = 1;
    if (producer) {
      const bool fin = ok && (t.nks == 0 || mbar_wait(smem_u32(done), it & 1));
      if (!fin) failed = 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int ch = part; ch < t.nepi && fin; ch += kSfParts) {
        const SfEpi ep = epi[ch];
        const uint32_t taddr = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + ep.col;
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        const uint2* ag = aops + ep.abase;
        // the a-tuples have at most d / 2 non-constant factors, first
        if (t.d <= 7) sf_epi_k<3>(K, r, ep.c0, ag, tabrow, sh, sl);
        else sf_epi_k<4>(K, r, ep.c0, ag, tabrow, sh, sl);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < K) partial[(part * kSfRows + row) * 8 + c] = make_float2(sh[c], sl[c]);
    }
    const int bad = __syncthreads_or(failed);   // partial sums complete
    if (producer && part == 0 && q < t.Q) {
      for (int c = 0; c < K; ++c) {
        float h = 0.0f, l = 0.0f;
#pragma unroll
        for (int p = 0; p < kSfParts; ++p) {
          const float2 v = partial[(p * kSfRows + row) * 8 + c];
          pair_add(h, l, v.x, v.y, h, l);
        }
        t.out[q * K + c] = bad ? NAN : static_cast<double>(h) + static_cast<double>(l);
      }
    }
  }
  // a wait timed out: this CTA's remaining queries get NaN
  for (; tile < ntiles; tile += gridDim.x) {
    const int64_t q = tile * kSfRows + row;
    if (producer && part == 0 && q < t.Q)
      for (int c = 0; c < K; ++c) t.out[q * K + c] = NAN;
  }
  if (__syncthreads_or(failed) && tid == 0) atomicExch(t.err, 1);
  if (warp == kSfProducers / 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(t.tmem_cols));
}

int eval_sf_tf32x3(const EvalArgs& e, const sg_surplus* s, cudaStream_t st) {
  SfArgs t{};
  t.xq = e.xq;
  t.Q = e.Q;
  t.d = s->d;
  t.nf = s->nf;
  t.level = s->level;
  t.k = s->k;
  t.side = s->sf_side;
  t.nks = s->sf_nks;
  t.nepi = s->sf_nepi;
  t.tmem_cols = s->sf_tmem;
  t.bbytes = static_cast<int>(s->sf_bbytes);
  t.lo = e.lo;
  t.width = e.width;
  t.xfdf = e.xfdf;
  t.meta_bytes = static_cast<int>(s->sf_meta_bytes);
  t.o_gops = static_cast<int>(s->sf_o_gops);
  t.ngemv = s->sf_ngemv;
  for (int i = 0; i < 5; ++i) t.gseg[i] = s->sf_gseg[i];
  t.kw = s->sf_kw;
  t.o_gw = static_cast<int>(s->sf_o_gw);
  t.o_aops = static_cast<int>(s->sf_o_aops);
  t.o_epi = static_cast<int>(s->sf_o_epi);
  t.o_prog = static_cast<int>(s->sf_o_prog);
  t.o_pstart = static_cast<int>(s->sf_o_pstart);
  t.meta = s->sf_meta;
  t.bpack = s->sf_b;
  t.out = e.out;
  t.err = s->tc_err;
  // one CTA per SM: the request also keeps a second CTA (and its tensor
  // memory) off the SM when the plan itself is small
  const size_t smem = std::max(s->sf_smem, size_t(116) * 1024);
  SG_CUDA_TRY(ensure_dynamic_smem(k_eval_sf_tf32x3, static_cast<int>(smem)));
  int dev = 0, nsm = 0;
  SG_CUDA_TRY(cudaGetDevice(&dev));
  SG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntiles = ceil_div(e.Q, kSfRows);
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(ntiles, nsm));
  SG_TIMED("k_eval_sf_tf32x3", st, (k_eval_sf_tf32x3<<<blocks, kSfThreads, smem, st>>>(t)));
  SG_LAUNCH_CHECK("k_eval_sf_tf32x3");
  return SG_OK;
}

}  // namespace sg
