// Host check of the sum-factorised evaluation plan (interp_sf.cu: sf_plan).
// For a Smolyak grid (d, L) and k outputs it enumerates the nodes, builds the
// plan with the library, and evaluates the interpolant's sum the way the
// kernel does, in FP64: the operand-A columns, the products of every K-step
// (tensor-core accumulators, with their overwrite/accumulate flags), the
// epilogue chunks and the CUDA-core columns.  The result must equal the
// direct sum over the nodes, sum_m w_m prod_j a_{m_j}(x_j), for random 1-D
// table values and surpluses; every table read must stay in range and every
// accumulator column read must have been written.
// Usage: sf_plan_check d L k  -> prints "ok <max rel diff>" or "FAIL <why>",
// exit status 0 on success, 2 when the plan does not fit (not an error).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <random>
#include <vector>

#include "../../paper_1507_04769_gb300/csrc/grid.cuh"
#include "../../paper_1507_04769_gb300/csrc/interp.cuh"

using namespace sg;

static int tile_float(int n, int k) { return ((n / 8) * 2 + k / 4) * 32 + (n % 8) * 4 + k % 4; }

int main(int argc, char** argv) {
  if (argc != 4) return 1;
  const int d = atoi(argv[1]), L = atoi(argv[2]), k = atoi(argv[3]);
  // Smolyak nodes: multi-indices i >= 1 with |i| <= d + L, tensor products of
  // the increment sets
  std::vector<uint16_t> fid;
  std::vector<int> lv(d);
  int64_t M = 0;
  std::function<void(int, int)> rec = [&](int a, int used) {
    if (a == d) {
      std::vector<int> j(d, 0);
      while (true) {
        for (int b = 0; b < d; ++b) fid.push_back(static_cast<uint16_t>(function_id(lv[b], delta_index(lv[b], j[b]))));
        ++M;
        int b = d - 1;
        while (b >= 0) {
          if (++j[b] < delta_count(lv[b])) break;
          j[b] = 0;
          --b;
        }
        if (b < 0) break;
      }
      return;
    }
    for (int l = 1; used + l + (d - a - 1) <= d + L; ++l) {
      lv[a] = l;
      rec(a + 1, used + l);
    }
  };
  rec(0, 0);
  const int nf = n_functions(L);
  SfPlan p;
  if (!sf_plan(d, L, nf, k, M, fid, p)) {
    printf("no plan (M=%lld)\n", static_cast<long long>(M));
    return 2;
  }
  const uint16_t* sops = reinterpret_cast<const uint16_t*>(p.meta.data());
  const uint16_t* gops = reinterpret_cast<const uint16_t*>(p.meta.data() + p.o_gops);
  const uint16_t* aops = reinterpret_cast<const uint16_t*>(p.meta.data() + p.o_aops);
  const SfEpi* epi = reinterpret_cast<const SfEpi*>(p.meta.data() + p.o_epi);
  const SfMma* prog = reinterpret_cast<const SfMma*>(p.meta.data() + p.o_prog);
  const int32_t* pstart = reinterpret_cast<const int32_t*>(p.meta.data() + p.o_pstart);
  const size_t naops = (p.o_epi - p.o_aops) / 2;
  const size_t ntab = (size_t(d) * nf + 1) * 128;
  auto fail = [](const char* why) {
    printf("FAIL %s\n", why);
    return 1;
  };
  std::mt19937_64 rng(1);
  std::uniform_real_distribution<double> U(-1, 1);
  double worst = 0;
  for (int trial = 0; trial < 4; ++trial) {
    std::vector<double> T(ntab, 0.0);   // T[(dim * nf + id) * 128] (one query row), the zero entry last
    for (int dim = 0; dim < d; ++dim)
      for (int id = 0; id < nf; ++id) T[size_t(dim * nf + id) * 128] = id == 0 ? 1.0 : U(rng);
    std::vector<double> W(M * k);
    for (auto& w : W) w = U(rng);
    std::vector<double> ref(k, 0.0), u(k, 0.0);
    for (int64_t m = 0; m < M; ++m) {
      double ph = 1;
      for (int dim = 0; dim < d; ++dim) ph *= T[size_t(dim * nf + fid[m * d + dim]) * 128];
      for (int c = 0; c < k; ++c) ref[c] += ph * W[m * k + c];
    }
    auto tab = [&](uint16_t o) { return o < ntab ? T[o] : NAN; };
    // operand A (hi part only: W's lo parts are zero here)
    std::vector<double> A(8 * p.nks);
    for (int c = 0; c < 8 * p.nks; ++c) {
      double v = 1;
      for (int j = 0; j < p.side; ++j) v *= tab(sops[c * 4 + j]);
      for (int j = p.side; j < 4; ++j)
        if (sops[c * 4 + j] != 0) return fail("operand column reads past its side");
      A[c] = v;
    }
    std::vector<double> B(p.bmap.size());
    for (size_t i = 0; i < B.size(); ++i) {
      const int32_t m = p.bmap[i];
      B[i] = m < 0 ? 0.0 : ((m & 3) == 1 ? 0.0 : W[m >> 2]);
    }
    std::vector<double> acc(p.tmem_cols, NAN);
    for (int ks = 0; ks < p.nks; ++ks)
      for (int e = pstart[ks]; e < pstart[ks + 1]; ++e) {
        const SfMma& m = prog[e];
        if (m.boff + 2 * m.n * 32 > p.bbytes || m.col + m.n > uint32_t(p.tmem_cols) || m.n % 16 || m.n > 256)
          return fail("product out of range");
        for (uint32_t n = 0; n < m.n; ++n) {
          double s = 0;
          for (int kk = 0; kk < 8; ++kk) s += A[8 * ks + kk] * B[m.boff / 4 + tile_float(n, kk)];
          acc[m.col + n] = m.accum ? acc[m.col + n] + s : s;
        }
      }
    for (int ie = 0; ie < p.nepi; ++ie) {
      const SfEpi& ep = epi[ie];
      for (int j = 0; j < 16; ++j) {
        const int col = ep.col + j, c = (ep.c0 + j) % k, a = (ep.c0 + j) / k;
        if (size_t(ep.abase + a) * 4 + 3 >= naops) return fail("epilogue tuple out of range");
        if (col >= p.tmem_cols || std::isnan(acc[col])) return fail("epilogue reads an unwritten column");
        double ph = 1;
        for (int i = 0; i < d / 2; ++i) ph *= tab(aops[(ep.abase + a) * 4 + i]);
        for (int i = d / 2; i < 4; ++i)
          if (aops[(ep.abase + a) * 4 + i] != 0) return fail("epilogue tuple reads past its half");
        u[c] += ph * acc[col];
      }
    }
    for (int S = 1; S <= 4; ++S) {
      if ((p.gseg[S] - p.gseg[S - 1]) % 24) return fail("CUDA-core segment not whole rounds");
      for (int j = p.gseg[S - 1]; j < p.gseg[S]; ++j) {
        double v = 1;
        for (int i = 0; i < S; ++i) v *= tab(gops[j * 4 + i]);
        for (int i = S; i < 4; ++i)
          if (gops[j * 4 + i] != 0) return fail("CUDA-core column reads past its factor count");
        for (int c = 0; c < k; ++c) {
          const int32_t m = p.bmap[p.o_gw / 4 + j * p.kw + c];
          if (m < 0) continue;
          if ((m & 3) != 2) return fail("CUDA-core column map");
          u[c] += v * W[m >> 2];
        }
      }
    }
    if (p.gseg[4] != p.ngemv) return fail("CUDA-core column count");
    for (int c = 0; c < k; ++c) worst = std::fmax(worst, std::fabs(u[c] - ref[c]) / (1e-300 + std::fabs(ref[c])));
  }
  if (!(worst < 1e-10)) {
    printf("FAIL max rel diff %.3e\n", worst);
    return 1;
  }
  printf("ok %.3e M=%lld nks=%d ngemv=%d tmem=%d smem=%zu\n", worst, static_cast<long long>(M), p.nks, p.ngemv,
         p.tmem_cols, p.smem);
  return 0;
}
