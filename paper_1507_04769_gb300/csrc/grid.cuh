// Sparse grid handle shared by the grid and interpolant translation units.
#pragma once

#include <vector>

#include "common.cuh"

struct sg_grid {
  int d = 0;
  int level = 0;
  int64_t M = 0;
  double* coords = nullptr;   // device, M x d
  int8_t* lev = nullptr;      // device, M x d
  int16_t* kidx = nullptr;    // device, M x d
  void* block = nullptr;      // the one device allocation the arrays above live in
  std::vector<int8_t> h_lev;  // host copies of the integer structure
  std::vector<int16_t> h_kidx;
  std::vector<double> h_lo, h_hi;
};

namespace sg {
int delta_count(int i);
int delta_index(int i, int j);
void enumerate_nodes(int d, int level, std::vector<int8_t>& lev, std::vector<int16_t>& kidx);
}  // namespace sg
