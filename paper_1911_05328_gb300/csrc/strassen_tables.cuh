// strassen_tables.cuh -- the bilinear coefficient tables of one Strassen-like
// level (Section 5 and its bilinear generalisation) and the operand sums they
// define, shared by the level passes and the fused-staging leaf.
#pragma once

#include <stdint.h>

namespace mmsr {

// ------------------------------------------------------ coefficient tables
// One source for host and device: alpha / beta are [variant][product r]
// [quadrant q], gamma is [variant][quadrant q][product r].  Kernels take the
// variant as a template argument, so every coefficient is a compile-time
// constant and the zero terms vanish from the generated code.
__host__ __device__ constexpr int coef_alpha(int v, int r, int q) {
  constexpr int8_t t[2][7][4] = {
      {{1, 0, 0, 1}, {0, 0, 1, 1}, {1, 0, 0, 0}, {0, 0, 0, 1}, {1, 1, 0, 0}, {-1, 0, 1, 0}, {0, 1, 0, -1}},
      {{1, 0, 0, 0}, {0, 1, 0, 0}, {1, 1, -1, -1}, {0, 0, 0, 1}, {0, 0, 1, 1}, {-1, 0, 1, 1}, {1, 0, -1, 0}}};
  return t[v][r][q];
}
__host__ __device__ constexpr int coef_beta(int v, int r, int q) {
  constexpr int8_t t[2][7][4] = {
      {{1, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, -1}, {-1, 0, 1, 0}, {0, 0, 0, 1}, {1, 1, 0, 0}, {0, 0, 1, 1}},
      {{1, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}, {1, -1, -1, 1}, {-1, 1, 0, 0}, {1, -1, 0, 1}, {0, -1, 0, 1}}};
  return t[v][r][q];
}
__host__ __device__ constexpr int coef_gamma(int v, int q, int r) {
  constexpr int8_t t[2][4][7] = {
      {{1, 0, 0, 1, -1, 0, 1}, {0, 0, 1, 0, 1, 0, 0}, {0, 1, 0, 1, 0, 0, 0}, {1, -1, 1, 0, 0, 1, 0}},
      {{1, 1, 0, 0, 0, 0, 0}, {1, 0, 1, 0, 1, 1, 0}, {1, 0, 0, -1, 0, 1, 1}, {1, 0, 0, 0, 1, 1, 1}}};
  return t[v][q][r];
}

template <typename T>
__device__ __forceinline__ T apply(int c, T acc, T x) {
  return c == 0 ? acc : (c > 0 ? acc + x : acc - x);
}

// Operand sum r of one side (0: alpha over A's quadrants, 1: beta over B's),
// terms in the fixed quadrant order 00, 01, 10, 11.
template <int VARIANT, int SIDE, typename T>
__device__ __forceinline__ T combo4(int r, T x0, T x1, T x2, T x3) {
  T acc = T(0);
  if constexpr (SIDE == 0) {
    acc = apply(coef_alpha(VARIANT, r, 0), acc, x0);
    acc = apply(coef_alpha(VARIANT, r, 1), acc, x1);
    acc = apply(coef_alpha(VARIANT, r, 2), acc, x2);
    acc = apply(coef_alpha(VARIANT, r, 3), acc, x3);
  } else {
    acc = apply(coef_beta(VARIANT, r, 0), acc, x0);
    acc = apply(coef_beta(VARIANT, r, 1), acc, x1);
    acc = apply(coef_beta(VARIANT, r, 2), acc, x2);
    acc = apply(coef_beta(VARIANT, r, 3), acc, x3);
  }
  return acc;
}

}  // namespace mmsr
