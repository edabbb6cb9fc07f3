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

// acc +- x for the j-th nonzero term: the first one starts the sum (+x or
// -x) instead of adding it to zero -- the same value up to the sign of a zero
// result, one addition fewer per sum.  With the coefficients compile-time
// constants (unrolled loops) the branches resolve at compile time, which
// matters where the sums run on this GPU's FP64 pipe (about two operations
// per clock per SM).
template <typename T>
__device__ __forceinline__ T accumulate_term(int c, bool& started, T acc, T x) {
  if (c == 0) return acc;
  if (!started) {
    started = true;
    return c > 0 ? x : -x;
  }
  return c > 0 ? acc + x : acc - x;
}

// Operand sum r of one side (0: alpha over A's quadrants, 1: beta over B's),
// terms in the fixed quadrant order 00, 01, 10, 11.
template <int VARIANT, int SIDE, typename T>
__device__ __forceinline__ T combo4(int r, T x0, T x1, T x2, T x3) {
  T acc = T(0);
  bool started = false;
  if constexpr (SIDE == 0) {
    acc = accumulate_term(coef_alpha(VARIANT, r, 0), started, acc, x0);
    acc = accumulate_term(coef_alpha(VARIANT, r, 1), started, acc, x1);
    acc = accumulate_term(coef_alpha(VARIANT, r, 2), started, acc, x2);
    acc = accumulate_term(coef_alpha(VARIANT, r, 3), started, acc, x3);
  } else {
    acc = accumulate_term(coef_beta(VARIANT, r, 0), started, acc, x0);
    acc = accumulate_term(coef_beta(VARIANT, r, 1), started, acc, x1);
    acc = accumulate_term(coef_beta(VARIANT, r, 2), started, acc, x2);
    acc = accumulate_term(coef_beta(VARIANT, r, 3), started, acc, x3);
  }
  return acc;
}

// Post-addition of quadrant q: sum_r gamma_qr P_r in product order.
template <int VARIANT, typename T>
__device__ __forceinline__ T combo7(int q, const T (&p)[7]) {
  T acc = T(0);
  bool started = false;
#pragma unroll
  for (int r = 0; r < 7; ++r) acc = accumulate_term(coef_gamma(VARIANT, q, r), started, acc, p[r]);
  return acc;
}

}  // namespace mmsr
