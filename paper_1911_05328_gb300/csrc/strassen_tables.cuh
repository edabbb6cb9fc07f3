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

// The first product r with gamma_qr != 0.
__host__ __device__ constexpr int first_gamma_term(int v, int q) {
  int r = 0;
  while (r < 7 && coef_gamma(v, q, r) == 0) ++r;
  return r;
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

// All seven operand sums of one side at one position (s[r] for product r).
// Strassen-Winograd's sums share terms -- A side: s4 = A10 + A11, s5 = s4 -
// A00, s6 = A00 - A10, s2 = A01 - s5; B side: s4 = B01 - B00, s5 = B11 - s4,
// s6 = B11 - B01, s3 = s5 - B10 -- four additions instead of seven; other
// variants sum each product's terms in quadrant order (combo4).
template <int VARIANT, int SIDE, typename T>
__device__ __forceinline__ void sums7(T x0, T x1, T x2, T x3, T (&s)[7]) {
  if constexpr (VARIANT == 1 && SIDE == 0) {
    s[0] = x0;
    s[1] = x1;
    s[3] = x3;
    s[4] = x2 + x3;
    s[5] = s[4] - x0;
    s[6] = x0 - x2;
    s[2] = x1 - s[5];
  } else if constexpr (VARIANT == 1 && SIDE == 1) {
    s[0] = x0;
    s[1] = x2;
    s[2] = x3;
    s[4] = x1 - x0;
    s[5] = x3 - s[4];
    s[6] = x3 - x1;
    s[3] = s[5] - x2;
  } else {
#pragma unroll
    for (int r = 0; r < 7; ++r) s[r] = combo4<VARIANT, SIDE>(r, x0, x1, x2, x3);
  }
}

// The four quadrant sums of seven products (c[q] = sum_r gamma_qr p[r]).
// Strassen-Winograd shares terms: u2 = p0 + p5, u3 = u2 + p6, u4 = u2 + p4;
// c0 = p0 + p1, c1 = u4 + p2, c2 = u3 - p3, c3 = u3 + p4 -- seven additions
// instead of ten.
template <int VARIANT, typename T>
__device__ __forceinline__ void post4(const T (&p)[7], T (&c)[4]) {
  if constexpr (VARIANT == 1) {
    const T u2 = p[0] + p[5];
    const T u3 = u2 + p[6];
    const T u4 = u2 + p[4];
    c[0] = p[0] + p[1];
    c[1] = u4 + p[2];
    c[2] = u3 - p[3];
    c[3] = u3 + p[4];
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = combo7<VARIANT>(q, p);
  }
}

}  // namespace mmsr
