// f64bits.cuh -- line maxima of finite FP64 values from their bit patterns
// (the FP64-accuracy split's row and column exponents), shared by the digit
// split and by the Strassen operand pass that can produce them on the way.
#pragma once
#include <cstdint>

namespace mmsr {

// |x| as a bit pattern: for finite doubles the unsigned order of these
// patterns is the numeric order of |x|.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// The high word of abs_bits(x): sign-free exponent field and the top 20
// significand bits.  The maximum of these words over a line has the same
// leading bit as the maximum of the full patterns whenever it is nonzero, so
// it fixes the line's exponent; a zero maximum (the line is zero or holds
// only subnormals below 2^-1042) needs the full patterns.
__device__ __forceinline__ uint32_t abs_hi_word(double x) {
  return (uint32_t)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7FFFFFFFu;
}

// Exponent E with max|x| < 2^E, from the bit pattern of max|x| (0 for an
// all-zero line): frexp's exponent, max|x| = f 2^E with f in [0.5, 1) --
// the exponent field minus 1022 for a normal number, the position of the
// leading significand bit for a subnormal one (value = b 2^-1074).
__device__ __forceinline__ int line_exponent(unsigned long long b) {
  if (b == 0) return 0;
  const int ex = (int)(b >> 52);
  if (ex != 0) return ex - 1022;
  return (63 - __clzll((long long)b)) - 1073;
}

}  // namespace mmsr
