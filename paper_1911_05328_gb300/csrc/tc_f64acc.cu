// tc_f64acc.cu -- FP64-accuracy (+,x) from 16-bit tensor-core products.
//
// Each row of A (column of B) is scaled by a power of two 2^-E so that its
// entries lie in (-1, 1), and every scaled entry is cut into seven signed
// digits of 7 bits:  a' = sum_{s=0..6} d_s 2^-7(s+1) + r,  |d_0| <= 128,
// |d_s| <= 64 (s >= 1), |r| <= 2^-50.  Digits are small integers, exact in
// bf16, and digit products are exact in the FP32 tensor-core accumulator.
// The product groups by digit order g = s + u:
//
//   a'b' ~ sum_{g=0..6} 2^-7(g+2) G_g,   G_g = sum_{s+u=g} sum_t d_s(i,t) d'_u(t,j)
//
// (28 slice products; the dropped orders g >= 7 and the residuals are below
// 2^-49 of the scaled magnitudes, which leaves room for the error growth of
// Strassen levels above these leaves).  Each G_g is an integer: it
// accumulates in its own TMEM accumulator over chunks of 256 k, where every
// partial sum is an integer of magnitude <= 256 * 36864 < 2^24 (per k, the
// digit products of one order sum to at most 2 * 128 * 64 + 5 * 64 * 64), so
// the FP32 accumulation is exact whatever its rounding, and drain warps move
// each chunk into two
// int64 registers per output (hi = G0 2^14 + G1 2^7 + G2, lo = G3 2^21 +
// G4 2^14 + G5 2^7 + G6).  The epilogue forms 2^(E_i+F_j) (hi 2^-28 +
// lo 2^-56) in FP64.  FP64 arithmetic is used only for that final sum and
// for split-K partials.
//
// Tile 128 x 64, k-blocks of 32 (64-byte swizzled rows), a TMA ring of the
// slice tiles, one 64-column TMEM accumulator per order (adjacent), warp
// roles as in the FP32 mode.  Within a k-step one MMA takes an A slice
// against several stacked B slices (N up to 256), so each A slice is read
// from shared memory once per four orders instead of once per product.
// Each group accumulator has its own full / empty mbarrier pair: the drain
// warps read group g as soon as its last product of a chunk has completed
// (while the tensor core still works on groups g+1..6), and the MMA issuer
// waits only for the group it is about to overwrite, so the drain runs
// under the next chunk's products instead of between chunks.
#include <cuda_bf16.h>
#include <string.h>

#include "f64bits.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace mmsr {
namespace {

__device__ int g_f64acc_status;
// One-shot test switch: the first CTA of the next launch skips the arrival
// and loads of its first ring stage, so its MMA wait runs out.
__device__ int g_f64acc_skip_signal;

// Two digit schemes.  Seven 7-bit slices (28 products, orders g <= 6): the
// dropped orders and the rounding sit below 2^-49 of the scaled magnitudes,
// room for the error growth of three or four Strassen levels above the
// leaves.  Six 8-bit slices (21 products, orders g <= 5; digits in
// [-128, 128], still exact in bf16): 2^-47, enough for up to two levels, with
// a quarter fewer products and a sixth less operand traffic.  kOrderBound
// bounds the digit products of one order at one k (7 bits: 2 x 128 x 64 +
// 5 x 64^2; 8 bits: 6 x 128^2), which fixes how many k a chunk may sum
// exactly in FP32.
template <int SL>
struct Scheme;
template <>
struct Scheme<7> {
  static constexpr int kBits = 7, kIntBits = 49, kChunk = 8, kStages = 2;  // chunk: 8 k-blocks = 256 k
  static constexpr int64_t kOrderBound = 36864;
  static constexpr int kHiShift = 28, kLoShift = 56;  // value = hi 2^-28 + lo 2^-56
};
template <>
struct Scheme<6> {
  static constexpr int kBits = 8, kIntBits = 47, kChunk = 5, kStages = 3;  // chunk: 5 k-blocks = 160 k
  static constexpr int64_t kOrderBound = 98304;
  static constexpr int kHiShift = 30, kLoShift = 54;  // value = hi 2^-30 + lo 2^-54
};

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int kDrain = 8, kThreads = 64 + 32 * kDrain;
constexpr uint32_t A_TILE = BM * BK * 2, B_TILE = BN * BK * 2;
constexpr uint32_t TMEM_COLS = 512;  // SL groups x 64 columns used
template <int SL>
struct FaCfg {
  using S = Scheme<SL>;
  static constexpr int STAGES = S::kStages, CHUNK = S::kChunk;  // CHUNK k-blocks per drain
  static constexpr uint32_t STAGE_BYTES = SL * (A_TILE + B_TILE);
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 256;
  static_assert((int64_t)CHUNK * BK * S::kOrderBound < (1 << 24), "chunk sums must stay exact in FP32");
  static_assert(SMEM <= 232448, "shared memory of one CTA");
  static_assert(SL * BN <= (int)TMEM_COLS, "one TMEM accumulator per digit order");
  // orders with a second accumulator in the TMEM columns the others leave
  // free (six slices: orders 0 and 1, all 512 columns in use; seven: none)
  static constexpr int PP = SL == 6 ? 2 : 0;
  static_assert(SL * BN + PP * BN <= (int)TMEM_COLS, "alternate buffers fit in TMEM");
  static_assert(PP == 0 || SL * BN == 384, "alternate buffer at column 384");
  static_assert((2 * STAGES + 2 * SL + 4 * PP + 1) * 8 + 16 <= 256, "barriers fit the reserved bytes");
};
static_assert(BK == 32, "the MMA issue loop covers two 16-deep k-steps per k-block");

// ----------------------------------------------------------- split kernels
// The split passes work on the bit patterns of the (finite) FP64 inputs in
// integer arithmetic: this GPU's FP64 pipe retires about 2 operations per
// clock per SM, so maxima, exponents and the scaled rounding are read from
// the exponent and significand fields instead.

// abs_bits and line_exponent: f64bits.cuh.

// Row maxima of A (one warp per row), stored as the exponent E of the row.
__global__ void __launch_bounds__(256) row_exponent_kernel(const double* __restrict__ A, int64_t m,
                                                           int64_t k, int* __restrict__ E) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  unsigned long long mx = 0;
  for (int64_t t = lane; t < k; t += 32) mx = max(mx, abs_bits(A[row * k + t]));
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) E[row] = line_exponent(mx);
}

// Column maxima of B (k x n, batch blockIdx.z of a contiguous stack): each
// thread scans 256 rows of one column and folds the bit pattern of its
// maximum |x| into Fmax with an atomic max (Fmax starts at 0 = +0.0).
__global__ void __launch_bounds__(256) col_max_kernel(const double* __restrict__ B, int64_t k,
                                                      int64_t n, unsigned long long* __restrict__ Fmax) {
  B += (int64_t)blockIdx.z * k * n;
  Fmax += (int64_t)blockIdx.z * n;
  const int64_t col = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (col >= n) return;
  const int64_t r0 = (int64_t)blockIdx.y * 256, r1 = min(k, r0 + 256);
  unsigned long long mx = 0;
  for (int64_t t = r0; t < r1; ++t) mx = max(mx, abs_bits(B[t * n + col]));
  if (mx) atomicMax(&Fmax[col], mx);
}

__global__ void __launch_bounds__(256) col_exponent_kernel(const unsigned long long* __restrict__ Fmax,
                                                           int64_t count, int* __restrict__ F) {
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (j < count) F[j] = line_exponent(Fmax[j]);
}

// x 2^(INT_BITS-E) rounded to the nearest integer, ties to even, for finite
// x with |x| < 2^E.  x = sig 2^e2 exactly (sig the significand with its
// implicit bit), so the scaling by a power of two is an exponent shift and
// the one rounding is a right shift of sig with round-half-even;
// |result| <= 2^INT_BITS.
template <int INT_BITS>
__device__ __forceinline__ long long scaled_round(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long sig = b & 0xFFFFFFFFFFFFFull;
  int e2;
  if (ex) {
    sig |= 1ull << 52;
    e2 = ex - 1075;
  } else {
    e2 = -1074;
  }
  const int sh = e2 + INT_BITS - E;
  long long M;
  if (sh >= 0) {
    M = (long long)(sig << sh);  // sig 2^sh < 2^INT_BITS since |x| < 2^E
  } else if (sh <= -54) {
    M = 0;  // |x 2^(INT_BITS-E)| < 2^53 2^-54 = 1/2
  } else {
    const int r = -sh;
    const unsigned long long q = sig >> r, rem = sig & ((1ull << r) - 1), half = 1ull << (r - 1);
    M = (long long)(q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0));
  }
  return (b >> 63) ? -M : M;
}

// Digits of x * 2^-E: one rounding of x * 2^(INT_BITS-E) to an integer M,
// then balanced digits.  Adding K (half the digit base in every position
// below the top one) makes them plain fields: below the top, digit + half is
// a field of M + K, and the top digit is (M + K) shifted down, arithmetically.
// The fields come from the two 32-bit halves of M + K, and each digit becomes
// an exact float by the 2^23 trick (2^23 + u has u as its low mantissa bits).
__device__ __forceinline__ float field_digit(uint32_t u, float bias) {
  return __int_as_float(0x4B000000 | (int)u) - bias;  // (2^23 + u) - (2^23 + offset), exact
}
template <int SL>
__device__ __forceinline__ void digits(double x, int E, float (&d)[SL]);
// Seven 7-bit digits: |M| <= 2^49, M = sum_s d_s 128^(6-s), d_1..d_6 in
// [-64, 63], |d_0| <= 128; K = 64 (1 + 128 + ... + 128^5).
template <>
__device__ __forceinline__ void digits<7>(double x, int E, float (&d)[7]) {
  constexpr long long kOffset = 64LL * (((1LL << 42) - 1) / 127);
  const long long Mk = scaled_round<49>(x, E) + kOffset;
  const uint32_t lo = (uint32_t)Mk, hi = (uint32_t)(Mk >> 32);
  constexpr float kB64 = 8388608.0f + 64.0f, kB128 = 8388608.0f + 128.0f;
  d[6] = field_digit(lo & 127u, kB64);
  d[5] = field_digit((lo >> 7) & 127u, kB64);
  d[4] = field_digit((lo >> 14) & 127u, kB64);
  d[3] = field_digit((lo >> 21) & 127u, kB64);
  d[2] = field_digit(__funnelshift_r(lo, hi, 28) & 127u, kB64);
  d[1] = field_digit((hi >> 3) & 127u, kB64);
  d[0] = field_digit((uint32_t)(((int)hi >> 10) + 128), kB128);  // d_0 + 128 in [0, 256]
}
// Six 8-bit digits: |M| <= 2^47, M = sum_s d_s 256^(5-s), d_1..d_5 in
// [-128, 127], |d_0| <= 128; K = 128 (1 + 256 + ... + 256^4).
template <>
__device__ __forceinline__ void digits<6>(double x, int E, float (&d)[6]) {
  constexpr long long kOffset = 128LL * (((1LL << 40) - 1) / 255);
  const long long Mk = scaled_round<47>(x, E) + kOffset;
  const uint32_t lo = (uint32_t)Mk, hi = (uint32_t)(Mk >> 32);
  constexpr float kB128 = 8388608.0f + 128.0f;
  d[5] = field_digit(lo & 255u, kB128);
  d[4] = field_digit((lo >> 8) & 255u, kB128);
  d[3] = field_digit((lo >> 16) & 255u, kB128);
  d[2] = field_digit(lo >> 24, kB128);
  d[1] = field_digit(hi & 255u, kB128);
  d[0] = field_digit((uint32_t)(((int)hi >> 8) + 128), kB128);  // d_0 + 128 in [0, 256]
}

// A (m x k) -> SL digit slices, slice s at S + s*m*Kp (row pitch Kp, zero
// pad).  Each thread converts four adjacent columns and stores 8 bytes per
// slice; blockIdx.x covers 1024 columns, blockIdx.y takes rows with the
// grid's y stride (a few thousand blocks in all, each walking many rows).
template <int SL>
__global__ void __launch_bounds__(256) digits_rows_kernel(const double* __restrict__ A, int64_t m,
                                                          int64_t k, int64_t Kp,
                                                          const int* __restrict__ E,
                                                          __nv_bfloat16* __restrict__ S, bool vec) {
  const int64_t slice = m * Kp;
  const int64_t t = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 4;  // Kp % 32 == 0: t + 3 < Kp
  if (t >= Kp) return;
  for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
    double x[4];
    const double* src = A + i * k + t;
    if (vec && t + 4 <= k) {  // rows 16-byte aligned (k even, A 16-byte aligned)
      const double2 a = __ldcs(reinterpret_cast<const double2*>(src));
      const double2 b = __ldcs(reinterpret_cast<const double2*>(src) + 1);
      x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = t + u < k ? __ldcs(src + u) : 0.0;
    }
    const int Ei = E[i];
    float d[4][SL];
#pragma unroll
    for (int u = 0; u < 4; ++u) digits<SL>(x[u], Ei, d[u]);
    const int64_t e = i * Kp + t;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const __nv_bfloat162 p0 = __floats2bfloat162_rn(d[0][s], d[1][s]);
      const __nv_bfloat162 p1 = __floats2bfloat162_rn(d[2][s], d[3][s]);
      *reinterpret_cast<uint2*>(S + s * slice + e) =
          make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
    }
  }
}

// B (k x n, batch blockIdx.z of a contiguous stack of `batches`) -> SL
// digit slices of B^T: slice s holds batches*n rows of pitch Kp, batch b at
// rows [b*n, (b+1)*n).  Via a 64 (k) x 32 (n) shared tile; each thread
// converts four adjacent k of one column and stores 8 bytes per slice, so a
// warp writes two full 128-byte rows of each slice.
template <int SL>
__global__ void __launch_bounds__(256) digits_cols_kernel(const double* __restrict__ B, int64_t k,
                                                          int64_t n, int64_t Kp,
                                                          const int* __restrict__ F,
                                                          __nv_bfloat16* __restrict__ S, int batches) {
  __shared__ double tile[64][33];
  const int64_t b = blockIdx.z;
  B += b * k * n;
  F += b * n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int pk = threadIdx.x & 15, pn = threadIdx.x >> 4;  // k quad, n row (of 16) when storing
  const int64_t k0 = (int64_t)blockIdx.x * 64;
  const int64_t slice = (int64_t)batches * n * Kp;
  const bool full_k = k0 + 64 <= Kp;  // Kp % 32 == 0: the last block may hold 32 k
  // n-tiles with stride gridDim.y (the grid's y extent is capped at 65535)
  for (int64_t n0 = (int64_t)blockIdx.y * 32; n0 < n; n0 += (int64_t)gridDim.y * 32) {
    __syncthreads();  // the previous n-tile's readers are done with `tile`
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int kk = ty + 8 * it;
      const int64_t gk = k0 + kk, gn = n0 + tx;
      tile[kk][tx] = (gk < k && gn < n) ? B[gk * n + gn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int nn = pn + 16 * it;
      const int64_t gn = n0 + nn, gk = k0 + 4 * pk;
      if (gn >= n || (!full_k && 4 * pk >= 32)) continue;
      float d[4][SL];
      const int Fj = F[gn];
#pragma unroll
      for (int u = 0; u < 4; ++u) digits<SL>(tile[4 * pk + u][nn], Fj, d[u]);
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        uint2 v;
        const __nv_bfloat162 p0 = __floats2bfloat162_rn(d[0][s], d[1][s]);
        const __nv_bfloat162 p1 = __floats2bfloat162_rn(d[2][s], d[3][s]);
        memcpy(&v.x, &p0, 4);
        memcpy(&v.y, &p1, 4);
        *reinterpret_cast<uint2*>(S + s * slice + (b * n + gn) * Kp + gk) = v;
      }
    }
  }
}

// ------------------------------------------------------------ GEMM kernel
// 2^-s as an exact double (s < 1023), folded at compile time.
__host__ __device__ constexpr double exp2_neg(int s) { return s == 0 ? 1.0 : 0.5 * exp2_neg(s - 1); }

// x 2^s with the result ldexp(x, s) gives, by one multiplication with the
// power of two built from its exponent field wherever 2^s is a normal double
// (this GPU's FP64 pipe retires about two operations per clock per SM, so
// the epilogue counts them).
__device__ __forceinline__ double scale_pow2(double x, int s) {
  if (s >= -1022 && s <= 1023) return x * __longlong_as_double((long long)(s + 1023) << 52);
  return ldexp(x, s);
}

// c + a b with a 64-bit sum, one instruction.
__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
// RN((hi + lo 2^-W) 2^sc) -- the value scale_pow2(fma((double)lo, 2^-W,
// (double)hi), sc) gives, bit for bit -- with one FP64 operation instead of
// four (this GPU's FP64 pipe retires about two per clock per SM, and the
// tile's tensor core idles while its epilogue runs).  With s = hi + (lo >> W)
// and r = lo mod 2^W the value is s + r 2^-W; c = s - 2^(52-W) is an integer
// below 2^53, so c 2^sc and (2^52 + r) 2^(sc-W) are doubles built exactly
// from their bits, and one fma of them forms (s + r 2^-W) 2^sc exactly and
// rounds it once.  Scales far from 1, or |c| >= 2^53, take the plain path.
template <int W>
__device__ __forceinline__ double combine_scaled(long long hi, long long lo, int sc) {
  const long long s = hi + (lo >> W);
  const long long r = lo & ((1ll << W) - 1);
  const long long c = s - (1ll << (52 - W));
  const unsigned long long a = c < 0 ? 0ull - (unsigned long long)c : (unsigned long long)c;
  if (sc < -900 || sc > 900 || a >= (1ull << 53))
    return scale_pow2(fma((double)lo, exp2_neg(W), (double)hi), sc);
  double cs = 0.0;
  if (a != 0) {
    const int lz = __clzll((long long)a);  // >= 11
    const unsigned long long mant = (a << (lz - 11)) & ((1ull << 52) - 1);
    const unsigned long long be = (unsigned long long)((63 - lz) + 1023 + sc);
    cs = __longlong_as_double((long long)((c < 0 ? (1ull << 63) : 0ull) | (be << 52) | mant));
  }
  const double drb = __longlong_as_double(0x4330000000000000ll | r);
  const double f = __longlong_as_double((long long)(sc - W + 1023) << 52);
  return fma(drb, f, cs);
}

__device__ __forceinline__ int exact_int(uint32_t fbits) {
  // fbits holds an integer-valued float of magnitude < 2^24: the conversion
  // is exact in any rounding mode.
  return __float2int_rn(__uint_as_float(fbits));
}

// QUAD: the TAR-Strassen epilogue -- batch entry b multiplies the stacked
// operands of leaf quad.leaf[b] and adds quad.sign[b][d] x its tile into up
// to four blocks quad.dst[b][d] of C (row pitch quad.ld), overwriting where
// quad.add[b][d] is 0.  Entries of one launch write disjoint blocks.
template <int SL, bool QUAD>
__global__ void __launch_bounds__(kThreads, 1)
    f64acc_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
                       const int* __restrict__ E, const int* __restrict__ F, double* __restrict__ C,
                       double* __restrict__ W, int64_t m, int64_t n, int64_t a_slice_rows,
                       int64_t b_slice_rows, int kb_total, int kb_per_slice, int kslices,
                       const __grid_constant__ QuadOut64 quad) {
  using Cfg = FaCfg<SL>;
  constexpr int kSlices = SL, kGroups = SL, STAGES = Cfg::STAGES, CHUNK = Cfg::CHUNK;
  // Orders below kPP alternate between two TMEM buffers from chunk to chunk
  // (columns g*64 in even chunks, 384 + g*64 in odd ones: the columns the
  // six orders leave free), so at a chunk boundary they restart at once in
  // the other buffer and only orders kPP.. wait for the drain.  Orders 0 and
  // 1 appear only in slice 0's and slice 1's products, so splitting the
  // stacked MMAs at order kPP costs no extra MMA.
  constexpr int kPP = Cfg::PP;
  constexpr uint32_t STAGE_BYTES = Cfg::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;       // [kGroups] (orders kPP.. only)
  uint64_t* acc_empty = acc_full + kGroups;   // [kGroups]
  uint64_t* pp_full = acc_empty + kGroups;    // [2][kPP]: alternating orders, per buffer
  uint64_t* pp_empty = pp_full + 2 * kPP;     // [2][kPP]
  uint64_t* quiesce = pp_empty + 2 * kPP;     // after an abort: all issued MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(quiesce + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  // producer state read after an abort (shared, so that no register stays
  // live through the other roles): [0] k-blocks issued, [1] k-block 0 skipped
  int* prod_state = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Banded rasterisation: consecutive CTAs walk bands of 8 tile rows column
  // by column, so a wave touches ~8 x 128 A rows and ~19 x 64 B rows (the
  // minimum of rows_a * 128 + 152 / rows_a * 64) instead of one A panel
  // and all of B.
  int64_t i0, j0;
  {
    constexpr int kBand = 8;
    const int tiles_n = gridDim.x, tiles_m = gridDim.y;
    const int pid = blockIdx.y * tiles_n + blockIdx.x;
    const int band = pid / (kBand * tiles_n);
    const int first_m = band * kBand;
    const int rows = min(kBand, tiles_m - first_m);
    const int in_band = pid - band * kBand * tiles_n;
    i0 = (int64_t)(first_m + in_band % rows) * BM;
    j0 = (int64_t)(in_band / rows) * BN;
  }
  // blockIdx.z = batch * kslices + k-slice; batch b uses rows [b*m, (b+1)*m)
  // of every A slice (and of E), rows [b*n, (b+1)*n) of every B^T slice
  const int z = blockIdx.z % kslices;
  const int batch = blockIdx.z / kslices;
  const int64_t leaf = QUAD ? (int64_t)quad.leaf[batch] : (int64_t)batch;
  const int64_t ra = leaf * m, rb = leaf * n;
  const int kb_begin = z * kb_per_slice;
  const int kb_end = min(kb_total, kb_begin + kb_per_slice);
  const int nkb = kb_end > kb_begin ? kb_end - kb_begin : 0;
  const int nchunks = (nkb + CHUNK - 1) / CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int g = 0; g < kGroups; ++g) {
      tc::mbar_init(&acc_full[g], 1);
      tc::mbar_init(&acc_empty[g], kDrain);
    }
    for (int i = 0; i < 2 * kPP; ++i) {
      tc::mbar_init(&pp_full[i], 1);
      tc::mbar_init(&pp_empty[i], kDrain);
    }
    tc::mbar_init(quiesce, 1);
    *abort_flag = 0;
    prod_state[0] = prod_state[1] = 0;
    tc::mbar_init_fence();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      tc::tma_prefetch(&tA);
      tc::tma_prefetch(&tB);
      bool skipped = false;  // the test switch took k-block 0 out
      int issued = 0;        // k-blocks whose loads were issued
      if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && nkb > 0)
        skipped = atomicExch(&g_f64acc_skip_signal, 0) != 0;
      for (int it = 0; it < nkb; ++it, issued = it) {
        const int s = it % STAGES;
        const uint32_t round = (uint32_t)(it / STAGES);
        if (it >= STAGES && !tc::mbar_wait(&empty[s], (round - 1) & 1u, abort_flag, &g_f64acc_status)) break;
        if (it == 0 && skipped) continue;
        tc::mbar_expect_tx(&full[s], STAGE_BYTES);
        uint8_t* st = smem + s * STAGE_BYTES;
        const int kx = (kb_begin + it) * BK;
#pragma unroll
        for (int sl = 0; sl < kSlices; ++sl) {
          tc::tma_load_2d(st + sl * A_TILE, &tA, &full[s], kx, (int)(sl * a_slice_rows + ra + i0));
          tc::tma_load_2d(st + kSlices * A_TILE + sl * B_TILE, &tB, &full[s], kx,
                          (int)(sl * b_slice_rows + rb + j0));
        }
      }
      prod_state[0] = issued;
      prod_state[1] = skipped ? 1 : 0;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f16(BM, BN, 1);
      constexpr uint32_t dhi = tc::desc_hi_sw64();
      // The first k-step of a chunk overwrites the accumulators order by
      // order, each as soon as the drain has read it: the 128 x 64 products
      // of order g one by one.  Descriptors are one 32-bit add of a
      // compile-time offset to a per-stage base word.
      auto issue_group = [&](uint32_t a_lo, uint32_t b_lo, int kk, int g, bool overwrite) {
#pragma unroll
        for (int sa = 0; sa <= g; ++sa) {
          const uint32_t aoff = (uint32_t)(sa * A_TILE + kk * 32) >> 4;
          const uint32_t boff = (uint32_t)((g - sa) * B_TILE + kk * 32) >> 4;
          tc::mma_f16(tmem + (uint32_t)(g * BN), tc::desc_join(a_lo + aoff, dhi),
                      tc::desc_join(b_lo + boff, dhi), idesc, (overwrite && sa == 0) ? 0u : 1u);
        }
      };
      // One 16-deep k-step of all the slice products with few, wide MMAs: A
      // slice sa meets B slices 0..SL-1-sa, which lie one after another in
      // the stage (one K-major operand of 64 (SL - sa) rows), and their
      // products belong to orders sa..SL-1, whose accumulators are adjacent
      // in TMEM (orders below kPP adjacent among themselves, in this chunk's
      // buffer `pp_col`).  So one MMA of N = 64 x (orders it covers) does up
      // to four of the 128 x 64 products and reads its A slice from shared
      // memory once for all of them (pieces of at most four orders:
      // N <= 256).  With six slices a k-step is 8 MMAs instead of 21 and
      // reads 74 KB of operands instead of 126 KB.  Order sa is complete once
      // the first piece of slice sa is issued (later slices do not reach
      // it), which is where the chunk's last k-step signals its drain.
      // parts: 1 = the pieces of the alternating orders, 2 = the others.  A
      // chunk's last k-step issues the others first, so the orders the next
      // chunk waits for are complete (and drained) a few products earlier.
      auto issue_stacked = [&](uint32_t a_lo, uint32_t b_lo, int kk, bool last_step, uint32_t pp_col,
                               uint64_t* ppf, int parts) {
        auto pp_piece = [&](int sa) {
          const uint32_t aoff = (uint32_t)(sa * A_TILE + kk * 32) >> 4;
          const uint32_t boff = (uint32_t)(kk * 32) >> 4;
          tc::mma_f16(tmem + pp_col + (uint32_t)(sa * BN), tc::desc_join(a_lo + aoff, dhi),
                      tc::desc_join(b_lo + boff, dhi), tc::idesc_f16(BM, BN * (kPP - sa), 1), 1u);
          if (last_step) tc::mma_commit(&ppf[sa]);
        };
        auto main_pieces = [&](int sa) {
          const uint32_t aoff = (uint32_t)(sa * A_TILE + kk * 32) >> 4;
#pragma unroll
          for (int g0 = sa < kPP ? kPP : sa; g0 < kGroups; g0 += 4) {
            const int cnt = min(4, kGroups - g0);
            const uint32_t boff = (uint32_t)((g0 - sa) * B_TILE + kk * 32) >> 4;
            tc::mma_f16(tmem + (uint32_t)(g0 * BN), tc::desc_join(a_lo + aoff, dhi),
                        tc::desc_join(b_lo + boff, dhi), tc::idesc_f16(BM, BN * cnt, 1), 1u);
            if (last_step && g0 == sa) tc::mma_commit(&acc_full[sa]);
          }
        };
        if (last_step || parts != 3) {
          if (parts & 2) {
#pragma unroll
            for (int sa = 0; sa < kSlices; ++sa) main_pieces(sa);
          }
          if (parts & 1) {
#pragma unroll
            for (int sa = 0; sa < kPP; ++sa) pp_piece(sa);
          }
        } else {
#pragma unroll
          for (int sa = 0; sa < kSlices; ++sa) {
            if (sa < kPP) pp_piece(sa);
            main_pieces(sa);
          }
        }
      };
      int it = 0;
      bool aborted = false;
      for (int c = 0; c < nchunks && !aborted; ++c) {
        const int first_it = it;
        const int last = min(nkb, (c + 1) * CHUNK);
        const int buf = c & 1;
        const uint32_t pp_col = buf ? (uint32_t)(kGroups * BN) : 0u;
        uint64_t* ppf = pp_full + buf * kPP;
        for (; it < last && !aborted; ++it) {
          const int s = it % STAGES;
          const uint32_t round = (uint32_t)(it / STAGES);
          if (!tc::mbar_wait(&full[s], round & 1u, abort_flag, &g_f64acc_status)) {
            aborted = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
          const uint32_t a_lo = tc::desc_lo(base), b_lo = tc::desc_lo(base + kSlices * A_TILE);
          if (it == first_it) {
            // first k-block of a chunk: the alternating orders restart in this
            // chunk's buffer (read by the drain two chunks ago), then every
            // other order once the drain has read its previous chunk
            if constexpr (kPP > 0) {
              if (c >= 2) {
#pragma unroll
                for (int g = 0; g < kPP; ++g)
                  if (!aborted && !tc::mbar_wait(&pp_empty[buf * kPP + g], (uint32_t)((c >> 1) - 1) & 1u, abort_flag,
                                                 &g_f64acc_status))
                    aborted = true;
                tc::fence_after_sync();
              }
              if (!aborted) {
#pragma unroll
                for (int sa = 0; sa < kPP; ++sa)
                  tc::mma_f16(tmem + pp_col + (uint32_t)(sa * BN), tc::desc_join(a_lo + ((uint32_t)(sa * A_TILE) >> 4), dhi),
                              tc::desc_join(b_lo, dhi), tc::idesc_f16(BM, BN * (kPP - sa), 1), sa == 0 ? 0u : 1u);
                // their second half-step too: more work for the tensor core
                // while the other orders drain
                issue_stacked(a_lo, b_lo, 1, it == last - 1, pp_col, ppf, 1);
              }
            }
#pragma unroll
            for (int g = kPP; g < kGroups; ++g) {
              if (c >= 1 && !aborted) {
                if (!tc::mbar_wait(&acc_empty[g], (c - 1) & 1u, abort_flag, &g_f64acc_status)) aborted = true;
                tc::fence_after_sync();
              }
              if (!aborted) issue_group(a_lo, b_lo, 0, g, true);
            }
            if (!aborted) issue_stacked(a_lo, b_lo, 1, it == last - 1, pp_col, ppf, kPP > 0 ? 2 : 3);
          } else {
            issue_stacked(a_lo, b_lo, 0, false, pp_col, ppf, 3);
            issue_stacked(a_lo, b_lo, 1, it == last - 1, pp_col, ppf, 3);
          }
          tc::mma_commit(&empty[s]);
        }
      }
    }
  } else {
    // drain warps: lane quarter q, column half h (32 of the 64 columns)
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    long long hi[32], lo[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) hi[e] = lo[e] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      // orders kPP.. first (the issuer waits for them), then the alternating
      // ones, whose buffer is not needed again until two chunks later
#pragma unroll
      for (int i = 0; i < kGroups; ++i) {
        const int g = i + kPP < kGroups ? i + kPP : i + kPP - kGroups;
        const bool alt = g < kPP;
        uint64_t* fbar = alt ? &pp_full[(c & 1) * kPP + g] : &acc_full[g];
        uint64_t* ebar = alt ? &pp_empty[(c & 1) * kPP + g] : &acc_empty[g];
        const uint32_t par = alt ? (uint32_t)(c >> 1) & 1u : (uint32_t)c & 1u;
        const uint32_t col = (alt && (c & 1)) ? (uint32_t)((kGroups + g) * BN) : (uint32_t)(g * BN);
        // warp-uniform verdict: the __syncwarp below needs every lane
        ok = __all_sync(0xffffffffu, tc::mbar_wait(fbar, par, abort_flag, &g_f64acc_status));
        if (!ok) break;
        tc::fence_after_sync();
        constexpr int kb = Scheme<SL>::kBits;
        const int wgt = g < 3 ? (1 << (kb * (2 - g))) : (1 << (kb * (SL - 1 - g)));
        {
          // The tensor core waits for this at every chunk boundary, so it is
          // kept to one 32-column TMEM load and one wait per order, and per
          // value one conversion and one 32 x 32 + 64-bit multiply-add.
          uint32_t r[32];
          tc::tmem_ld_32x32b_x32(tmem + lane_base + col + (uint32_t)(h * 32), r);
          tc::tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            if (g < 3)
              hi[e] = mad_wide(exact_int(r[e]), wgt, hi[e]);
            else
              lo[e] = mad_wide(exact_int(r[e]), wgt, lo[e]);
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(ebar);
      }
    }
    const int64_t row = i0 + q * 32 + lane;
    if (row < m) {
      // C_ij = 2^(E_i + F_j) (hi 2^-kHiShift + lo 2^-kLoShift), rounded once
      // (combine_scaled: one fma of exact operands)
      constexpr int kHi = Scheme<SL>::kHiShift;
      const int Ei = E[ra + row];
      double v[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int64_t col = j0 + h * 32 + e;
        v[e] = (ok && col < n) ? combine_scaled<Scheme<SL>::kLoShift - kHi>(hi[e], lo[e], Ei + F[rb + col] - kHi) : 0.0;
      }
      const int64_t c0 = j0 + h * 32;
      if constexpr (QUAD) {
#pragma unroll 1
        for (int d = 0; d < 4; ++d) {
          double* base = quad.dst[batch][d];
          if (base == nullptr) continue;
          const bool neg = quad.sign[batch][d] < 0;
          const bool add = quad.add[batch][d] != 0;
          double* dst = base + row * quad.ld + c0;
          if (c0 + 32 <= n && aligned16(dst)) {
            // eight 16-byte reads of the old values in flight, then the sums
            // and their stores
#pragma unroll
            for (int u0 = 0; u0 < 16; u0 += 8) {
              double2 o[8];
#pragma unroll
              for (int u = 0; u < 8; ++u)
                o[u] = add ? reinterpret_cast<const double2*>(dst)[u0 + u] : make_double2(0.0, 0.0);
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int e = 2 * (u0 + u);
                const double x0 = neg ? -v[e] : v[e], x1 = neg ? -v[e + 1] : v[e + 1];
                reinterpret_cast<double2*>(dst)[u0 + u] =
                    add ? make_double2(o[u].x + x0, o[u].y + x1) : make_double2(x0, x1);
              }
            }
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              if (c0 + e < n) {
                const double x = neg ? -v[e] : v[e];
                dst[e] = add ? dst[e] + x : x;
              }
            }
          }
        }
      } else {
        double* out = ((z == 0) ? C + ra * n : W + (int64_t)(z - 1) * m * n) + row * n + c0;
        if (c0 + 32 <= n && aligned16(out)) {
#pragma unroll
          for (int u = 0; u < 16; ++u) reinterpret_cast<double2*>(out)[u] = make_double2(v[2 * u], v[2 * u + 1]);
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e)
            if (c0 + e < n) out[e] = v[e];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(abort_flag)) {
    // Aborted: let this CTA's own TMA loads (the last ring round issued) and
    // issued MMAs land before shared memory and TMEM are released; both waits
    // are bounded and ignore the abort flag.
    if (warp == 0 && lane == 0) {
      const int issued = prod_state[0], skipped = prod_state[1];
      for (int it = max(0, issued - STAGES); it < issued; ++it)
        if (!(it == 0 && skipped)) tc::mbar_wait_quiesce(&full[it % STAGES], (uint32_t)(it / STAGES) & 1u);
    }
    if (warp == 1 && lane == 0) {
      tc::mma_commit(quiesce);
      tc::mbar_wait_quiesce(quiesce, 0);
    }
    __syncwarp();
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct F64AccLayout {
  int64_t Kp, a_bytes, b_bytes, off_b, off_e, off_f, off_fmax, off_part, min_bytes;
  int slices;
};

F64AccLayout layout(int64_t m, int64_t n, int64_t k, int slices, int64_t batches = 1) {
  F64AccLayout L;
  L.slices = slices;
  L.Kp = align_up(k > 0 ? k : 1, BK);
  L.a_bytes = align_up((int64_t)slices * batches * m * L.Kp * 2, 1024);
  L.b_bytes = align_up((int64_t)slices * batches * n * L.Kp * 2, 1024);
  L.off_b = L.a_bytes;
  L.off_e = L.a_bytes + L.b_bytes;
  L.off_f = L.off_e + align_up(batches * m * 4, 256);
  L.off_fmax = L.off_f + align_up(batches * n * 4, 256);
  L.off_part = L.off_fmax + align_up(batches * n * 8, 1024);
  L.min_bytes = L.off_part;
  return L;
}

// Digit slices and the tensor-core product for one scheme.
// Exponents and digit slices of `batches` stacked products (A: batches x m
// rows, B: batches matrices of k x n).
template <int SL>
int f64acc_prepare_t(int64_t m, int64_t n, int64_t k, const double* A, const double* B, uint8_t* w,
                     const F64AccLayout& L, int batches, cudaStream_t st, bool maxima_ready = false) {
  auto* SA = reinterpret_cast<__nv_bfloat16*>(w);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(w + L.off_b);
  int* E = reinterpret_cast<int*>(w + L.off_e);
  int* F = reinterpret_cast<int*>(w + L.off_f);
  const int64_t rows_a = (int64_t)batches * m;
  TraceScope tr(kTrSplitF64Slices, st);
  auto* Fmax = reinterpret_cast<unsigned long long*>(w + L.off_fmax);
  if (!maxima_ready) {
    // (otherwise the operand pass that wrote A and B left E and Fmax)
    row_exponent_kernel<<<(unsigned)((rows_a + 7) / 8), 256, 0, st>>>(A, rows_a, k, E);
    MMSR_TRY_STATUS(cudaMemsetAsync(Fmax, 0, (size_t)batches * n * 8, st));
    col_max_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)(k > 0 ? (k + 255) / 256 : 1), (unsigned)batches), 256,
                     0, st>>>(B, k, n, Fmax);
  }
  col_exponent_kernel<<<(unsigned)(((int64_t)batches * n + 255) / 256), 256, 0, st>>>(Fmax, (int64_t)batches * n, F);
  {
    const int64_t gx = std::max<int64_t>(1, (L.Kp + 1023) / 1024);
    const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(rows_a, std::max<int64_t>(1, 4096 / gx)));
    digits_rows_kernel<SL><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(A, rows_a, k, L.Kp, E, SA,
                                                                            aligned16(A) && k % 2 == 0);
  }
  // n-tiles per block: enough blocks to fill the GPU a few times over, each
  // walking several tiles
  const int64_t tiles_n = (n + 31) / 32;
  const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(tiles_n, std::max<int64_t>(1, 8192 / ((L.Kp + 63) / 64 * batches))));
  dim3 g((unsigned)((L.Kp + 63) / 64), (unsigned)std::min<int64_t>(gy, kMaxGridY), (unsigned)batches);
  digits_cols_kernel<SL><<<g, 256, 0, st>>>(B, k, n, L.Kp, F, SB, batches);
  MMSR_TRY_STATUS(cudaGetLastError());
  return MM_OK;
}

// The tensor-core products over prepared slices: `entries` products (k-split
// s), each writing C (ordinary) or adding into the blocks `quad` names.
template <int SL, bool QUAD>
int f64acc_gemm_t(int64_t m, int64_t n, uint8_t* w, const F64AccLayout& L, int batches, int entries, int s,
                  double* C, double* part, const QuadOut64& quad, cudaStream_t st) {
  auto* SA = reinterpret_cast<__nv_bfloat16*>(w);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(w + L.off_b);
  const int* E = reinterpret_cast<const int*>(w + L.off_e);
  const int* F = reinterpret_cast<const int*>(w + L.off_f);
  const int64_t rows_a = (int64_t)batches * m;
  CUtensorMap tA, tB;
  MMSR_TRY_STATUS(make_tmap_2d_16bit(&tA, SA, SL * rows_a, L.Kp, L.Kp, BM, true, BK));
  MMSR_TRY_STATUS(make_tmap_2d_16bit(&tB, SB, SL * (int64_t)batches * n, L.Kp, L.Kp, BN, true, BK));
  static std::atomic<uint64_t> configured{0};
  MMSR_TRY_STATUS(smem_limit_once(f64acc_gemm_kernel<SL, QUAD>, FaCfg<SL>::SMEM, configured));
  const int kb_total = (int)(L.Kp / BK);
  const int kbs = (kb_total + s - 1) / s;
  TraceScope tr(kTrTcF64Acc, st);
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)(s * entries));
  f64acc_gemm_kernel<SL, QUAD><<<grid, kThreads, FaCfg<SL>::SMEM, st>>>(tA, tB, E, F, C, part, m, n, rows_a,
                                                                       (int64_t)batches * n, kb_total, kbs, s,
                                                                       quad);
  MMSR_TRY_STATUS(cudaGetLastError());
  return MM_OK;
}

template <int SL>
int f64acc_core_t(int64_t m, int64_t n, int64_t k, const double* A, const double* B, double* C,
                  uint8_t* w, const F64AccLayout& L, int batches, int s, double* part, cudaStream_t st,
                  bool maxima_ready) {
  int rc = f64acc_prepare_t<SL>(m, n, k, A, B, w, L, batches, st, maxima_ready);
  if (rc != MM_OK) return rc;
  QuadOut64 none;
  memset(&none, 0, sizeof(none));
  rc = f64acc_gemm_t<SL, false>(m, n, w, L, batches, batches, s, C, part, none, st);
  if (rc != MM_OK) return rc;
  if (s > 1) MMSR_TRY_STATUS(launch_sum_reduce_f64(m * n, C, part, s - 1, st));
  return MM_OK;
}

int f64acc_core(int64_t m, int64_t n, int64_t k, const double* A, const double* B, double* C, uint8_t* w,
                const F64AccLayout& L, int batches, int s, double* part, cudaStream_t st,
                bool maxima_ready = false) {
  return L.slices == 6 ? f64acc_core_t<6>(m, n, k, A, B, C, w, L, batches, s, part, st, maxima_ready)
                       : f64acc_core_t<7>(m, n, k, A, B, C, w, L, batches, s, part, st, maxima_ready);
}

}  // namespace

int g_f64acc_slices = 0;  // mm_set_option(MM_OPT_F64ACC_SLICES, ...): 0 = by Strassen depth

int f64acc_slices_for_levels(int levels) {
  if (g_f64acc_slices == 6 || g_f64acc_slices == 7) return g_f64acc_slices;
  return levels <= 2 ? 6 : 7;
}

int plan_f64acc(int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  const F64AccLayout L = layout(m, n, k, f64acc_slices_for_levels(0));
  p->tile_m = BM;
  p->tile_n = BN;
  p->tile_k = BK;
  p->kernel = f64acc_slices_for_levels(0) == 6 ? 7 : 3;
  p->workspace_min = L.min_bytes;
  if (budget < (size_t)L.min_bytes) {
    p->split_k = 1;
    p->workspace_used = L.min_bytes;
    return MM_OK;
  }
  int s = 1, kbs = 0;
  int64_t used = 0;
  split_plan(m, n, L.Kp, BK, 8, budget - (size_t)L.min_bytes, &s, &kbs, &used);
  p->split_k = s;
  p->workspace_used = L.min_bytes + used;
  return MM_OK;
}

int run_f64acc(int64_t m, int64_t n, int64_t k, const double* A, const double* B, double* C,
               void* ws, size_t ws_bytes, cudaStream_t st) {
  mm_plan_t p;
  plan_f64acc(m, n, k, ws_bytes, &p);
  if ((size_t)p.workspace_min > ws_bytes) return MM_ERR_WORKSPACE;
  const F64AccLayout L = layout(m, n, k, f64acc_slices_for_levels(0));
  uint8_t* w = static_cast<uint8_t*>(ws);
  double* part = p.split_k > 1 ? reinterpret_cast<double*>(w + L.off_part) : nullptr;
  return f64acc_core(m, n, k, A, B, C, w, L, 1, p.split_k, part, st);
}

size_t f64acc_batched_bytes(int64_t m, int64_t n, int64_t k, int batches, int slices) {
  return (size_t)layout(m, n, k, slices, batches).min_bytes;
}

int run_f64acc_batched(const double* A, const double* B, double* C, int64_t m, int64_t n, int64_t k,
                       int batches, int slices, void* ws, cudaStream_t st, bool maxima_ready) {
  const F64AccLayout L = layout(m, n, k, slices, batches);
  return f64acc_core(m, n, k, A, B, C, static_cast<uint8_t*>(ws), L, batches, 1, nullptr, st, maxima_ready);
}

int f64acc_prepare_batched(const double* A, const double* B, int64_t m, int64_t n, int64_t k, int batches,
                           int slices, void* ws, cudaStream_t st, bool maxima_ready) {
  const F64AccLayout L = layout(m, n, k, slices, batches);
  return slices == 6 ? f64acc_prepare_t<6>(m, n, k, A, B, static_cast<uint8_t*>(ws), L, batches, st, maxima_ready)
                     : f64acc_prepare_t<7>(m, n, k, A, B, static_cast<uint8_t*>(ws), L, batches, st, maxima_ready);
}

void f64acc_maxima_buffers(int64_t m, int64_t n, int64_t k, int batches, int slices, void* ws, int** E,
                           unsigned long long** Fmax) {
  const F64AccLayout L = layout(m, n, k, slices, batches);
  *E = reinterpret_cast<int*>(static_cast<uint8_t*>(ws) + L.off_e);
  *Fmax = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(ws) + L.off_fmax);
}

int f64acc_gemm_quad(int64_t m, int64_t n, int64_t k, int batches, int slices, void* ws, const QuadOut64& quad,
                     cudaStream_t st) {
  const F64AccLayout L = layout(m, n, k, slices, batches);
  auto* w = static_cast<uint8_t*>(ws);
  return slices == 6 ? f64acc_gemm_t<6, true>(m, n, w, L, batches, quad.entries, 1, nullptr, nullptr, quad, st)
                     : f64acc_gemm_t<7, true>(m, n, w, L, batches, quad.entries, 1, nullptr, nullptr, quad, st);
}

int arm_f64acc_skip_signal(int on) {
  return cudaMemcpyToSymbol(g_f64acc_skip_signal, &on, sizeof(int)) == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

int read_f64acc_status(int* status) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_f64acc_status, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_f64acc_status, &zero, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  *status = v;
  return MM_OK;
}

}  // namespace mmsr
