// strassen.cu -- Strassen-like recursions (Section 5) on the GPU.
//
// Both variants are written in the bilinear form of the paper's
// generalisation: product r multiplies S_r = sum_q alpha[r][q] A_q by
// T_r = sum_q beta[r][q] B_q (quadrants q = 00, 01, 10, 11), and quadrant q
// of C is sum_r gamma[q][r] P_r.  MM_STRASSEN_PAPER uses the paper's printed
// S/T/C formulas; MM_STRASSEN_WINOGRAD is Strassen-Winograd (7 products,
// 15 additions when intermediates are shared) expanded into the same form.
//
// Schedule.  The top `levels` levels run breadth-first, in the spirit of the
// parallel Strassen of Lemma par-strassen / Theorem star-strassen-2: level l
// holds a stack of 7^l operand matrices of size (n/2^l)^2.  One pre-combine
// pass per level reads the four quadrants of every level-(l-1) operand once
// and writes its seven combinations; at the last level the pass writes the
// leaf operands directly in the layout the leaf kernel consumes (bf16 hi/lo
// split, B transposed, for the FP32 mode).  All 7^L leaf products then run in
// ONE batched leaf launch (the leaves are independent, so they fill the GPU
// together), and post-combine passes fold seven products into four
// quadrants level by level, bottom-up.  Temporaries are carved from the
// caller's workspace; the total is O(n^2) for a fixed number of levels
// ((7/4)^L n^2 per operand stack) and is reported by mm_plan_query.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "f64bits.cuh"
#include "internal.h"
#include "strassen_tables.cuh"

namespace mmsr {

namespace {

// ------------------------------------------------------- vector helpers
// V consecutive elements through one 16- or 8-byte access when V * sizeof(T)
// is 16 or 8 (the caller checks alignment), element by element otherwise.
template <typename T, int V>
__device__ __forceinline__ void vload(const T* __restrict__ p, T (&x)[V]) {
  if constexpr (V * sizeof(T) == 16) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    memcpy(x, &u, 16);
  } else if constexpr (V * sizeof(T) == 8) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    memcpy(x, &u, 8);
  } else {
#pragma unroll
    for (int t = 0; t < V; ++t) x[t] = p[t];
  }
}
template <typename T, int V>
__device__ __forceinline__ void vstore(T* __restrict__ p, const T (&x)[V]) {
  if constexpr (V * sizeof(T) == 16) {
    uint4 u;
    memcpy(&u, x, 16);
    *reinterpret_cast<uint4*>(p) = u;
  } else if constexpr (V * sizeof(T) == 8) {
    uint2 u;
    memcpy(&u, x, 8);
    *reinterpret_cast<uint2*>(p) = u;
  } else {
#pragma unroll
    for (int t = 0; t < V; ++t) p[t] = x[t];
  }
}

// Level transition for one operand side: source stack matrix r (2h x 2w,
// row pitch src_ld, matrices src_stride apart) -> seven (h x w) matrices
// 7r..7r+6 of the destination stack (contiguous).  Blocks walk rows, threads
// walk V-element column groups: each position's four quadrant values are
// read once and its seven sums written once.
template <typename T, int V, int VARIANT, int SIDE>
__global__ void __launch_bounds__(256) pre_combine_kernel(const T* __restrict__ src, int64_t src_ld,
                                                          int64_t src_stride, int h, int w,
                                                          T* __restrict__ dst) {
  const int r = blockIdx.y;
  const T* s = src + (int64_t)r * src_stride;
  const int64_t total = (int64_t)h * w;
  T* d = dst + (int64_t)r * 7 * total;
  const int wv = w / V;
  for (int i = blockIdx.x; i < h; i += gridDim.x) {
    const T* top = s + (int64_t)i * src_ld;
    const T* bot = s + (int64_t)(h + i) * src_ld;
    for (int jv = threadIdx.x; jv < wv; jv += blockDim.x) {
      const int j = jv * V;
      T x0[V], x1[V], x2[V], x3[V];
      vload<T, V>(top + j, x0);
      vload<T, V>(top + w + j, x1);
      vload<T, V>(bot + j, x2);
      vload<T, V>(bot + w + j, x3);
      T sv[V][7];
#pragma unroll
      for (int t = 0; t < V; ++t) sums7<VARIANT, SIDE>(x0[t], x1[t], x2[t], x3[t], sv[t]);
#pragma unroll
      for (int p = 0; p < 7; ++p) {
        T y[V];
#pragma unroll
        for (int t = 0; t < V; ++t) y[t] = sv[t][p];
        vstore<T, V>(d + (int64_t)p * total + (int64_t)i * w + j, y);
      }
    }
  }
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Last level, A side, FP32 mode: seven (h x w) sums written as bf16 hi/lo
// rows of pitch Kp (columns w..Kp-1 zero), product p into stack slot 7 r + p.
// Blocks walk rows, threads walk 8-column groups; `vec` = the source rows
// allow 16-byte loads.
template <int VARIANT>
__global__ void __launch_bounds__(256) pre_combine_split_rows_kernel(
    const float* __restrict__ src, int64_t src_ld, int64_t src_stride, int h, int w, int Kp,
    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int vec) {
  const int r = blockIdx.y;
  const float* s = src + (int64_t)r * src_stride;
  for (int i = blockIdx.x; i < h; i += gridDim.x) {
    for (int c8 = threadIdx.x * 8; c8 < Kp; c8 += blockDim.x * 8) {
      float x[4][8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* row = s + (int64_t)((q >> 1) * h + i) * src_ld + (q & 1) * w;
        if (vec && c8 + 8 <= w) {
          const float4 a = *reinterpret_cast<const float4*>(row + c8);
          const float4 b = *reinterpret_cast<const float4*>(row + c8 + 4);
          x[q][0] = a.x; x[q][1] = a.y; x[q][2] = a.z; x[q][3] = a.w;
          x[q][4] = b.x; x[q][5] = b.y; x[q][6] = b.z; x[q][7] = b.w;
        } else {
#pragma unroll
          for (int t = 0; t < 8; ++t) x[q][t] = (c8 + t < w) ? row[c8 + t] : 0.f;
        }
      }
#pragma unroll
      for (int p = 0; p < 7; ++p) {
        __align__(16) __nv_bfloat16 hh[8], ll[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
          split_bf16(combo4<VARIANT, 0>(p, x[0][t], x[1][t], x[2][t], x[3][t]), hh[t], ll[t]);
        const int64_t off = ((int64_t)(r * 7 + p) * h + i) * Kp + c8;
        *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(hh);
        *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(ll);
      }
    }
  }
}

// Last level, B side, FP32 mode: source stack matrix r is (2h x 2w) = (k x n);
// the seven sums T_p (h x w) are written transposed as bf16 hi/lo (w x Kp),
// product p into stack slot 7 r + p.  Tile: 64 k x 32 n of each quadrant
// through shared memory.
template <int VARIANT>
__global__ void __launch_bounds__(256) pre_combine_split_transpose_kernel(
    const float* __restrict__ src, int64_t src_ld, int64_t src_stride, int64_t h, int64_t w,
    int64_t Kp, __nv_bfloat16* __restrict__ hiT, __nv_bfloat16* __restrict__ loT) {
  __shared__ float tile[4][64][33];
  const int r = blockIdx.z;
  const float* s = src + (int64_t)r * src_stride;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t k0 = (int64_t)blockIdx.x * 64;
  // n-tiles with stride gridDim.y (the grid's y extent is capped at 65535)
  for (int64_t n0 = (int64_t)blockIdx.y * 32; n0 < w; n0 += (int64_t)gridDim.y * 32) {
  __syncthreads();  // the previous n-tile's readers are done with `tile`
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int kk = ty + 8 * it;
      const int64_t gk = k0 + kk, gn = n0 + tx;
      tile[q][kk][tx] = (gk < h && gn < w) ? s[((q >> 1) * h + gk) * src_ld + (q & 1) * w + gn] : 0.f;
    }
  }
  __syncthreads();
  const int row = threadIdx.x >> 3, chunk = threadIdx.x & 7;
  const int64_t gn = n0 + row;
  if (gn >= w) continue;
#pragma unroll
  for (int p = 0; p < 7; ++p) {
    __align__(16) __nv_bfloat16 hh[8], ll[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int kk = chunk * 8 + t;
      split_bf16(combo4<VARIANT, 1>(p, tile[0][kk][row], tile[1][kk][row], tile[2][kk][row], tile[3][kk][row]),
                 hh[t], ll[t]);
    }
    const int64_t off = ((int64_t)(r * 7 + p) * w + gn) * Kp + k0 + chunk * 8;
    *reinterpret_cast<uint4*>(hiT + off) = *reinterpret_cast<const uint4*>(hh);
    *reinterpret_cast<uint4*>(loT + off) = *reinterpret_cast<const uint4*>(ll);
  }
  }
}

// How a post-addition pass sums: in the products' own type, in FP64
// arithmetic, or (FP32 products) as an error-free double-float sum.
enum PostSum { kSumPlain = 0, kSumF64 = 1, kSumDoubleFloat = 2 };

// s + e = a + b exactly (Knuth's TwoSum; round-to-nearest adds, no
// contraction or reassociation).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Running sum of one post-addition output in the pass's summation mode.
// kSumDoubleFloat is Sum2 of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005): the running sum carries its exact
// rounding errors separately, so the result is as accurate as a sum in twice
// the precision, rounded once.  Zero coefficients add nothing.
template <typename TP, int MODE>
struct PostAcc {
  TP v;
  __device__ __forceinline__ void init(TP x0) { v = x0; }
  __device__ __forceinline__ void add(int g, TP x) { v = apply(g, v, x); }
  __device__ __forceinline__ void set(int g, TP x) { v = g > 0 ? x : -x; }  // first term, no old value
  __device__ __forceinline__ TP get() const { return v; }
};
template <typename TP>
struct PostAcc<TP, kSumF64> {
  double v;
  __device__ __forceinline__ void init(TP x0) { v = (double)x0; }
  __device__ __forceinline__ void add(int g, TP x) { v = apply(g, v, (double)x); }
  __device__ __forceinline__ void set(int g, TP x) { v = g > 0 ? (double)x : -(double)x; }
  __device__ __forceinline__ TP get() const { return (TP)v; }
};
template <typename TP>
struct PostAcc<TP, kSumDoubleFloat> {
  float s, e;
  __device__ __forceinline__ void init(TP x0) {
    s = (float)x0;
    e = 0.f;
  }
  __device__ __forceinline__ void set(int g, TP x) {
    s = g > 0 ? (float)x : -(float)x;
    e = 0.f;
  }
  __device__ __forceinline__ void add(int g, TP x) {
    if (g == 0) return;
    float s2, e2;
    two_sum(s, g > 0 ? (float)x : -(float)x, s2, e2);
    s = s2;
    e = __fadd_rn(e, e2);
  }
  __device__ __forceinline__ TP get() const { return (TP)__fadd_rn(s, e); }
};

// Post-additions: products 7r..7r+6 (h x w each, contiguous) -> the four
// quadrants of destination matrix r (2h x 2w, pitch dst_ld, dst_stride
// apart).  Terms are added in product order, after the destination's old
// value when `accumulate` is set.
template <typename TP, int V, int MODE, int VARIANT>
__global__ void __launch_bounds__(256) post_combine_kernel(const TP* __restrict__ P, int h, int w,
                                                           TP* __restrict__ dst, int64_t dst_ld,
                                                           int64_t dst_stride, int accumulate) {
  const int r = blockIdx.y;
  const int64_t total = (int64_t)h * w;
  const TP* pp = P + (int64_t)r * 7 * total;
  TP* d = dst + (int64_t)r * dst_stride;
  const int wv = w / V;
  for (int i = blockIdx.x; i < h; i += gridDim.x) {
    for (int jv = threadIdx.x; jv < wv; jv += blockDim.x) {
      const int64_t e = (int64_t)i * w + jv * V;
      TP x[7][V];
#pragma unroll
      for (int p = 0; p < 7; ++p) vload<TP, V>(pp + (int64_t)p * total + e, x[p]);
      if constexpr (MODE == kSumPlain) {
        // plain sums: the variant's shared form of the four quadrant sums,
        // then the old value where it is accumulated into
        TP c[V][4];
#pragma unroll
        for (int t = 0; t < V; ++t) {
          TP xt[7];
#pragma unroll
          for (int p = 0; p < 7; ++p) xt[p] = x[p][t];
          post4<VARIANT>(xt, c[t]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          TP* out = d + (int64_t)((q >> 1) * h + i) * dst_ld + (q & 1) * w + jv * V;
          TP y[V];
          if (accumulate) vload<TP, V>(out, y);
#pragma unroll
          for (int t = 0; t < V; ++t) y[t] = accumulate ? y[t] + c[t][q] : c[t][q];
          vstore<TP, V>(out, y);
        }
        continue;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        TP* out = d + (int64_t)((q >> 1) * h + i) * dst_ld + (q & 1) * w + jv * V;
        TP y[V];
        if (accumulate) vload<TP, V>(out, y);
#pragma unroll
        for (int t = 0; t < V; ++t) {
          PostAcc<TP, MODE> acc;
          acc.init(accumulate ? y[t] : TP(0));
#pragma unroll
          for (int p = 0; p < 7; ++p) {
            const int g = coef_gamma(VARIANT, q, p);
            if (!accumulate && p == first_gamma_term(VARIANT, q))
              acc.set(g, x[p][t]);
            else
              acc.add(g, x[p][t]);
          }
          y[t] = acc.get();
        }
        vstore<TP, V>(out, y);
      }
    }
  }
}

// ------------------------------------------------- two levels in one pass
// The 49 two-level operand sums at one element position: x[a][b] is the
// (a, b) sub-block (a, b in 0..3) of a 4h x 4w source matrix, i.e. sub-
// quadrant (a & 1, b & 1) of level-1 quadrant (a >> 1, b >> 1).  The level-1
// sums S1 are formed in registers and never stored; every addition is the one
// two single-level passes make, in the same order, so the results are
// identical.  emit(7 r1 + r2, value) receives each level-2 sum.
template <int VARIANT, int SIDE, typename T, typename Emit>
__device__ __forceinline__ void combine2(const T (&x)[4][4], Emit&& emit) {
  // level-1 sums of the four sub-positions, then level-2 sums of each
  T s1[4][7];
#pragma unroll
  for (int q2 = 0; q2 < 4; ++q2) {
    const int u = q2 >> 1, v = q2 & 1;
    sums7<VARIANT, SIDE>(x[u][v], x[u][2 + v], x[2 + u][v], x[2 + u][2 + v], s1[q2]);
  }
#pragma unroll
  for (int r1 = 0; r1 < 7; ++r1) {
    T s2[7];
    sums7<VARIANT, SIDE>(s1[0][r1], s1[1][r1], s1[2][r1], s1[3][r1], s2);
#pragma unroll
    for (int r2 = 0; r2 < 7; ++r2) emit(7 * r1 + r2, s2[r2]);
  }
}

// Two operand levels: source matrix r (4h x 4w, pitch src_ld, src_stride
// apart) -> matrices 49r..49r+48 (h x w, contiguous) of the stack two levels
// down.  Blocks walk rows, threads walk columns.
template <typename T, int VARIANT, int SIDE>
__global__ void __launch_bounds__(256) pre_combine2_kernel(const T* __restrict__ src, int64_t src_ld,
                                                           int64_t src_stride, int h, int w,
                                                           T* __restrict__ dst) {
  const int r = blockIdx.y;
  const T* s = src + (int64_t)r * src_stride;
  const int64_t total = (int64_t)h * w;
  T* d = dst + (int64_t)r * 49 * total;
  for (int i = blockIdx.x; i < h; i += gridDim.x) {
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
      T x[4][4];
      const T* row = s + (int64_t)i * src_ld + j;
#pragma unroll
      for (int a = 0; a < 4; ++a, row += (int64_t)h * src_ld)
#pragma unroll
        for (int b = 0; b < 4; ++b) x[a][b] = row[b * w];
      // the 49 sums arrive in output order: one running pointer
      T* o = d + (int64_t)i * w + j;
      combine2<VARIANT, SIDE>(x, [&](int, T v) {
        *o = v;
        o += total;
      });
    }
  }
}

// The last two operand levels of the FP64-accuracy mode, also producing
// what the digit split needs first: frexp's exponent of each leaf row's
// max |a| (A side) or each leaf column's max |b| (B side), bit-identical to
// the split's own passes over the leaf operands, which are then skipped.
// Each thread keeps, per leaf, the maximum of the high words of |x|
// (abs_hi_word); a line whose maximum high word is zero is re-scanned in
// full from the values just written.

// A side: each block owns whole rows of the 49 leaf operands, so it reduces
// each row's maximum itself and stores the row exponent E[leaf][row].
template <int VARIANT>
__global__ void __launch_bounds__(256) pre_combine2_rowexp_kernel(const double* __restrict__ src, int64_t src_ld,
                                                                  int64_t src_stride, int h, int w,
                                                                  double* __restrict__ dst, int* __restrict__ E) {
  __shared__ uint32_t red[8][49];
  __shared__ uint32_t hi_max[49];
  __shared__ unsigned long long rescan_max[49];
  const int r = blockIdx.y;
  const double* s = src + (int64_t)r * src_stride;
  const int64_t total = (int64_t)h * w;
  double* d = dst + (int64_t)r * 49 * total;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int i = blockIdx.x; i < h; i += gridDim.x) {
    uint32_t mx[49];
#pragma unroll
    for (int q = 0; q < 49; ++q) mx[q] = 0;
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
      double x[4][4];
      const double* row = s + (int64_t)i * src_ld + j;
#pragma unroll
      for (int a = 0; a < 4; ++a, row += (int64_t)h * src_ld)
#pragma unroll
        for (int b = 0; b < 4; ++b) x[a][b] = row[b * w];
      double* o = d + (int64_t)i * w + j;
      combine2<VARIANT, 0>(x, [&](int q, double v) {
        *o = v;
        o += total;
        mx[q] = max(mx[q], abs_hi_word(v));
      });
    }
#pragma unroll
    for (int q = 0; q < 49; ++q) {
      uint32_t v = mx[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
      if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();  // also orders this block's stores of row i before the re-scan below
    for (int q = threadIdx.x; q < 49; q += blockDim.x) {
      uint32_t v = 0;
      for (int u = 0; u < nwarps; ++u) v = max(v, red[u][q]);
      hi_max[q] = v;
      rescan_max[q] = 0;
    }
    __syncthreads();
    // rows whose high words are all zero: the exact maximum of the patterns
    // (hi_max is not written below, so every warp takes the same branches)
    for (int q = 0; q < 49; ++q) {
      if (hi_max[q] != 0) continue;
      const double* line = d + (int64_t)q * total + (int64_t)i * w;
      unsigned long long b = 0;
      for (int j = threadIdx.x; j < w; j += blockDim.x) b = max(b, abs_bits(line[j]));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, off));
      if (lane == 0 && b != 0) atomicMax(&rescan_max[q], b);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 49; q += blockDim.x)
      E[(int64_t)(49 * r + q) * h + i] =
          line_exponent(hi_max[q] != 0 ? (unsigned long long)hi_max[q] << 32 : rescan_max[q]);
    __syncthreads();
  }
}

// B side: a thread owns one column of a band of rows and folds each leaf
// column's maximum pattern into Fmax[leaf][column] (zeroed beforehand) with
// an atomic max.
template <int VARIANT>
__global__ void __launch_bounds__(256) pre_combine2_colmax_kernel(const double* __restrict__ src, int64_t src_ld,
                                                                  int64_t src_stride, int h, int w, int band,
                                                                  double* __restrict__ dst,
                                                                  unsigned long long* __restrict__ Fmax) {
  const int r = blockIdx.z;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= w) return;
  const double* s = src + (int64_t)r * src_stride;
  const int64_t total = (int64_t)h * w;
  double* d = dst + (int64_t)r * 49 * total;
  const int i0 = blockIdx.y * band, i1 = min(h, i0 + band);
  uint32_t mx[49];
#pragma unroll
  for (int q = 0; q < 49; ++q) mx[q] = 0;
  for (int i = i0; i < i1; ++i) {
    double x[4][4];
    const double* row = s + (int64_t)i * src_ld + j;
#pragma unroll
    for (int a = 0; a < 4; ++a, row += (int64_t)h * src_ld)
#pragma unroll
      for (int b = 0; b < 4; ++b) x[a][b] = row[b * w];
    double* o = d + (int64_t)i * w + j;
    combine2<VARIANT, 1>(x, [&](int q, double v) {
      *o = v;
      o += total;
      mx[q] = max(mx[q], abs_hi_word(v));
    });
  }
  unsigned long long* fm = Fmax + (int64_t)49 * r * w + j;
#pragma unroll
  for (int q = 0; q < 49; ++q) {
    unsigned long long b = (unsigned long long)mx[q] << 32;
    if (b == 0)  // the thread's own stores, re-read in full
      for (int i = i0; i < i1; ++i) b = max(b, abs_bits(d[(int64_t)q * total + (int64_t)i * w + j]));
    if (b != 0) atomicMax(fm + (int64_t)q * w, b);
  }
}

// bf16 hi/lo of four consecutive values, as two 8-byte words.
__device__ __forceinline__ void split4(const float (&v)[4], uint2& hi, uint2& lo) {
  __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) split_bf16(v[t], h[t], l[t]);
  memcpy(&hi, h, 8);
  memcpy(&lo, l, 8);
}

// Two operand levels ending at the leaves, A side, FP32 mode: the 49 sums
// are written as bf16 hi/lo rows of pitch Kp (columns w..Kp-1 zero).  Each
// thread takes four consecutive columns (16-byte loads where `vec` allows,
// 8-byte stores).
template <int VARIANT>
__global__ void __launch_bounds__(256) pre_combine2_split_rows_kernel(
    const float* __restrict__ src, int64_t src_ld, int64_t src_stride, int h, int w, int Kp,
    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int vec) {
  const int r = blockIdx.y;
  const float* s = src + (int64_t)r * src_stride;
  const int64_t step = (int64_t)h * Kp;  // one leaf operand
  for (int i = blockIdx.x; i < h; i += gridDim.x) {
    for (int j = threadIdx.x * 4; j < Kp; j += blockDim.x * 4) {
      float x[4][4][4];  // [a][b][column]
      const float* row = s + (int64_t)i * src_ld + j;
#pragma unroll
      for (int a = 0; a < 4; ++a, row += (int64_t)h * src_ld)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (vec && j + 4 <= w) {
            const float4 q = *reinterpret_cast<const float4*>(row + b * w);
            x[a][b][0] = q.x; x[a][b][1] = q.y; x[a][b][2] = q.z; x[a][b][3] = q.w;
          } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) x[a][b][t] = j + t < w ? row[b * w + t] : 0.f;
          }
        }
      int64_t off = ((int64_t)49 * r * h + i) * Kp + j;
#pragma unroll
      for (int r1 = 0; r1 < 7; ++r1) {
        float s1[4][4];  // [q2][column]
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
          const int u = q2 >> 1, v = q2 & 1;
#pragma unroll
          for (int t = 0; t < 4; ++t)
            s1[q2][t] = combo4<VARIANT, 0>(r1, x[u][v][t], x[u][2 + v][t], x[2 + u][v][t], x[2 + u][2 + v][t]);
        }
#pragma unroll
        for (int r2 = 0; r2 < 7; ++r2, off += step) {
          float y[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) y[t] = combo4<VARIANT, 0>(r2, s1[0][t], s1[1][t], s1[2][t], s1[3][t]);
          uint2 vh, vl;
          split4(y, vh, vl);
          *reinterpret_cast<uint2*>(hi + off) = vh;
          *reinterpret_cast<uint2*>(lo + off) = vl;
        }
      }
    }
  }
}

// Two operand levels ending at the leaves, B side, FP32 mode: source matrix r
// is (4h x 4w) = (k x n); the 49 sums (h x w) are written transposed as bf16
// hi/lo (w x Kp).  A 32 k x 16 n tile of each of the 16 sub-blocks goes
// through shared memory (reads run along n); each of the 128 threads then
// takes four consecutive k of one column (8-byte stores along k).
template <int VARIANT>
__global__ void __launch_bounds__(128) pre_combine2_split_transpose_kernel(
    const float* __restrict__ src, int64_t src_ld, int64_t src_stride, int h, int w, int Kp,
    __nv_bfloat16* __restrict__ hiT, __nv_bfloat16* __restrict__ loT) {
  __shared__ float tile[16][32][17];
  const int r = blockIdx.z;
  const float* s = src + (int64_t)r * src_stride;
  const int k0 = blockIdx.x * 32;
  // n-tiles with stride gridDim.y (the grid's y extent is capped at 65535)
  for (int n0 = blockIdx.y * 16; n0 < w; n0 += gridDim.y * 16) {
  __syncthreads();  // the previous n-tile's readers are done with `tile`
  {
    const int jj = threadIdx.x & 15;
    const int gn = n0 + jj;
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int kk = (threadIdx.x >> 4) + 8 * it;
      const int gk = k0 + kk;
      const bool in = gk < h && gn < w;
      const float* p = s + (int64_t)gk * src_ld + gn;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) tile[a * 4 + b][kk][jj] = in ? p[(int64_t)a * h * src_ld + b * w] : 0.f;
    }
  }
  __syncthreads();
  const int kq = threadIdx.x & 7, jj = threadIdx.x >> 3;
  const int gn = n0 + jj;
  if (gn >= w) continue;
  float x[4][4][4];  // [a][b][k]
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int t = 0; t < 4; ++t) x[a][b][t] = tile[a * 4 + b][kq * 4 + t][jj];
  const int64_t step = (int64_t)w * Kp;  // one leaf operand
  int64_t off = ((int64_t)49 * r * w + gn) * Kp + k0 + kq * 4;
#pragma unroll
  for (int r1 = 0; r1 < 7; ++r1) {
    float s1[4][4];
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) {
      const int u = q2 >> 1, v = q2 & 1;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        s1[q2][t] = combo4<VARIANT, 1>(r1, x[u][v][t], x[u][2 + v][t], x[2 + u][v][t], x[2 + u][2 + v][t]);
    }
#pragma unroll
    for (int r2 = 0; r2 < 7; ++r2, off += step) {
      float y[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) y[t] = combo4<VARIANT, 1>(r2, s1[0][t], s1[1][t], s1[2][t], s1[3][t]);
      uint2 vh, vl;
      split4(y, vh, vl);
      *reinterpret_cast<uint2*>(hiT + off) = vh;
      *reinterpret_cast<uint2*>(loT + off) = vl;
    }
  }
  }
}

// Two post-addition levels: products 49r..49r+48 (h x w each, contiguous) ->
// the 16 sub-blocks of destination matrix r (4h x 4w, pitch dst_ld,
// dst_stride apart).  For each level-1 product r1 the level-2 sums T (four
// values) are formed in registers in the order of a single-level pass, then
// folded into the 16 outputs in r1 order, so the results equal two separate
// passes (the second in the `MODE` summation, after the old value when
// `accumulate` is set).  Each thread takes V consecutive columns.
template <typename TP, int V, int MODE, int VARIANT>
__global__ void __launch_bounds__(256) post_combine2_kernel(const TP* __restrict__ P, int h, int w,
                                                            TP* __restrict__ dst, int64_t dst_ld,
                                                            int64_t dst_stride, int accumulate) {
  const int r = blockIdx.y;
  const int64_t total = (int64_t)h * w;
  const TP* pp = P + (int64_t)r * 49 * total;
  TP* d = dst + (int64_t)r * dst_stride;
  const int wv = w / V;
  for (int i = blockIdx.x; i < h; i += gridDim.x) {
    for (int jv = threadIdx.x; jv < wv; jv += blockDim.x) {
      const int j = jv * V;
      if constexpr (MODE == kSumPlain) {
        // plain sums: the variant's shared form at both levels -- the level-2
        // quadrant sums of each r1's seven products, then the level-1 sums of
        // those over r1 -- and the old value where it is accumulated into
        TP* drow = d + (int64_t)i * dst_ld + j;
        const TP* src = pp + (int64_t)i * w + j;
        TP t2[V][4][7];  // [column][level-2 quadrant][r1]
#pragma unroll
        for (int r1 = 0; r1 < 7; ++r1) {
          TP p7[7][V];
#pragma unroll
          for (int r2 = 0; r2 < 7; ++r2, src += total) vload<TP, V>(src, p7[r2]);
#pragma unroll
          for (int t = 0; t < V; ++t) {
            TP pr[7], c[4];
#pragma unroll
            for (int r2 = 0; r2 < 7; ++r2) pr[r2] = p7[r2][t];
            post4<VARIANT>(pr, c);
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) t2[t][q2][r1] = c[q2];
          }
        }
        TP c1[V][4][4];  // [column][level-2 quadrant][level-1 quadrant]
#pragma unroll
        for (int t = 0; t < V; ++t)
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) post4<VARIANT>(t2[t][q2], c1[t][q2]);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            TP* out = drow + (int64_t)a * h * dst_ld + b * w;
            const int q1 = (a >> 1) * 2 + (b >> 1), q2 = (a & 1) * 2 + (b & 1);
            TP y[V];
            if (accumulate) vload<TP, V>(out, y);
#pragma unroll
            for (int t = 0; t < V; ++t) y[t] = accumulate ? y[t] + c1[t][q2][q1] : c1[t][q2][q1];
            vstore<TP, V>(out, y);
          }
        continue;
      }
      PostAcc<TP, MODE> acc[4][4][V];  // [level-1 quadrant][level-2 quadrant][column]
      // sub-block (a, b) of the destination = level-1 quadrant
      // (a >> 1, b >> 1), level-2 quadrant (a & 1, b & 1)
      TP* drow = d + (int64_t)i * dst_ld + j;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          TP y[V];
          if (accumulate) vload<TP, V>(drow + (int64_t)a * h * dst_ld + b * w, y);
#pragma unroll
          for (int t = 0; t < V; ++t)
            acc[(a >> 1) * 2 + (b >> 1)][(a & 1) * 2 + (b & 1)][t].init(accumulate ? y[t] : TP(0));
        }
      const TP* src = pp + (int64_t)i * w + j;
#pragma unroll
      for (int r1 = 0; r1 < 7; ++r1) {
        TP p7[7][V];
#pragma unroll
        for (int r2 = 0; r2 < 7; ++r2, src += total) vload<TP, V>(src, p7[r2]);
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2)
#pragma unroll
          for (int t = 0; t < V; ++t) {
            TP pr[7];
#pragma unroll
            for (int r2 = 0; r2 < 7; ++r2) pr[r2] = p7[r2][t];
            const TP tq = combo7<VARIANT>(q2, pr);
#pragma unroll
            for (int q1 = 0; q1 < 4; ++q1) {
              // the first product of quadrant q1 sets the sum where there is
              // no old value to add to (one FP64 addition fewer per output)
              const int g = coef_gamma(VARIANT, q1, r1);
              if (!accumulate && r1 == first_gamma_term(VARIANT, q1))
                acc[q1][q2][t].set(g, tq);
              else
                acc[q1][q2][t].add(g, tq);
            }
          }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          TP y[V];
#pragma unroll
          for (int t = 0; t < V; ++t) y[t] = acc[(a >> 1) * 2 + (b >> 1)][(a & 1) * 2 + (b & 1)][t].get();
          vstore<TP, V>(drow + (int64_t)a * h * dst_ld + b * w, y);
        }
    }
  }
}

// Blocks per matrix for a row-walking pass over R matrices of h rows with
// `threads`-thread blocks: about one full wave of the GPU in total.
unsigned rows_grid(int64_t h, int64_t R, int threads) {
  const int64_t per_sm = 2048 / threads < 32 ? 2048 / threads : 32;
  int64_t b = ((int64_t)num_sms() * per_sm + R - 1) / R;
  if (b > h) b = h;
  return (unsigned)(b < 1 ? 1 : b);
}

// Threads per block for rows of `groups` column groups (a multiple of 32,
// at most 256).
int row_threads(int64_t groups) {
  if (groups >= 256) return 256;
  const int64_t t = (groups + 31) / 32 * 32;
  return (int)(t < 32 ? 32 : t);
}

bool aligned_to(const void* p, int64_t bytes) {
  return (reinterpret_cast<uintptr_t>(p) % (uintptr_t)bytes) == 0;
}

template <typename T, int VARIANT, int SIDE>
void pre_combine_v(bool vec, dim3 g, int threads, cudaStream_t st, const T* src, int64_t src_ld,
                   int64_t src_stride, int h, int w, T* dst) {
  if (vec)
    pre_combine_kernel<T, 16 / sizeof(T), VARIANT, SIDE><<<g, threads, 0, st>>>(src, src_ld, src_stride, h, w, dst);
  else
    pre_combine_kernel<T, 1, VARIANT, SIDE><<<g, threads, 0, st>>>(src, src_ld, src_stride, h, w, dst);
}

template <typename T>
cudaError_t launch_pre_combine(const T* src, int64_t src_ld, int64_t src_stride, int64_t h, int64_t w,
                               int64_t R, T* dst, int variant, int side, cudaStream_t st) {
  constexpr int V = 16 / sizeof(T);
  const bool vec = w % V == 0 && src_ld % V == 0 && src_stride % V == 0 && aligned_to(src, 16) &&
                   aligned_to(dst, 16);
  const int threads = row_threads(vec ? w / V : w);
  const dim3 g(rows_grid(h, R, threads), (unsigned)R);
  const int hh = (int)h, ww = (int)w;
  if (variant == 0 && side == 0) pre_combine_v<T, 0, 0>(vec, g, threads, st, src, src_ld, src_stride, hh, ww, dst);
  if (variant == 0 && side == 1) pre_combine_v<T, 0, 1>(vec, g, threads, st, src, src_ld, src_stride, hh, ww, dst);
  if (variant == 1 && side == 0) pre_combine_v<T, 1, 0>(vec, g, threads, st, src, src_ld, src_stride, hh, ww, dst);
  if (variant == 1 && side == 1) pre_combine_v<T, 1, 1>(vec, g, threads, st, src, src_ld, src_stride, hh, ww, dst);
  return cudaGetLastError();
}

template <typename TP, int MODE, int VARIANT>
void post_combine_v(bool vec, dim3 g, int threads, cudaStream_t st, const TP* P, int h, int w, TP* dst,
                    int64_t dst_ld, int64_t dst_stride, int accumulate) {
  if (vec)
    post_combine_kernel<TP, 16 / sizeof(TP), MODE, VARIANT><<<g, threads, 0, st>>>(P, h, w, dst, dst_ld,
                                                                                   dst_stride, accumulate);
  else
    post_combine_kernel<TP, 1, MODE, VARIANT><<<g, threads, 0, st>>>(P, h, w, dst, dst_ld, dst_stride,
                                                                     accumulate);
}

template <typename TP, int MODE>
cudaError_t launch_post_combine(const TP* P, int64_t h, int64_t w, int64_t R, TP* dst, int64_t dst_ld,
                                int64_t dst_stride, int variant, int accumulate, cudaStream_t st) {
  constexpr int V = 16 / sizeof(TP);
  const bool vec = w % V == 0 && dst_ld % V == 0 && dst_stride % V == 0 && aligned_to(P, 16) &&
                   aligned_to(dst, 16);
  const int threads = row_threads(vec ? w / V : w);
  const dim3 g(rows_grid(h, R, threads), (unsigned)R);
  if (variant == 0)
    post_combine_v<TP, MODE, 0>(vec, g, threads, st, P, (int)h, (int)w, dst, dst_ld, dst_stride, accumulate);
  else
    post_combine_v<TP, MODE, 1>(vec, g, threads, st, P, (int)h, (int)w, dst, dst_ld, dst_stride, accumulate);
  return cudaGetLastError();
}

int64_t pw7(int l) {
  int64_t p = 1;
  for (int i = 0; i < l; ++i) p *= 7;
  return p;
}

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct StrassenLayout {
  int64_t pp_bytes;   // each of the two ping-pong stack buffers
  int64_t off_pp1, off_ahi, off_alo, off_bhi, off_blo, off_p, off_leafws, total;
  int64_t mL, nL, kL, KpL, leaves;
};

// Workspace carve-up.  The level passes go two levels at a time (see
// below), so with at most four levels only the first operand pass and the
// first post pass can write an intermediate stack: one level down on the
// operand side (level 1 when L = 3, level 2 when L = 4; none when L <= 2)
// and one level up on the post side (the same levels).  The operand side is
// finished before the post side starts, so one buffer holds either.  FP32
// mode then holds the last level's split operands (bf16 hi/lo, B transposed)
// and the leaf products; FP64 modes the FP64 leaf operands and products.  In
// FP64-accuracy mode the leaf products overlay the FP64 leaf operands of A,
// which are dead once their digit slices are written.
int intermediate_level(int L) { return L >= 3 ? L - 2 : 0; }

bool fused_level(int L, int sr, int64_t m, int64_t n, int64_t k) {
  return L == 1 && sr == MM_SR_PLUS_TIMES_F32 && g_strassen_fused && strassen_fused_shape_ok(m, n, k);
}

StrassenLayout strassen_layout(int L, int sr, int64_t m, int64_t n, int64_t k) {
  StrassenLayout s;
  if (fused_level(L, sr, m, n, k)) {
    // operand sums formed in the leaf's staging: the product stack only
    memset(&s, 0, sizeof(s));
    s.mL = m / 2;
    s.nL = n / 2;
    s.kL = k / 2;
    s.leaves = 7;
    s.total = align_up(7 * s.mL * s.nL * 4, 1024);
    return s;
  }
  const int esz = (sr == MM_SR_PLUS_TIMES_F32) ? 4 : 8;
  s.mL = m >> L;
  s.nL = n >> L;
  s.kL = k >> L;
  s.leaves = pw7(L);
  int64_t pp = 0;
  if (const int l = intermediate_level(L)) {
    const int64_t ml = m >> l, nl = n >> l, kl = k >> l;
    int64_t e = ml * kl;
    if (kl * nl > e) e = kl * nl;
    if (ml * nl > e) e = ml * nl;
    pp = pw7(l) * e * esz;
  }
  s.pp_bytes = align_up(pp, 1024);
  s.off_pp1 = 0;  // the second ping-pong buffer is never needed (see above)
  int64_t off = s.pp_bytes;
  if (sr == MM_SR_PLUS_TIMES_F32) {
    s.KpL = align_up(s.kL > 0 ? s.kL : 1, 64);
    const int64_t a = align_up(s.leaves * s.mL * s.KpL * 2, 1024);
    const int64_t b = align_up(s.leaves * s.nL * s.KpL * 2, 1024);
    s.off_ahi = off;
    s.off_alo = off + a;
    s.off_bhi = off + 2 * a;
    s.off_blo = off + 2 * a + b;
    off += 2 * a + 2 * b;
  } else {
    s.KpL = s.kL;
    const int64_t a = align_up(s.leaves * s.mL * s.kL * 8, 1024);
    const int64_t b = align_up(s.leaves * s.kL * s.nL * 8, 1024);
    s.off_ahi = off;       // A leaf stack (FP64)
    s.off_alo = off;
    s.off_bhi = off + a;   // B leaf stack (FP64)
    s.off_blo = off + a;
    off += a + b;
  }
  const int64_t pbytes = align_up(s.leaves * s.mL * s.nL * esz, 1024);
  if (sr == MM_SR_PLUS_TIMES_F64ACC && pbytes <= s.off_bhi - s.off_ahi) {
    s.off_p = s.off_ahi;
  } else {
    s.off_p = off;
    off += pbytes;
  }
  s.off_leafws = off;  // FP64-accuracy leaves: digit slices and exponents
  if (sr == MM_SR_PLUS_TIMES_F64ACC)
    off += align_up((int64_t)f64acc_batched_bytes(s.mL, s.nL, s.kL, (int)s.leaves, f64acc_slices_for_levels(L)), 1024);
  s.total = off;
  return s;
}

// Level passes.  Two levels run as one pass wherever possible (half the
// stack traffic of two single-level passes), paired where the stacks are
// largest: operand expansion pairs the LAST levels ((L-1, L), (L-3, L-2),
// ...; a single first level when L is odd), post-addition pairs the
// deepest levels ((L, L-1), ...; a single top level when L is odd).
template <typename T>
cudaError_t launch_pre_combine2(const T* src, int64_t src_ld, int64_t src_stride, int64_t h, int64_t w,
                                int64_t R, T* dst, int variant, int side, cudaStream_t st) {
  const int threads = row_threads(w);
  const dim3 g(rows_grid(h, R, threads), (unsigned)R);
  const int hh = (int)h, ww = (int)w;
  if (variant == 0 && side == 0) pre_combine2_kernel<T, 0, 0><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, dst);
  if (variant == 0 && side == 1) pre_combine2_kernel<T, 0, 1><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, dst);
  if (variant == 1 && side == 0) pre_combine2_kernel<T, 1, 0><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, dst);
  if (variant == 1 && side == 1) pre_combine2_kernel<T, 1, 1><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, dst);
  return cudaGetLastError();
}

// The last two FP64 operand levels with the split's line maxima (above):
// side 0 stores row exponents E, side 1 folds column maxima into Fmax.
cudaError_t launch_pre_combine2_maxima(const double* src, int64_t src_ld, int64_t src_stride, int64_t h,
                                       int64_t w, int64_t R, double* dst, int variant, int side, int* E,
                                       unsigned long long* Fmax, cudaStream_t st) {
  const int hh = (int)h, ww = (int)w;
  if (side == 0) {
    const int threads = row_threads(w);
    const dim3 g(rows_grid(h, R, threads), (unsigned)R);
    if (variant == 0)
      pre_combine2_rowexp_kernel<0><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, dst, E);
    else
      pre_combine2_rowexp_kernel<1><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, dst, E);
  } else {
    // column blocks x bands of rows: about four blocks per SM in all
    const int threads = row_threads(w);
    const int64_t gx = (w + threads - 1) / threads;
    int64_t gy = ((int64_t)num_sms() * 4 + gx * R - 1) / (gx * R);
    gy = gy < 1 ? 1 : (gy > h ? h : gy);
    const int band = (int)((h + gy - 1) / gy);
    gy = (h + band - 1) / band;
    const dim3 g((unsigned)gx, (unsigned)gy, (unsigned)R);
    if (variant == 0)
      pre_combine2_colmax_kernel<0><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, band, dst, Fmax);
    else
      pre_combine2_colmax_kernel<1><<<g, threads, 0, st>>>(src, src_ld, src_stride, hh, ww, band, dst, Fmax);
  }
  return cudaGetLastError();
}

template <typename TP, int MODE>
cudaError_t launch_post_combine2(const TP* P, int64_t h, int64_t w, int64_t R, TP* dst, int64_t dst_ld,
                                 int64_t dst_stride, int variant, int accumulate, cudaStream_t st) {
  // One column per thread: with 49 product streams per thread, wider
  // accesses measured slower (fewer threads in flight).
  const int threads = row_threads(w);
  const dim3 g(rows_grid(h, R, threads), (unsigned)R);
  if (variant == 0)
    post_combine2_kernel<TP, 1, MODE, 0><<<g, threads, 0, st>>>(P, (int)h, (int)w, dst, dst_ld, dst_stride, accumulate);
  else
    post_combine2_kernel<TP, 1, MODE, 1><<<g, threads, 0, st>>>(P, (int)h, (int)w, dst, dst_ld, dst_stride, accumulate);
  return cudaGetLastError();
}

// First level of each operand pass: pairs (l, l+1) ending at L, a single
// level 1 first when L is odd.
inline int pass_first_level(int L, int l) { return (L & 1) && l == 1 ? 1 : 2; }

// Operand side of the breadth-first expansion (FP32 mode).  X is rows x
// cols with row pitch ld.
cudaError_t expand_f32(int L, int variant, int side, const float* X, int64_t rows, int64_t cols,
                       int64_t ld, uint8_t* ws, const StrassenLayout& S, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, cudaStream_t st) {
  const float* src = X;
  int64_t src_ld = ld, src_stride = 0;
  int pass = 0;
  for (int l = 1; l <= L;) {
    const int span = pass_first_level(L, l);  // levels l .. l+span-1 in this pass
    const int lend = l + span - 1;
    const int64_t h = rows >> lend, w = cols >> lend, R = pw7(l - 1);
    if (lend < L) {
      float* dst = reinterpret_cast<float*>(ws + ((pass & 1) ? S.off_pp1 : 0));
      if (span == 2)
        MMSR_CUDA_TRY(launch_pre_combine2<float>(src, src_ld, src_stride, h, w, R, dst, variant, side, st));
      else
        MMSR_CUDA_TRY(launch_pre_combine<float>(src, src_ld, src_stride, h, w, R, dst, variant, side, st));
      src = dst;
      src_ld = w;
      src_stride = h * w;  // stacks hold contiguous (h x w) matrices
    } else if (side == 0) {
      if (span == 2) {
        const int vec = (w % 4 == 0 && src_ld % 4 == 0 && src_stride % 4 == 0 && aligned_to(src, 16)) ? 1 : 0;
        const int threads = row_threads(S.KpL / 4);
        const dim3 g(rows_grid(h, R, threads), (unsigned)R);
        if (variant == 0)
          pre_combine2_split_rows_kernel<0><<<g, threads, 0, st>>>(src, src_ld, src_stride, (int)h, (int)w,
                                                                  (int)S.KpL, hi, lo, vec);
        else
          pre_combine2_split_rows_kernel<1><<<g, threads, 0, st>>>(src, src_ld, src_stride, (int)h, (int)w,
                                                                  (int)S.KpL, hi, lo, vec);
      } else {
        const int vec = (w % 4 == 0 && src_ld % 4 == 0 && src_stride % 4 == 0 && aligned_to(src, 16)) ? 1 : 0;
        const int threads = row_threads(S.KpL / 8);
        const dim3 g(rows_grid(h, R, threads), (unsigned)R);
        if (variant == 0)
          pre_combine_split_rows_kernel<0><<<g, threads, 0, st>>>(src, src_ld, src_stride, (int)h, (int)w,
                                                                 (int)S.KpL, hi, lo, vec);
        else
          pre_combine_split_rows_kernel<1><<<g, threads, 0, st>>>(src, src_ld, src_stride, (int)h, (int)w,
                                                                 (int)S.KpL, hi, lo, vec);
      }
      MMSR_CUDA_TRY(cudaGetLastError());
    } else {
      if (span == 2) {
        const dim3 g((unsigned)(S.KpL / 32), (unsigned)std::min<int64_t>((w + 15) / 16, kMaxGridY), (unsigned)R);
        if (variant == 0)
          pre_combine2_split_transpose_kernel<0><<<g, 128, 0, st>>>(src, src_ld, src_stride, (int)h, (int)w,
                                                                   (int)S.KpL, hi, lo);
        else
          pre_combine2_split_transpose_kernel<1><<<g, 128, 0, st>>>(src, src_ld, src_stride, (int)h, (int)w,
                                                                   (int)S.KpL, hi, lo);
      } else {
        const dim3 g((unsigned)(S.KpL / 64), (unsigned)std::min<int64_t>((w + 31) / 32, kMaxGridY), (unsigned)R);
        if (variant == 0)
          pre_combine_split_transpose_kernel<0><<<g, 256, 0, st>>>(src, src_ld, src_stride, h, w, S.KpL, hi, lo);
        else
          pre_combine_split_transpose_kernel<1><<<g, 256, 0, st>>>(src, src_ld, src_stride, h, w, S.KpL, hi, lo);
      }
      MMSR_CUDA_TRY(cudaGetLastError());
    }
    l += span;
    ++pass;
  }
  return cudaSuccess;
}

// Operand side, FP64 mode: FP64 stacks all the way to the leaves.  With E
// (side 0) or Fmax (side 1) given, a last pass of two levels also leaves the
// FP64-accuracy split's row exponents or column maxima and sets *maxima.
cudaError_t expand_f64(int L, int variant, int side, const double* X, int64_t rows, int64_t cols,
                       int64_t ld, uint8_t* ws, const StrassenLayout& S, double* leaf,
                       cudaStream_t st, int* E = nullptr, unsigned long long* Fmax = nullptr,
                       bool* maxima = nullptr) {
  if (maxima) *maxima = false;
  const double* src = X;
  int64_t src_ld = ld, src_stride = 0;
  int pass = 0;
  for (int l = 1; l <= L;) {
    const int span = pass_first_level(L, l);
    const int lend = l + span - 1;
    const int64_t h = rows >> lend, w = cols >> lend, R = pw7(l - 1);
    double* dst = (lend < L) ? reinterpret_cast<double*>(ws + ((pass & 1) ? S.off_pp1 : 0)) : leaf;
    if (span == 2 && lend == L && maxima && (side == 0 ? E != nullptr : Fmax != nullptr)) {
      if (side == 1) MMSR_CUDA_TRY(cudaMemsetAsync(Fmax, 0, (size_t)(R * 49) * (size_t)w * 8, st));
      MMSR_CUDA_TRY(launch_pre_combine2_maxima(src, src_ld, src_stride, h, w, R, dst, variant, side, E, Fmax, st));
      *maxima = true;
    } else if (span == 2)
      MMSR_CUDA_TRY(launch_pre_combine2<double>(src, src_ld, src_stride, h, w, R, dst, variant, side, st));
    else
      MMSR_CUDA_TRY(launch_pre_combine<double>(src, src_ld, src_stride, h, w, R, dst, variant, side, st));
    src = dst;
    src_ld = w;
    src_stride = h * w;
    l += span;
    ++pass;
  }
  return cudaSuccess;
}

template <typename TP>
cudaError_t post_pass(int span, const TP* src, int64_t h, int64_t w, int64_t R, TP* dst, int64_t dst_ld,
                      int64_t dst_stride, int variant, int accumulate, int mode, cudaStream_t st) {
  if (span == 2) {
    if (mode == kSumDoubleFloat)
      return launch_post_combine2<TP, kSumDoubleFloat>(src, h, w, R, dst, dst_ld, dst_stride, variant, accumulate, st);
    if (mode == kSumF64)
      return launch_post_combine2<TP, kSumF64>(src, h, w, R, dst, dst_ld, dst_stride, variant, accumulate, st);
    return launch_post_combine2<TP, kSumPlain>(src, h, w, R, dst, dst_ld, dst_stride, variant, accumulate, st);
  }
  if (mode == kSumDoubleFloat)
    return launch_post_combine<TP, kSumDoubleFloat>(src, h, w, R, dst, dst_ld, dst_stride, variant, accumulate, st);
  if (mode == kSumF64)
    return launch_post_combine<TP, kSumF64>(src, h, w, R, dst, dst_ld, dst_stride, variant, accumulate, st);
  return launch_post_combine<TP, kSumPlain>(src, h, w, R, dst, dst_ld, dst_stride, variant, accumulate, st);
}

// Bottom-up post-additions from the leaf products to C (pitch ldc).  The
// top level adds into C's old values when `accumulate` is set and sums in
// `top_mode` (PostSum); lower levels sum plainly.
template <typename TP>
cudaError_t fold(int L, int variant, const TP* P, int64_t m, int64_t n, uint8_t* ws,
                 const StrassenLayout& S, TP* C, int64_t ldc, int accumulate, int top_mode,
                 cudaStream_t st) {
  const TP* src = P;
  int pass = 0;
  for (int l = L; l >= 1;) {
    const int span = l >= 2 ? 2 : 1;  // levels l .. l-span+1 in this pass
    const int ltop = l - span + 1;
    const int64_t h = m >> l, w = n >> l, R = pw7(ltop - 1);
    const int64_t side = (int64_t)1 << span;  // destination matrices are side*h x side*w
    if (ltop > 1) {
      TP* dst = reinterpret_cast<TP*>(ws + ((pass & 1) ? S.off_pp1 : 0));
      MMSR_CUDA_TRY(post_pass<TP>(span, src, h, w, R, dst, side * w, side * side * h * w, variant, 0,
                                  kSumPlain, st));
      src = dst;
    } else {
      MMSR_CUDA_TRY(post_pass<TP>(span, src, h, w, R, C, ldc, 0, variant, accumulate, top_mode, st));
    }
    l -= span;
    ++pass;
  }
  return cudaSuccess;
}

// One Strassen product on strided views: C (pitch ldc) := [C +] A (pitch
// lda) x B (pitch ldb), `levels` >= 1 levels, workspace laid out by S.
int run_view(int levels, int variant, int sr, int64_t m, int64_t n, int64_t k, const void* A,
             int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc, int accumulate, uint8_t* w,
             const StrassenLayout& S, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (fused_level(levels, sr, m, n, k)) {
    float* P = reinterpret_cast<float*>(w + S.off_p);
    e = launch_strassen_fused_leaves(variant, static_cast<const float*>(A), static_cast<const float*>(B), P, m, n, k,
                                     lda, ldb, st);
    if (e == cudaSuccess) {
      TraceScope tr(kTrStrassenPost, st);
      e = fold<float>(1, variant, P, m, n, w, S, static_cast<float*>(C), ldc, accumulate, kSumPlain, st);
    }
    return e == cudaSuccess ? MM_OK : report_cuda(e, "fused Strassen level");
  }
  if (sr == MM_SR_PLUS_TIMES_F32) {
    auto* ahi = reinterpret_cast<__nv_bfloat16*>(w + S.off_ahi);
    auto* alo = reinterpret_cast<__nv_bfloat16*>(w + S.off_alo);
    auto* bhi = reinterpret_cast<__nv_bfloat16*>(w + S.off_bhi);
    auto* blo = reinterpret_cast<__nv_bfloat16*>(w + S.off_blo);
    float* P = reinterpret_cast<float*>(w + S.off_p);
    {
      TraceScope tr(kTrStrassenCombine, st);
      e = expand_f32(levels, variant, 0, static_cast<const float*>(A), m, k, lda, w, S, ahi, alo, st);
      if (e == cudaSuccess)
        e = expand_f32(levels, variant, 1, static_cast<const float*>(B), k, n, ldb, w, S, bhi, blo, st);
    }
    if (e == cudaSuccess) e = launch_bf16x3_batched(ahi, alo, bhi, blo, P, S.mL, S.nL, S.KpL, (int)S.leaves, st);
    if (e == cudaSuccess) {
      TraceScope tr(kTrStrassenPost, st);
      // Wide top-level sums once the operand and product sums of three or
      // more levels have grown the cancellation error.
      const int top = levels >= 3 ? (g_strassen_top_f64 ? kSumF64 : kSumDoubleFloat) : kSumPlain;
      e = fold<float>(levels, variant, P, m, n, w, S, static_cast<float*>(C), ldc, accumulate, top, st);
    }
  } else {
    double* la = reinterpret_cast<double*>(w + S.off_ahi);
    double* lb = reinterpret_cast<double*>(w + S.off_bhi);
    double* P = reinterpret_cast<double*>(w + S.off_p);
    // FP64-accuracy leaves: the last operand pass leaves the digit split's
    // line maxima where the split reads them
    const bool fa = sr == MM_SR_PLUS_TIMES_F64ACC;
    const int slices = f64acc_slices_for_levels(levels);
    int* E = nullptr;
    unsigned long long* Fmax = nullptr;
    if (fa) f64acc_maxima_buffers(S.mL, S.nL, S.kL, (int)S.leaves, slices, w + S.off_leafws, &E, &Fmax);
    bool max_a = false, max_b = false;
    {
      TraceScope tr(kTrStrassenCombine, st);
      e = expand_f64(levels, variant, 0, static_cast<const double*>(A), m, k, lda, w, S, la, st, E, nullptr,
                     fa ? &max_a : nullptr);
      if (e == cudaSuccess)
        e = expand_f64(levels, variant, 1, static_cast<const double*>(B), k, n, ldb, w, S, lb, st, nullptr, Fmax,
                       fa ? &max_b : nullptr);
    }
    if (e == cudaSuccess) {
      if (fa) {
        const int rc = run_f64acc_batched(la, lb, P, S.mL, S.nL, S.kL, (int)S.leaves, slices, w + S.off_leafws, st,
                                          max_a && max_b);
        if (rc != MM_OK) return rc;
      } else {
        e = launch_dfma_batched(la, lb, P, S.mL, S.nL, S.kL, (int)S.leaves, st);
      }
    }
    if (e == cudaSuccess) {
      TraceScope tr(kTrStrassenPost, st);
      e = fold<double>(levels, variant, P, m, n, w, S, static_cast<double*>(C), ldc, accumulate, kSumPlain, st);
    }
  }
  return e == cudaSuccess ? MM_OK : report_cuda(e, "Strassen level pass");
}

bool strassen_semiring(int sr) {
  return sr == MM_SR_PLUS_TIMES_F32 || sr == MM_SR_PLUS_TIMES_F64 || sr == MM_SR_PLUS_TIMES_F64ACC;
}

void fill_plan(int levels, int sr, int64_t total, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  p->levels = levels;
  p->split_k = 1;
  p->tile_m = sr == MM_SR_PLUS_TIMES_F64 ? 64 : 128;
  p->tile_n = sr == MM_SR_PLUS_TIMES_F32 ? 256 : 64;
  p->tile_k = sr == MM_SR_PLUS_TIMES_F32 ? 64 : (sr == MM_SR_PLUS_TIMES_F64 ? 16 : 32);
  p->kernel = sr == MM_SR_PLUS_TIMES_F32 ? 2
              : sr == MM_SR_PLUS_TIMES_F64 ? 0
                                           : (f64acc_slices_for_levels(levels) == 6 ? 7 : 3);
  p->workspace_min = total;
  p->workspace_used = total;
}

}  // namespace

int g_strassen_top_f64 = 0;  // mm_set_option(MM_OPT_STRASSEN_TOP_F64, ...)
int g_strassen_fused = 0;    // mm_set_option(MM_OPT_STRASSEN_FUSED, ...)


void strassen_tables(int variant, int8_t* alpha, int8_t* beta, int8_t* gamma) {
  for (int r = 0; r < 7; ++r)
    for (int q = 0; q < 4; ++q) {
      alpha[r * 4 + q] = (int8_t)coef_alpha(variant, r, q);
      beta[r * 4 + q] = (int8_t)coef_beta(variant, r, q);
      gamma[q * 7 + r] = (int8_t)coef_gamma(variant, q, r);
    }
}

int plan_strassen(int levels, int sr, int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  if (!strassen_semiring(sr)) return MM_ERR_UNSUPPORTED;
  fill_plan(levels, sr, strassen_layout(levels, sr, m, n, k).total, p);
  (void)budget;
  return MM_OK;
}

// Depth for MM_LEVELS_AUTO: the preferred depth of the semiring (measured at
// n >= 8192: FP32 mode and FP64-accuracy mode are fastest at two levels;
// the FP64 DFMA leaves are bound by the FP64 pipe, so every level saves an
// eighth of the time), lowered until every leaf dimension stays at least
// 1024 (512 for FP64), the shape divides by 2^L and the workspace fits the
// budget.  0 means the classic product.
int choose_strassen_levels(int sr, int64_t m, int64_t n, int64_t k, size_t budget) {
  int L = sr == MM_SR_PLUS_TIMES_F32 ? 2 : (sr == MM_SR_PLUS_TIMES_F64ACC ? 2 : 4);
  const int64_t floor_dim = sr == MM_SR_PLUS_TIMES_F64 ? 512 : 1024;
  for (; L > 0; --L) {
    const int64_t mask = ((int64_t)1 << L) - 1;
    if ((m & mask) || (n & mask) || (k & mask)) continue;
    if ((m >> L) < floor_dim || (n >> L) < floor_dim || (k >> L) < floor_dim) continue;
    if ((size_t)strassen_layout(L, sr, m, n, k).total <= budget) break;
  }
  return L;
}

int run_strassen(int levels, int variant, int sr, int64_t m, int64_t n, int64_t k, const void* A,
                 const void* B, void* C, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!strassen_semiring(sr)) return MM_ERR_UNSUPPORTED;
  const StrassenLayout S = strassen_layout(levels, sr, m, n, k);
  if ((size_t)S.total > ws_bytes) return MM_ERR_WORKSPACE;
  return run_view(levels, variant, sr, m, n, k, A, k, B, n, C, n, 0, static_cast<uint8_t*>(ws), S, st);
}

// TAR-Strassen (the zero-temporary Strassen schedule the paper sketches in
// Section 5), one or two levels: the leaf products are not stored; the leaf
// epilogue adds each one, times its +-1 coefficient, straight into the
// blocks of C it contributes to.  Leaf product p = 7 r1 + r2 (r1 the top
// level's product, the order of the operand passes) goes to block (q1, q2)
// with coefficient gamma(q1, r1) gamma(q2, r2).  Products run in waves in
// which no two touch the same block, so the read-modify-writes of one launch
// never collide; a block's first writer overwrites it.  The waves are a
// greedy colouring (one level of the paper's formulas: exactly P1;
// P2 || P5; P3 || P4; P6 || P7).  A product may reach at most four
// blocks (the epilogue's limit): every product of the paper's formulas at
// one or two levels and of Winograd's at one level; two Winograd levels
// (P1 x P1 reaches all sixteen blocks) are refused.  FP32 mode (bf16x3 leaf)
// and FP64-accuracy mode (digit-slice leaf).  Workspace: the operand sums.
struct TarPlan {
  int levels = 0, products = 0, waves = 0;
  bool fits = true;  // every product reaches at most four blocks
  int wave_of[49];
  int ndst[49];
  int block[49][4];  // block index br * 2^L + bc
  int sign[49][4];
};

TarPlan tar_plan(int L, int variant) {
  TarPlan T;
  T.levels = L;
  T.products = pw7(L);
  const int side = 1 << L;
  uint32_t used[49], mask_of[49];
  memset(used, 0, sizeof(used));
  for (int p = 0; p < T.products; ++p) {
    const int r1 = L == 2 ? p / 7 : p, r2 = L == 2 ? p % 7 : 0;
    T.ndst[p] = 0;
    uint32_t mask = 0;
    for (int q1 = 0; q1 < 4; ++q1) {
      const int g1 = coef_gamma(variant, q1, r1);
      if (g1 == 0) continue;
      for (int q2 = 0; q2 < (L == 2 ? 4 : 1); ++q2) {
        const int g2 = L == 2 ? coef_gamma(variant, q2, r2) : 1;
        if (g2 == 0) continue;
        const int br = (q1 >> 1) * (side / 2) + (L == 2 ? (q2 >> 1) : 0);
        const int bc = (q1 & 1) * (side / 2) + (L == 2 ? (q2 & 1) : 0);
        const int b = br * side + bc;
        mask |= 1u << b;
        if (T.ndst[p] < 4) {
          T.block[p][T.ndst[p]] = b;
          T.sign[p][T.ndst[p]] = g1 * g2;
        }
        ++T.ndst[p];
      }
    }
    if (T.ndst[p] > 4) T.fits = false;
    mask_of[p] = mask;
  }
  // greedy colouring, products with more blocks first (ties in product
  // order): one Winograd level then takes four waves, {P1}, {P6, P2},
  // {P5, P4}, {P7, P3}, instead of five in plain product order; the paper's
  // formulas keep their printed order
  int order[49];
  for (int p = 0; p < T.products; ++p) order[p] = p;
  std::stable_sort(order, order + T.products, [&](int a, int b) { return T.ndst[a] > T.ndst[b]; });
  for (int i = 0; i < T.products; ++i) {
    const int p = order[i];
    int w = 0;
    while (w < T.waves && (used[w] & mask_of[p])) ++w;
    if (w == T.waves) ++T.waves;
    used[w] |= mask_of[p];
    T.wave_of[p] = w;
  }
  return T;
}

size_t tar_workspace(int L, int sr, int64_t m, int64_t n, int64_t k) {
  const StrassenLayout S = strassen_layout(L, sr, m, n, k);
  // FP32 mode: everything before the product stack; FP64-accuracy mode: the
  // FP64 leaf operands and their digit slices (its products overlay the A
  // leaf stack in mm_strassen too, so the two need the same)
  return (size_t)(sr == MM_SR_PLUS_TIMES_F32 ? S.off_p : S.total);
}

template <typename T, typename Launch>
cudaError_t tar_waves_run(const TarPlan& TP, const StrassenLayout& S, T* C, int64_t ldc, Launch&& launch) {
  const int side = 1 << TP.levels;
  bool written[16] = {false};
  for (int v = 0; v < TP.waves; ++v) {
    QuadOutT<T> qo;
    memset(&qo, 0, sizeof(qo));
    qo.ld = ldc;
    bool wrote[16] = {false};
    auto flush = [&]() -> cudaError_t {
      if (qo.entries == 0) return cudaSuccess;
      cudaError_t e = launch(qo);
      memset(&qo, 0, sizeof(qo));
      qo.ld = ldc;
      return e;
    };
    for (int p = 0; p < TP.products; ++p) {
      if (TP.wave_of[p] != v) continue;
      const int i = qo.entries++;
      qo.leaf[i] = (int16_t)p;
      for (int d = 0; d < TP.ndst[p]; ++d) {
        const int b = TP.block[p][d];
        qo.dst[i][d] = C + (int64_t)(b / side) * S.mL * ldc + (int64_t)(b % side) * S.nL;
        qo.sign[i][d] = (int8_t)TP.sign[p][d];
        qo.add[i][d] = written[b] ? 1 : 0;
        wrote[b] = true;
      }
      if (qo.entries == kQuadEntries) MMSR_CUDA_TRY(flush());
    }
    MMSR_CUDA_TRY(flush());
    for (int b = 0; b < 16; ++b) written[b] = written[b] || wrote[b];
  }
  return cudaSuccess;
}

int run_tar_view(int L, int variant, int sr, int64_t m, int64_t n, int64_t k, const void* A, int64_t lda,
                 const void* B, int64_t ldb, void* C, int64_t ldc, uint8_t* w, cudaStream_t st) {
  const StrassenLayout S = strassen_layout(L, sr, m, n, k);
  const TarPlan TP = tar_plan(L, variant);
  if (!TP.fits) return MM_ERR_UNSUPPORTED;
  cudaError_t e;
  if (sr == MM_SR_PLUS_TIMES_F32) {
    auto* ahi = reinterpret_cast<__nv_bfloat16*>(w + S.off_ahi);
    auto* alo = reinterpret_cast<__nv_bfloat16*>(w + S.off_alo);
    auto* bhi = reinterpret_cast<__nv_bfloat16*>(w + S.off_bhi);
    auto* blo = reinterpret_cast<__nv_bfloat16*>(w + S.off_blo);
    {
      TraceScope tr(kTrStrassenCombine, st);
      e = expand_f32(L, variant, 0, static_cast<const float*>(A), m, k, lda, w, S, ahi, alo, st);
      if (e == cudaSuccess) e = expand_f32(L, variant, 1, static_cast<const float*>(B), k, n, ldb, w, S, bhi, blo, st);
    }
    if (e != cudaSuccess) return report_cuda(e, "TAR-Strassen operand pass");
    e = tar_waves_run<float>(TP, S, static_cast<float*>(C), ldc, [&](const QuadOut& qo) {
      return launch_bf16x3_batched(ahi, alo, bhi, blo, nullptr, S.mL, S.nL, S.KpL, qo.entries, st, &qo,
                                   (int)S.leaves);
    });
    return e == cudaSuccess ? MM_OK : report_cuda(e, "TAR-Strassen leaf wave");
  }
  double* la = reinterpret_cast<double*>(w + S.off_ahi);
  double* lb = reinterpret_cast<double*>(w + S.off_bhi);
  const int slices = f64acc_slices_for_levels(L);
  int* E = nullptr;
  unsigned long long* Fmax = nullptr;
  f64acc_maxima_buffers(S.mL, S.nL, S.kL, (int)S.leaves, slices, w + S.off_leafws, &E, &Fmax);
  bool max_a = false, max_b = false;
  {
    TraceScope tr(kTrStrassenCombine, st);
    e = expand_f64(L, variant, 0, static_cast<const double*>(A), m, k, lda, w, S, la, st, E, nullptr, &max_a);
    if (e == cudaSuccess)
      e = expand_f64(L, variant, 1, static_cast<const double*>(B), k, n, ldb, w, S, lb, st, nullptr, Fmax, &max_b);
  }
  if (e != cudaSuccess) return report_cuda(e, "TAR-Strassen operand pass");
  int rc = f64acc_prepare_batched(la, lb, S.mL, S.nL, S.kL, (int)S.leaves, slices, w + S.off_leafws, st,
                                  max_a && max_b);
  if (rc != MM_OK) return rc;
  e = tar_waves_run<double>(TP, S, static_cast<double*>(C), ldc, [&](const QuadOut64& qo) {
    return f64acc_gemm_quad(S.mL, S.nL, S.kL, (int)S.leaves, slices, w + S.off_leafws, qo, st) == MM_OK
               ? cudaSuccess
               : cudaErrorLaunchFailure;
  });
  return e == cudaSuccess ? MM_OK : report_cuda(e, "TAR-Strassen leaf wave");
}

bool tar_semiring(int sr) { return sr == MM_SR_PLUS_TIMES_F32 || sr == MM_SR_PLUS_TIMES_F64ACC; }

int plan_strassen_tar(int L, int sr, int64_t m, int64_t n, int64_t k, mm_plan_t* p) {
  if (!tar_semiring(sr)) return MM_ERR_UNSUPPORTED;
  fill_plan(L, sr, (int64_t)tar_workspace(L, sr, m, n, k), p);
  return MM_OK;
}

int run_strassen_tar(int L, int variant, int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                     void* C, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!tar_semiring(sr)) return MM_ERR_UNSUPPORTED;
  if (!tar_plan(L, variant).fits) return MM_ERR_UNSUPPORTED;
  if (tar_workspace(L, sr, m, n, k) > ws_bytes) return MM_ERR_WORKSPACE;
  return run_tar_view(L, variant, sr, m, n, k, A, k, B, n, C, n, static_cast<uint8_t*>(ws), st);
}

int strassen_tar_waves(int L, int variant, int* wave_of_product) {
  const TarPlan T = tar_plan(L, variant);
  for (int p = 0; p < T.products; ++p) wave_of_product[p] = T.wave_of[p];
  return T.fits ? T.waves : MM_ERR_UNSUPPORTED;
}

// STAR-Strassen-1 (Theorem star-strassen-1): the top `classic` levels are
// the classic 8-way recursion of Eq. mm-dac run in place (no temporaries:
// every block product adds into its C block, the k-halves one after the
// other as in CO2), and each of the 8^classic block products runs `levels`
// Strassen levels.  The Strassen temporaries are those of one block product,
// reused by the next, so the workspace shrinks by 4^classic while the work
// grows by (8/7)^classic against Strassen on all classic + levels levels.
int plan_star_strassen(int classic, int levels, int sr, int64_t m, int64_t n, int64_t k,
                       size_t budget, mm_plan_t* p) {
  if (!strassen_semiring(sr)) return MM_ERR_UNSUPPORTED;
  if (levels == 0) return plan_semiring(sr, m, n, k, budget, p);
  fill_plan(levels, sr, strassen_layout(levels, sr, m >> classic, n >> classic, k >> classic).total, p);
  return MM_OK;
}

int run_star_strassen(int classic, int levels, int variant, int sr, int64_t m, int64_t n, int64_t k,
                      const void* A, const void* B, void* C, void* ws, size_t ws_bytes,
                      cudaStream_t st) {
  if (!strassen_semiring(sr)) return MM_ERR_UNSUPPORTED;
  if (levels == 0) return run_semiring(sr, m, n, k, A, B, C, ws, ws_bytes, st);
  const int64_t g = (int64_t)1 << classic;
  const int64_t bm = m >> classic, bn = n >> classic, bk = k >> classic;
  const StrassenLayout S = strassen_layout(levels, sr, bm, bn, bk);
  if ((size_t)S.total > ws_bytes) return MM_ERR_WORKSPACE;
  const int64_t eb = sr == MM_SR_PLUS_TIMES_F32 ? 4 : 8;
  const uint8_t* a = static_cast<const uint8_t*>(A);
  const uint8_t* b = static_cast<const uint8_t*>(B);
  uint8_t* c = static_cast<uint8_t*>(C);
  for (int64_t t = 0; t < g; ++t)
    for (int64_t I = 0; I < g; ++I)
      for (int64_t J = 0; J < g; ++J) {
        const int rc = run_view(levels, variant, sr, bm, bn, bk, a + (I * bm * k + t * bk) * eb, k,
                                b + (t * bk * n + J * bn) * eb, n, c + (I * bm * n + J * bn) * eb, n,
                                t > 0 ? 1 : 0, static_cast<uint8_t*>(ws), S, st);
        if (rc != MM_OK) return rc;
      }
  return MM_OK;
}

}  // namespace mmsr

extern "C" int mm_strassen_tables(int variant, int8_t* alpha, int8_t* beta, int8_t* gamma) {
  if (variant != MM_STRASSEN_PAPER && variant != MM_STRASSEN_WINOGRAD) return MM_ERR_ARG;
  if (!alpha || !beta || !gamma) return MM_ERR_ARG;
  mmsr::strassen_tables(variant, alpha, beta, gamma);
  return MM_OK;
}
