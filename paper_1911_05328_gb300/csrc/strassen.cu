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

#include "common.cuh"
#include "internal.h"

namespace mmsr {

// ------------------------------------------------------ coefficient tables
// [variant][product r][quadrant q]
static const int8_t kAlphaHost[2][7][4] = {
    {{1, 0, 0, 1}, {0, 0, 1, 1}, {1, 0, 0, 0}, {0, 0, 0, 1}, {1, 1, 0, 0}, {-1, 0, 1, 0}, {0, 1, 0, -1}},
    {{1, 0, 0, 0}, {0, 1, 0, 0}, {1, 1, -1, -1}, {0, 0, 0, 1}, {0, 0, 1, 1}, {-1, 0, 1, 1}, {1, 0, -1, 0}}};
static const int8_t kBetaHost[2][7][4] = {
    {{1, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, -1}, {-1, 0, 1, 0}, {0, 0, 0, 1}, {1, 1, 0, 0}, {0, 0, 1, 1}},
    {{1, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}, {1, -1, -1, 1}, {-1, 1, 0, 0}, {1, -1, 0, 1}, {0, -1, 0, 1}}};
// [variant][quadrant q][product r]
static const int8_t kGammaHost[2][4][7] = {
    {{1, 0, 0, 1, -1, 0, 1}, {0, 0, 1, 0, 1, 0, 0}, {0, 1, 0, 1, 0, 0, 0}, {1, -1, 1, 0, 0, 1, 0}},
    {{1, 1, 0, 0, 0, 0, 0}, {1, 0, 1, 0, 1, 1, 0}, {1, 0, 0, -1, 0, 1, 1}, {1, 0, 0, 0, 1, 1, 1}}};

__constant__ int8_t kAlpha[2][7][4] = {
    {{1, 0, 0, 1}, {0, 0, 1, 1}, {1, 0, 0, 0}, {0, 0, 0, 1}, {1, 1, 0, 0}, {-1, 0, 1, 0}, {0, 1, 0, -1}},
    {{1, 0, 0, 0}, {0, 1, 0, 0}, {1, 1, -1, -1}, {0, 0, 0, 1}, {0, 0, 1, 1}, {-1, 0, 1, 1}, {1, 0, -1, 0}}};
__constant__ int8_t kBeta[2][7][4] = {
    {{1, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, -1}, {-1, 0, 1, 0}, {0, 0, 0, 1}, {1, 1, 0, 0}, {0, 0, 1, 1}},
    {{1, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}, {1, -1, -1, 1}, {-1, 1, 0, 0}, {1, -1, 0, 1}, {0, -1, 0, 1}}};
__constant__ int8_t kGamma[2][4][7] = {
    {{1, 0, 0, 1, -1, 0, 1}, {0, 0, 1, 0, 1, 0, 0}, {0, 1, 0, 1, 0, 0, 0}, {1, -1, 1, 0, 0, 1, 0}},
    {{1, 1, 0, 0, 0, 0, 0}, {1, 0, 1, 0, 1, 1, 0}, {1, 0, 0, -1, 0, 1, 1}, {1, 0, 0, 0, 1, 1, 1}}};

namespace {

template <typename T>
__device__ __forceinline__ T apply(int8_t c, T acc, T x) {
  return c == 0 ? acc : (c > 0 ? acc + x : acc - x);
}

// Sum of +-1/0 terms in the fixed quadrant order 00, 01, 10, 11.
template <typename T>
__device__ __forceinline__ T combo4(const int8_t* c, T x0, T x1, T x2, T x3) {
  T acc = T(0);
  acc = apply(c[0], acc, x0);
  acc = apply(c[1], acc, x1);
  acc = apply(c[2], acc, x2);
  acc = apply(c[3], acc, x3);
  return acc;
}

__device__ __forceinline__ const int8_t* coef_row(int variant, int side, int j) {
  return side == 0 ? kAlpha[variant][j] : kBeta[variant][j];
}

// Level transition for one operand side: source stack matrix r (2h x 2w,
// row pitch src_ld, matrices src_stride apart) -> seven (h x w) matrices
// 7r..7r+6 of the destination stack (contiguous).  One thread per element
// position reads the four quadrants once and writes seven sums.
template <typename T>
__global__ void __launch_bounds__(256) pre_combine_kernel(const T* __restrict__ src, int64_t src_ld,
                                                          int64_t src_stride, int64_t h, int64_t w,
                                                          T* __restrict__ dst, int variant, int side) {
  const int r = blockIdx.y;
  const T* s = src + (int64_t)r * src_stride;
  T* d = dst + (int64_t)r * 7 * h * w;
  const int64_t total = h * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w, j = e - i * w;
    const T x0 = s[i * src_ld + j], x1 = s[i * src_ld + w + j];
    const T x2 = s[(h + i) * src_ld + j], x3 = s[(h + i) * src_ld + w + j];
#pragma unroll
    for (int p = 0; p < 7; ++p) d[(int64_t)p * total + e] = combo4(coef_row(variant, side, p), x0, x1, x2, x3);
  }
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Last level, A side, FP32 mode: seven (h x w) sums written as bf16 hi/lo
// rows of pitch Kp (columns w..Kp-1 zero).  One thread per 8 columns.
__global__ void __launch_bounds__(256) pre_combine_split_rows_kernel(
    const float* __restrict__ src, int64_t src_ld, int64_t src_stride, int64_t h, int64_t w,
    int64_t Kp, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int variant) {
  const int r = blockIdx.y;
  const float* s = src + (int64_t)r * src_stride;
  const int64_t cpr = Kp / 8;
  const int64_t total = h * cpr;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cpr, c8 = (e - i * cpr) * 8;
    float x[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float* row = s + ((q >> 1) * h + i) * src_ld + (q & 1) * w;
#pragma unroll
      for (int t = 0; t < 8; ++t) x[q][t] = (c8 + t < w) ? row[c8 + t] : 0.f;
    }
#pragma unroll
    for (int p = 0; p < 7; ++p) {
      const int8_t* c = kAlpha[variant][p];
      __align__(16) __nv_bfloat16 hh[8], ll[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) split_bf16(combo4(c, x[0][t], x[1][t], x[2][t], x[3][t]), hh[t], ll[t]);
      const int64_t off = ((int64_t)(r * 7 + p) * h + i) * Kp + c8;
      *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(hh);
      *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(ll);
    }
  }
}

// Last level, B side, FP32 mode: source stack matrix r is (2h x 2w) = (k x n);
// the seven sums T_p (h x w) are written transposed as bf16 hi/lo (w x Kp).
// Tile: 64 k x 32 n of each quadrant through shared memory.
__global__ void __launch_bounds__(256) pre_combine_split_transpose_kernel(
    const float* __restrict__ src, int64_t src_ld, int64_t src_stride, int64_t h, int64_t w,
    int64_t Kp, __nv_bfloat16* __restrict__ hiT, __nv_bfloat16* __restrict__ loT, int variant) {
  __shared__ float tile[4][64][33];
  const int r = blockIdx.z;
  const float* s = src + (int64_t)r * src_stride;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t k0 = (int64_t)blockIdx.x * 64, n0 = (int64_t)blockIdx.y * 32;
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
  if (gn >= w) return;
#pragma unroll
  for (int p = 0; p < 7; ++p) {
    const int8_t* c = kBeta[variant][p];
    __align__(16) __nv_bfloat16 hh[8], ll[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int kk = chunk * 8 + t;
      split_bf16(combo4(c, tile[0][kk][row], tile[1][kk][row], tile[2][kk][row], tile[3][kk][row]), hh[t], ll[t]);
    }
    const int64_t off = ((int64_t)(r * 7 + p) * w + gn) * Kp + k0 + chunk * 8;
    *reinterpret_cast<uint4*>(hiT + off) = *reinterpret_cast<const uint4*>(hh);
    *reinterpret_cast<uint4*>(loT + off) = *reinterpret_cast<const uint4*>(ll);
  }
}

// Post-additions: products 7r..7r+6 (h x w each, contiguous) -> the four
// quadrants of destination matrix r (2h x 2w, pitch dst_ld, dst_stride
// apart).  Sums run in ACC precision in product order; one thread per
// element position reads each product once and writes four quadrants.
template <typename TP, typename ACC, typename TOUT>
__global__ void __launch_bounds__(256) post_combine_kernel(const TP* __restrict__ P, int64_t h, int64_t w,
                                                           TOUT* __restrict__ dst, int64_t dst_ld,
                                                           int64_t dst_stride, int variant) {
  const int r = blockIdx.y;
  const TP* pp = P + (int64_t)r * 7 * h * w;
  TOUT* d = dst + (int64_t)r * dst_stride;
  const int64_t total = h * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w, j = e - i * w;
    ACC x[7];
#pragma unroll
    for (int p = 0; p < 7; ++p) x[p] = (ACC)pp[(int64_t)p * total + e];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ACC acc = ACC(0);
#pragma unroll
      for (int p = 0; p < 7; ++p) acc = apply(kGamma[variant][q][p], acc, x[p]);
      d[((q >> 1) * h + i) * dst_ld + (q & 1) * w + j] = (TOUT)acc;
    }
  }
}

unsigned grid_for(int64_t work) {
  int64_t b = (work + 255) / 256;
  const int64_t cap = (int64_t)kNumSMs * 16;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
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

// Workspace carve-up.  FP32 mode: FP32 stacks for levels 1..L-1 (ping-pong),
// the last level's split operands (bf16 hi/lo, B transposed) and the leaf
// products.  FP64 mode: FP64 stacks, FP64 leaf operands and products.
StrassenLayout strassen_layout(int L, int sr, int64_t m, int64_t n, int64_t k) {
  StrassenLayout s;
  const int esz = (sr == MM_SR_PLUS_TIMES_F32) ? 4 : 8;
  s.mL = m >> L;
  s.nL = n >> L;
  s.kL = k >> L;
  s.leaves = pw7(L);
  int64_t pp = 0;
  for (int l = 1; l <= L - 1; ++l) {
    const int64_t ml = m >> l, nl = n >> l, kl = k >> l;
    int64_t e = ml * kl;
    if (kl * nl > e) e = kl * nl;
    if (ml * nl > e) e = ml * nl;
    const int64_t b = pw7(l) * e * esz;
    if (b > pp) pp = b;
  }
  s.pp_bytes = align_up(pp, 1024);
  s.off_pp1 = s.pp_bytes;
  int64_t off = 2 * s.pp_bytes;
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
  s.off_p = off;
  off += align_up(s.leaves * s.mL * s.nL * esz, 1024);
  s.off_leafws = off;  // FP64-accuracy leaves: digit slices and exponents
  if (sr == MM_SR_PLUS_TIMES_F64ACC)
    off += align_up((int64_t)f64acc_batched_bytes(s.mL, s.nL, s.kL, (int)s.leaves), 1024);
  s.total = off;
  return s;
}

// Operand side of the breadth-first expansion (FP32 mode).
cudaError_t expand_f32(int L, int variant, int side, const float* X, int64_t rows, int64_t cols,
                       uint8_t* ws, const StrassenLayout& S, __nv_bfloat16* hi, __nv_bfloat16* lo,
                       cudaStream_t st) {
  const float* src = X;
  int64_t src_ld = cols, src_stride = 0;
  for (int l = 1; l <= L; ++l) {
    const int64_t h = rows >> l, w = cols >> l, R = pw7(l - 1);
    if (l < L) {
      float* dst = reinterpret_cast<float*>(ws + ((l & 1) ? S.off_pp1 : 0));
      pre_combine_kernel<float><<<dim3(grid_for(h * w), (unsigned)R), 256, 0, st>>>(
          src, src_ld, src_stride, h, w, dst, variant, side);
      src = dst;
      src_ld = w;
      src_stride = h * w;  // stacks hold contiguous (h x w) matrices
    } else if (side == 0) {
      pre_combine_split_rows_kernel<<<dim3(grid_for(h * (S.KpL / 8)), (unsigned)R), 256, 0, st>>>(
          src, src_ld, src_stride, h, w, S.KpL, hi, lo, variant);
    } else {
      dim3 g((unsigned)(S.KpL / 64), (unsigned)((w + 31) / 32), (unsigned)R);
      pre_combine_split_transpose_kernel<<<g, 256, 0, st>>>(src, src_ld, src_stride, h, w, S.KpL, hi, lo,
                                                            variant);
    }
    MMSR_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// Operand side, FP64 mode: FP64 stacks all the way to the leaves.
cudaError_t expand_f64(int L, int variant, int side, const double* X, int64_t rows, int64_t cols,
                       uint8_t* ws, const StrassenLayout& S, double* leaf, cudaStream_t st) {
  const double* src = X;
  int64_t src_ld = cols, src_stride = 0;
  for (int l = 1; l <= L; ++l) {
    const int64_t h = rows >> l, w = cols >> l, R = pw7(l - 1);
    double* dst = (l < L) ? reinterpret_cast<double*>(ws + ((l & 1) ? S.off_pp1 : 0)) : leaf;
    pre_combine_kernel<double><<<dim3(grid_for(h * w), (unsigned)R), 256, 0, st>>>(
        src, src_ld, src_stride, h, w, dst, variant, side);
    MMSR_CUDA_TRY(cudaGetLastError());
    src = dst;
    src_ld = w;
    src_stride = h * w;
  }
  return cudaSuccess;
}

// Bottom-up post-additions from the leaf products to C.
template <typename TP>
cudaError_t fold(int L, int variant, const TP* P, int64_t m, int64_t n, uint8_t* ws,
                 const StrassenLayout& S, TP* C, bool top_f64, cudaStream_t st) {
  const TP* src = P;
  for (int l = L; l >= 1; --l) {
    const int64_t h = m >> l, w = n >> l, R = pw7(l - 1);
    dim3 g(grid_for(h * w), (unsigned)R);
    if (l > 1) {
      TP* dst = reinterpret_cast<TP*>(ws + (((l - 1) & 1) ? S.off_pp1 : 0));
      post_combine_kernel<TP, TP, TP><<<g, 256, 0, st>>>(src, h, w, dst, 2 * w, 4 * h * w, variant);
      src = dst;
    } else if (top_f64) {
      post_combine_kernel<TP, double, TP><<<g, 256, 0, st>>>(src, h, w, C, n, 0, variant);
    } else {
      post_combine_kernel<TP, TP, TP><<<g, 256, 0, st>>>(src, h, w, C, n, 0, variant);
    }
    MMSR_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

void strassen_tables(int variant, int8_t* alpha, int8_t* beta, int8_t* gamma) {
  memcpy(alpha, kAlphaHost[variant], 28);
  memcpy(beta, kBetaHost[variant], 28);
  memcpy(gamma, kGammaHost[variant], 28);
}

int plan_strassen(int levels, int sr, int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  if (sr != MM_SR_PLUS_TIMES_F32 && sr != MM_SR_PLUS_TIMES_F64 && sr != MM_SR_PLUS_TIMES_F64ACC)
    return MM_ERR_UNSUPPORTED;
  const StrassenLayout S = strassen_layout(levels, sr, m, n, k);
  p->levels = levels;
  p->split_k = 1;
  p->tile_m = sr == MM_SR_PLUS_TIMES_F64 ? 64 : 128;
  p->tile_n = sr == MM_SR_PLUS_TIMES_F32 ? 256 : 64;
  p->tile_k = sr == MM_SR_PLUS_TIMES_F32 ? 64 : (sr == MM_SR_PLUS_TIMES_F64 ? 16 : 32);
  p->kernel = sr == MM_SR_PLUS_TIMES_F32 ? 2 : (sr == MM_SR_PLUS_TIMES_F64 ? 0 : 3);
  p->workspace_min = S.total;
  p->workspace_used = S.total;
  (void)budget;
  return MM_OK;
}

int run_strassen(int levels, int variant, int sr, int64_t m, int64_t n, int64_t k, const void* A,
                 const void* B, void* C, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (sr != MM_SR_PLUS_TIMES_F32 && sr != MM_SR_PLUS_TIMES_F64 && sr != MM_SR_PLUS_TIMES_F64ACC)
    return MM_ERR_UNSUPPORTED;
  const StrassenLayout S = strassen_layout(levels, sr, m, n, k);
  if ((size_t)S.total > ws_bytes) return MM_ERR_WORKSPACE;
  uint8_t* w = static_cast<uint8_t*>(ws);
  cudaError_t e = cudaSuccess;
  if (sr == MM_SR_PLUS_TIMES_F32) {
    auto* ahi = reinterpret_cast<__nv_bfloat16*>(w + S.off_ahi);
    auto* alo = reinterpret_cast<__nv_bfloat16*>(w + S.off_alo);
    auto* bhi = reinterpret_cast<__nv_bfloat16*>(w + S.off_bhi);
    auto* blo = reinterpret_cast<__nv_bfloat16*>(w + S.off_blo);
    float* P = reinterpret_cast<float*>(w + S.off_p);
    {
      TraceScope tr(kTrStrassenCombine, st);
      e = expand_f32(levels, variant, 0, static_cast<const float*>(A), m, k, w, S, ahi, alo, st);
      if (e == cudaSuccess)
        e = expand_f32(levels, variant, 1, static_cast<const float*>(B), k, n, w, S, bhi, blo, st);
    }
    if (e == cudaSuccess) e = launch_bf16x3_batched(ahi, alo, bhi, blo, P, S.mL, S.nL, S.KpL, (int)S.leaves, st);
    if (e == cudaSuccess) {
      TraceScope tr(kTrStrassenPost, st);
      e = fold<float>(levels, variant, P, m, n, w, S, static_cast<float*>(C), levels >= 3, st);
    }
  } else {
    double* la = reinterpret_cast<double*>(w + S.off_ahi);
    double* lb = reinterpret_cast<double*>(w + S.off_bhi);
    double* P = reinterpret_cast<double*>(w + S.off_p);
    {
      TraceScope tr(kTrStrassenCombine, st);
      e = expand_f64(levels, variant, 0, static_cast<const double*>(A), m, k, w, S, la, st);
      if (e == cudaSuccess)
        e = expand_f64(levels, variant, 1, static_cast<const double*>(B), k, n, w, S, lb, st);
    }
    if (e == cudaSuccess) {
      if (sr == MM_SR_PLUS_TIMES_F64ACC) {
        const int rc = run_f64acc_batched(la, lb, P, S.mL, S.nL, S.kL, (int)S.leaves, w + S.off_leafws, st);
        if (rc != MM_OK) return rc;
      } else {
        e = launch_dfma_batched(la, lb, P, S.mL, S.nL, S.kL, (int)S.leaves, st);
      }
    }
    if (e == cudaSuccess) {
      TraceScope tr(kTrStrassenPost, st);
      e = fold<double>(levels, variant, P, m, n, w, S, static_cast<double*>(C), false, st);
    }
  }
  return e == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

}  // namespace mmsr

extern "C" int mm_strassen_tables(int variant, int8_t* alpha, int8_t* beta, int8_t* gamma) {
  if (variant != MM_STRASSEN_PAPER && variant != MM_STRASSEN_WINOGRAD) return MM_ERR_ARG;
  if (!alpha || !beta || !gamma) return MM_ERR_ARG;
  mmsr::strassen_tables(variant, alpha, beta, gamma);
  return MM_OK;
}
