// strassen_fused.cu -- one FP32-mode Strassen level whose operand sums are
// formed inside the leaf's own staging instead of by separate level passes
// (the "computed on the fly" operands of the SAR-Strassen lemma, Section 5).
//
// Converter warps read, for leaf r, the FP32 quadrant tiles of A and B that
// the level's coefficient tables name, add them in FP32 in the order the
// level passes use (quadrants 00, 01, 10, 11, from zero), split each sum into
// bf16 (hi, lo) and write the tensor core's K-major 64-byte-swizzled operand
// tiles straight into the shared-memory ring -- no S_r / T_r stacks in global
// memory.  An MMA warp and eight drain warps run the bf16x3 product as in the
// FP32-mode leaf (hh + hl + lh into 256-k TMEM chunks, drained with
// round-to-nearest adds), and the drain writes P_r to the product stack; the
// ordinary post-addition pass then folds the seven products into C.  Because
// the sums, the split and the k order match the materialised path, the
// result is bit-identical to it.
//
// Layout: 128 x 128 output tile per CTA, 32-wide k-blocks, six ring stages of
// 32 KB (A hi, A lo, B^T hi, B^T lo), one converter warp per stage (warp w
// converts the k-blocks congruent to w mod 6, so six k-blocks are in flight
// while each warp waits on its own loads), TMEM 2 x 128 columns.
#include <cuda_bf16.h>

#include "internal.h"
#include "strassen_tables.cuh"
#include "tcgen05.cuh"

namespace mmsr {
namespace {

__device__ int g_fused_status;

constexpr int FBM = 128, FBN = 128, FBK = 32, FSTAGES = 6, FCHUNK = 8;
constexpr int kConv = FSTAGES, kFDrain = 8;
constexpr int kFThreads = 32 * (1 + kConv + kFDrain);
constexpr uint32_t FA_BYTES = FBM * FBK * 2, FB_BYTES = FBN * FBK * 2;
constexpr uint32_t FSTAGE = 2 * FA_BYTES + 2 * FB_BYTES;
constexpr size_t FSMEM = 1024 + (size_t)FSTAGES * FSTAGE + 256;
constexpr uint32_t FTMEM_COLS = 2 * FBN;
static_assert(FSMEM <= 232448, "shared memory of one CTA");

// Byte offset of 16-byte chunk c (eight bf16 of k) of row r in a tile of
// 64-byte rows with the 64-byte swizzle the MMA descriptors name: the chunk
// index is XORed with address bits 7-8, i.e. with (r >> 1) & 3.
__device__ __forceinline__ uint32_t sw64(int r, int c) { return (uint32_t)(r * 64 + 16 * (c ^ ((r >> 1) & 3))); }

// hi / lo bf16 of eight FP32 sums, as two 16-byte words.
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    h[e] = __float2bfloat16_rn(x[e]);
    l[e] = __float2bfloat16_rn(x[e] - __bfloat162float(h[e]));
  }
  hi = *reinterpret_cast<const uint4*>(h);
  lo = *reinterpret_cast<const uint4*>(l);
}

template <int VARIANT>
__global__ void __launch_bounds__(kFThreads, 1)
    fused_leaf_kernel(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ P, int64_t h,
                      int64_t w, int64_t kh, int64_t lda, int64_t ldb) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + FSTAGES * FSTAGE);
  uint64_t* empty = full + FSTAGES;
  uint64_t* acc_full = empty + FSTAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* quiesce = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(quiesce + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.z;  // leaf (product) index
  const int64_t i0 = (int64_t)blockIdx.y * FBM, j0 = (int64_t)blockIdx.x * FBN;
  const int nkb = (int)(kh / FBK);
  const int nchunks = (nkb + FCHUNK - 1) / FCHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < FSTAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kFDrain);
    }
    tc::mbar_init(quiesce, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, FTMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f16(FBM, FBN, 1);
      bool aborted = false;
      for (int c = 0; c < nchunks && !aborted; ++c) {
        const int b = c & 1;
        if (c >= 2 && !tc::mbar_wait(&acc_empty[b], ((c >> 1) - 1) & 1u, abort_flag, &g_fused_status)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(b * FBN);
        const int last = min(nkb, (c + 1) * FCHUNK);
        for (int kb = c * FCHUNK; kb < last; ++kb) {
          const int s = kb % FSTAGES;
          if (!tc::mbar_wait(&full[s], (uint32_t)(kb / FSTAGES) & 1u, abort_flag, &g_fused_status)) {
            aborted = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t base = smem_u32(smem + s * FSTAGE);
#pragma unroll
          for (int kk = 0; kk < FBK / 16; ++kk) {
            const uint64_t ahi = tc::desc_sw64(base + kk * 32);
            const uint64_t alo = tc::desc_sw64(base + FA_BYTES + kk * 32);
            const uint64_t bhi = tc::desc_sw64(base + 2 * FA_BYTES + kk * 32);
            const uint64_t blo = tc::desc_sw64(base + 2 * FA_BYTES + FB_BYTES + kk * 32);
            tc::mma_f16(d, ahi, bhi, idesc, (kb == c * FCHUNK && kk == 0) ? 0u : 1u);
            tc::mma_f16(d, ahi, blo, idesc, 1);
            tc::mma_f16(d, alo, bhi, idesc, 1);
          }
          tc::mma_commit(&empty[s]);  // the converter may refill the stage once these finish
        }
        if (aborted) break;  // no chunk signal: the drain must not read a partial chunk
        tc::mma_commit(&acc_full[b]);
      }
    }
  } else if (warp <= kConv) {
    // -------------------------------------------- converters (one per stage)
    const int s = warp - 1;
    uint8_t* st = smem + s * FSTAGE;
    for (int kb = s, round = 0; kb < nkb; kb += FSTAGES, ++round) {
      if (round > 0 &&
          !__all_sync(0xffffffffu, tc::mbar_wait(&empty[s], (uint32_t)(round - 1) & 1u, abort_flag, &g_fused_status)))
        break;
      const int64_t k0 = (int64_t)kb * FBK;
      // S_r tile (128 rows x 32 k): item = (row, 8-k chunk), 16 per lane
#pragma unroll 2
      for (int i = 0; i < 16; ++i) {
        const int item = lane + 32 * i, row = item >> 2, c = item & 3;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cf = coef_alpha(VARIANT, r, q);
          if (cf == 0) continue;
          const float* src = A + ((q >> 1) * h + i0 + row) * lda + (q & 1) * kh + k0 + c * 8;
          const float4 u = *reinterpret_cast<const float4*>(src);
          const float4 v = *reinterpret_cast<const float4*>(src + 4);
          const float y[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 8; ++e) x[e] = apply(cf, x[e], y[e]);
        }
        uint4 hv, lv;
        split8(x, hv, lv);
        *reinterpret_cast<uint4*>(st + sw64(row, c)) = hv;
        *reinterpret_cast<uint4*>(st + FA_BYTES + sw64(row, c)) = lv;
      }
      // T_r^T tile (128 n-rows x 32 k): lane takes columns lane + 32 e, one
      // 8-k chunk at a time (loads along n are warp-coalesced)
#pragma unroll 1
      for (int e = 0; e < 4; ++e) {
        const int nrow = lane + 32 * e;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          float x[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) x[t] = 0.f;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int cf = coef_beta(VARIANT, r, q);
            if (cf == 0) continue;
            const float* src = B + ((q >> 1) * kh + k0 + c * 8) * ldb + (q & 1) * w + j0 + nrow;
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = apply(cf, x[t], src[t * ldb]);
          }
          uint4 hv, lv;
          split8(x, hv, lv);
          *reinterpret_cast<uint4*>(st + 2 * FA_BYTES + sw64(nrow, c)) = hv;
          *reinterpret_cast<uint4*>(st + 2 * FA_BYTES + FB_BYTES + sw64(nrow, c)) = lv;
        }
      }
      // the generic-proxy stores must be visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full[s]);
    }
  } else {
    // ------------------------------------------------------------ drain
    // a warp reads only its own TMEM lane quarter, warp % 4; the first four
    // drain warps take columns 0..63, the next four columns 64..127
    const int dw = warp - 1 - kConv;  // 0..7
    const int q = warp & 3, half = dw >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float sum[FBN / 2];
#pragma unroll
    for (int e = 0; e < FBN / 2; ++e) sum[e] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int b = c & 1;
      ok = __all_sync(0xffffffffu, tc::mbar_wait(&acc_full[b], (c >> 1) & 1u, abort_flag, &g_fused_status));
      tc::fence_after_sync();
#pragma unroll
      for (int cc = 0; cc < FBN / 2; cc += 32) {
        uint32_t rr[32];
        tc::tmem_ld_32x32b_x32(tmem + lane_base + (uint32_t)(b * FBN + half * (FBN / 2) + cc), rr);
        tc::tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 32; ++e) sum[cc + e] = __fadd_rn(sum[cc + e], __uint_as_float(rr[e]));
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
    }
    const int64_t row = i0 + q * 32 + lane;
    float* dst = P + (int64_t)r * h * w + row * w + j0 + half * (FBN / 2);
#pragma unroll
    for (int e = 0; e < FBN / 2; e += 4)
      *reinterpret_cast<float4*>(dst + e) =
          ok ? make_float4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(abort_flag)) {
    // Aborted: every product the issuer started lands before TMEM is freed
    // (the converters' stores are synchronous).
    if (warp == 0 && lane == 0) {
      tc::mma_commit(quiesce);
      tc::mbar_wait_quiesce(quiesce, 0);
    }
    __syncwarp();
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, FTMEM_COLS);
  }
}

}  // namespace

bool strassen_fused_shape_ok(int64_t m, int64_t n, int64_t k) {
  return m % (2 * FBM) == 0 && n % (2 * FBN) == 0 && k % (2 * FBK) == 0 && k > 0;
}

// Leaf products P_r (7 stacked (m/2) x (n/2) FP32 matrices at P) of one
// level with the operand sums formed in the staging; A is m x k (pitch lda),
// B is k x n (pitch ldb).
cudaError_t launch_strassen_fused_leaves(int variant, const float* A, const float* B, float* P, int64_t m, int64_t n,
                                         int64_t k, int64_t lda, int64_t ldb, cudaStream_t st) {
  static std::atomic<uint64_t> conf0{0}, conf1{0};
  MMSR_CUDA_TRY(smem_limit_once(fused_leaf_kernel<0>, FSMEM, conf0));
  MMSR_CUDA_TRY(smem_limit_once(fused_leaf_kernel<1>, FSMEM, conf1));
  const int64_t h = m / 2, w = n / 2, kh = k / 2;
  dim3 grid((unsigned)(w / FBN), (unsigned)(h / FBM), 7);
  TraceScope tr(kTrTcBf16x3, st);
  if (variant == 0)
    fused_leaf_kernel<0><<<grid, kFThreads, FSMEM, st>>>(A, B, P, h, w, kh, lda, ldb);
  else
    fused_leaf_kernel<1><<<grid, kFThreads, FSMEM, st>>>(A, B, P, h, w, kh, lda, ldb);
  return cudaGetLastError();
}

int read_fused_status(int* status) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_fused_status, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_fused_status, &zero, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  *status = v;
  return MM_OK;
}

}  // namespace mmsr
