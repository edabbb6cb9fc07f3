// tc_bf16.cu -- FP32-mode (+,x) on tcgen05 tensor cores: each FP32 operand
// is split into a bf16 pair (hi, lo) and C = A_hi B_hi + A_hi B_lo + A_lo B_hi
// is accumulated in FP32 (the lo*lo term, ~2^-16 relative, is dropped).
//
// Leaf = the paper's base-kernel (Section 3) as a 128 x BN output tile of
// one CTA: a TMA producer thread streams 64-wide k-blocks of the four split
// operands into a STAGES-deep shared-memory ring, a single thread issues the
// tcgen05.mma instructions into short chunk accumulators in tensor memory,
// and eight drain warps add each finished chunk into FP32 registers and
// finally write the tile to global memory.  Split-K slices (the budgeted k-parallel CO3/SAR
// form, Figs. mm-n3, sar-mm) write FP32 partials that a fixed-order sum
// folds into C.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"
#include "tcgen05.cuh"

namespace mmsr {

namespace {
__device__ int g_tc_status;  // device status word of this translation unit
// One-shot test switch: when set, the first CTA of the next GEMM launch skips
// the arrival and loads of its first ring stage, so its MMA wait runs out
// (the bounded-wait timeout path, exercised without any fault).
__device__ int g_tc_skip_signal;
}

// ------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

cudaError_t make_tmap_2d_16bit(CUtensorMap* map, const void* base, int64_t rows, int64_t cols,
                               int64_t ld, int box_rows, bool bf16, int box_cols) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : (box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

constexpr int BM = 128, BK = 64;  // BK: k alignment of the split operands

// GEMM k-block (64: 128-byte swizzled rows, 32: 64-byte rows), ring depth
// and TMEM chunk length (in k-blocks).  Measured at n = 8192 / 16384: 32-wide
// blocks in a 4-deep ring beat 64-wide blocks in a 2-deep ring (the ring
// hides three blocks of TMA latency instead of one), and 256-k chunks beat
// 128-k chunks (fewer drain handshakes) at 4.52e-6 vs 4.46e-6 error; chunks
// of 512 k / 1024 k gain ~1-2% more but raise the error to 4.8e-6 / 5.6e-6.
#ifndef MMSR_TC_BK
#define MMSR_TC_BK 32
#endif
#ifndef MMSR_TC_STAGES
#define MMSR_TC_STAGES 4
#endif
#ifndef MMSR_TC_CHUNK
#define MMSR_TC_CHUNK 8
#endif
constexpr int kTcBK = MMSR_TC_BK;
static_assert(BK % kTcBK == 0, "the GEMM k-block must divide the operand k alignment");

// ----------------------------------------------------------- split kernels
__device__ __forceinline__ void split1(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));  // exact difference in fp32
}

// X (rows x cols fp32, row-major) -> hi, lo (rows x ld bf16), zero padded.
__global__ void __launch_bounds__(256) split_rows_kernel(const float* __restrict__ X, int64_t rows,
                                                         int64_t cols, int64_t ld,
                                                         __nv_bfloat16* __restrict__ hi,
                                                         __nv_bfloat16* __restrict__ lo, bool vec) {
  const int64_t cpr = ld / 8;
  const int64_t total = rows * cpr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const int64_t r = idx / cpr, c8 = (idx - r * cpr) * 8;
    float v[8];
    const float* src = X + r * cols + c8;
    if (vec && c8 + 8 <= cols) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(src));
      const float4 b = __ldcs(reinterpret_cast<const float4*>(src) + 1);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (c8 + e < cols) ? src[e] : 0.f;
    }
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split1(v[e], h[e], l[e]);
    *reinterpret_cast<uint4*>(hi + r * ld + c8) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo + r * ld + c8) = *reinterpret_cast<const uint4*>(l);
  }
}

// B (k x n fp32, row-major) -> hiT, loT (n x ld bf16): transposed so both
// MMA operands are K-major.  Tile: 64 k x 64 n through shared memory (256-byte
// row segments read, 128-byte row segments written); the blocks of one grid
// row walk the n-tiles with stride gridDim.y.
__global__ void __launch_bounds__(256) split_transpose_kernel(const float* __restrict__ Bm,
                                                              int64_t k, int64_t n, int64_t ld,
                                                              __nv_bfloat16* __restrict__ hiT,
                                                              __nv_bfloat16* __restrict__ loT) {
  __shared__ float tile[64][65];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t k0 = (int64_t)blockIdx.x * 64;
  for (int64_t n0 = (int64_t)blockIdx.y * 64; n0 < n; n0 += (int64_t)gridDim.y * 64) {
    __syncthreads();  // the previous n-tile's readers are done with `tile`
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int kk = ty + 4 * i;
      const int64_t gk = k0 + kk, gn = n0 + tx;
      tile[kk][tx] = (gk < k && gn < n) ? __ldcs(Bm + gk * n + gn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int item = threadIdx.x + 256 * h;
      const int row = item >> 3, chunk = item & 7;
      const int64_t gn = n0 + row;
      if (gn < n) {
        __align__(16) __nv_bfloat16 hv[8], lv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) split1(tile[chunk * 8 + e][row], hv[e], lv[e]);
        *reinterpret_cast<uint4*>(hiT + gn * ld + k0 + chunk * 8) = *reinterpret_cast<const uint4*>(hv);
        *reinterpret_cast<uint4*>(loT + gn * ld + k0 + chunk * 8) = *reinterpret_cast<const uint4*>(lv);
      }
    }
  }
}

// ------------------------------------------------------------ GEMM kernel
// Warp roles (320 threads): warp 0 = TMA producer, warp 1 = MMA issuer (and
// TMEM owner), warps 2..9 = drain/epilogue.  The tensor core's FP32
// accumulation over long chains is biased (its relative error grows with the
// chain length), so the k-loop is cut into chunks of CHUNK k-blocks: each
// chunk accumulates in one of two TMEM buffers while the drain warps add the
// other, finished chunk into FP32 registers with round-to-nearest adds.  The
// chain inside TMEM is then at most CHUNK*BK/16*3 MMAs long, whatever k is.
constexpr int kDrainWarps = 8;
constexpr int kGroupM = 16;  // tile rows per rasterisation band
constexpr int kTcThreads = 64 + 32 * kDrainWarps;

// Shared-memory descriptor for a K-major tile whose rows are KB bf16 wide.
template <int KB>
__device__ __forceinline__ uint64_t desc_kb(uint32_t saddr) {
  return KB == 64 ? tc::desc_sw128(saddr) : tc::desc_sw64(saddr);
}

template <int BN, int STAGES>
struct Bf16x3Cfg {
  static constexpr int KB = kTcBK;
  static constexpr uint32_t A_BYTES = BM * KB * 2;
  static constexpr uint32_t B_BYTES = BN * KB * 2;
  static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 256;
  static constexpr uint32_t TMEM_COLS = 2 * BN;  // double-buffered chunk accumulator
  static constexpr int COLS_PER_WARP = BN / 2;   // two drain warps share each lane quarter
};

// QUAD epilogue: instead of writing its tile to C, batch entry b multiplies
// the stacked operands of leaf[b] and adds sign[b][d] x tile into up to four
// destinations dst[b][d] (row pitch ld), overwriting where add[b][d] is 0 --
// the leaf epilogue of Strassen levels whose products go straight into the
// blocks of C (no product temporaries).  Entries of one launch must write
// disjoint destinations.
template <int BN, int STAGES, int CHUNK, bool QUAD>
__global__ void __launch_bounds__(kTcThreads, 1)
    bf16x3_gemm_kernel(const __grid_constant__ CUtensorMap tAhi, const __grid_constant__ CUtensorMap tAlo,
                       const __grid_constant__ CUtensorMap tBhi, const __grid_constant__ CUtensorMap tBlo,
                       float* __restrict__ C, float* __restrict__ W, int64_t m, int64_t n,
                       int kb_total, int kb_per_slice, int slices, int64_t a_batch_rows,
                       int64_t b_batch_rows, int64_t c_batch_stride, const __grid_constant__ QuadOut quad) {
  using Cfg = Bf16x3Cfg<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;  // [2]: chunk accumulated (MMA -> drain)
  uint64_t* acc_empty = acc_full + 2;   // [2]: chunk drained (drain -> MMA)
  uint64_t* quiesce = acc_empty + 2;    // after an abort: all issued MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(quiesce + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  // producer state read after an abort (shared, so that no register stays
  // live through the other roles): [0] k-blocks issued, [1] k-block 0 skipped
  int* prod_state = abort_flag + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Grouped rasterisation: consecutive CTAs walk a band of kGroupM tile rows
  // column by column, so a wave shares its A and B panels through L2 instead
  // of streaming all of B once per band of rows.
  int64_t i0, j0;
  {
    const int tiles_n = gridDim.x, units_m = gridDim.y, band_h = kGroupM;
    const int pid = blockIdx.y * tiles_n + blockIdx.x;
    const int band = pid / (band_h * tiles_n);
    const int first_m = band * band_h;
    const int rows = min(band_h, units_m - first_m);
    const int in_band = pid - band * band_h * tiles_n;
    i0 = (int64_t)(first_m + in_band % rows) * BM;
    j0 = (int64_t)(in_band / rows) * BN;
  }
  // blockIdx.z = batch * slices + k-slice; a batch is one independent product
  // whose operands sit at row offset batch * {a,b}_batch_rows of the stacks
  const int z = blockIdx.z % slices;
  const int batch = blockIdx.z / slices;
  const int64_t leaf = QUAD ? (int64_t)quad.leaf[batch] : (int64_t)batch;  // stacked operands of this entry
  const int ya = (int)(leaf * a_batch_rows + i0), yb = (int)(leaf * b_batch_rows + j0);
  const int kb_begin = z * kb_per_slice;
  const int kb_end = min(kb_total, kb_begin + kb_per_slice);
  const int nkb = kb_end > kb_begin ? kb_end - kb_begin : 0;
  const int nchunks = (nkb + CHUNK - 1) / CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kDrainWarps);
    }
    tc::mbar_init(quiesce, 1);
    *abort_flag = 0;
    prod_state[0] = prod_state[1] = 0;
    tc::mbar_init_fence();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      tc::tma_prefetch(&tAhi);
      tc::tma_prefetch(&tAlo);
      tc::tma_prefetch(&tBhi);
      tc::tma_prefetch(&tBlo);
      bool skipped = false;  // the test switch took k-block 0 out
      int issued = 0;        // k-blocks whose loads were issued
      if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && nkb > 0)
        skipped = atomicExch(&g_tc_skip_signal, 0) != 0;
      for (int it = 0; it < nkb; ++it, issued = it) {
        const int s = it % STAGES;
        const uint32_t round = (uint32_t)(it / STAGES);
        if (it >= STAGES && !tc::mbar_wait(&empty[s], (round - 1) & 1u, abort_flag, &g_tc_status)) break;
        if (it == 0 && skipped) continue;
        tc::mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
        uint8_t* st = smem + s * Cfg::STAGE_BYTES;
        const int kx = (kb_begin + it) * Cfg::KB;
        tc::tma_load_2d(st, &tAhi, &full[s], kx, ya);
        tc::tma_load_2d(st + Cfg::A_BYTES, &tAlo, &full[s], kx, ya);
        tc::tma_load_2d(st + 2 * Cfg::A_BYTES, &tBhi, &full[s], kx, yb);
        tc::tma_load_2d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, &tBlo, &full[s], kx, yb);
      }
      prod_state[0] = issued;
      prod_state[1] = skipped ? 1 : 0;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f16(BM, BN, 1);
      int it = 0;
      for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        if (c >= 2 && !tc::mbar_wait(&acc_empty[b], ((c >> 1) - 1) & 1u, abort_flag, &g_tc_status)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(b * BN);
        const int last = min(nkb, (c + 1) * CHUNK);
        bool aborted = false;
        for (int first = 1; it < last; ++it, first = 0) {
          const int s = it % STAGES;
          const uint32_t round = (uint32_t)(it / STAGES);
          if (!tc::mbar_wait(&full[s], round & 1u, abort_flag, &g_tc_status)) { aborted = true; break; }
          tc::fence_after_sync();
          const uint32_t base = smem_u32(smem + s * Cfg::STAGE_BYTES);
#pragma unroll
          for (int kk = 0; kk < Cfg::KB / 16; ++kk) {
            const uint64_t ahi = desc_kb<Cfg::KB>(base + kk * 32);
            const uint64_t alo = desc_kb<Cfg::KB>(base + Cfg::A_BYTES + kk * 32);
            const uint64_t bhi = desc_kb<Cfg::KB>(base + 2 * Cfg::A_BYTES + kk * 32);
            const uint64_t blo = desc_kb<Cfg::KB>(base + 2 * Cfg::A_BYTES + Cfg::B_BYTES + kk * 32);
            tc::mma_f16(d, ahi, bhi, idesc, (first && kk == 0) ? 0u : 1u);
            tc::mma_f16(d, ahi, blo, idesc, 1);
            tc::mma_f16(d, alo, bhi, idesc, 1);
          }
          tc::mma_commit(&empty[s]);
        }
        if (aborted) break;  // no chunk signal: the drain must not read a partial chunk
        tc::mma_commit(&acc_full[b]);
      }
    }
  } else {
    // drain warps: lane quarter = warp % 4, column half = (warp - 2) / 4
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float sum[Cfg::COLS_PER_WARP];
#pragma unroll
    for (int e = 0; e < Cfg::COLS_PER_WARP; ++e) sum[e] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int b = c & 1;
      // warp-uniform verdict: the TMEM loads below are warp-collective (after
      // an abort they read a discarded chunk; the tile is written as zeros)
      ok = __all_sync(0xffffffffu, tc::mbar_wait(&acc_full[b], (c >> 1) & 1u, abort_flag, &g_tc_status));
      tc::fence_after_sync();
#pragma unroll
      for (int cc = 0; cc < Cfg::COLS_PER_WARP; cc += 32) {
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tmem + lane_base + (uint32_t)(b * BN + half * Cfg::COLS_PER_WARP + cc), r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 32; ++e) sum[cc + e] = __fadd_rn(sum[cc + e], __uint_as_float(r[e]));
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
    }
    float* out = (z == 0) ? C + (int64_t)batch * c_batch_stride : W + (int64_t)(z - 1) * m * n;
    const int64_t row = i0 + q * 32 + lane;
    if constexpr (QUAD) {
      if (row < m) {
      const int64_t c0 = j0 + half * Cfg::COLS_PER_WARP;
      const int64_t cols_left = n - c0;
      if (!ok) {
#pragma unroll
        for (int e = 0; e < Cfg::COLS_PER_WARP; ++e) sum[e] = 0.f;
      }
#pragma unroll 1
      for (int d = 0; d < 4; ++d) {
        float* base = quad.dst[batch][d];
        if (base == nullptr) continue;
        const float sg = (float)quad.sign[batch][d];
        const bool add = quad.add[batch][d] != 0;
        float* dst = base + row * quad.ld + c0;
        if ((quad.ld % 4 == 0) && aligned16(base) && cols_left >= Cfg::COLS_PER_WARP) {
          // four 16-byte reads in flight per round trip, then their stores
#pragma unroll
          for (int e0 = 0; e0 < Cfg::COLS_PER_WARP; e0 += 16) {
            float4 o[4];
            if (add) {
#pragma unroll
              for (int u = 0; u < 4; ++u) o[u] = *reinterpret_cast<const float4*>(dst + e0 + 4 * u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int e = e0 + 4 * u;
              float4 v = make_float4(sg * sum[e], sg * sum[e + 1], sg * sum[e + 2], sg * sum[e + 3]);
              if (add) {
                v.x = __fadd_rn(o[u].x, v.x); v.y = __fadd_rn(o[u].y, v.y);
                v.z = __fadd_rn(o[u].z, v.z); v.w = __fadd_rn(o[u].w, v.w);
              }
              *reinterpret_cast<float4*>(dst + e) = v;
            }
          }
        } else {
#pragma unroll
          for (int e = 0; e < Cfg::COLS_PER_WARP; ++e)
            if (e < cols_left) dst[e] = add ? __fadd_rn(dst[e], sg * sum[e]) : sg * sum[e];
        }
      }
      }
    } else if (row < m) {
      const int64_t c0 = j0 + half * Cfg::COLS_PER_WARP;
      float* dst = out + row * n + c0;
      const int64_t cols_left = n - c0;
      if (!ok) {
#pragma unroll
        for (int e = 0; e < Cfg::COLS_PER_WARP; ++e) sum[e] = 0.f;
      }
      if ((n % 4 == 0) && cols_left >= Cfg::COLS_PER_WARP) {
#pragma unroll
        for (int e = 0; e < Cfg::COLS_PER_WARP; e += 4)
          *reinterpret_cast<float4*>(dst + e) = make_float4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < Cfg::COLS_PER_WARP; ++e)
          if (e < cols_left) dst[e] = sum[e];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(abort_flag)) {
    // Aborted: before shared memory and TMEM are released, let this CTA's
    // own asynchronous work land -- the TMA loads of the last ring round the
    // producer issued and every MMA the issuer started.  Both waits are
    // bounded and ignore the abort flag.
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
    tc::tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// ------------------------------------------------------------ stream-K
// The zero-temporary k-parallel form of Fig. tar-mm for the FP32 mode, as a
// data-parallel + stream-K hybrid.  One persistent CTA per SM first takes
// whole tiles cta, cta + P, ... below dp_tiles: those waves run in lockstep,
// so CTAs at the same k-block share their operand panels through L2.  The
// units (128 x BN tile, k-block) of the tiles left over are then split into
// equal contiguous ranges over the first P_sk CTAs.  The three roles walk the
// same sequence of segments (the part of one tile inside the CTA's work);
// the ring of operand stages and the two TMEM chunk buffers keep running
// phase counters across segments.  A segment that is a whole tile goes to C;
// a partial one is stored in one of the CTA's two slots (its first or its
// last stream-K segment -- the p b^2 temporaries), and the CTA that
// completes a tile's counter folds the slots in k order and writes C.
// Nothing waits on another CTA, and the fold order is fixed, so results
// repeat exactly.
__device__ __forceinline__ int64_t skf_begin(int64_t c, int64_t total, int P) { return total * c / P; }
__device__ __forceinline__ int skf_owner(int64_t i, int64_t total, int P) {
  int64_t c = i * P / total;
  while (c + 1 < P && skf_begin(c + 1, total, P) <= i) ++c;
  while (c > 0 && skf_begin(c, total, P) > i) --c;
  return (int)c;
}
// Next segment of [it, end): tile t, k-blocks [j0, j1); advances it.
__device__ __forceinline__ bool skf_next(int64_t& it, int64_t end, int64_t kbt, int64_t& t, int64_t& j0,
                                         int64_t& j1) {
  if (it >= end) return false;
  t = it / kbt;
  j0 = it - t * kbt;
  j1 = min(kbt, j0 + (end - it));
  it = t * kbt + j1;
  return true;
}
// One CTA's walk: its whole tiles (stride P below dp_end), then its
// stream-K range [it, end) of units.
struct SkfWalk {
  int64_t dp, dp_end, it, end;
  int P;
  __device__ __forceinline__ bool next(int64_t kbt, int64_t& t, int64_t& j0, int64_t& j1) {
    if (dp < dp_end) {
      t = dp;
      j0 = 0;
      j1 = kbt;
      dp += P;
      return true;
    }
    return skf_next(it, end, kbt, t, j0, j1);
  }
};

template <int BN, int STAGES, int CHUNK>
__global__ void __launch_bounds__(kTcThreads, 1)
    bf16x3_streamk_kernel(const __grid_constant__ CUtensorMap tAhi, const __grid_constant__ CUtensorMap tAlo,
                          const __grid_constant__ CUtensorMap tBhi, const __grid_constant__ CUtensorMap tBlo,
                          float* __restrict__ C, float* __restrict__ slots, int* __restrict__ counters, int64_t m,
                          int64_t n, int64_t tiles_n, int64_t kbt, int64_t dp_tiles, int64_t sk_total, int P,
                          int P_sk) {
  using Cfg = Bf16x3Cfg<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* quiesce = acc_empty + 2;
  // drain-warp rendezvous of a partial tile (bounded waits, unlike a named
  // barrier): every drain warp has stored its slot rows / the verdict is out
  uint64_t* seg_stored = quiesce + 1;
  uint64_t* seg_decided = seg_stored + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(seg_decided + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* prod_state = abort_flag + 1;  // [0] k-blocks issued
  int* fold = prod_state + 2;        // [0] last arriver, [1] first contributor, [2] last contributor
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cta = blockIdx.x;
  // stream-K units are numbered from the first tile after the whole-tile
  // waves; CTAs from P_sk on have no stream-K range
  const int64_t sk_base = dp_tiles * kbt;
  const int64_t begin = cta < P_sk ? sk_base + skf_begin(cta, sk_total, P_sk) : sk_base;
  const int64_t end = cta < P_sk ? sk_base + skf_begin(cta + 1, sk_total, P_sk) : sk_base;
  const SkfWalk walk0{cta, dp_tiles, begin, end, P};

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kDrainWarps);
    }
    tc::mbar_init(quiesce, 1);
    tc::mbar_init(seg_stored, kDrainWarps);
    tc::mbar_init(seg_decided, 1);
    *abort_flag = 0;
    prod_state[0] = 0;
    tc::mbar_init_fence();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      tc::tma_prefetch(&tAhi);
      tc::tma_prefetch(&tAlo);
      tc::tma_prefetch(&tBhi);
      tc::tma_prefetch(&tBlo);
      SkfWalk walk = walk0;
      int64_t t, j0, j1;
      uint32_t g = 0;  // k-blocks issued so far (ring position)
      bool stop = false;
      while (!stop && walk.next(kbt, t, j0, j1)) {
        const int ya = (int)((t / tiles_n) * BM), yb = (int)((t % tiles_n) * BN);
        for (int64_t j = j0; j < j1; ++j, ++g) {
          const int s = (int)(g % STAGES);
          const uint32_t round = g / STAGES;
          if (g >= STAGES && !tc::mbar_wait(&empty[s], (round - 1) & 1u, abort_flag, &g_tc_status)) {
            stop = true;
            break;
          }
          tc::mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
          uint8_t* st = smem + s * Cfg::STAGE_BYTES;
          const int kx = (int)(j * Cfg::KB);
          tc::tma_load_2d(st, &tAhi, &full[s], kx, ya);
          tc::tma_load_2d(st + Cfg::A_BYTES, &tAlo, &full[s], kx, ya);
          tc::tma_load_2d(st + 2 * Cfg::A_BYTES, &tBhi, &full[s], kx, yb);
          tc::tma_load_2d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, &tBlo, &full[s], kx, yb);
        }
      }
      prod_state[0] = (int)g;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f16(BM, BN, 1);
      SkfWalk walk = walk0;
      int64_t t, j0, j1;
      uint32_t g = 0, gc = 0;  // k-blocks and chunks consumed so far
      bool aborted = false;
      while (!aborted && walk.next(kbt, t, j0, j1)) {
        for (int64_t cs = j0; cs < j1 && !aborted; cs += CHUNK, ++gc) {
          const int b = (int)(gc & 1);
          if (gc >= 2 && !tc::mbar_wait(&acc_empty[b], ((gc >> 1) - 1) & 1u, abort_flag, &g_tc_status)) {
            aborted = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t d = tmem + (uint32_t)(b * BN);
          const int64_t ce = min(j1, cs + CHUNK);
          for (int64_t j = cs; j < ce; ++j, ++g) {
            const int s = (int)(g % STAGES);
            if (!tc::mbar_wait(&full[s], (g / STAGES) & 1u, abort_flag, &g_tc_status)) {
              aborted = true;
              break;
            }
            tc::fence_after_sync();
            const uint32_t base = smem_u32(smem + s * Cfg::STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < Cfg::KB / 16; ++kk) {
              const uint64_t ahi = desc_kb<Cfg::KB>(base + kk * 32);
              const uint64_t alo = desc_kb<Cfg::KB>(base + Cfg::A_BYTES + kk * 32);
              const uint64_t bhi = desc_kb<Cfg::KB>(base + 2 * Cfg::A_BYTES + kk * 32);
              const uint64_t blo = desc_kb<Cfg::KB>(base + 2 * Cfg::A_BYTES + Cfg::B_BYTES + kk * 32);
              tc::mma_f16(d, ahi, bhi, idesc, (j == cs && kk == 0) ? 0u : 1u);
              tc::mma_f16(d, ahi, blo, idesc, 1);
              tc::mma_f16(d, alo, bhi, idesc, 1);
            }
            tc::mma_commit(&empty[s]);
          }
          if (aborted) break;  // no chunk signal: the drain must not read a partial chunk
          tc::mma_commit(&acc_full[b]);
        }
      }
    }
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int tr = q * 32 + lane;  // tile row of this thread
    const int tcol = half * Cfg::COLS_PER_WARP;
    SkfWalk walk = walk0;
    int64_t t, j0, j1;
    uint32_t gc = 0, ps = 0;  // chunks drained, partial segments met
    bool ok = true;
    while (ok && walk.next(kbt, t, j0, j1)) {
      float sum[Cfg::COLS_PER_WARP];
#pragma unroll
      for (int e = 0; e < Cfg::COLS_PER_WARP; ++e) sum[e] = 0.f;
      for (int64_t cs = j0; cs < j1 && ok; cs += CHUNK, ++gc) {
        const int b = (int)(gc & 1);
        ok = __all_sync(0xffffffffu, tc::mbar_wait(&acc_full[b], (gc >> 1) & 1u, abort_flag, &g_tc_status));
        if (!ok) break;
        tc::fence_after_sync();
#pragma unroll
        for (int cc = 0; cc < Cfg::COLS_PER_WARP; cc += 32) {
          uint32_t r[32];
          tc::tmem_ld_32x32b_x32(tmem + lane_base + (uint32_t)(b * BN + tcol + cc), r);
          tc::tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; ++e) sum[cc + e] = __fadd_rn(sum[cc + e], __uint_as_float(r[e]));
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
      }
      if (!ok) break;
      const int64_t row = (t / tiles_n) * BM + tr, c0 = (t % tiles_n) * BN + tcol;
      const int64_t cols_left = n - c0;
      if (j0 == 0 && j1 == kbt) {
        if (row < m) {
          float* dst = C + row * n + c0;
          if ((n % 4 == 0) && cols_left >= Cfg::COLS_PER_WARP) {
#pragma unroll
            for (int e = 0; e < Cfg::COLS_PER_WARP; e += 4)
              *reinterpret_cast<float4*>(dst + e) = make_float4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < Cfg::COLS_PER_WARP; ++e)
              if (e < cols_left) dst[e] = sum[e];
          }
        }
        continue;
      }
      // partial tile: this CTA's slot (0: its first stream-K segment, 1: its
      // last), stored thread-major (float4 i of drain thread d at i * 256 + d)
      // so that every warp-wide store and load is 512 contiguous bytes
      const int mine = (t * kbt + j0 == begin) ? 0 : 1;
      const int dt = threadIdx.x - 2 * 32;  // drain thread 0..255
      float4* slot = reinterpret_cast<float4*>(slots + ((int64_t)cta * 2 + mine) * (BM * BN)) + dt;
#pragma unroll
      for (int e = 0; e < Cfg::COLS_PER_WARP; e += 4)
        __stcg(slot + (e / 4) * (kDrainWarps * 32), make_float4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3]));
      __threadfence();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(seg_stored);
      ok = __all_sync(0xffffffffu, tc::mbar_wait(seg_stored, ps & 1u, abort_flag, &g_tc_status));
      if (!ok) break;
      if (warp == 2) {
        if (lane == 0) {
          // every drain warp's slot part is stored and fenced: count this CTA
          const int64_t u = t * kbt - sk_base;
          const int cf = skf_owner(u, sk_total, P_sk), cl = skf_owner(u + kbt - 1, sk_total, P_sk);
          fold[0] = atomicAdd(&counters[t], 1) == cl - cf;
          fold[1] = cf;
          fold[2] = cl;
          tc::mbar_arrive(seg_decided);  // release: the verdict is visible to the waiters
        }
        __syncwarp();
      }
      ok = __all_sync(0xffffffffu, tc::mbar_wait(seg_decided, ps & 1u, abort_flag, &g_tc_status));
      ++ps;
      if (!ok) break;
      if (fold[0]) {
        __threadfence();
#pragma unroll
        for (int e = 0; e < Cfg::COLS_PER_WARP; ++e) sum[e] = 0.f;
        for (int qc = fold[1]; qc <= fold[2]; ++qc) {
          const int which = ((sk_base + skf_begin(qc, sk_total, P_sk)) / kbt == t) ? 0 : 1;
          const float4* src = reinterpret_cast<const float4*>(slots + ((int64_t)qc * 2 + which) * (BM * BN)) + dt;
#pragma unroll
          for (int e0 = 0; e0 < Cfg::COLS_PER_WARP; e0 += 64) {
            float4 v[16];  // sixteen 16-byte loads in flight per thread
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = __ldcg(src + (e0 / 4 + u) * (kDrainWarps * 32));
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int e = e0 + 4 * u;
              sum[e] = __fadd_rn(sum[e], v[u].x);
              sum[e + 1] = __fadd_rn(sum[e + 1], v[u].y);
              sum[e + 2] = __fadd_rn(sum[e + 2], v[u].z);
              sum[e + 3] = __fadd_rn(sum[e + 3], v[u].w);
            }
          }
        }
        if (row < m) {
          float* dst = C + row * n + c0;
          if ((n % 4 == 0) && cols_left >= Cfg::COLS_PER_WARP) {
#pragma unroll
            for (int e = 0; e < Cfg::COLS_PER_WARP; e += 4)
              *reinterpret_cast<float4*>(dst + e) = make_float4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < Cfg::COLS_PER_WARP; ++e)
              if (e < cols_left) dst[e] = sum[e];
          }
        }
        if (threadIdx.x == 64) counters[t] = 0;
      }
      // fold[] is rewritten only after the next partial segment's
      // seg_stored completes, i.e. after every drain warp has read it here
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(abort_flag)) {
    if (warp == 0 && lane == 0) {
      const int issued = prod_state[0];
      for (int g = max(0, issued - STAGES); g < issued; ++g)
        tc::mbar_wait_quiesce(&full[g % STAGES], (uint32_t)(g / STAGES) & 1u);
    }
    if (warp == 1 && lane == 0) {
      tc::mma_commit(quiesce);
      tc::mbar_wait_quiesce(quiesce, 0);
    }
    __syncwarp();
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

__global__ void __launch_bounds__(256) sum_reduce_f32_kernel(int64_t count, float* __restrict__ C,
                                                             const float* __restrict__ W, int parts,
                                                             bool vec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    for (int64_t v = t; v < count / 4; v += stride) {
      float4 c = reinterpret_cast<const float4*>(C)[v];
      for (int p = 0; p < parts; ++p) {
        const float4 w = __ldcs(reinterpret_cast<const float4*>(W + (int64_t)p * count) + v);
        c.x += w.x; c.y += w.y; c.z += w.z; c.w += w.w;
      }
      reinterpret_cast<float4*>(C)[v] = c;
    }
  } else {
    for (int64_t e = t; e < count; e += stride) {
      float c = C[e];
      for (int p = 0; p < parts; ++p) c += W[(int64_t)p * count + e];
      C[e] = c;
    }
  }
}

template <int BN, int STAGES, int CHUNK>
cudaError_t launch_gemm(const CUtensorMap& a_hi, const CUtensorMap& a_lo, const CUtensorMap& b_hi,
                        const CUtensorMap& b_lo, float* C, float* W, int64_t m, int64_t n,
                        int kb_total, int kbs, int s, cudaStream_t st, int batches = 1,
                        int64_t a_batch_rows = 0, int64_t b_batch_rows = 0,
                        int64_t c_batch_stride = 0, const QuadOut* quad = nullptr) {
  QuadOut qo;
  if (quad) qo = *quad; else memset(&qo, 0, sizeof(qo));
  using Cfg = Bf16x3Cfg<BN, STAGES>;
  static std::atomic<uint64_t> conf_plain{0}, conf_quad{0};
  MMSR_CUDA_TRY(smem_limit_once(bf16x3_gemm_kernel<BN, STAGES, CHUNK, false>, Cfg::SMEM, conf_plain));
  MMSR_CUDA_TRY(smem_limit_once(bf16x3_gemm_kernel<BN, STAGES, CHUNK, true>, Cfg::SMEM, conf_quad));
  const bool q = qo.entries > 0;
  const unsigned tiles_m = (unsigned)((m + BM - 1) / BM), tiles_n = (unsigned)((n + BN - 1) / BN);
  TraceScope tr(kTrTcBf16x3, st);
  dim3 grid(tiles_n, tiles_m, (unsigned)(s * batches));
  if (q)
    bf16x3_gemm_kernel<BN, STAGES, CHUNK, true><<<grid, kTcThreads, Cfg::SMEM, st>>>(
        a_hi, a_lo, b_hi, b_lo, C, W, m, n, kb_total, kbs, s, a_batch_rows, b_batch_rows, c_batch_stride, qo);
  else
    bf16x3_gemm_kernel<BN, STAGES, CHUNK, false><<<grid, kTcThreads, Cfg::SMEM, st>>>(
        a_hi, a_lo, b_hi, b_lo, C, W, m, n, kb_total, kbs, s, a_batch_rows, b_batch_rows, c_batch_stride, qo);
  return cudaGetLastError();
}

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct F32Layout {
  int64_t Kp, a_bytes, b_bytes, off_alo, off_bhi, off_blo, off_part, min_bytes;
};

F32Layout f32_layout(int64_t m, int64_t n, int64_t k) {
  F32Layout L;
  L.Kp = align_up(k > 0 ? k : 1, BK);
  L.a_bytes = align_up(m * L.Kp * 2, 1024);
  L.b_bytes = align_up(n * L.Kp * 2, 1024);
  L.off_alo = L.a_bytes;
  L.off_bhi = 2 * L.a_bytes;
  L.off_blo = 2 * L.a_bytes + L.b_bytes;
  L.off_part = 2 * L.a_bytes + 2 * L.b_bytes;
  L.min_bytes = L.off_part;
  return L;
}

constexpr int kTcBN = 256, kTcStages = MMSR_TC_STAGES, kTcChunk = MMSR_TC_CHUNK;

}  // namespace

// Split an FP32 operand pair into the bf16 hi/lo layout the GEMM expects.
cudaError_t launch_split_bf16(const float* A, const float* B, int64_t m, int64_t n, int64_t k,
                              int64_t Kp, __nv_bfloat16* ahi, __nv_bfloat16* alo,
                              __nv_bfloat16* bhi, __nv_bfloat16* blo, cudaStream_t st) {
  TraceScope tr(kTrSplitBf16, st);
  const bool vec = (k % 4 == 0) && aligned16(A);
  int64_t blocks = (m * (Kp / 8) + 255) / 256;
  if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
  if (blocks < 1) blocks = 1;
  split_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, m, k, Kp, ahi, alo, vec);
  // a few thousand blocks, each walking several n-tiles
  const int64_t tiles_n = (n + 63) / 64;
  const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(tiles_n, std::max<int64_t>(1, 4096 / (Kp / 64))));
  dim3 g((unsigned)(Kp / 64), (unsigned)std::min<int64_t>(gy, kMaxGridY));
  split_transpose_kernel<<<g, 256, 0, st>>>(B, k, n, Kp, bhi, blo);
  return cudaGetLastError();
}

// `batches` independent bf16x3 products on stacked split operands:
// A stack (batches*m) x Kp, B stack (batches*n) x Kp (both K-major, hi/lo),
// output P + b*m*n (row-major m x n each).
cudaError_t launch_bf16x3_batched(const __nv_bfloat16* ahi, const __nv_bfloat16* alo,
                                  const __nv_bfloat16* bhi, const __nv_bfloat16* blo, float* P,
                                  int64_t m, int64_t n, int64_t Kp, int batches, cudaStream_t st,
                                  const QuadOut* quad, int map_batches) {
  const int64_t mb = map_batches > 0 ? map_batches : batches;
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  MMSR_CUDA_TRY(make_tmap_2d_16bit(&ta_hi, ahi, mb * m, Kp, Kp, BM, true, kTcBK));
  MMSR_CUDA_TRY(make_tmap_2d_16bit(&ta_lo, alo, mb * m, Kp, Kp, BM, true, kTcBK));
  MMSR_CUDA_TRY(make_tmap_2d_16bit(&tb_hi, bhi, mb * n, Kp, Kp, kTcBN, true, kTcBK));
  MMSR_CUDA_TRY(make_tmap_2d_16bit(&tb_lo, blo, mb * n, Kp, Kp, kTcBN, true, kTcBK));
  const int kb_total = (int)(Kp / kTcBK);
  return launch_gemm<kTcBN, kTcStages, kTcChunk>(ta_hi, ta_lo, tb_hi, tb_lo, P, nullptr, m, n,
                                                 kb_total, kb_total, 1, st, batches, m, n, m * n, quad);
}

int g_f32_streamk = 1;  // mm_set_option(MM_OPT_F32_STREAMK, ...)

// Stream-K geometry: one CTA per SM (fewer when the product has under four
// k-blocks per CTA), two BM x BN FP32 slots per CTA and one counter per tile.
// With whole waves first (MM_OPT_F32_STREAMK 3) the tiles of the whole waves
// (dp_tiles = P * floor(tiles / P)) run as plain tiles and the units of the
// tiles left over go to the first P_sk CTAs, at least eight k-blocks each,
// so that a small remainder is not split into slivers whose fold costs more
// than their products; otherwise every tile's units are split over P CTAs.
struct F32Sk {
  int64_t tiles_n, tiles, kbt, total, dp_tiles, sk_total, slot_bytes, bytes;
  int P, P_sk;
};
F32Sk f32_sk(int64_t m, int64_t n, int64_t k) {
  F32Sk g;
  g.tiles_n = (n + kTcBN - 1) / kTcBN;
  g.tiles = ((m + BM - 1) / BM) * g.tiles_n;
  g.kbt = align_up(k > 0 ? k : 1, BK) / kTcBK;
  g.total = g.tiles * g.kbt;
  int64_t P = std::min<int64_t>(num_sms(), g.total / 4);
  g.P = (int)std::max<int64_t>(P, 1);
  g.dp_tiles = g_f32_streamk == 3 ? (g.tiles / g.P) * g.P : 0;
  g.sk_total = (g.tiles - g.dp_tiles) * g.kbt;
  g.P_sk = (int)std::max<int64_t>(1, std::min<int64_t>(g.P, g.dp_tiles > 0 ? g.sk_total / 8 : g.P));
  g.slot_bytes = (int64_t)g.P * 2 * BM * kTcBN * 4;
  g.bytes = g.slot_bytes + align_up(g.tiles * 4, 256);
  return g;
}
// Shapes the stream-K form takes: one to four waves of tiles, at least eight
// k-blocks per tile.
bool f32_sk_eligible(int64_t m, int64_t n, int64_t k) {
  const F32Sk g = f32_sk(m, n, k);
  return k > 0 && g.tiles >= (int64_t)num_sms() && g.tiles < 4 * (int64_t)num_sms() && g.kbt >= 8 &&
         g.total < ((int64_t)1 << 40);
}
// The planner's rule: stream-K when the grid's last wave would be nearly
// empty.  Its ranges give up the classic grid's lockstep waves, whose CTAs
// share each k-block's operand panels through L2, and a split tile costs a
// slot store and a fold; measured against the classic grid (2048 x 256c x k,
// k = 2048 and 8192) it won only where the last wave held at most ~30% of P
// tiles after one whole wave (~15% after two) and never past three waves.
bool f32_sk_wanted(int64_t m, int64_t n, int64_t k) {
  if (g_f32_streamk == 0 || !f32_sk_eligible(m, n, k)) return false;
  if (g_f32_streamk >= 2) return true;
  const F32Sk g = f32_sk(m, n, k);
  const int64_t whole = g.tiles / g.P, rest = g.tiles - whole * g.P;
  return whole >= 1 && whole <= 2 && rest > 0 && rest * 10 * whole <= 3 * (int64_t)g.P;
}

int plan_f32(int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  const F32Layout L = f32_layout(m, n, k);
  p->tile_m = BM;
  p->tile_n = kTcBN;
  p->tile_k = kTcBK;
  p->kernel = 2;
  p->workspace_min = L.min_bytes;
  if (budget < (size_t)L.min_bytes) {
    p->split_k = 1;
    p->workspace_used = L.min_bytes;
    return MM_OK;
  }
  // A nearly empty last wave and room for the per-CTA partial tiles: the
  // stream-K form evens out the last wave.  Under one wave the same budget
  // always buys enough split-K slices to fill the GPU, and split-K is the
  // faster of the two there (its CTAs of one slice share their operands
  // through L2, stream-K's ranges spread over all of k: 1024 x 1024 x 16384
  // took 129 us in stream-K against 72 + 7 us with s = 4).
  if (f32_sk_wanted(m, n, k) && budget >= (size_t)(L.min_bytes + f32_sk(m, n, k).bytes)) {
    p->kernel = 5;
    p->split_k = 1;
    p->workspace_used = L.min_bytes + f32_sk(m, n, k).bytes;
    return MM_OK;
  }
  int s = 1, kbs = 0;
  int64_t used = 0;
  split_plan(m, n, L.Kp, kTcBK, 4, budget - (size_t)L.min_bytes, &s, &kbs, &used);
  // The budget bounds the slices; like the paper's bound of min{p, 4^d}
  // temporaries per depth (Section 4), more copies than the processors can
  // use buy nothing.  Take the s' <= s with the least modelled time: waves of
  // CTAs (ceil(s' tiles / P) of them, each 1/s' of a tile's k) plus the
  // reduction's HBM traffic.  At 1.7 waves of tiles a second slice keeps two
  // waves and only adds the reduction (measured 0.364 against 0.326 ms on
  // 2048 x 4096 x 8192), at 1.05 waves it saves a quarter.
  if (s > 1) {
    const int64_t tiles = ((m + BM - 1) / BM) * ((n + kTcBN - 1) / kTcBN);
    const double P = (double)num_sms();
    const double t_tile = 6.0 * BM * kTcBN * (double)L.Kp / 1.2e13;  // s, bf16x3 at ~1.8 PFLOP/s
    const double t_slice = (double)m * (double)n * 8.0 / 6.5e12;    // write + read back one slice
    int best = 1;
    double best_t = std::ceil((double)tiles / P) * t_tile;
    for (int c = 2; c <= s; ++c) {
      const double t = std::ceil((double)c * (double)tiles / P) / c * t_tile + (c - 1) * t_slice;
      if (t < best_t) {
        best = c;
        best_t = t;
      }
    }
    if (best < s) {
      const int64_t kb_total = L.Kp / kTcBK;
      kbs = (int)((kb_total + best - 1) / best);
      s = (int)((kb_total + kbs - 1) / kbs);
      used = (int64_t)(s - 1) * m * n * 4;
    }
  }
  p->split_k = s;
  p->workspace_used = L.min_bytes + used;
  return MM_OK;
}

int run_f32(int64_t m, int64_t n, int64_t k, const float* A, const float* B, float* C, void* ws,
            size_t ws_bytes, cudaStream_t st) {
  mm_plan_t p;
  plan_f32(m, n, k, ws_bytes, &p);
  if ((size_t)p.workspace_min > ws_bytes) return MM_ERR_WORKSPACE;
  const F32Layout L = f32_layout(m, n, k);
  uint8_t* w = static_cast<uint8_t*>(ws);
  auto* ahi = reinterpret_cast<__nv_bfloat16*>(w);
  auto* alo = reinterpret_cast<__nv_bfloat16*>(w + L.off_alo);
  auto* bhi = reinterpret_cast<__nv_bfloat16*>(w + L.off_bhi);
  auto* blo = reinterpret_cast<__nv_bfloat16*>(w + L.off_blo);
  float* part = p.split_k > 1 ? reinterpret_cast<float*>(w + L.off_part) : nullptr;
  cudaError_t e = launch_split_bf16(A, B, m, n, k, L.Kp, ahi, alo, bhi, blo, st);
  if (e != cudaSuccess) return MM_ERR_CUDA;
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  if (make_tmap_2d_16bit(&ta_hi, ahi, m, L.Kp, L.Kp, BM, true, kTcBK) != cudaSuccess ||
      make_tmap_2d_16bit(&ta_lo, alo, m, L.Kp, L.Kp, BM, true, kTcBK) != cudaSuccess ||
      make_tmap_2d_16bit(&tb_hi, bhi, n, L.Kp, L.Kp, kTcBN, true, kTcBK) != cudaSuccess ||
      make_tmap_2d_16bit(&tb_lo, blo, n, L.Kp, L.Kp, kTcBN, true, kTcBK) != cudaSuccess)
    return MM_ERR_CUDA;
  const int kb_total = (int)(L.Kp / kTcBK);
  if (p.kernel == 5) {
    const F32Sk g = f32_sk(m, n, k);
    float* slots = reinterpret_cast<float*>(w + L.off_part);
    int* counters = reinterpret_cast<int*>(w + L.off_part + g.slot_bytes);
    using Cfg = Bf16x3Cfg<kTcBN, kTcStages>;
    static std::atomic<uint64_t> conf_sk{0};
    if (smem_limit_once(bf16x3_streamk_kernel<kTcBN, kTcStages, kTcChunk>, Cfg::SMEM, conf_sk) != cudaSuccess ||
        cudaMemsetAsync(counters, 0, (size_t)g.tiles * 4, st) != cudaSuccess)
      return MM_ERR_CUDA;
    TraceScope tr(kTrTcBf16x3, st);
    bf16x3_streamk_kernel<kTcBN, kTcStages, kTcChunk><<<(unsigned)g.P, kTcThreads, Cfg::SMEM, st>>>(
        ta_hi, ta_lo, tb_hi, tb_lo, C, slots, counters, m, n, g.tiles_n, g.kbt, g.dp_tiles, g.sk_total, g.P, g.P_sk);
    return cudaGetLastError() == cudaSuccess ? MM_OK : MM_ERR_CUDA;
  }
  const int s = p.split_k;
  const int kbs = (kb_total + s - 1) / s;
  e = launch_gemm<kTcBN, kTcStages, kTcChunk>(ta_hi, ta_lo, tb_hi, tb_lo, C, part, m, n, kb_total, kbs, s, st);
  if (e == cudaSuccess && s > 1) {
    TraceScope tr(kTrSumReduceF32, st);
    const bool vec = aligned16(C) && aligned16(part) && (m * n) % 4 == 0;
    int64_t blocks = ((vec ? m * n / 4 : m * n) + 255) / 256;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    sum_reduce_f32_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(m * n, C, part, s - 1, vec);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

int arm_tc_skip_signal(int on) {
  return cudaMemcpyToSymbol(g_tc_skip_signal, &on, sizeof(int)) == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

int read_tc_status(int* status) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  *status = v;
  return MM_OK;
}

}  // namespace mmsr
