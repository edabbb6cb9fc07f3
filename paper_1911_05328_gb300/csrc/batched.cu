// batched.cu -- many independent products of mixed shapes and semirings in
// one persistent launch (the dynamic load balancing a processor-oblivious
// schedule relies on, Section 6: idle workers take the next available task).
//
// Host side: problems are sorted by tile cost (k, longest first) and cut
// into output tiles; the sorted problem table is copied into the workspace
// by small launches that carry it as kernel parameters.  One pre-pass, its
// work cut into equal blocks over the whole batch, splits the FP32 problems
// into bf16 hi/lo operands in stacked buffers with a common row pitch (so
// four tensor maps describe every FP32 problem of the batch) and decides,
// per (min,+) problem, whether the exact packed 2 x 16-bit leaf applies.
//
// Device side: FP32 tiles run in one persistent tcgen05 kernel -- one CTA
// per SM pops tile indices from an atomic counter and runs the pipeline
// (TMA producer warp, MMA warp, eight drain warps, chunked TMEM
// accumulation); the shared-memory ring and the TMEM accumulators persist
// across tiles with running phase counters, so no barrier is ever
// re-initialised while an asynchronous arrive may be pending.  (min,+) tiles
// run in a second launch, one 128 x 256 packed tile per CTA and two CTAs per
// SM: the packed mainloop needs sixteen warps per SM to keep the ALU pipe
// busy, which does not fit beside the tensor pipeline's register budget
// (inside the persistent kernel eight warps reached half its rate).  Both
// lists run longest problem first; a 32-bit launch takes (min,+) problems
// outside the packed range.  The whole call is capturable in one CUDA graph.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <numeric>
#include <string.h>
#include <vector>

#include "internal.h"
#include "minplus_tile.cuh"
#include "strassen_tables.cuh"
#include "tcgen05.cuh"

namespace mmsr {
namespace {

__device__ int g_batched_status;
// One-shot test switch: the CTA that claims tile 0 in the next launch skips
// the arrival and loads of its first ring position, so its MMA wait runs out.
__device__ int g_batched_skip_signal;

constexpr int kMaxBatch = 1 << 20;  // problems per call (tile counts stay in int32)
// FP32 tiles: 128 x 128, 64-wide k-blocks (128-byte swizzled rows) in a
// 3-deep TMA ring, TMEM chunks of 8 k-blocks (512 k).  On the 512-problem
// workload (median k ~ 340) this measured 0.68 ms for the kernel against
// 0.76 ms with the standalone GEMM's 32-wide blocks in a 6-deep ring (same
// 192 KB): half as many TMA boxes and ring handshakes per tile.  Split
// operands are padded to TKA columns.
#ifndef MMSR_B_BK
#define MMSR_B_BK 64
#endif
#ifndef MMSR_B_STAGES
#define MMSR_B_STAGES 3
#endif
#ifndef MMSR_B_CHUNK
#define MMSR_B_CHUNK 8
#endif
#ifndef MMSR_B_BN
#define MMSR_B_BN 128
#endif
constexpr int TBM = 128, TBN = MMSR_B_BN, TBK = MMSR_B_BK, TSTAGES = MMSR_B_STAGES, TCHUNK = MMSR_B_CHUNK, TKA = 64;
static_assert(TKA % TBK == 0 && (TBK == 32 || TBK == 64), "k-block / swizzle");
// warp 0: TMA producer, warp 1: MMA issuer, warps 2..9: drain, warp 10:
// tile scheduler (claims tile indices and finds their problems ahead of the
// other roles, so the claim's atomic and the table search stay off the
// producer's path between two tiles)
constexpr int kDrainW = 8, kSchedWarp = 2 + kDrainW, kBThreads = 64 + 32 * kDrainW + 32;
constexpr uint32_t TA_BYTES = TBM * TBK * 2, TB_BYTES = TBN * TBK * 2;
constexpr uint32_t TSTAGE = 2 * TA_BYTES + 2 * TB_BYTES;
constexpr int kTileQ = 4;  // tile indices the producer may claim ahead of the consumers
constexpr size_t BSMEM = 1024 + (size_t)TSTAGES * TSTAGE + 256;
constexpr uint32_t BTMEM_COLS = 2 * TBN;
constexpr int MPN = 256;  // (min,+) tile: 128 x 256

// Per-problem row of the batch table.  The table lives in the caller's
// workspace (written at the start of every call by small upload kernels that
// carry it as a kernel parameter, so the call stays capturable), which
// leaves the batch size free of the kernel-parameter limit.
struct BatchRow {
  int kind;  // 0: FP32 (+,x) on tensor cores, 1: (min,+) 256-wide tiles, 2: 128-wide,
             // 3: a Strassen-Winograd parent (its post pass only)
  int m, n, k;
  int row0a, row0b;  // FP32: first row of this A / B^T in the stacked split buffers
  const void* A;
  const void* B;
  void* C;
  int s, kbs;        // FP32: k-slices per tile and k-blocks per slice
  int64_t slot_off;  // FP32, s > 1: first float of this problem's partial tiles
  int cnt_off;       // FP32, s > 1: first of this problem's per-tile counters
  int prep_a;        // pre-pass blocks of A (the rest of the problem's blocks are B's)
  int lda, ldb;      // row pitches of A and B (a Strassen leaf reads its parent's)
  int sr;            // Strassen leaf: its product r (operands sum the parent's
                     // quadrants by alpha_r / beta_r, output is P_r); -1 otherwise
  int8_t ca[4], cb[4];  // Strassen leaf: alpha_r and beta_r over quadrants 00, 01, 10, 11
  int64_t p_off;     // Strassen leaf: first float of P_r; parent: of P_0
};
// What the kernels take by value: sizes and the device addresses of the
// table (rows in cost order and three prefix sums of tile counts).
struct BatchHeader {
  int count;
  int total_tiles;  // FP32 tile slices (persistent kernel)
  int mp16_total;   // packed (min,+) tiles
  int mp_total;     // 32-bit (min,+) tiles
  const BatchRow* rows;
  const int* tile_start;       // [count + 1] 128 x 128 tile slices of FP32 problems
  const int* mp16_tile_start;  // [count + 1] packed tiles of (min,+) problems
  const int* mp_tile_start;    // [count + 1] 128 x 128 tiles of (min,+) problems (fallback)
  const int* prep_start;       // [count + 1] pre-pass blocks
  const int* post_start;       // [count + 1] post-pass blocks (Strassen parents)
  int prep_total, post_total;
  float* pstack;               // the leaf products of the Strassen problems
};
constexpr int kUploadBytes = 30720;  // table bytes per upload launch (kernel parameter)
struct UploadChunk {
  uint32_t len;
  uint32_t pad[3];
  uint8_t bytes[kUploadBytes];
};

__global__ void __launch_bounds__(256) batched_upload_kernel(const __grid_constant__ UploadChunk c,
                                                             uint8_t* __restrict__ dst) {
  for (uint32_t i = threadIdx.x * 16; i < c.len; i += blockDim.x * 16)
    *reinterpret_cast<uint4*>(dst + i) = *reinterpret_cast<const uint4*>(c.bytes + i);
}

// ----------------------------------------------------------- pre-passes
__device__ __forceinline__ void split1(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// One pre-pass over the whole batch, its work cut into equal blocks so that
// a few large problems do not leave most SMs idle (with a fixed number of
// blocks per problem, 8 products of 256 x 384 x 32768 among 56 small ones
// took 1.07 ms at 16% of the HBM bandwidth).  Block b works for the problem
// p with prep_start[p] <= b < prep_start[p + 1]:
//  - FP32: A -> stacked hi/lo rows (pitch KP), kPrepA items of 8 columns per
//    block; then B -> stacked hi/lo of B^T, kPrepB tiles of 64 (k) x 64 (n)
//    per block through shared memory; columns k..roundup(k, 64) are zero;
//  - (min,+): kPrepR entries of A, then of B, per block, any entry outside
//    the packed range flags violation[p] (zeroed by the call's memset).
constexpr int kPrepA = 4096, kPrepB = 4, kPrepR = 4096;

// Eight consecutive entries of a row starting at column c8 (zero past column
// k), by 16-byte loads where the row allows them.
__device__ __forceinline__ void load8(const float* __restrict__ row, int64_t c8, int64_t k, bool vec, float* x) {
  const float* src = row + c8;
  if (vec && c8 + 8 <= k) {
    const float4 u = __ldcs(reinterpret_cast<const float4*>(src));
    const float4 w = __ldcs(reinterpret_cast<const float4*>(src + 4));
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w; x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
  } else {
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = c8 + t < k ? src[t] : 0.f;
  }
}

__global__ void __launch_bounds__(256, 4) batched_prepass_kernel(const BatchHeader T, int64_t KP,
                                                              __nv_bfloat16* __restrict__ ahi,
                                                              __nv_bfloat16* __restrict__ alo,
                                                              __nv_bfloat16* __restrict__ bhi,
                                                              __nv_bfloat16* __restrict__ blo,
                                                              int* __restrict__ violation) {
  __shared__ float tile[64][65];
  for (int blk = blockIdx.x; blk < T.prep_total; blk += gridDim.x) {
    int lo = 0, hi = T.count - 1;  // last p with prep_start[p] <= blk
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&T.prep_start[mid]) <= blk) lo = mid; else hi = mid - 1;
    }
    const int p = lo;
    // the row in registers: the stores below could alias the table as far as
    // the compiler knows, which would reload its fields every iteration
    const BatchRow R = T.rows[p];
    const int lb = blk - __ldg(&T.prep_start[p]);
    const int64_t m = R.m, n = R.n, k = R.k;
    if (R.kind == 0) {
      const int64_t kp = (k + TKA - 1) / TKA * TKA;
      if (lb < R.prep_a) {
        // A rows: items of 8 columns, four per thread in flight (a streaming
        // pass needs many bytes in flight per SM to approach the HBM rate)
        const float* __restrict__ A = static_cast<const float*>(R.A);
        const int64_t cpr = kp / 8, items = m * cpr, lda = R.lda;
        const int64_t e0 = (int64_t)lb * kPrepA, e_end = min(items, e0 + kPrepA);
        const bool vec = (k & 3) == 0 && (lda & 3) == 0;
        for (int64_t e = e0 + threadIdx.x; e < e_end; e += 4 * 256) {
          float x[4][8];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int64_t ej = e + j * 256;
            if (ej < e_end) {
              const int64_t r = ej / cpr, c8 = (ej - r * cpr) * 8;
              if (R.sr < 0) {
                load8(A + r * lda, c8, k, vec, x[j]);
              } else {
                // S_r = sum_q alpha_rq A_q over the parent's quadrants (Section 5)
#pragma unroll
                for (int t = 0; t < 8; ++t) x[j][t] = 0.f;
#pragma unroll
                for (int qd = 0; qd < 4; ++qd) {
                  const int c = R.ca[qd];
                  if (c == 0) continue;
                  float y[8];
                  load8(A + ((qd >> 1) * m + r) * lda + (qd & 1) * k, c8, k, vec, y);
#pragma unroll
                  for (int t = 0; t < 8; ++t) x[j][t] = c > 0 ? x[j][t] + y[t] : x[j][t] - y[t];
                }
              }
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int64_t ej = e + j * 256;
            if (ej < e_end) {
              const int64_t r = ej / cpr, c8 = (ej - r * cpr) * 8;
              __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
              for (int t = 0; t < 8; ++t) split1(x[j][t], h[t], l[t]);
              const int64_t off = (R.row0a + r) * KP + c8;
              *reinterpret_cast<uint4*>(ahi + off) = *reinterpret_cast<const uint4*>(h);
              *reinterpret_cast<uint4*>(alo + off) = *reinterpret_cast<const uint4*>(l);
            }
          }
        }
      } else {
        // B^T: 64 (k) x 64 (n) tiles through shared memory, sixteen loads
        // per thread in flight
        const float* __restrict__ B = static_cast<const float*>(R.B);
        const int64_t tk = kp / 64, tn = (n + 63) / 64;
        const int64_t t_begin = (int64_t)(lb - R.prep_a) * kPrepB, t_end = min(tk * tn, t_begin + kPrepB);
        const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
        for (int64_t tt = t_begin; tt < t_end; ++tt) {
          const int64_t k0 = (tt / tn) * 64, n0 = (tt % tn) * 64;
          const int64_t gn = n0 + tx;
          float v[16];
          const int64_t ldb = R.ldb;
          if (R.sr < 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int64_t gk = k0 + ty + 4 * i;
              v[i] = (gk < k && gn < n) ? __ldcs(B + gk * ldb + gn) : 0.f;
            }
          } else {
            // T_r = sum_q beta_rq B_q over the parent's quadrants
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
            for (int qd = 0; qd < 4; ++qd) {
              const int c = R.cb[qd];
              if (c == 0) continue;
              const float* Bq = B + (qd >> 1) * k * ldb + (qd & 1) * n;
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const int64_t gk = k0 + ty + 4 * i;
                const float y = (gk < k && gn < n) ? __ldcs(Bq + gk * ldb + gn) : 0.f;
                v[i] = c > 0 ? v[i] + y : v[i] - y;
              }
            }
          }
          __syncthreads();  // the previous tile's readers are done
#pragma unroll
          for (int i = 0; i < 16; ++i) tile[ty + 4 * i][tx] = v[i];
          __syncthreads();
          // B^T row n0 + row, k0 + 16 q .. +15: four threads per row
          const int row = threadIdx.x >> 2, q = threadIdx.x & 3;
          const int64_t gr = n0 + row;
          if (gr < n) {
            __align__(16) __nv_bfloat16 h[16], l[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) split1(tile[q * 16 + e][row], h[e], l[e]);
            const int64_t off = (R.row0b + gr) * KP + k0 + q * 16;
            *reinterpret_cast<uint4*>(bhi + off) = *reinterpret_cast<const uint4*>(h);
            *reinterpret_cast<uint4*>(bhi + off + 8) = *reinterpret_cast<const uint4*>(h + 8);
            *reinterpret_cast<uint4*>(blo + off) = *reinterpret_cast<const uint4*>(l);
            *reinterpret_cast<uint4*>(blo + off + 8) = *reinterpret_cast<const uint4*>(l + 8);
          }
        }
      }
    } else {
      const bool second = lb >= R.prep_a;
      const int32_t* X = static_cast<const int32_t*>(second ? R.B : R.A);
      const int64_t cnt = second ? k * n : m * k;
      const int64_t i0 = (int64_t)(second ? lb - R.prep_a : lb) * kPrepR, i1 = min(cnt, i0 + kPrepR);
      int bad = 0;
      // i0 is a multiple of 4 and X is 16-byte aligned (checked on the host)
#pragma unroll 4
      for (int64_t v = i0 / 4 + threadIdx.x; v < i1 / 4; v += 256) {
        const int4 q = __ldcs(reinterpret_cast<const int4*>(X) + v);
        bad |= mp::out_of_pack_range(q.x) | mp::out_of_pack_range(q.y) | mp::out_of_pack_range(q.z) |
               mp::out_of_pack_range(q.w);
      }
      for (int64_t e = max(i0, i1 / 4 * 4) + threadIdx.x; e < i1; e += 256) bad |= mp::out_of_pack_range(X[e]);
      bad = __syncthreads_or(bad);
      if (bad && threadIdx.x == 0) atomicOr(&violation[p], 1);
    }
    __syncthreads();  // the next block of work may reuse `tile`
  }
}

// Post pass of the Strassen-Winograd problems (one level, Section 5's
// bilinear form): C_q = sum_r gamma_qr P_r for the four quadrants, products
// in order r = 0..6, kPostE entries of the half-size blocks per block.
constexpr int kPostE = 4096;
constexpr int kBatchVariant = 1;  // Strassen-Winograd

__global__ void __launch_bounds__(256) batched_post_kernel(const BatchHeader T) {
  for (int blk = blockIdx.x; blk < T.post_total; blk += gridDim.x) {
    int lo = 0, hi = T.count - 1;  // last p with post_start[p] <= blk
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&T.post_start[mid]) <= blk) lo = mid; else hi = mid - 1;
    }
    const BatchRow R = T.rows[lo];
    const int64_t m2 = R.m / 2, n2 = R.n / 2, n = R.n, ps = m2 * n2;
    const float* __restrict__ P0 = T.pstack + R.p_off;
    float* __restrict__ C = static_cast<float*>(R.C);
    const int64_t e0 = (int64_t)(blk - __ldg(&T.post_start[lo])) * kPostE, e1 = min(ps, e0 + kPostE);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += 256) {
      const int64_t i = e / n2, j = e - i * n2;
      float pr[7];
#pragma unroll
      for (int r = 0; r < 7; ++r) pr[r] = __ldcs(P0 + r * ps + e);
#pragma unroll
      for (int qd = 0; qd < 4; ++qd) {
        C[((qd >> 1) * m2 + i) * n + (qd & 1) * n2 + j] = combo7<kBatchVariant>(qd, pr);
      }
    }
  }
}

// 32-bit fallback for (min,+) problems whose inputs fall outside the packed
// range: one 128 x 128 tile per CTA over a compact list of those problems'
// tiles; CTAs of in-range problems exit at once.  Kept out of the persistent
// kernel so its register demand does not press on the kernel's main paths.
__global__ void __launch_bounds__(256, 2)
    batched_minplus32_kernel(const BatchHeader T, const int* __restrict__ violation) {
  const int t = blockIdx.x;
  int lo = 0, hi = T.count - 1;  // last p with mp_tile_start[p] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (T.mp_tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int p = lo;
  if (T.rows[p].kind == 0 || __ldcg(&violation[p]) == 0) return;
  extern __shared__ __align__(16) int32_t fsmem[];
  const int64_t m = T.rows[p].m, n = T.rows[p].n, k = T.rows[p].k;
  const int local = t - T.mp_tile_start[p];
  const int tiles_n = (int)((n + mp::BN - 1) / mp::BN);
  const int32_t* A = static_cast<const int32_t*>(T.rows[p].A);
  const int32_t* B = static_cast<const int32_t*>(T.rows[p].B);
  int32_t* C = static_cast<int32_t*>(T.rows[p].C);
  const bool vec = (k % 4 == 0) && (n % 4 == 0) && aligned16(A) && aligned16(B) && aligned16(C);
  mp::minplus32_tile(A, B, C, (int32_t*)nullptr, 0, m, n, k, (int64_t)(local / tiles_n) * mp::BM,
                     (int64_t)(local % tiles_n) * mp::BN, (int64_t)0, (int)((k + mp::BK - 1) / mp::BK), vec,
                     (int)threadIdx.x, fsmem, mp::SyncCta());
}

// Packed (min,+) tiles: one tile per CTA over the compact list of (min,+)
// problems' tiles (longest first); a problem uses 128 x 256 tiles, or
// 128 x 128 tiles where that pads its width less.  CTAs of problems outside
// the packed range exit at once.
template <int NP>
__device__ __forceinline__ void batched_packed_tile(const BatchHeader& T, int p, int local, uint32_t* psmem) {
  const int64_t m = T.rows[p].m, n = T.rows[p].n, k = T.rows[p].k;
  constexpr int TN = mp::PackTile<NP>::TN;
  const int tiles_n = (int)((n + TN - 1) / TN);
  const int32_t* A = static_cast<const int32_t*>(T.rows[p].A);
  const int32_t* B = static_cast<const int32_t*>(T.rows[p].B);
  int32_t* C = static_cast<int32_t*>(T.rows[p].C);
  const bool vec = (k % 4 == 0) && (n % 4 == 0) && aligned16(A) && aligned16(B) && aligned16(C);
  mp::minplus16_tile<mp::SyncCta, NP>(A, B, C, (int32_t*)nullptr, 0, m, n, k, (int64_t)(local / tiles_n) * mp::PBM,
                                      (int64_t)(local % tiles_n) * TN, (int64_t)0, k, vec, (int)threadIdx.x,
                                      psmem, mp::SyncCta());
}

__global__ void __launch_bounds__(256, 2)
    batched_minplus16_kernel(const BatchHeader T, const int* __restrict__ violation) {
  const int t = blockIdx.x;
  int lo = 0, hi = T.count - 1;  // last p with mp16_tile_start[p] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (T.mp16_tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int p = lo;
  if (T.rows[p].kind == 0 || __ldcg(&violation[p]) != 0) return;
  __shared__ __align__(16) uint32_t psmem[mp::PSMEM_BYTES / 4];
  const int local = t - T.mp16_tile_start[p];
  if (T.rows[p].kind == 1)
    batched_packed_tile<8>(T, p, local, psmem);
  else
    batched_packed_tile<4>(T, p, local, psmem);
}

// Shared-memory descriptor of a K-major operand tile with TBK-wide rows.
__device__ __forceinline__ uint64_t kdesc(uint32_t saddr) {
  return TBK == 64 ? tc::desc_sw128(saddr) : tc::desc_sw64(saddr);
}

// ------------------------------------------------------ persistent kernel
__global__ void __launch_bounds__(kBThreads, 1)
    batched_kernel(const BatchHeader T, const __grid_constant__ CUtensorMap tAhi,
                   const __grid_constant__ CUtensorMap tAlo, const __grid_constant__ CUtensorMap tBhi,
                   const __grid_constant__ CUtensorMap tBlo, int* __restrict__ counter,
                   float* __restrict__ slots, int* __restrict__ split_cnt) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TSTAGES * TSTAGE);
  uint64_t* empty = full + TSTAGES;
  uint64_t* acc_full = empty + TSTAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* tile_full = acc_empty + 2;         // [kTileQ]
  uint64_t* tile_empty = tile_full + kTileQ;   // [kTileQ]
  uint64_t* quiesce = tile_empty + kTileQ;     // after an abort: all issued MMAs done
  // drain-warp rendezvous of a k-slice (bounded waits): every drain warp has
  // stored its part of the partial tile / the fold verdict is out
  uint64_t* seg_stored = quiesce + 1;
  uint64_t* seg_decided = seg_stored + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(seg_decided + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* tile_q = abort_flag + 1;                // [kTileQ]
  int* fold_flag = tile_q + kTileQ;            // this CTA folds the tile's slices
  int* tile_qp = fold_flag + 1;                // [kTileQ] problem of each queued tile

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kDrainW);
    }
    for (int q = 0; q < kTileQ; ++q) {
      tc::mbar_init(&tile_full[q], 1);
      tc::mbar_init(&tile_empty[q], 2 + kDrainW);  // producer, MMA thread and drain warps
    }
    tc::mbar_init(quiesce, 1);
    tc::mbar_init(seg_stored, kDrainW);
    tc::mbar_init(seg_decided, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, BTMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // running positions of the TMA ring and of the TMEM chunk buffers; each
  // role advances its own copy over the same sequence of tensor-core tiles.
  // Tile indices travel through a small mbarrier queue instead of a CTA
  // barrier: the producer claims tiles ahead (and starts their TMA loads)
  // while the tensor core and the drain warps still work on earlier ones.
  uint32_t ring = 0, chunk = 0, ps = 0;  // ps: k-sliced tiles drained (rendezvous phase)
  // warps 0, 1 and the scheduler work through one lane
  const bool active = (warp >= 2 && warp < kSchedWarp) || lane == 0;
  bool skipped = false;  // producer: the test switch took ring position 0 out

  for (uint32_t j = 0; active; ++j) {
    const int slot = (int)(j % kTileQ);
    const uint32_t ph = (j / kTileQ) & 1u;
    int t = INT_MAX, p = 0;
    if (warp == kSchedWarp) {
      if (j < kTileQ || tc::mbar_wait(&tile_empty[slot], ph ^ 1u, abort_flag, &g_batched_status)) {
        t = atomicAdd(counter, 1);
        if (t < T.total_tiles) {
          int lo = 0, hi = T.count - 1;  // last p with tile_start[p] <= t
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (T.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
          }
          p = lo;
        }
        tile_q[slot] = t;
        tile_qp[slot] = p;
        tc::mbar_arrive(&tile_full[slot]);  // release: the entry is visible to the waiters
      }
      if (t >= T.total_tiles) break;
      continue;
    }
    {
      const bool drain = warp >= 2;
      bool ok = tc::mbar_wait(&tile_full[slot], ph, abort_flag, &g_batched_status);
      if (drain) ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        t = *reinterpret_cast<volatile int*>(&tile_q[slot]);
        p = *reinterpret_cast<volatile int*>(&tile_qp[slot]);
      }
      if (drain) __syncwarp();
      if (ok && lane == 0) tc::mbar_arrive(&tile_empty[slot]);
      // tile 0 is always its CTA's first tile, so the ring is at position 0
      if (warp == 0 && t == 0) skipped = atomicExch(&g_batched_skip_signal, 0) != 0;
    }
    if (t >= T.total_tiles) break;
    const int local = t - T.tile_start[p];
    const int64_t m = T.rows[p].m, n = T.rows[p].n, k = T.rows[p].k;
    // unit = (tile, k-slice), the slices of one tile adjacent in the queue
    const int nsl = T.rows[p].s, tile = local / nsl, z = local - tile * nsl;

    {
      // ------------------------------------------------ FP32 tensor-core tile
      const int tiles_n = (int)((n + TBN - 1) / TBN);
      const int64_t i0 = (int64_t)(tile / tiles_n) * TBM, j0 = (int64_t)(tile % tiles_n) * TBN;
      const int nkb_all = (int)((k + TBK - 1) / TBK);
      const int kb0 = z * T.rows[p].kbs;
      const int nkb = max(0, min(nkb_all - kb0, T.rows[p].kbs));
      const int nchunks = (nkb + TCHUNK - 1) / TCHUNK;
      if (warp == 0) {
        if (lane == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const int ya = T.rows[p].row0a + (int)i0, yb = T.rows[p].row0b + (int)j0;
          for (int it = 0; it < nkb; ++it, ++ring) {
            const int s = ring % TSTAGES;
            const uint32_t round = ring / TSTAGES;
            if (round > 0 && !tc::mbar_wait(&empty[s], (round - 1) & 1u, abort_flag, &g_batched_status)) break;
            if (ring == 0 && skipped) continue;
            tc::mbar_expect_tx(&full[s], TSTAGE);
            uint8_t* st = smem + s * TSTAGE;
            const int kx = (kb0 + it) * TBK;
            tc::tma_load_2d(st, &tAhi, &full[s], kx, ya);
            tc::tma_load_2d(st + TA_BYTES, &tAlo, &full[s], kx, ya);
            tc::tma_load_2d(st + 2 * TA_BYTES, &tBhi, &full[s], kx, yb);
            tc::tma_load_2d(st + 2 * TA_BYTES + TB_BYTES, &tBlo, &full[s], kx, yb);
          }
        }
      } else if (warp == 1) {
        if (lane == 0) {
          constexpr uint32_t idesc = tc::idesc_f16(TBM, TBN, 1);
          int it = 0;
          for (int c = 0; c < nchunks; ++c, ++chunk) {
            const int b = chunk & 1;
            if (chunk >= 2 && !tc::mbar_wait(&acc_empty[b], ((chunk >> 1) - 1) & 1u, abort_flag, &g_batched_status)) break;
            tc::fence_after_sync();
            const uint32_t d = tmem + (uint32_t)(b * TBN);
            const int last = min(nkb, (c + 1) * TCHUNK);
            bool aborted = false;
            for (int first = 1; it < last; ++it, ++ring, first = 0) {
              const int s = ring % TSTAGES;
              if (!tc::mbar_wait(&full[s], (ring / TSTAGES) & 1u, abort_flag, &g_batched_status)) {
                aborted = true;
                break;
              }
              tc::fence_after_sync();
              const uint32_t base = smem_u32(smem + s * TSTAGE);
#pragma unroll
              for (int kk = 0; kk < TBK / 16; ++kk) {
                const uint64_t ahi = kdesc(base + kk * 32);
                const uint64_t alo = kdesc(base + TA_BYTES + kk * 32);
                const uint64_t bhi = kdesc(base + 2 * TA_BYTES + kk * 32);
                const uint64_t blo = kdesc(base + 2 * TA_BYTES + TB_BYTES + kk * 32);
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
        const int q = warp & 3, half = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        float sum[TBN / 2];
#pragma unroll
        for (int e = 0; e < TBN / 2; ++e) sum[e] = 0.f;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c, ++chunk) {
          const int b = chunk & 1;
          // warp-uniform verdict: the __syncwarp below needs every lane
          ok = __all_sync(0xffffffffu, ok && tc::mbar_wait(&acc_full[b], (chunk >> 1) & 1u, abort_flag,
                                                           &g_batched_status));
          if (!ok) break;
          tc::fence_after_sync();
#pragma unroll
          for (int cc = 0; cc < TBN / 2; cc += 16) {
            uint32_t r[16];
            tc::tmem_ld_32x32b_x16(tmem + lane_base + (uint32_t)(b * TBN + half * (TBN / 2) + cc), r);
            tc::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e) sum[cc + e] = __fadd_rn(sum[cc + e], __uint_as_float(r[e]));
          }
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
        }
        // a Strassen leaf writes its product P_r into the stack, else C
        float* C = T.rows[p].sr >= 0 ? T.pstack + T.rows[p].p_off : static_cast<float*>(T.rows[p].C);
        const int64_t row = i0 + q * 32 + lane;
        if (nsl > 1) {
          // One k-slice of a split tile: store the partial tile thread-major
          // (float4 i of drain thread d at i x 256 + d, so warp-wide stores
          // and the fold's loads are 512 contiguous bytes), count the slice on
          // the tile's counter, and the slice that completes it folds all
          // slices in slice order and writes C.  No CTA waits on another.
          const int dt = threadIdx.x - 64;
          float* tile_slots = slots + T.rows[p].slot_off + (int64_t)tile * nsl * (TBM * TBN);
          float4* mine = reinterpret_cast<float4*>(tile_slots + (int64_t)z * (TBM * TBN)) + dt;
#pragma unroll
          for (int e = 0; e < TBN / 2; e += 4)
            __stcg(mine + (e / 4) * (kDrainW * 32), ok ? make_float4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3])
                                                        : make_float4(0.f, 0.f, 0.f, 0.f));
          __threadfence();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(seg_stored);
          bool go = __all_sync(0xffffffffu, tc::mbar_wait(seg_stored, ps & 1u, abort_flag, &g_batched_status));
          if (go && warp == 2) {
            if (lane == 0) {
              *fold_flag = atomicAdd(&split_cnt[T.rows[p].cnt_off + tile], 1) == nsl - 1;
              tc::mbar_arrive(seg_decided);  // release: the verdict is visible to the waiters
            }
            __syncwarp();
          }
          go = go && __all_sync(0xffffffffu, tc::mbar_wait(seg_decided, ps & 1u, abort_flag, &g_batched_status));
          ++ps;
          if (go && *reinterpret_cast<volatile int*>(fold_flag)) {
            __threadfence();
#pragma unroll
            for (int e = 0; e < TBN / 2; ++e) sum[e] = 0.f;
            for (int zz = 0; zz < nsl; ++zz) {
              const float4* src = reinterpret_cast<const float4*>(tile_slots + (int64_t)zz * (TBM * TBN)) + dt;
              float4 v[TBN / 8];  // all sixteen 16-byte loads in flight
#pragma unroll
              for (int u = 0; u < TBN / 8; ++u) v[u] = __ldcg(src + u * (kDrainW * 32));
#pragma unroll
              for (int u = 0; u < TBN / 8; ++u) {
                sum[4 * u] = __fadd_rn(sum[4 * u], v[u].x);
                sum[4 * u + 1] = __fadd_rn(sum[4 * u + 1], v[u].y);
                sum[4 * u + 2] = __fadd_rn(sum[4 * u + 2], v[u].z);
                sum[4 * u + 3] = __fadd_rn(sum[4 * u + 3], v[u].w);
              }
            }
          } else {
            continue;  // another slice folds this tile (or the call aborted)
          }
        }
        if (row < m) {
          const int64_t c0 = j0 + half * (TBN / 2);
          float* dst = C + row * n + c0;
          // 16-byte stores where the row allows them (n % 4 == 0 keeps every
          // row 16-byte aligned), element stores at the ragged edge
          const bool vec = (n % 4 == 0) && aligned16(C);
#pragma unroll
          for (int e = 0; e < TBN / 2; e += 4) {
            if (vec && c0 + e + 4 <= n) {
              *reinterpret_cast<float4*>(dst + e) =
                  ok ? make_float4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (c0 + e + u < n) dst[e + u] = ok ? sum[e + u] : 0.f;
            }
          }
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
    if (warp == 0 && lane == 0)
      for (uint32_t r = ring > (uint32_t)TSTAGES ? ring - TSTAGES : 0u; r < ring; ++r)
        if (!(r == 0 && skipped)) tc::mbar_wait_quiesce(&full[r % TSTAGES], (r / TSTAGES) & 1u);
    if (warp == 1 && lane == 0) {
      tc::mma_commit(quiesce);
      tc::mbar_wait_quiesce(quiesce, 0);
    }
    __syncwarp();
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, BTMEM_COLS);
  }
}

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct BatchPlan {
  int count = 0, total_tiles = 0, mp16_total = 0, mp_total = 0, prep_total = 0, post_total = 0;
  std::vector<uint8_t> table;  // rows, then the three prefix sums (uploaded to off_table)
  int64_t rows_bytes = 0, starts_bytes = 0;
  int64_t KP = 0, rows_a = 0, rows_b = 0;
  int64_t split_tiles = 0, slot_floats = 0;  // k-sliced FP32 tiles: counters and partial tiles
  int64_t pstack_floats = 0;                 // Strassen leaf products
  int64_t off_viol = 256, off_cnt = 0, off_table = 0, off_slots = 0, off_pstack = 0, off_ahi = 0, off_alo = 0,
          off_bhi = 0, off_blo = 0, total = 0;

  // The kernels' view of the table once it sits at `w + off_table`.
  BatchHeader header(uint8_t* w) const {
    BatchHeader H;
    H.count = count;
    H.total_tiles = total_tiles;
    H.mp16_total = mp16_total;
    H.mp_total = mp_total;
    H.rows = reinterpret_cast<const BatchRow*>(w + off_table);
    const int* st = reinterpret_cast<const int*>(w + off_table + rows_bytes);
    H.tile_start = st;
    H.mp16_tile_start = st + (count + 1);
    H.mp_tile_start = st + 2 * (count + 1);
    H.prep_start = st + 3 * (count + 1);
    H.post_start = st + 4 * (count + 1);
    H.prep_total = prep_total;
    H.post_total = post_total;
    H.pstack = reinterpret_cast<float*>(w + off_pstack);
    return H;
  }
};

// One row of the table before sorting: a problem, or for a problem with one
// Strassen-Winograd level its seven leaf products and the parent row whose
// post pass folds them into C.
struct Item {
  int kind;  // as BatchRow::kind
  int64_t m, n, k, lda, ldb;
  const void* A;
  const void* B;
  void* C;
  int sr;         // Strassen leaf r, or -1
  int64_t p_off;  // leaf: its product's first float; parent: P_0's
  int split;      // split_k hint
};

int make_plan(int count, const mm_problem_t* probs, BatchPlan* P) {
  if (count < 0 || count > kMaxBatch || (count > 0 && !probs)) return MM_ERR_ARG;
  std::vector<Item> items;
  items.reserve(count);
  int64_t pfl = 0;  // floats of the leaf-product stack
  for (int i = 0; i < count; ++i) {
    const mm_problem_t& q = probs[i];
    if (q.semiring != MM_SR_PLUS_TIMES_F32 && q.semiring != MM_SR_MIN_PLUS_I32) return MM_ERR_UNSUPPORTED;
    if (q.reserved != 0) return MM_ERR_UNSUPPORTED;
    if (q.levels < 0 || q.levels > 1) return MM_ERR_ARG;
    if (q.levels == 1 && q.semiring != MM_SR_PLUS_TIMES_F32) return MM_ERR_UNSUPPORTED;  // no (min,+) Strassen
    if (q.split_k < 0 || (q.split_k != 0 && q.semiring != MM_SR_PLUS_TIMES_F32)) return MM_ERR_ARG;
    if (q.m < 0 || q.n < 0 || q.k < 0 || q.m > (1 << 20) || q.n > (1 << 20) || q.k > (1 << 20))
      return MM_ERR_SHAPE;
    if (q.levels == 1 && ((q.m | q.n | q.k) & 1)) return MM_ERR_SHAPE;
    if (q.m > 0 && q.n > 0 && (!q.C || (q.k > 0 && (!q.A || !q.B)))) return MM_ERR_ARG;
    if (!aligned16(q.C) || !aligned16(q.A) || !aligned16(q.B)) return MM_ERR_ALIGN;
    const bool f32 = q.semiring == MM_SR_PLUS_TIMES_F32;
    if (q.levels == 1 && q.m > 0 && q.n > 0 && q.k > 0) {
      const int64_t m2 = q.m / 2, n2 = q.n / 2, k2 = q.k / 2;
      items.push_back({3, q.m, q.n, q.k, q.k, q.n, nullptr, nullptr, q.C, -1, pfl, 0});
      for (int r = 0; r < 7; ++r)
        items.push_back({0, m2, n2, k2, q.k, q.n, q.A, q.B, nullptr, r, pfl + r * m2 * n2, q.split_k});
      pfl += 7 * m2 * n2;
    } else {
      // (min,+): 128-wide tiles where they pad the width less than 256-wide ones
      const bool narrow = ((q.n + 127) / 128) * 128 < ((q.n + 255) / 256) * 256;
      items.push_back({f32 ? 0 : (narrow ? 2 : 1), q.m, q.n, q.k, q.k, q.n, q.A, q.B, q.C, -1, 0, q.split_k});
    }
  }
  if ((int64_t)items.size() > kMaxBatch * 4) return MM_ERR_SHAPE;
  const int rows_n = (int)items.size();
  std::vector<int> order(rows_n);
  std::iota(order.begin(), order.end(), 0);
  // Longest tiles first: every tile of a problem costs ~k (tiles have a fixed
  // size), so descending k is longest-processing-time order for the tile
  // queues; ties by m n (more tiles first), then by index for determinism.
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (items[a].k != items[b].k) return items[a].k > items[b].k;
    return (double)items[a].m * items[a].n > (double)items[b].m * items[b].n;
  });
  // k-slices of FP32 tiles (Section 3's k-split inside the batch).  The
  // library's rule: a tile whose k-blocks exceed an eighth of one SM's share
  // of the batch's FP32 work holds back the end of the batch, so it is cut
  // into slices of about that size (at least 8 k-blocks, at most 16 slices);
  // a hint s > 1 asks for s slices.
  int64_t fp_work = 0;  // FP32 (tile, 64-wide k-block) units
  for (const Item& it : items)
    if (it.kind == 0 && it.m > 0 && it.n > 0)
      fp_work += ((it.m + TBM - 1) / TBM) * ((it.n + TBN - 1) / TBN) * ((it.k + TBK - 1) / TBK);
  const int64_t slice_target = std::max<int64_t>(8, fp_work / (8 * (int64_t)num_sms()));
  auto slices_of = [&](const Item& q, int* kbs) {
    const int64_t nkb = (q.k + TBK - 1) / TBK;
    int64_t s = 1;
    if (q.split > 1)
      s = std::min<int64_t>({(int64_t)q.split, 64, nkb});
    else if (q.split == 0 && nkb > slice_target)
      s = std::min<int64_t>(16, (nkb + slice_target - 1) / slice_target);
    if (s < 1) s = 1;
    int64_t per = (nkb + s - 1) / s;
    if (per < 1) per = 1;
    s = std::max<int64_t>(1, (nkb + per - 1) / per);  // no empty tail slices
    *kbs = (int)per;
    return (int)s;
  };
  std::vector<BatchRow> rows(rows_n);
  std::vector<int> starts(5 * (size_t)(rows_n + 1));
  int* tile_start = starts.data();
  int* mp16_start = tile_start + (rows_n + 1);
  int* mp_start = mp16_start + (rows_n + 1);
  int* prep_start = mp_start + (rows_n + 1);
  int* post_start = prep_start + (rows_n + 1);
  int64_t prep = 0, post = 0;
  int64_t kp_max = 0, ra = 0, rb = 0, tiles = 0, mp_tiles = 0, mp16_tiles = 0, split_tiles = 0, slot_floats = 0;
  for (int i = 0; i < rows_n; ++i) {
    const Item& q = items[order[i]];
    BatchRow& r = rows[i];
    memset(&r, 0, sizeof(r));
    r.kind = q.kind;
    r.m = (int)q.m;
    r.n = (int)q.n;
    r.k = (int)q.k;
    r.A = q.A;
    r.B = q.B;
    r.C = q.C;
    r.lda = (int)q.lda;
    r.ldb = (int)q.ldb;
    r.sr = q.sr;
    r.p_off = q.p_off;
    for (int qd = 0; qd < 4; ++qd) {
      r.ca[qd] = (int8_t)(q.sr >= 0 ? coef_alpha(kBatchVariant, q.sr, qd) : 0);
      r.cb[qd] = (int8_t)(q.sr >= 0 ? coef_beta(kBatchVariant, q.sr, qd) : 0);
    }
    r.s = 1;
    r.kbs = (int)std::max<int64_t>(1, (q.k + TBK - 1) / TBK);
    prep_start[i] = (int)prep;
    post_start[i] = (int)post;
    if (r.kind == 3) {
      post += (q.m / 2 * (q.n / 2) + kPostE - 1) / kPostE;
    } else if (q.m > 0 && q.n > 0 && q.k > 0) {
      if (r.kind == 0) {
        const int64_t kp = align_up(q.k, TKA);
        r.prep_a = (int)((q.m * (kp / 8) + kPrepA - 1) / kPrepA);
        prep += r.prep_a + ((kp / 64) * ((q.n + 63) / 64) + kPrepB - 1) / kPrepB;
      } else {
        r.prep_a = (int)((q.m * q.k + kPrepR - 1) / kPrepR);
        prep += r.prep_a + (q.k * q.n + kPrepR - 1) / kPrepR;
      }
    }
    tile_start[i] = (int)tiles;
    mp16_start[i] = (int)mp16_tiles;
    mp_start[i] = (int)mp_tiles;
    if ((r.kind == 1 || r.kind == 2) && q.m > 0 && q.n > 0) {
      mp_tiles += ((q.m + mp::BM - 1) / mp::BM) * ((q.n + mp::BN - 1) / mp::BN);
      const int64_t tn = r.kind == 2 ? 128 : MPN;
      mp16_tiles += ((q.m + mp::PBM - 1) / mp::PBM) * ((q.n + tn - 1) / tn);
    }
    if (r.kind == 0 && q.m > 0 && q.n > 0) {
      const int64_t pt = ((q.m + TBM - 1) / TBM) * ((q.n + TBN - 1) / TBN);
      r.s = slices_of(q, &r.kbs);
      if (r.s > 1) {
        r.slot_off = slot_floats;
        r.cnt_off = (int)split_tiles;
        slot_floats += pt * r.s * TBM * TBN;
        split_tiles += pt;
      }
      tiles += pt * r.s;
    }
    if (r.kind == 0) {
      r.row0a = (int)ra;
      r.row0b = (int)rb;
      ra += q.m;
      rb += q.n;
      kp_max = std::max<int64_t>(kp_max, align_up(q.k > 0 ? q.k : 1, TKA));
    }
    if (tiles > (int64_t)1 << 30 || mp_tiles > (int64_t)1 << 30 || mp16_tiles > (int64_t)1 << 30 ||
        ra > (int64_t)1 << 30 || rb > (int64_t)1 << 30 || split_tiles > (int64_t)1 << 30 ||
        prep > (int64_t)1 << 30 || post > (int64_t)1 << 30)
      return MM_ERR_SHAPE;
  }
  tile_start[rows_n] = (int)tiles;
  mp16_start[rows_n] = (int)mp16_tiles;
  mp_start[rows_n] = (int)mp_tiles;
  prep_start[rows_n] = (int)prep;
  post_start[rows_n] = (int)post;
  P->prep_total = (int)prep;
  P->post_total = (int)post;
  P->count = rows_n;
  P->total_tiles = (int)tiles;
  P->mp16_total = (int)mp16_tiles;
  P->mp_total = (int)mp_tiles;
  P->rows_bytes = align_up((int64_t)rows_n * (int64_t)sizeof(BatchRow), 16);
  P->starts_bytes = align_up((int64_t)starts.size() * 4, 16);
  P->table.assign((size_t)(P->rows_bytes + P->starts_bytes), 0);
  if (rows_n > 0) memcpy(P->table.data(), rows.data(), (size_t)rows_n * sizeof(BatchRow));
  memcpy(P->table.data() + P->rows_bytes, starts.data(), starts.size() * 4);
  P->KP = kp_max;
  P->rows_a = ra;
  P->rows_b = rb;
  P->split_tiles = split_tiles;
  P->slot_floats = slot_floats;
  P->pstack_floats = pfl;
  // workspace: [0] tile counter, [256] per-row (min,+) range verdicts, the
  // per-tile counters of k-sliced tiles (all zeroed by one memset per call),
  // then the table, the partial tiles, the Strassen leaf products and the
  // stacked split operands
  P->off_cnt = align_up(P->off_viol + 4 * (int64_t)rows_n, 16);
  P->off_table = align_up(P->off_cnt + 4 * split_tiles, 256);
  P->off_slots = align_up(P->off_table + (int64_t)P->table.size(), 1024);
  P->off_pstack = align_up(P->off_slots + 4 * slot_floats, 1024);
  P->off_ahi = align_up(P->off_pstack + 4 * pfl, 1024);
  P->off_alo = P->off_ahi + align_up(ra * kp_max * 2, 1024);
  P->off_bhi = P->off_alo + align_up(ra * kp_max * 2, 1024);
  P->off_blo = P->off_bhi + align_up(rb * kp_max * 2, 1024);
  P->total = P->off_blo + align_up(rb * kp_max * 2, 1024);
  return MM_OK;
}

}  // namespace

int arm_batched_skip_signal(int on) {
  return cudaMemcpyToSymbol(g_batched_skip_signal, &on, sizeof(int)) == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

int read_batched_status(int* status) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_batched_status, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_batched_status, &zero, sizeof(int)) != cudaSuccess) return MM_ERR_CUDA;
  *status = v;
  return MM_OK;
}

}  // namespace mmsr

using namespace mmsr;

extern "C" size_t mm_batched_query(int count, const mm_problem_t* problems) {
  BatchPlan local;  // planning is host-only and cheap
  if (make_plan(count, problems, &local) != MM_OK) return 0;
  return (size_t)local.total;
}

extern "C" int mm_batched(int count, const mm_problem_t* problems, void* workspace,
                          size_t workspace_bytes, void* stream) {
  BatchPlan P;
  int rc = make_plan(count, problems, &P);
  if (rc != MM_OK) return rc;
  if (count == 0 || (P.total_tiles == 0 && P.mp_total == 0)) return MM_OK;
  if (!workspace) return MM_ERR_ARG;
  if (!aligned16(workspace)) return MM_ERR_ALIGN;
  if ((size_t)P.total > workspace_bytes) return MM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w = static_cast<uint8_t*>(workspace);
  int* counter = reinterpret_cast<int*>(w);
  int* violation = reinterpret_cast<int*>(w + P.off_viol);
  auto* ahi = reinterpret_cast<__nv_bfloat16*>(w + P.off_ahi);
  auto* alo = reinterpret_cast<__nv_bfloat16*>(w + P.off_alo);
  auto* bhi = reinterpret_cast<__nv_bfloat16*>(w + P.off_bhi);
  auto* blo = reinterpret_cast<__nv_bfloat16*>(w + P.off_blo);
  MMSR_TRY_STATUS(cudaMemsetAsync(w, 0, (size_t)(P.off_cnt + 4 * P.split_tiles), st));
  const BatchHeader H = P.header(w);
  {
    TraceScope tr(kTrSplitBf16, st);
    // the table: kernel parameters of a few launches (captured by value)
    UploadChunk chunk;
    for (size_t off = 0; off < P.table.size(); off += kUploadBytes) {
      chunk.len = (uint32_t)std::min<size_t>(kUploadBytes, P.table.size() - off);
      memcpy(chunk.bytes, P.table.data() + off, chunk.len);
      batched_upload_kernel<<<1, 256, 0, st>>>(chunk, w + P.off_table + off);
    }
    if (P.prep_total > 0)
      batched_prepass_kernel<<<(unsigned)std::min(P.prep_total, 64 * num_sms()), 256, 0, st>>>(
          H, P.KP, ahi, alo, bhi, blo, violation);
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  const int64_t ra = std::max<int64_t>(P.rows_a, 1), rb = std::max<int64_t>(P.rows_b, 1);
  const int64_t kp = std::max<int64_t>(P.KP, TKA);
  MMSR_TRY_STATUS(make_tmap_2d_16bit(&ta_hi, ahi, ra, kp, kp, TBM, true, TBK));
  MMSR_TRY_STATUS(make_tmap_2d_16bit(&ta_lo, alo, ra, kp, kp, TBM, true, TBK));
  MMSR_TRY_STATUS(make_tmap_2d_16bit(&tb_hi, bhi, rb, kp, kp, TBN, true, TBK));
  MMSR_TRY_STATUS(make_tmap_2d_16bit(&tb_lo, blo, rb, kp, kp, TBN, true, TBK));
  static std::atomic<uint64_t> configured{0};
  MMSR_TRY_STATUS(smem_limit_once(batched_kernel, BSMEM, configured));
  const int sms = num_sms();
  if (P.total_tiles > 0) {
    TraceScope tr(kTrBatched, st);
    const int grid = std::min(sms, P.total_tiles);
    batched_kernel<<<grid, kBThreads, BSMEM, st>>>(H, ta_hi, ta_lo, tb_hi, tb_lo, counter,
                                                   reinterpret_cast<float*>(w + P.off_slots),
                                                   reinterpret_cast<int*>(w + P.off_cnt));
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  if (P.post_total > 0) {
    TraceScope tr(kTrStrassenPost, st);
    batched_post_kernel<<<(unsigned)std::min(P.post_total, 16 * sms), 256, 0, st>>>(H);
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  if (P.mp16_total > 0) {
    TraceScope tr(kTrMinplus16Leaf, st);
    batched_minplus16_kernel<<<(unsigned)P.mp16_total, 256, 0, st>>>(H, violation);
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  if (P.mp_total > 0) {
    TraceScope tr(kTrMinplusLeaf, st);
    static std::atomic<uint64_t> fb_configured{0};
    MMSR_TRY_STATUS(smem_limit_once(batched_minplus32_kernel, mp::SMEM_BYTES, fb_configured));
    batched_minplus32_kernel<<<(unsigned)P.mp_total, 256, mp::SMEM_BYTES, st>>>(H, violation);
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  return MM_OK;
}
