// orand.cu -- boolean (or, and) semiring: C[i][j] = OR_t (A[i][t] AND B[t][j]).
//
// Operands are bit-packed along k into the workspace (A as m x KW words,
// B transposed as n x KW words, KW = ceil(k / 32), bit t % 32 of word t / 32
// set iff the entry is nonzero), so one 32-bit AND/OR covers 32 terms of the
// (+)-sum.  The leaf is the paper's base-kernel (Section 3) on this semiring:
// a 128 x 128 CTA tile, 256 threads with 8 x 8 register accumulators, words
// staged through shared memory, k-serial within a slice (Fig. mm-n2).  Split-K
// slices write byte partials that an OR folds into C (the madd of Fig. mm-n3).
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace mmsr {
namespace {

constexpr int OBM = 128, OBN = 128, OBW = 32;  // tile rows, cols, words per stage (1024 k)
// Shared tiles are stored k-major ([word][row]) with a 132-word pitch: a
// thread's four consecutive rows are one 16-byte load, and the staging
// stores (4 rows x 8 words per warp) fall in 32 distinct banks.
constexpr int OLD = OBM + 4;

// Four bytes -> four bits: bit b of the result is set iff byte b of v is
// nonzero.  The 0/1 flags sit at bits 0, 8, 16, 24; the multiplier copies
// them to bits 21..24 without overlapping partial products (no carries).
__device__ __forceinline__ uint32_t nonzero_nibble(uint32_t v) {
  const uint32_t f = __vcmpne4(v, 0u) & 0x01010101u;
  return ((f * 0x204081u) >> 21) & 0xFu;
}

__global__ void __launch_bounds__(256) pack_rows_kernel(const uint8_t* __restrict__ A, int64_t m,
                                                        int64_t k, int64_t KW,
                                                        uint32_t* __restrict__ P, bool vec) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * KW;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / KW, w = e - i * KW;
    uint32_t word = 0;
    const int64_t t0 = w * 32;
    if (vec && t0 + 32 <= k) {
      // rows are 16-byte aligned (k % 16 == 0): two 16-byte loads per word
      const uint4* src = reinterpret_cast<const uint4*>(A + i * k + t0);
      const uint4 lo = __ldcs(src), hi = __ldcs(src + 1);
      const uint32_t v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) word |= nonzero_nibble(v[q]) << (4 * q);
    } else {
      for (int b = 0; b < 32; ++b) {
        const int64_t t = t0 + b;
        if (t < k && A[i * k + t]) word |= 1u << b;
      }
    }
    P[e] = word;
  }
}

// B (k x n) -> bits of B^T (n x KW).  A block covers 32 columns and 8 words
// (256 rows of B); warp q takes word w = 8 * blockIdx.y + q: lane l loads the
// 32 bytes of row 32 w + l, and one ballot per column gathers that column's
// word (bit l = row 32 w + l).  The words go through shared memory so that
// each column's 8 words are stored as one 32-byte run.
__global__ void __launch_bounds__(256) pack_cols_kernel(const uint8_t* __restrict__ B, int64_t k,
                                                        int64_t n, int64_t KW,
                                                        uint32_t* __restrict__ P, bool vec) {
  __shared__ uint32_t words[32][9];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int64_t w = (int64_t)blockIdx.y * 8 + q;
  const int64_t t = w * 32 + lane;
  uint32_t v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = 0u;
  if (w < KW && t < k) {
    const uint8_t* row = B + t * n + j0;
    if (vec && j0 + 32 <= n) {
      // rows are 16-byte aligned (n % 16 == 0) and j0 is a multiple of 32
      const uint4 a = __ldcs(reinterpret_cast<const uint4*>(row));
      const uint4 b = __ldcs(reinterpret_cast<const uint4*>(row) + 1);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (j0 + c < n) v[c >> 2] |= (uint32_t)row[c] << (8 * (c & 3));
    }
  }
  uint32_t mine = 0;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const uint32_t bits = __ballot_sync(0xffffffffu, ((v[c >> 2] >> (8 * (c & 3))) & 0xFFu) != 0u);
    if (lane == c) mine = bits;
  }
  words[lane][q] = mine;  // column j0 + lane, word w
  __syncthreads();
  const int col = threadIdx.x >> 3, wi = threadIdx.x & 7;
  const int64_t jj = j0 + col, ww = (int64_t)blockIdx.y * 8 + wi;
  if (jj < n && ww < KW) P[jj * KW + ww] = words[col][wi];
}

// 4-byte asynchronous copy global -> shared; a word outside the operand is
// zero-filled (src-size 0: nothing is read, the address is only a valid one).
__device__ __forceinline__ void cp_async4_zfill(uint32_t* smem, const uint32_t* gmem, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(valid ? 4 : 0));
}

// Shared memory: two stages x (A, B) x OBW words x OLD rows; the next stage's
// words are copied asynchronously while the current one is consumed.
constexpr size_t kOrSmem = (size_t)2 * 2 * OBW * OLD * sizeof(uint32_t);

__global__ void __launch_bounds__(256, 2)
    orand_leaf_kernel(int64_t m, int64_t n, int64_t KW, const uint32_t* __restrict__ PA,
                      const uint32_t* __restrict__ PB, uint8_t* __restrict__ C,
                      uint8_t* __restrict__ W, int words_per_slice, bool vec_out) {
  extern __shared__ __align__(16) uint32_t osm[];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * OBM, j0 = (int64_t)blockIdx.x * OBN;
  const int z = blockIdx.z;
  const int64_t wb = (int64_t)z * words_per_slice;
  const int64_t we = min(KW, wb + words_per_slice);
  const int nblk = we > wb ? (int)((we - wb + OBW - 1) / OBW) : 0;
  // staging map: a warp copies 4 rows x 8 consecutive words (whole 32-byte
  // sectors); this thread's word column c is fixed, its rows are r0 + 8 q
  const int lane = tid & 31, wrp = tid >> 5;
  const int c = (wrp & 3) * 8 + (lane & 7);
  const int r0 = 4 * (wrp >> 2) + (lane >> 3);
  auto issue = [&](int b) {
    uint32_t* As = osm + (size_t)(b & 1) * 2 * OBW * OLD;
    uint32_t* Bs = As + OBW * OLD;
    const int64_t gw = wb + (int64_t)b * OBW + c;
    const bool wok = gw < we;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int r = r0 + 8 * q;
      const int64_t ga = i0 + r, gb = j0 + r;
      const bool va = wok && ga < m, vb = wok && gb < n;
      cp_async4_zfill(&As[c * OLD + r], va ? PA + ga * KW + gw : PA, va);
      cp_async4_zfill(&Bs[c * OLD + r], vb ? PB + gb * KW + gw : PB, vb);
    }
  };
  uint32_t acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0u;
  if (nblk > 0) issue(0);
  cp_async_commit();
  for (int b = 0; b < nblk; ++b) {
    if (b + 1 < nblk) issue(b + 1);  // into the stage read in iteration b - 1
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of stage b have landed
    __syncthreads();     // ... and every other thread's
    const uint32_t* As = osm + (size_t)(b & 1) * 2 * OBW * OLD;
    const uint32_t* Bs = As + OBW * OLD;
#pragma unroll 4
    for (int cc = 0; cc < OBW; ++cc) {
      uint32_t a[8], bb[8];
      *reinterpret_cast<uint4*>(a) = *reinterpret_cast<const uint4*>(&As[cc * OLD + ty * 4]);
      *reinterpret_cast<uint4*>(a + 4) = *reinterpret_cast<const uint4*>(&As[cc * OLD + 64 + ty * 4]);
      *reinterpret_cast<uint4*>(bb) = *reinterpret_cast<const uint4*>(&Bs[cc * OLD + tx * 4]);
      *reinterpret_cast<uint4*>(bb + 4) = *reinterpret_cast<const uint4*>(&Bs[cc * OLD + 64 + tx * 4]);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] |= a[i] & bb[j];
    }
    __syncthreads();  // stage b is read out before iteration b + 1 refills it
  }
  cp_async_wait<0>();
  uint8_t* out = (z == 0) ? C : W + (int64_t)(z - 1) * m * n;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gi = i0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + i - 4));
    if (gi >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gj = j0 + h * 64 + tx * 4;  // four consecutive outputs
      uint8_t* dst = out + gi * n + gj;
      if (vec_out && gj + 4 <= n) {
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) v |= (acc[i][h * 4 + j] ? 1u : 0u) << (8 * j);
        *reinterpret_cast<uint32_t*>(dst) = v;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (gj + j < n) dst[j] = acc[i][h * 4 + j] ? 1 : 0;
      }
    }
  }
}

__global__ void __launch_bounds__(256) or_reduce_kernel(int64_t count, uint8_t* __restrict__ C,
                                                        const uint8_t* __restrict__ W, int parts) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint8_t c = C[e];
    for (int p = 0; p < parts; ++p) c |= W[(int64_t)p * count + e];
    C[e] = c;
  }
}

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

unsigned grid_for(int64_t work) {
  int64_t b = (work + 255) / 256;
  if (b > (int64_t)num_sms() * 16) b = (int64_t)num_sms() * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

struct OrLayout {
  int64_t KW, off_b, off_part, min_bytes;
};

OrLayout or_layout(int64_t m, int64_t n, int64_t k) {
  OrLayout L;
  L.KW = (k + 31) / 32;
  L.off_b = align_up(m * L.KW * 4, 1024);
  L.off_part = L.off_b + align_up(n * L.KW * 4, 1024);
  L.min_bytes = L.off_part;
  return L;
}

}  // namespace

int plan_orand(int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  const OrLayout L = or_layout(m, n, k);
  p->tile_m = OBM;
  p->tile_n = OBN;
  p->tile_k = OBW * 32;
  p->kernel = 4;
  p->workspace_min = L.min_bytes;
  if (budget < (size_t)L.min_bytes) {
    p->split_k = 1;
    p->workspace_used = L.min_bytes;
    return MM_OK;
  }
  int s = 1, kbs = 0;
  int64_t used = 0;
  // k-blocks of OBW words (1024 terms); partials are one byte per output
  split_plan(m, n, L.KW * 32, OBW * 32, 1, budget - (size_t)L.min_bytes, &s, &kbs, &used);
  p->split_k = s;
  p->workspace_used = L.min_bytes + used;
  return MM_OK;
}

int run_orand(int64_t m, int64_t n, int64_t k, const uint8_t* A, const uint8_t* B, uint8_t* C,
              void* ws, size_t ws_bytes, cudaStream_t st) {
  mm_plan_t p;
  plan_orand(m, n, k, ws_bytes, &p);
  if ((size_t)p.workspace_min > ws_bytes) return MM_ERR_WORKSPACE;
  const OrLayout L = or_layout(m, n, k);
  uint8_t* w = static_cast<uint8_t*>(ws);
  uint32_t* PA = reinterpret_cast<uint32_t*>(w);
  uint32_t* PB = reinterpret_cast<uint32_t*>(w + L.off_b);
  uint8_t* part = p.split_k > 1 ? w + L.off_part : nullptr;
  const int s = p.split_k;
  const int64_t kb_total = (L.KW + OBW - 1) / OBW;
  const int words_per_slice = (int)(((kb_total + s - 1) / s) * OBW);
  {
    TraceScope tr(kTrOrPack, st);
    if (L.KW > 0) {
      pack_rows_kernel<<<grid_for(m * L.KW), 256, 0, st>>>(A, m, k, L.KW, PA, aligned16(A) && k % 16 == 0);
      pack_cols_kernel<<<dim3((unsigned)((n + 31) / 32), (unsigned)((L.KW + 7) / 8)), 256, 0, st>>>(
          B, k, n, L.KW, PB, aligned16(B) && n % 16 == 0);
    }
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  {
    TraceScope tr(kTrOrAndLeaf, st);
    dim3 grid((unsigned)((n + OBN - 1) / OBN), (unsigned)((m + OBM - 1) / OBM), (unsigned)s);
    static std::atomic<uint64_t> configured{0};
    MMSR_TRY_STATUS(smem_limit_once(orand_leaf_kernel, kOrSmem, configured));
    // 4-byte output stores need n % 4 == 0 and 4-byte aligned outputs
    const bool vec_out = n % 4 == 0 && ((uintptr_t)C % 4 == 0) && (part == nullptr || (uintptr_t)part % 4 == 0);
    orand_leaf_kernel<<<grid, 256, kOrSmem, st>>>(m, n, L.KW, PA, PB, C, part,
                                                  words_per_slice > 0 ? words_per_slice : OBW, vec_out);
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  if (s > 1) {
    TraceScope tr(kTrOrReduce, st);
    or_reduce_kernel<<<grid_for(m * n), 256, 0, st>>>(m * n, C, part, s - 1);
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  return MM_OK;
}

}  // namespace mmsr
