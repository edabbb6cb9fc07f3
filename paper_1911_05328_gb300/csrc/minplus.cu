// minplus.cu -- (min,+) tropical leaf kernel and the min-reduction of
// split-K partials.
//
// Leaf (the paper's base-kernel, Section 3, applied to the closed semiring
// of Section 2 with (+) = min, (x) = +): one CTA owns a BM x BN tile of C
// and walks its k-slice in BK-wide blocks, keeping the tile's accumulators
// in registers -- the k-serial, in-place CO2 order inside a slice (Fig.
// mm-n2).  Split-K slices beyond the first write whole m x n buffers that
// the reduction folds into C, the madd of CO3 (Fig. mm-n3); min is exact
// and order-free, so any number of slices gives bit-identical C.
//
// Sentinel arithmetic: values are in [0, 2^30] with 2^30 = +inf.  Sums are
// formed in uint32 (<= 2^31, no wrap) and the accumulator starts at 2^30,
// so min(acc, a + b) never exceeds the sentinel and needs no clamp.  Padding
// outside the matrix (k tail) is filled with the sentinel, which can never
// win a min.
#include <atomic>

#include "common.cuh"

namespace mmsr {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3, THREADS = 256;
constexpr int LDA = BK + 4;  // padded row of the A stage (ints), keeps 16B alignment
constexpr int SMEM_A = STAGES * BM * LDA;
constexpr int SMEM_B = STAGES * BK * BN;
constexpr size_t SMEM_BYTES = (SMEM_A + SMEM_B) * sizeof(int32_t);

// Load one BM x BK block of A and BK x BN block of B into stage `st`.
// Interior blocks use 16-byte cp.async; blocks that cross an edge (or when
// rows are not 16-byte aligned) take guarded scalar loads with +inf fill.
__device__ __forceinline__ void load_stage(int32_t* As, int32_t* Bs, const int32_t* __restrict__ A,
                                           const int32_t* __restrict__ B, int64_t m, int64_t n,
                                           int64_t k, int64_t i0, int64_t j0, int64_t k0,
                                           bool vec, int tid) {
  const bool a_full = vec && (i0 + BM <= m) && (k0 + BK <= k);
  const bool b_full = vec && (k0 + BK <= k) && (j0 + BN <= n);
  // A: 128 rows x 32 ints = 1024 16-byte chunks, 4 per thread.
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = tid + q * THREADS;
    const int row = idx >> 3, c4 = idx & 7;
    int32_t* dst = As + row * LDA + c4 * 4;
    if (a_full) {
      cp_async16(dst, A + (i0 + row) * k + k0 + c4 * 4);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t gi = i0 + row, gk = k0 + c4 * 4 + e;
        dst[e] = (gi < m && gk < k) ? A[gi * k + gk] : kInf;
      }
    }
  }
  // B: 32 rows x 128 ints = 1024 chunks, 4 per thread.
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = tid + q * THREADS;
    const int row = idx >> 5, c4 = idx & 31;
    int32_t* dst = Bs + row * BN + c4 * 4;
    if (b_full) {
      cp_async16(dst, B + (k0 + row) * n + j0 + c4 * 4);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t gk = k0 + row, gj = j0 + c4 * 4 + e;
        dst[e] = (gk < k && gj < n) ? B[gk * n + gj] : kInf;
      }
    }
  }
}

// ------------------------------------------------------------------------
// Packed 2 x 16-bit fast path.
//
// When every finite entry of A and B is <= kPackMax (and everything else is
// the sentinel), the product is exact in 16-bit lanes: entries map to
// min(v, 32767), so the sentinel becomes 32767 and finite sums stay
// <= 2 * 16383 = 32766 < 32767; any sum that involves a sentinel is >= 32767
// and can never beat the accumulator, which starts at 32767.  A result of
// 32767 therefore means +inf and maps back to 2^30.  One __viaddmin_u16x2
// computes two outputs, twice the 32-bit rate.  A range scan decides the path
// on the device (no host round trip); the loser kernel exits at once.
constexpr int kPackMax = 16383;
constexpr uint32_t kInf16 = 32767u;
constexpr int kPackSlots = 4096;

struct PackSlot {
  int viol;
  unsigned int done;
  int verdict;  // 1: packed path valid for this call's inputs
  int pad;
};
__device__ PackSlot g_pack[kPackSlots];

__device__ __forceinline__ int pack_verdict(int slot) { return __ldcg(&g_pack[slot].verdict); }

__device__ __forceinline__ int out_of_pack_range(int v) {
  return (v < 0) | ((v > kPackMax) & (v != kInf));
}

// Scans A and B; the last block to finish publishes the verdict and resets
// the slot's scratch (so the slot is clean for its next use).
__global__ void __launch_bounds__(256) range_scan_kernel(const int32_t* __restrict__ A, int64_t na,
                                                         const int32_t* __restrict__ B, int64_t nb,
                                                         int slot, bool vec) {
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int pass = 0; pass < 2; ++pass) {
    const int32_t* X = pass ? B : A;
    const int64_t cnt = pass ? nb : na;
    if (vec) {
      for (int64_t v = t0; v < cnt / 4; v += stride) {
        const int4 q = __ldcs(reinterpret_cast<const int4*>(X) + v);
        bad |= out_of_pack_range(q.x) | out_of_pack_range(q.y) | out_of_pack_range(q.z) |
               out_of_pack_range(q.w);
      }
    } else {
      for (int64_t e = t0; e < cnt; e += stride) bad |= out_of_pack_range(X[e]);
    }
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    PackSlot* ps = &g_pack[slot];
    if (bad) atomicOr(&ps->viol, 1);
    __threadfence();
    const unsigned prev = atomicAdd(&ps->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const int v = atomicExch(&ps->viol, 0);
      atomicExch(&ps->verdict, v ? 0 : 1);
      atomicExch(&ps->done, 0u);
    }
  }
}

constexpr int PBM = 128, PBN = 256, PBK = 16, PTHREADS = 256;  // k sub-blocks of 16
constexpr int PBNP = PBN / 2;  // packed column pairs per tile row
constexpr size_t PSMEM_BYTES = 2 * (size_t)(PBK * PBM + PBK * PBNP) * sizeof(uint32_t);

__device__ __forceinline__ uint32_t to16(int v) { return min((uint32_t)v, kInf16); }

struct PackStage {
  int4 a[2];
  int4 b[4];
};

// Loads the 16-wide k sub-block at k0; columns at or past `kend` (the end
// of this CTA's k-slice, or k) read as the sentinel.
__device__ __forceinline__ void packed_load(PackStage& r, const int32_t* __restrict__ A,
                                            const int32_t* __restrict__ B, int64_t m, int64_t n,
                                            int64_t k, int64_t kend, int64_t i0, int64_t j0,
                                            int64_t k0, bool vec, int tid) {
  const bool a_full = vec && (i0 + PBM <= m) && (k0 + PBK <= kend);
  const bool b_full = vec && (k0 + PBK <= kend) && (j0 + PBN <= n);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int row = tid & 127, c4 = (tid >> 7) + 2 * q;
    if (a_full) {
      r.a[q] = __ldg(reinterpret_cast<const int4*>(A + (i0 + row) * k + k0 + c4 * 4));
    } else {
      int v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t gi = i0 + row, gk = k0 + c4 * 4 + e;
        v[e] = (gi < m && gk < kend) ? A[gi * k + gk] : kInf;
      }
      r.a[q] = make_int4(v[0], v[1], v[2], v[3]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = tid + q * PTHREADS;
    const int row = idx >> 6, c4 = idx & 63;
    if (b_full) {
      r.b[q] = __ldg(reinterpret_cast<const int4*>(B + (k0 + row) * n + j0 + c4 * 4));
    } else {
      int v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t gk = k0 + row, gj = j0 + c4 * 4 + e;
        v[e] = (gk < kend && gj < n) ? B[gk * n + gj] : kInf;
      }
      r.b[q] = make_int4(v[0], v[1], v[2], v[3]);
    }
  }
}

// A goes to smem k-major with each value duplicated into both halves; B as
// packed (even, odd) column pairs.
__device__ __forceinline__ void packed_store(const PackStage& r, uint32_t* As, uint32_t* Bs, int tid) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int row = tid & 127, c4 = (tid >> 7) + 2 * q;
    const int v[4] = {r.a[q].x, r.a[q].y, r.a[q].z, r.a[q].w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t h = to16(v[e]);
      As[(c4 * 4 + e) * PBM + row] = h | (h << 16);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int idx = tid + q * PTHREADS;
    const int row = idx >> 6, c4 = idx & 63;
    const uint32_t p0 = to16(r.b[q].x) | (to16(r.b[q].y) << 16);
    const uint32_t p1 = to16(r.b[q].z) | (to16(r.b[q].w) << 16);
    *reinterpret_cast<uint2*>(Bs + row * PBNP + c4 * 2) = make_uint2(p0, p1);
  }
}

__global__ void __launch_bounds__(PTHREADS, 2)
    minplus16_leaf_kernel(int64_t m, int64_t n, int64_t k, const int32_t* __restrict__ A,
                          const int32_t* __restrict__ B, int32_t* __restrict__ C,
                          int32_t* __restrict__ W, int kb_per_slice, bool vec, int slot) {
  if (pack_verdict(slot) != 1) return;
  extern __shared__ __align__(16) uint32_t psmem[];
  uint32_t* As = psmem;                      // [2][PBK][PBM]
  uint32_t* Bs = psmem + 2 * PBK * PBM;      // [2][PBK][PBNP]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * PBM, j0 = (int64_t)blockIdx.x * PBN;
  const int z = blockIdx.z;
  // slices are counted in the 32-wide k-blocks of the 32-bit leaf; this
  // kernel walks each slice in 16-wide sub-blocks
  const int64_t kbeg = (int64_t)z * kb_per_slice * BK;
  const int64_t kend = min(k, kbeg + (int64_t)kb_per_slice * BK);
  const int nkb = kend > kbeg ? (int)((kend - kbeg + PBK - 1) / PBK) : 0;

  uint32_t acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = kInf16 | (kInf16 << 16);

  PackStage stg;
  if (nkb > 0) {
    packed_load(stg, A, B, m, n, k, kend, i0, j0, kbeg, vec, tid);
    packed_store(stg, As, Bs, tid);
  }
  __syncthreads();
  for (int kb = 0; kb < nkb; ++kb) {
    const int cur = kb & 1;
    if (kb + 1 < nkb) packed_load(stg, A, B, m, n, k, kend, i0, j0, kbeg + (int64_t)(kb + 1) * PBK, vec, tid);
    const uint32_t* as = As + cur * PBK * PBM;
    const uint32_t* bs = Bs + cur * PBK * PBNP;
#pragma unroll
    for (int kk = 0; kk < PBK; ++kk) {
      const uint4 a0 = *reinterpret_cast<const uint4*>(as + kk * PBM + ty * 4);
      const uint4 a1 = *reinterpret_cast<const uint4*>(as + kk * PBM + 64 + ty * 4);
      const uint4 b0 = *reinterpret_cast<const uint4*>(bs + kk * PBNP + tx * 4);
      const uint4 b1 = *reinterpret_cast<const uint4*>(bs + kk * PBNP + 64 + tx * 4);
      const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const uint32_t b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = __viaddmin_u16x2(a[i], b[j], acc[i][j]);
    }
    if (kb + 1 < nkb) packed_store(stg, As + (cur ^ 1) * PBK * PBM, Bs + (cur ^ 1) * PBK * PBNP, tid);
    __syncthreads();
  }

  int32_t* out = (z == 0) ? C : W + (int64_t)(z - 1) * m * n;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gi = i0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + (i - 4)));
    if (gi >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gj = j0 + 2 * (h * 64 + tx * 4);  // 8 consecutive output columns
      int v[8];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const uint32_t w = acc[i][h * 4 + p];
        const uint32_t lo = w & 0xFFFFu, hi = w >> 16;
        v[2 * p] = lo >= kInf16 ? kInf : (int)lo;
        v[2 * p + 1] = hi >= kInf16 ? kInf : (int)hi;
      }
      int32_t* dst = out + gi * n + gj;
      if (vec && gj + 8 <= n) {
        *reinterpret_cast<int4*>(dst) = make_int4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<int4*>(dst + 4) = make_int4(v[4], v[5], v[6], v[7]);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (gj + e < n) dst[e] = v[e];
      }
    }
  }
}

__global__ void __launch_bounds__(THREADS, 2)
    minplus_leaf_kernel(int64_t m, int64_t n, int64_t k, const int32_t* __restrict__ A,
                        const int32_t* __restrict__ B, int32_t* __restrict__ C,
                        int32_t* __restrict__ W, int kb_per_slice, bool vec, int slot) {
  // The packed 2 x 16-bit leaf already produced C when the range scan of
  // this call found every finite input small enough.
  if (slot >= 0 && pack_verdict(slot) == 1) return;
  extern __shared__ __align__(16) int32_t smem[];
  int32_t* As = smem;
  int32_t* Bs = smem + SMEM_A;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  const int z = blockIdx.z;
  const int64_t kb_total = (k + BK - 1) / BK;
  const int64_t kb_begin = (int64_t)z * kb_per_slice;
  const int64_t kb_end = min(kb_total, kb_begin + kb_per_slice);
  const int nkb = kb_end > kb_begin ? (int)(kb_end - kb_begin) : 0;

  uint32_t acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = (uint32_t)kInf;

#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nkb)
      load_stage(As + s * BM * LDA, Bs + s * BK * BN, A, B, m, n, k, i0, j0,
                 (kb_begin + s) * BK, vec, tid);
    cp_async_commit();
  }

  for (int kb = 0; kb < nkb; ++kb) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    {
      const int nxt = kb + STAGES - 1;
      if (nxt < nkb) {
        const int sn = nxt % STAGES;
        load_stage(As + sn * BM * LDA, Bs + sn * BK * BN, A, B, m, n, k, i0, j0,
                   (kb_begin + nxt) * BK, vec, tid);
      }
      cp_async_commit();
    }
    const int sc = kb % STAGES;
    const int32_t* as = As + sc * BM * LDA;
    const int32_t* bs = Bs + sc * BK * BN;
#pragma unroll
    for (int kq = 0; kq < BK; kq += 4) {
      uint4 a4[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = (i < 4) ? (ty * 4 + i) : (64 + ty * 4 + (i - 4));
        a4[i] = *reinterpret_cast<const uint4*>(as + row * LDA + kq);
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint4 b0 = *reinterpret_cast<const uint4*>(bs + (kq + kk) * BN + tx * 4);
        const uint4 b1 = *reinterpret_cast<const uint4*>(bs + (kq + kk) * BN + 64 + tx * 4);
        const uint32_t b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint32_t a = kk == 0 ? a4[i].x : kk == 1 ? a4[i].y : kk == 2 ? a4[i].z : a4[i].w;
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = __viaddmin_u32(a, b[j], acc[i][j]);
        }
      }
    }
  }
  cp_async_wait<0>();

  int32_t* out = (z == 0) ? C : W + (int64_t)(z - 1) * m * n;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gi = i0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + (i - 4)));
    if (gi >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gj = j0 + h * 64 + tx * 4;
      int32_t* dst = out + gi * n + gj;
      if (vec && gj + 4 <= n) {
        *reinterpret_cast<uint4*>(dst) =
            make_uint4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (gj + e < n) dst[e] = (int32_t)acc[i][h * 4 + e];
      }
    }
  }
}

// C = min(C, W_0, ..., W_{parts-1}), element-wise, 16-byte vectors.
__global__ void __launch_bounds__(256) min_reduce_kernel(int64_t count, int32_t* __restrict__ C,
                                                         const int32_t* __restrict__ W, int parts,
                                                         bool vec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const int64_t nv = count >> 2;
    for (int64_t v = t; v < nv; v += stride) {
      int4 c = reinterpret_cast<const int4*>(C)[v];
      for (int p = 0; p < parts; ++p) {
        const int4 w = __ldcs(reinterpret_cast<const int4*>(W + (int64_t)p * count) + v);
        c.x = min(c.x, w.x);
        c.y = min(c.y, w.y);
        c.z = min(c.z, w.z);
        c.w = min(c.w, w.w);
      }
      reinterpret_cast<int4*>(C)[v] = c;
    }
    for (int64_t e = (nv << 2) + t; e < count; e += stride) {
      int32_t c = C[e];
      for (int p = 0; p < parts; ++p) c = min(c, W[(int64_t)p * count + e]);
      C[e] = c;
    }
  } else {
    for (int64_t e = t; e < count; e += stride) {
      int32_t c = C[e];
      for (int p = 0; p < parts; ++p) c = min(c, W[(int64_t)p * count + e]);
      C[e] = c;
    }
  }
}

}  // namespace

int minplus_tile_k() { return BK; }

int g_packed_mode = 1;  // 1: use the packed path when the range scan allows, 0: never

cudaError_t launch_minplus_leaf(int64_t m, int64_t n, int64_t k, const int32_t* A,
                                const int32_t* B, int32_t* C, int32_t* W, int s,
                                int kb_per_slice, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    MMSR_CUDA_TRY(cudaFuncSetAttribute(minplus_leaf_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES));
    MMSR_CUDA_TRY(cudaFuncSetAttribute(minplus16_leaf_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)PSMEM_BYTES));
    configured = true;
  }
  const bool vec = (k % 4 == 0) && (n % 4 == 0) && aligned16(A) && aligned16(B) && aligned16(C) &&
                   (W == nullptr || aligned16(W));
  int slot = -1;
  if (g_packed_mode && k > 0) {
    // the packed tile and the 32-bit tile split k into the same 32-wide blocks
    static std::atomic<unsigned> counter{0};
    slot = (int)(counter.fetch_add(1u) % (unsigned)kPackSlots);
    {
      TraceScope tr(kTrRangeScan, st);
      const bool svec = aligned16(A) && aligned16(B) && ((m * k) % 4 == 0) && ((k * n) % 4 == 0);
      int64_t blocks = ((m * k + k * n) / (svec ? 4 : 1) + 255) / 256;
      if (blocks > (int64_t)kNumSMs * 4) blocks = (int64_t)kNumSMs * 4;
      if (blocks < 1) blocks = 1;
      range_scan_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, m * k, B, k * n, slot, svec);
      MMSR_CUDA_TRY(cudaGetLastError());
    }
    {
      TraceScope tr(kTrMinplus16Leaf, st);
      dim3 pgrid((unsigned)((n + PBN - 1) / PBN), (unsigned)((m + PBM - 1) / PBM), (unsigned)s);
      minplus16_leaf_kernel<<<pgrid, PTHREADS, PSMEM_BYTES, st>>>(m, n, k, A, B, C, W, kb_per_slice,
                                                                   vec, slot);
      MMSR_CUDA_TRY(cudaGetLastError());
    }
  }
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)s);
  TraceScope tr(kTrMinplusLeaf, st);
  minplus_leaf_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(m, n, k, A, B, C, W, kb_per_slice, vec,
                                                         slot);
  return cudaGetLastError();
}

cudaError_t launch_min_reduce(int64_t count, int32_t* C, const int32_t* W, int parts,
                              cudaStream_t st) {
  if (parts <= 0 || count <= 0) return cudaSuccess;
  const bool vec = aligned16(C) && aligned16(W) && (count % 4 == 0);
  const int64_t work = vec ? count / 4 : count;
  int64_t blocks = (work + 255) / 256;
  const int64_t cap = (int64_t)kNumSMs * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  TraceScope tr(kTrMinReduce, st);
  min_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(count, C, W, parts, vec);
  return cudaGetLastError();
}

}  // namespace mmsr

// ---------------------------------------------------------------------------
// Allocation-free split-K entry point.
//
// Some callers cannot hand the library a workspace: code running inside a
// host framework whose memory pool owns the device (a raw cudaMalloc there
// bypasses the pool's accounting and may synchronise the whole device), or
// callers with a fixed memory footprint decided at start-up.  For them the
// split-K partials of the (min,+) product live in a file-scope device array
// that is part of the library image, so this entry point allocates nothing.
#include <mutex>

namespace mmsr {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB, per GPU, held until exit
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int32_t g_minplus_scratch[kStaticScratchBytes / sizeof(int32_t)];

std::mutex g_scratch_mu;
int32_t* g_scratch_addr[kMaxDevices] = {};

// Device address of g_minplus_scratch on the current device.  In host code
// the symbol name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
cudaError_t scratch_address(int32_t** out) {
  int dev = 0;
  MMSR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    MMSR_CUDA_TRY(cudaGetSymbolAddress(&p, g_minplus_scratch));
    g_scratch_addr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace mmsr

extern "C" int mm_minplus_noalloc(int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                                  void* C, int split_k, void* stream) {
  using namespace mmsr;
  if (m < 0 || n < 0 || k < 0 || split_k < 1) return MM_ERR_ARG;
  if (m == 0 || n == 0) return MM_OK;
  if (!C || (k > 0 && (!A || !B))) return MM_ERR_ARG;
  if (!aligned16(C) || (k > 0 && (!aligned16(A) || !aligned16(B)))) return MM_ERR_ALIGN;
  if (m > (int64_t(1) << 22) || n > (int64_t(1) << 22) || k > (int64_t(1) << 22)) return MM_ERR_SHAPE;
  const int64_t kb_total = (k + BK - 1) / BK;
  int64_t s = split_k;
  if (s > 64) s = 64;
  if (kb_total > 0 && s > kb_total) s = kb_total;
  if (kb_total == 0) s = 1;
  const int64_t kbs = kb_total > 0 ? (kb_total + s - 1) / s : 0;
  if (kbs > 0) s = (kb_total + kbs - 1) / kbs;
  const uint64_t need = (uint64_t)(s - 1) * (uint64_t)m * (uint64_t)n * sizeof(int32_t);
  if (need > kStaticScratchBytes) return MM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* W = nullptr;
  if (s > 1) {
    cudaError_t e = scratch_address(&W);
    if (e != cudaSuccess) return MM_ERR_CUDA;
  }
  // Every element of each used partial slice is written by the leaf before
  // the reduction reads it, so stale contents from an earlier call are never
  // observed and nothing needs clearing.
  cudaError_t e = launch_minplus_leaf(m, n, k, static_cast<const int32_t*>(A),
                                      static_cast<const int32_t*>(B), static_cast<int32_t*>(C), W,
                                      (int)s, (int)kbs, st);
  if (e == cudaSuccess && s > 1) e = launch_min_reduce(m * n, static_cast<int32_t*>(C), W, (int)(s - 1), st);
  return e == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}
