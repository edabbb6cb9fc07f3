// minplus_tile.cuh -- device-side (min,+) tile mainloops shared by the
// standalone leaf kernels (minplus.cu) and the persistent batched kernel.
//
// Leaf (the paper's base-kernel, Section 3, on the closed semiring of
// Section 2 with (+) = min, (x) = +): a 256-thread group owns one output tile
// and walks its k-range keeping the accumulators in registers -- the
// k-serial, in-place CO2 order (Fig. mm-n2).
//
// Sentinel arithmetic: values are in [0, 2^30] with 2^30 = +inf.  Sums are
// formed in uint32 (<= 2^31, no wrap) and the accumulator starts at 2^30,
// so min(acc, a + b) never exceeds the sentinel and needs no clamp.  Padding
// outside the matrix (k tail) is filled with the sentinel, which can never
// win a min.
//
// Packed 2 x 16-bit variant: when every finite entry of A and B is
// <= kPackMax (and everything else is the sentinel), the product is exact in
// 16-bit lanes: entries map to min(v, 32767), so the sentinel becomes 32767
// and finite sums stay <= 2 * 16383 = 32766 < 32767; any sum that involves
// a sentinel is >= 32767 and can never beat the accumulator, which starts at
// 32767.  A result of 32767 therefore means +inf and maps back to 2^30.  One
// __viaddmin_u16x2 computes two outputs, twice the 32-bit rate.
#pragma once

#include "common.cuh"

namespace mmsr {
namespace mp {

// Barrier for the whole CTA, or for the 256 threads of named barrier 1.
struct SyncCta {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncNamed256 {
  __device__ __forceinline__ void operator()() const { asm volatile("bar.sync 1, 256;" ::: "memory"); }
};

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

constexpr int kPackMax = 16383;
constexpr uint32_t kInf16 = 32767u;

__device__ __forceinline__ int out_of_pack_range(int v) {
  return (v < 0) | ((v > kPackMax) & (v != kInf));
}

constexpr int PBM = 128, PBN = 256, PBK = 16, PTHREADS = 256;  // k sub-blocks of 16
constexpr int PBNP = PBN / 2;  // packed column pairs per tile row
constexpr size_t PSMEM_BYTES = 2 * (size_t)(PBK * PBM + PBK * PBNP) * sizeof(uint32_t);

__device__ __forceinline__ uint32_t to16(int v) { return min((uint32_t)v, kInf16); }

// Tile shapes of the packed leaf: 128 rows x 32 NP columns, each of the 256
// threads holding 8 rows x NP column pairs.  NP = 8 (256 columns) is the
// standard tile; NP = 4 (128 columns) serves narrow products.
template <int NP>
struct PackTile {
  static_assert(NP == 4 || NP == 8, "column pairs per thread");
  static constexpr int TN = 32 * NP;   // output columns
  static constexpr int TNP = TN / 2;   // packed column pairs
  static constexpr int BQ = NP / 2;    // 16-byte B loads per thread and k sub-block
  static constexpr int BROW = TN / 4;  // 16-byte chunks per B row
  static constexpr int BROW_LOG2 = NP == 8 ? 6 : 5;
  static constexpr size_t SMEM = 2 * (size_t)(PBK * PBM + PBK * TNP) * sizeof(uint32_t);
};

template <int NP>
struct PackStage {
  int4 a[2];
  int4 b[NP / 2];
};

// Loads the 16-wide k sub-block at k0; columns at or past `kend` (the end
// of this CTA's k-slice, or k) read as the sentinel.
template <int NP>
__device__ __forceinline__ void packed_load(PackStage<NP>& r, const int32_t* __restrict__ A,
                                            const int32_t* __restrict__ B, int64_t m, int64_t n,
                                            int64_t k, int64_t kend, int64_t i0, int64_t j0,
                                            int64_t k0, bool vec, int tid) {
  using T = PackTile<NP>;
  const bool a_full = vec && (i0 + PBM <= m) && (k0 + PBK <= kend);
  const bool b_full = vec && (k0 + PBK <= kend) && (j0 + T::TN <= n);
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
  for (int q = 0; q < T::BQ; ++q) {
    const int idx = tid + q * PTHREADS;
    const int row = idx >> T::BROW_LOG2, c4 = idx & (T::BROW - 1);
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
template <int NP>
__device__ __forceinline__ void packed_store(const PackStage<NP>& r, uint32_t* As, uint32_t* Bs, int tid) {
  using T = PackTile<NP>;
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
  for (int q = 0; q < T::BQ; ++q) {
    const int idx = tid + q * PTHREADS;
    const int row = idx >> T::BROW_LOG2, c4 = idx & (T::BROW - 1);
    const uint32_t p0 = to16(r.b[q].x) | (to16(r.b[q].y) << 16);
    const uint32_t p1 = to16(r.b[q].z) | (to16(r.b[q].w) << 16);
    *reinterpret_cast<uint2*>(Bs + row * T::TNP + c4 * 2) = make_uint2(p0, p1);
  }
}

// One 128 x 32 NP output tile of the packed leaf over k in [kbeg, kend),
// executed by 256 threads (tid 0..255) that synchronise with `bar`.  With
// `merge` the tile is folded into C by an atomic min (C must already hold
// the semiring's 0 or another partial of the same product) instead of stored.
template <class Bar, int NP = 8>
__device__ __forceinline__ void minplus16_tile(const int32_t* __restrict__ A, const int32_t* __restrict__ B,
                                               int32_t* __restrict__ C, int32_t* __restrict__ W, int z,
                                               int64_t m, int64_t n, int64_t k,
                                               int64_t i0, int64_t j0, int64_t kbeg, int64_t kend,
                                               bool vec, int tid, uint32_t* psmem, Bar bar,
                                               bool merge = false) {
  using T = PackTile<NP>;
  uint32_t* As = psmem;                      // [2][PBK][PBM]
  uint32_t* Bs = psmem + 2 * PBK * PBM;      // [2][PBK][TNP]
  const int tx = tid & 15, ty = tid >> 4;
  const int nkb = kend > kbeg ? (int)((kend - kbeg + PBK - 1) / PBK) : 0;

  uint32_t acc[8][NP];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[i][j] = kInf16 | (kInf16 << 16);

  PackStage<NP> stg;
  if (nkb > 0) {
    packed_load<NP>(stg, A, B, m, n, k, kend, i0, j0, kbeg, vec, tid);
    packed_store<NP>(stg, As, Bs, tid);
  }
  bar();
  for (int kb = 0; kb < nkb; ++kb) {
    const int cur = kb & 1;
    if (kb + 1 < nkb)
      packed_load<NP>(stg, A, B, m, n, k, kend, i0, j0, kbeg + (int64_t)(kb + 1) * PBK, vec, tid);
    const uint32_t* as = As + cur * PBK * PBM;
    const uint32_t* bs = Bs + cur * PBK * T::TNP;
#pragma unroll
    for (int kk = 0; kk < PBK; ++kk) {
      const uint4 a0 = *reinterpret_cast<const uint4*>(as + kk * PBM + ty * 4);
      const uint4 a1 = *reinterpret_cast<const uint4*>(as + kk * PBM + 64 + ty * 4);
      const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const uint4 b0 = *reinterpret_cast<const uint4*>(bs + kk * T::TNP + tx * 4);
      if constexpr (NP == 8) {
        const uint4 b1 = *reinterpret_cast<const uint4*>(bs + kk * T::TNP + 64 + tx * 4);
        const uint32_t b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = __viaddmin_u16x2(a[i], b[j], acc[i][j]);
      } else {
        const uint32_t b[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = __viaddmin_u16x2(a[i], b[j], acc[i][j]);
      }
    }
    if (kb + 1 < nkb) packed_store<NP>(stg, As + (cur ^ 1) * PBK * PBM, Bs + (cur ^ 1) * PBK * T::TNP, tid);
    bar();
  }

  // slice 0 accumulates in C, slice z > 0 in the z-th workspace buffer
  int32_t* out = (z == 0) ? C : W + (int64_t)(z - 1) * m * n;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gi = i0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + (i - 4)));
    if (gi >= m) continue;
#pragma unroll
    for (int h = 0; h < NP / 4; ++h) {
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
      if (merge) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (gj + e < n) atomicMin(reinterpret_cast<unsigned int*>(dst + e), (unsigned int)v[e]);
      } else if (vec && gj + 8 <= n) {
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

// One 128 x 128 output tile of the 32-bit leaf over k-blocks
// [kb_begin, kb_begin + nkb), executed by 256 threads that synchronise with `bar`.
// With `merge` the tile is folded into C by an atomic min (C must already
// hold the sentinel or a partial result), otherwise it is stored.
template <class Bar>
__device__ __forceinline__ void minplus32_tile(const int32_t* __restrict__ A, const int32_t* __restrict__ B,
                                               int32_t* __restrict__ C, int32_t* __restrict__ W, int z,
                                               int64_t m, int64_t n, int64_t k,
                                               int64_t i0, int64_t j0, int64_t kb_begin, int nkb,
                                               bool vec, int tid, int32_t* smem, Bar bar, bool merge = false) {
  int32_t* As = smem;
  int32_t* Bs = smem + SMEM_A;
  const int tx = tid & 15, ty = tid >> 4;

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
    bar();
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

  // slice 0 accumulates in C, slice z > 0 in the z-th workspace buffer
  int32_t* out = (z == 0) ? C : W + (int64_t)(z - 1) * m * n;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gi = i0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + (i - 4)));
    if (gi >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gj = j0 + h * 64 + tx * 4;
      int32_t* dst = out + gi * n + gj;
      if (merge) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (gj + e < n) atomicMin(reinterpret_cast<unsigned int*>(dst + e), acc[i][h * 4 + e]);
      } else if (vec && gj + 4 <= n) {
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

}  // namespace mp
}  // namespace mmsr
