// dfma.cu -- plain FP64 (+,x) leaf on CUDA cores and the fixed-order FP64
// sum of split-K partials.
//
// This is the paper's classic base-kernel (Section 3) in FP64 with the
// k-serial CO2 order inside each k-slice (Fig. mm-n2); slices beyond the first
// write m x n FP64 buffers and the reduction adds them into C in slice order
// (the madd of CO3, Fig. mm-n3), so results are deterministic run to run.
#include <algorithm>

#include "common.cuh"

namespace mmsr {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, STAGES = 3, THREADS = 256;
constexpr int LDA = BK + 2;  // doubles; keeps 16-byte alignment of each row
constexpr int SMEM_A = STAGES * BM * LDA;
constexpr int SMEM_B = STAGES * BK * BN;
constexpr size_t SMEM_BYTES = (SMEM_A + SMEM_B) * sizeof(double);

__device__ __forceinline__ void load_stage(double* As, double* Bs, const double* __restrict__ A,
                                           const double* __restrict__ B, int64_t m, int64_t n,
                                           int64_t k, int64_t i0, int64_t j0, int64_t k0,
                                           bool vec, int tid) {
  const bool a_full = vec && (i0 + BM <= m) && (k0 + BK <= k);
  const bool b_full = vec && (k0 + BK <= k) && (j0 + BN <= n);
  // A: 64 rows x 16 doubles = 512 chunks of 2 doubles, 2 per thread.
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int idx = tid + q * THREADS;
    const int row = idx >> 3, c2 = idx & 7;
    double* dst = As + row * LDA + c2 * 2;
    if (a_full) {
      cp_async16(dst, A + (i0 + row) * k + k0 + c2 * 2);
    } else {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t gi = i0 + row, gk = k0 + c2 * 2 + e;
        dst[e] = (gi < m && gk < k) ? A[gi * k + gk] : 0.0;
      }
    }
  }
  // B: 16 rows x 64 doubles = 512 chunks, 2 per thread.
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int idx = tid + q * THREADS;
    const int row = idx >> 5, c2 = idx & 31;
    double* dst = Bs + row * BN + c2 * 2;
    if (b_full) {
      cp_async16(dst, B + (k0 + row) * n + j0 + c2 * 2);
    } else {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t gk = k0 + row, gj = j0 + c2 * 2 + e;
        dst[e] = (gk < k && gj < n) ? B[gk * n + gj] : 0.0;
      }
    }
  }
}

__global__ void __launch_bounds__(THREADS)
    dfma_leaf_kernel(int64_t m, int64_t n, int64_t k, const double* __restrict__ A,
                     const double* __restrict__ B, double* __restrict__ C,
                     double* __restrict__ W, int kb_per_slice, bool vec, int slices,
                     int64_t a_bs, int64_t b_bs, int64_t c_bs, int64_t flat_tiles_n) {
  extern __shared__ __align__(16) double smem_d[];
  // blockIdx.z = batch * slices + k-slice (batches: independent products)
  const int batch = blockIdx.z / slices;
  A += (int64_t)batch * a_bs;
  B += (int64_t)batch * b_bs;
  C += (int64_t)batch * c_bs;
  double* As = smem_d;
  double* Bs = smem_d + SMEM_A;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // tile (row, column) = (blockIdx.y, blockIdx.x); with flat_tiles_n > 0 the
  // tiles run along x alone (more row tiles than a grid's y extent allows)
  int64_t tile_r = blockIdx.y, tile_c = blockIdx.x;
  if (flat_tiles_n > 0) {
    tile_r = (int64_t)blockIdx.x / flat_tiles_n;
    tile_c = (int64_t)blockIdx.x - tile_r * flat_tiles_n;
  }
  const int64_t i0 = tile_r * BM, j0 = tile_c * BN;
  const int z = blockIdx.z % slices;
  const int64_t kb_total = (k + BK - 1) / BK;
  const int64_t kb_begin = (int64_t)z * kb_per_slice;
  const int64_t kb_end = min(kb_total, kb_begin + kb_per_slice);
  const int nkb = kb_end > kb_begin ? (int)(kb_end - kb_begin) : 0;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

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
    const double* as = As + sc * BM * LDA;
    const double* bs = Bs + sc * BK * BN;
#pragma unroll
    for (int kq = 0; kq < BK; kq += 2) {
      double2 a2[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        a2[i] = *reinterpret_cast<const double2*>(as + (ty * 4 + i) * LDA + kq);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const double2 b0 = *reinterpret_cast<const double2*>(bs + (kq + kk) * BN + tx * 2);
        const double2 b1 = *reinterpret_cast<const double2*>(bs + (kq + kk) * BN + 32 + tx * 2);
        const double b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double a = kk == 0 ? a2[i].x : a2[i].y;
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a, b[j], acc[i][j]);
        }
      }
    }
  }
  cp_async_wait<0>();

  double* out = (z == 0) ? C : W + (int64_t)(z - 1) * m * n;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gi = i0 + ty * 4 + i;
    if (gi >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gj = j0 + h * 32 + tx * 2;
      double* dst = out + gi * n + gj;
      if (vec && gj + 2 <= n) {
        *reinterpret_cast<double2*>(dst) = make_double2(acc[i][h * 2], acc[i][h * 2 + 1]);
      } else {
        if (gj < n) dst[0] = acc[i][h * 2];
        if (gj + 1 < n) dst[1] = acc[i][h * 2 + 1];
      }
    }
  }
}

// Small-tile variant for products whose 64 x 64 grid would leave most SMs
// idle (n = 256 gives 16 CTAs): an SB x SB tile per CTA, one output per
// thread, k staged through shared memory in blocks of 32.  The FP64 pipe
// (2 FMA per SM per clock) bounds these products, so an SM's time grows with
// the CTAs it holds: SB = 8 gives n = 256 1024 CTAs (6 or 7 per SM) where
// SB = 16 gave 256 (1 or 2 per SM).
constexpr int SBK = 32;

template <int SB>
__global__ void __launch_bounds__(SB * SB)
    dfma_small_kernel(int64_t m, int64_t n, int64_t k, const double* __restrict__ A,
                      const double* __restrict__ B, double* __restrict__ C, double* __restrict__ W,
                      int kb_per_slice) {
  constexpr int T = SB * SB, PER = SBK * SB / T;  // staged elements per thread and operand
  __shared__ double As[SB][SBK + 1];
  __shared__ double Bs[SBK][SB + 1];
  const int tx = threadIdx.x % SB, ty = threadIdx.x / SB;
  const int64_t i0 = (int64_t)blockIdx.y * SB, j0 = (int64_t)blockIdx.x * SB;
  const int z = blockIdx.z;
  // slices are counted in the 16-wide k-blocks of the 64 x 64 leaf
  const int64_t kbeg = (int64_t)z * kb_per_slice * BK;
  const int64_t kend = min(k, kbeg + (int64_t)kb_per_slice * BK);
  double acc = 0.0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += SBK) {
    // SB x 32 elements of each operand block, PER per thread
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + T * q;
      const int ar = e / SBK, ac = e % SBK;  // A block SB x 32
      const int br = e / SB, bc = e % SB;    // B block 32 x SB
      const int64_t ga = i0 + ar, gk = k0 + ac;
      As[ar][ac] = (ga < m && gk < kend) ? A[ga * k + gk] : 0.0;
      const int64_t gkb = k0 + br, gb = j0 + bc;
      Bs[br][bc] = (gkb < kend && gb < n) ? B[gkb * n + gb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < SBK; ++t) acc = fma(As[ty][t], Bs[t][tx], acc);
    __syncthreads();
  }
  const int64_t gi = i0 + ty, gj = j0 + tx;
  if (gi < m && gj < n) ((z == 0) ? C : W + (int64_t)(z - 1) * m * n)[gi * n + gj] = acc;
}

__global__ void __launch_bounds__(256) sum_reduce_f64_kernel(int64_t count, double* __restrict__ C,
                                                             const double* __restrict__ W,
                                                             int parts, bool vec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const int64_t nv = count >> 1;
    for (int64_t v = t; v < nv; v += stride) {
      double2 c = reinterpret_cast<const double2*>(C)[v];
      for (int p = 0; p < parts; ++p) {
        const double2 w = __ldcs(reinterpret_cast<const double2*>(W + (int64_t)p * count) + v);
        c.x += w.x;
        c.y += w.y;
      }
      reinterpret_cast<double2*>(C)[v] = c;
    }
  } else {
    for (int64_t e = t; e < count; e += stride) {
      double c = C[e];
      for (int p = 0; p < parts; ++p) c += W[(int64_t)p * count + e];
      C[e] = c;
    }
  }
}

// ------------------------------------------------------------ stream-K
// The zero-temporary k-parallel form of Fig. tar-mm / Theorem tar-mm for
// the FP64 semiring: a grid of P persistent CTAs takes equal contiguous
// ranges of the (tile, k-block) iteration space, tile-major.  A tile covered
// by one CTA is written straight to C; a tile shared by several CTAs has each
// of them store its register tile in a per-CTA slot (at most two per CTA:
// its first and its last segment, the p b^2 temporaries of the theorem) and
// count itself on the tile's counter.  The CTA that arrives last folds the
// slots into C in k order (contributor order), so the sum -- and the result
// -- is the same whatever order the CTAs finish in; nothing waits.
constexpr int SKT = 32, SKBK = 8, SK_THREADS = 256, SK_LDA = SKBK + 2;

__device__ __forceinline__ int64_t sk_begin(int64_t c, int64_t total, int P) { return total * c / P; }

// The CTA whose range holds iteration i.
__device__ __forceinline__ int sk_owner(int64_t i, int64_t total, int P) {
  int64_t c = i * P / total;
  while (c + 1 < P && sk_begin(c + 1, total, P) <= i) ++c;
  while (c > 0 && sk_begin(c, total, P) > i) --c;
  return (int)c;
}

__device__ __forceinline__ void sk_load(double (*As)[SK_LDA], double (*Bs)[SKT], const double* __restrict__ A,
                                        const double* __restrict__ B, int64_t m, int64_t n, int64_t k,
                                        int64_t i0, int64_t j0, int64_t k0, bool vec, int tid) {
  // A: 32 rows x 8 doubles = 128 chunks of 2; B: 8 rows x 32 doubles = 128
  // chunks of 2 -- one chunk of each per thread of the first half / second half
  if (tid < 128) {
    const int row = tid >> 2, c2 = tid & 3;
    const int64_t gi = i0 + row, gk = k0 + c2 * 2;
    double* dst = &As[row][c2 * 2];
    if (vec && gi < m && gk + 2 <= k) {
      cp_async16(dst, A + gi * k + gk);
    } else {
      dst[0] = (gi < m && gk < k) ? A[gi * k + gk] : 0.0;
      dst[1] = (gi < m && gk + 1 < k) ? A[gi * k + gk + 1] : 0.0;
    }
  } else {
    const int u = tid - 128, row = u >> 4, c2 = u & 15;
    const int64_t gk = k0 + row, gj = j0 + c2 * 2;
    double* dst = &Bs[row][c2 * 2];
    if (vec && gk < k && gj + 2 <= n) {
      cp_async16(dst, B + gk * n + gj);
    } else {
      dst[0] = (gk < k && gj < n) ? B[gk * n + gj] : 0.0;
      dst[1] = (gk < k && gj + 1 < n) ? B[gk * n + gj + 1] : 0.0;
    }
  }
}

__global__ void __launch_bounds__(SK_THREADS)
    dfma_streamk_kernel(int64_t m, int64_t n, int64_t k, const double* __restrict__ A, const double* __restrict__ B,
                        double* __restrict__ C, double* __restrict__ slots, int* __restrict__ counters,
                        int64_t tiles_n, int64_t ki, int64_t total, int P, bool vec) {
  __shared__ __align__(16) double As[2][SKT][SK_LDA];
  __shared__ __align__(16) double Bs[2][SKBK][SKT];
  __shared__ int s_last, s_first_c, s_last_c;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // outputs (2 ty + i, 2 tx + j)
  const int c = blockIdx.x;
  int64_t it = sk_begin(c, total, P);
  const int64_t end = sk_begin(c + 1, total, P);
  for (int seg = 0; it < end; ++seg) {
    const int64_t t = it / ki, j0 = it - t * ki;
    const int64_t j1 = min(ki, j0 + (end - it));
    const int64_t ti = t / tiles_n;
    const int64_t i0 = ti * SKT, c0 = (t - ti * tiles_n) * SKT;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    __syncthreads();  // the previous segment's readers are done with the stages
    sk_load(As[0], Bs[0], A, B, m, n, k, i0, c0, j0 * SKBK, vec, tid);
    cp_async_commit();
    for (int64_t j = j0; j < j1; ++j) {
      const int cur = (int)((j - j0) & 1);
      if (j + 1 < j1) sk_load(As[cur ^ 1], Bs[cur ^ 1], A, B, m, n, k, i0, c0, (j + 1) * SKBK, vec, tid);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < SKBK; kk += 2) {
        const double2 a0 = *reinterpret_cast<const double2*>(&As[cur][2 * ty][kk]);
        const double2 a1 = *reinterpret_cast<const double2*>(&As[cur][2 * ty + 1][kk]);
        const double2 b0 = *reinterpret_cast<const double2*>(&Bs[cur][kk][2 * tx]);
        const double2 b1 = *reinterpret_cast<const double2*>(&Bs[cur][kk + 1][2 * tx]);
        acc[0][0] = fma(a0.x, b0.x, acc[0][0]);
        acc[0][1] = fma(a0.x, b0.y, acc[0][1]);
        acc[1][0] = fma(a1.x, b0.x, acc[1][0]);
        acc[1][1] = fma(a1.x, b0.y, acc[1][1]);
        acc[0][0] = fma(a0.y, b1.x, acc[0][0]);
        acc[0][1] = fma(a0.y, b1.y, acc[0][1]);
        acc[1][0] = fma(a1.y, b1.x, acc[1][0]);
        acc[1][1] = fma(a1.y, b1.y, acc[1][1]);
      }
      __syncthreads();  // stage `cur` is refilled two iterations on
    }
    cp_async_wait<0>();
    const bool whole = (j0 == 0 && j1 == ki);
    if (whole) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int64_t gi = i0 + 2 * ty + i, gj = c0 + 2 * tx + jj;
          if (gi < m && gj < n) C[gi * n + gj] = acc[i][jj];
        }
    } else {
      double* slot = slots + ((int64_t)c * 2 + (seg == 0 ? 0 : 1)) * (SKT * SKT);
#pragma unroll
      for (int i = 0; i < 2; ++i)
        *reinterpret_cast<double2*>(slot + (2 * ty + i) * SKT + 2 * tx) = make_double2(acc[i][0], acc[i][1]);
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        const int cf = sk_owner(t * ki, total, P), cl = sk_owner(t * ki + ki - 1, total, P);
        const int prev = atomicAdd(&counters[t], 1);
        s_last = prev == cl - cf;
        s_first_c = cf;
        s_last_c = cl;
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        double sum[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int q = s_first_c; q <= s_last_c; ++q) {
          // contributor q keeps tile t in slot 0 when t is its first segment
          const int which = (sk_begin(q, total, P) / ki == t) ? 0 : 1;
          const double* src = slots + ((int64_t)q * 2 + which) * (SKT * SKT);
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const double2 v = __ldcg(reinterpret_cast<const double2*>(src + (2 * ty + i) * SKT + 2 * tx));
            sum[i][0] += v.x;
            sum[i][1] += v.y;
          }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int64_t gi = i0 + 2 * ty + i, gj = c0 + 2 * tx + jj;
            if (gi < m && gj < n) C[gi * n + gj] = sum[i][jj];
          }
        if (tid == 0) counters[t] = 0;
      }
    }
    it = t * ki + j1;
  }
}

// Stream-K geometry of one product on this device.
struct SkGeom {
  int64_t tiles_n, tiles, ki, total;
  int P;
};

SkGeom sk_geom(int64_t m, int64_t n, int64_t k) {
  SkGeom g;
  g.tiles_n = (n + SKT - 1) / SKT;
  g.tiles = ((m + SKT - 1) / SKT) * g.tiles_n;
  g.ki = (k + SKBK - 1) / SKBK;
  g.total = g.tiles * g.ki;
  // the same number of CTAs on every SM (up to four), each with at least
  // sixteen k-blocks where the product has that many (shorter ranges leave
  // each CTA's load latency exposed): every SM then gets the same share of
  // the iteration space, to within one k-block per CTA
  const int64_t sms = num_sms();
  int64_t per = g.total / (16 * sms);
  if (per > 4) per = 4;
  int64_t P = per >= 1 ? per * sms : std::max<int64_t>(1, std::min<int64_t>(sms, g.total / 4));
  g.P = (int)P;
  return g;
}

}  // namespace

int dfma_tile_k() { return BK; }

size_t dfma_streamk_bytes(int64_t m, int64_t n, int64_t k) {
  const SkGeom g = sk_geom(m, n, k);
  return (size_t)g.P * 2 * SKT * SKT * sizeof(double) + (size_t)((g.tiles * 4 + 255) / 256 * 256);
}

int g_f64_streamk = 1;  // mm_set_option(MM_OPT_F64_STREAMK, ...)

bool dfma_streamk_wanted(int64_t m, int64_t n, int64_t k) {
  // shapes it takes: the 64 x 64 grid fills less than four waves of two CTAs
  // per SM, and the k-split has room (index arithmetic in int64 without
  // overflow)
  const int64_t tiles64 = ((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  const SkGeom g = sk_geom(m, n, k);
  if (g_f64_streamk == 0 || !(k > 0 && tiles64 < 8 * (int64_t)num_sms() && g.total < ((int64_t)1 << 40) && g.ki >= 4))
    return false;
  if (g_f64_streamk == 2) return true;
  // The planner's rule.  The FP64 pipe bounds both forms, so the classic
  // grid takes ceil(tiles / SMs) tile-times and stream-K tiles / SMs plus its
  // folds (1024 x 64c x 4096: 304 tiles 8.18 against 8.25 ms, 320 tiles 12.24
  // against 8.69).  Under two CTAs per SM of 64 x 64 tiles the classic path
  // runs 16 x 16 or 8 x 8 tiles, many per SM, which balance without slots
  // (n = 256: 33 against 43 us).  So: at least two tiles per SM, and a last
  // wave empty enough to save 5%.
  const int64_t sms = num_sms();
  const int64_t waves = (tiles64 + sms - 1) / sms;
  return tiles64 >= 2 * sms && waves * sms * 100 >= 105 * tiles64;
}

cudaError_t launch_dfma_streamk(int64_t m, int64_t n, int64_t k, const double* A, const double* B, double* C,
                                void* ws, cudaStream_t st) {
  const SkGeom g = sk_geom(m, n, k);
  double* slots = static_cast<double*>(ws);
  int* counters = reinterpret_cast<int*>(static_cast<uint8_t*>(ws) + (size_t)g.P * 2 * SKT * SKT * sizeof(double));
  TraceScope tr(kTrDfmaLeaf, st);
  MMSR_CUDA_TRY(cudaMemsetAsync(counters, 0, (size_t)g.tiles * 4, st));
  const bool vec = (k % 2 == 0) && (n % 2 == 0) && aligned16(A) && aligned16(B);
  dfma_streamk_kernel<<<(unsigned)g.P, SK_THREADS, 0, st>>>(m, n, k, A, B, C, slots, counters, g.tiles_n, g.ki,
                                                            g.total, g.P, vec);
  return cudaGetLastError();
}

cudaError_t launch_dfma_leaf(int64_t m, int64_t n, int64_t k, const double* A, const double* B,
                             double* C, double* W, int s, int kb_per_slice, cudaStream_t st) {
  static std::atomic<uint64_t> configured{0};
  MMSR_CUDA_TRY(smem_limit_once(dfma_leaf_kernel, SMEM_BYTES, configured));
  const bool vec = (k % 2 == 0) && (n % 2 == 0) && aligned16(A) && aligned16(B) && aligned16(C) &&
                   (W == nullptr || aligned16(W));
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)s);
  TraceScope tr(kTrDfmaLeaf, st);
  if ((int64_t)grid.x * grid.y * s < 2 * (int64_t)num_sms()) {
    // too few 64 x 64 tiles to occupy the GPU: 16 x 16 tiles, or 8 x 8 when
    // 16 x 16 tiles would still leave fewer than four CTAs per SM
    const int64_t tiles16 = ((n + 15) / 16) * ((m + 15) / 16) * s;
    if (tiles16 < 4 * (int64_t)num_sms()) {
      dim3 sg((unsigned)((n + 7) / 8), (unsigned)((m + 7) / 8), (unsigned)s);
      dfma_small_kernel<8><<<sg, 64, 0, st>>>(m, n, k, A, B, C, W, kb_per_slice);
    } else {
      dim3 sg((unsigned)((n + 15) / 16), (unsigned)((m + 15) / 16), (unsigned)s);
      dfma_small_kernel<16><<<sg, 256, 0, st>>>(m, n, k, A, B, C, W, kb_per_slice);
    }
    return cudaGetLastError();
  }
  if (grid.y > kMaxGridY) {
    const int64_t tiles_n = grid.x;
    dim3 flat((unsigned)(tiles_n * grid.y), 1, (unsigned)s);
    dfma_leaf_kernel<<<flat, THREADS, SMEM_BYTES, st>>>(m, n, k, A, B, C, W, kb_per_slice, vec, s, 0, 0, 0,
                                                        tiles_n);
    return cudaGetLastError();
  }
  dfma_leaf_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(m, n, k, A, B, C, W, kb_per_slice, vec, s, 0, 0, 0, 0);
  return cudaGetLastError();
}

cudaError_t launch_dfma_batched(const double* A, const double* B, double* C, int64_t m, int64_t n,
                                int64_t k, int batches, cudaStream_t st) {
  static std::atomic<uint64_t> configured{0};
  MMSR_CUDA_TRY(smem_limit_once(dfma_leaf_kernel, SMEM_BYTES, configured));
  const bool vec = (k % 2 == 0) && (n % 2 == 0) && aligned16(A) && aligned16(B) && aligned16(C) &&
                   ((m * k) % 2 == 0) && ((k * n) % 2 == 0) && ((m * n) % 2 == 0);
  const int kb = (int)((k + BK - 1) / BK);
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)batches);
  TraceScope tr(kTrDfmaLeaf, st);
  dfma_leaf_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(m, n, k, A, B, C, nullptr, kb > 0 ? kb : 1, vec, 1,
                                                      m * k, k * n, m * n, 0);
  return cudaGetLastError();
}

cudaError_t launch_sum_reduce_f64(int64_t count, double* C, const double* W, int parts,
                                  cudaStream_t st) {
  if (parts <= 0 || count <= 0) return cudaSuccess;
  const bool vec = aligned16(C) && aligned16(W) && (count % 2 == 0);
  const int64_t work = vec ? count / 2 : count;
  int64_t blocks = (work + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  TraceScope tr(kTrSumReduceF64, st);
  sum_reduce_f64_kernel<<<(unsigned)blocks, 256, 0, st>>>(count, C, W, parts, vec);
  return cudaGetLastError();
}

}  // namespace mmsr
