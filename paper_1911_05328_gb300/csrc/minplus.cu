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

__global__ void __launch_bounds__(THREADS, 2)
    minplus_leaf_kernel(int64_t m, int64_t n, int64_t k, const int32_t* __restrict__ A,
                        const int32_t* __restrict__ B, int32_t* __restrict__ C,
                        int32_t* __restrict__ W, int kb_per_slice, bool vec) {
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

cudaError_t launch_minplus_leaf(int64_t m, int64_t n, int64_t k, const int32_t* A,
                                const int32_t* B, int32_t* C, int32_t* W, int s,
                                int kb_per_slice, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    MMSR_CUDA_TRY(cudaFuncSetAttribute(minplus_leaf_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES));
    configured = true;
  }
  const bool vec = (k % 4 == 0) && (n % 4 == 0) && aligned16(A) && aligned16(B) && aligned16(C) &&
                   (W == nullptr || aligned16(W));
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)s);
  TraceScope tr(kTrMinplusLeaf, st);
  minplus_leaf_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(m, n, k, A, B, C, W, kb_per_slice, vec);
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
