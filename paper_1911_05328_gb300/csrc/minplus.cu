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
#include "minplus_tile.cuh"

namespace mmsr {
namespace {

using namespace mp;

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
// Slots 0 .. kEagerSlots-1 are reused round-robin by calls made outside
// stream capture; each captured call gets a slot of its own from the rest,
// never reused, so a replayed graph cannot share its slot with a later eager
// call (replays of one graph still share theirs, like their workspace).
// Once the captured slots run out, captured calls take the 32-bit leaf.
constexpr int kEagerSlots = 4096, kCapturedSlots = 4096;
constexpr int kPackSlots = kEagerSlots + kCapturedSlots;

struct PackSlot {
  int viol;
  unsigned int done;
  int verdict;  // 1: packed path valid for this call's inputs
  int pad;
};
__device__ PackSlot g_pack[kPackSlots];

__device__ __forceinline__ int pack_verdict(int slot) { return __ldcg(&g_pack[slot].verdict); }

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
      // four 16-byte loads in flight per thread
      const int4* X4 = reinterpret_cast<const int4*>(X);
      const int64_t nv = cnt / 4;
      int64_t v = t0;
      for (; v + 3 * stride < nv; v += 4 * stride) {
        int4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldcs(X4 + v + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          bad |= out_of_pack_range(q[u].x) | out_of_pack_range(q[u].y) | out_of_pack_range(q[u].z) |
                 out_of_pack_range(q[u].w);
      }
      for (; v < nv; v += stride) {
        const int4 q = __ldcs(X4 + v);
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

__global__ void __launch_bounds__(PTHREADS, 2)
    minplus16_leaf_kernel(int64_t m, int64_t n, int64_t k, const int32_t* __restrict__ A,
                          const int32_t* __restrict__ B, int32_t* __restrict__ C,
                          int32_t* __restrict__ W, int kb_per_slice, bool vec, int slot) {
  if (pack_verdict(slot) != 1) return;
  extern __shared__ __align__(16) uint32_t psmem[];
  const int z = blockIdx.z;
  // slices are counted in the 32-wide k-blocks of the 32-bit leaf; the
  // packed tile walks each slice in 16-wide sub-blocks
  const int64_t kbeg = (int64_t)z * kb_per_slice * BK;
  const int64_t kend = min(k, kbeg + (int64_t)kb_per_slice * BK);
  minplus16_tile(A, B, C, W, z, m, n, k, (int64_t)blockIdx.y * PBM, (int64_t)blockIdx.x * PBN, kbeg, kend,
                 vec, (int)threadIdx.x, psmem, SyncCta());
}

// Zero-workspace k-parallel form (the TAR-MM of Fig. tar-mm: every worker
// keeps a tile-sized temporary -- here the register tile -- and merges it
// into C with an atomic (+), here min, which is exact and order-free).  The
// persistent CTAs split the (tile, 16-wide k sub-block) units of the whole
// product evenly (stream-K), so no wave of CTAs runs half empty; a segment
// that covers a whole tile stores it, partial segments merge into C, which
// a fill kernel sets to the sentinel first.
__global__ void __launch_bounds__(PTHREADS, 2)
    minplus16_streamk_kernel(int64_t m, int64_t n, int64_t k, const int32_t* __restrict__ A,
                             const int32_t* __restrict__ B, int32_t* __restrict__ C, bool vec,
                             int slot, int64_t units, int64_t nsub, int64_t tiles_n) {
  if (pack_verdict(slot) != 1) return;
  extern __shared__ __align__(16) uint32_t psmem[];
  const int64_t G = gridDim.x;
  int64_t u = units * blockIdx.x / G;
  const int64_t end = units * (blockIdx.x + 1) / G;
  while (u < end) {
    const int64_t tile = u / nsub, s0 = u - tile * nsub;
    const int64_t s1 = min(nsub, s0 + (end - u));
    const bool whole = (s0 == 0 && s1 == nsub);
    minplus16_tile(A, B, C, (int32_t*)nullptr, 0, m, n, k, (tile / tiles_n) * PBM, (tile % tiles_n) * PBN,
                   s0 * PBK, min(k, s1 * PBK), vec, (int)threadIdx.x, psmem, SyncCta(), !whole);
    __syncthreads();  // the next segment restages shared memory
    u += s1 - s0;
  }
}

__global__ void __launch_bounds__(256) fill_inf_kernel(int32_t* __restrict__ C, int64_t count, int slot) {
  if (pack_verdict(slot) != 1) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    C[e] = kInf;
}

// The same zero-workspace form for the exact 32-bit leaf, over (128 x 128
// tile, 32-wide k-block) units; it runs when the packed leaf did not.
__global__ void __launch_bounds__(THREADS, 2)
    minplus32_streamk_kernel(int64_t m, int64_t n, int64_t k, const int32_t* __restrict__ A,
                             const int32_t* __restrict__ B, int32_t* __restrict__ C, bool vec, int slot,
                             int64_t units, int64_t nkb, int64_t tiles_n) {
  if (slot >= 0 && pack_verdict(slot) == 1) return;
  extern __shared__ __align__(16) int32_t smem[];
  const int64_t G = gridDim.x;
  int64_t u = units * blockIdx.x / G;
  const int64_t end = units * (blockIdx.x + 1) / G;
  while (u < end) {
    const int64_t tile = u / nkb, b0 = u - tile * nkb;
    const int64_t b1 = min(nkb, b0 + (end - u));
    const bool whole = (b0 == 0 && b1 == nkb);
    minplus32_tile(A, B, C, (int32_t*)nullptr, 0, m, n, k, (tile / tiles_n) * BM, (tile % tiles_n) * BN, b0,
                   (int)(b1 - b0), vec, (int)threadIdx.x, smem, SyncCta(), !whole);
    __syncthreads();  // the next segment restages shared memory
    u += b1 - b0;
  }
}

// C = +inf before the 32-bit stream-K merges (skipped when the packed leaf ran).
__global__ void __launch_bounds__(256) fill_inf32_kernel(int32_t* __restrict__ C, int64_t count, int slot) {
  if (slot >= 0 && pack_verdict(slot) == 1) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    C[e] = kInf;
}

__global__ void __launch_bounds__(THREADS, 2)
    minplus_leaf_kernel(int64_t m, int64_t n, int64_t k, const int32_t* __restrict__ A,
                        const int32_t* __restrict__ B, int32_t* __restrict__ C,
                        int32_t* __restrict__ W, int kb_per_slice, bool vec, int slot) {
  // The packed 2 x 16-bit leaf already produced C when the range scan of
  // this call found every finite input small enough.
  if (slot >= 0 && pack_verdict(slot) == 1) return;
  extern __shared__ __align__(16) int32_t smem[];
  const int z = blockIdx.z;
  const int64_t kb_total = (k + BK - 1) / BK;
  const int64_t kb_begin = (int64_t)z * kb_per_slice;
  const int64_t kb_end = min(kb_total, kb_begin + kb_per_slice);
  const int nkb = kb_end > kb_begin ? (int)(kb_end - kb_begin) : 0;
  minplus32_tile(A, B, C, W, z, m, n, k, (int64_t)blockIdx.y * BM, (int64_t)blockIdx.x * BN, kb_begin, nkb,
                 vec, (int)threadIdx.x, smem, SyncCta());
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
int g_streamk_mode = 1;  // 1: stream-K for unsplit packed products with few waves, 0: never

cudaError_t launch_minplus_leaf(int64_t m, int64_t n, int64_t k, const int32_t* A,
                                const int32_t* B, int32_t* C, int32_t* W, int s,
                                int kb_per_slice, cudaStream_t st) {
  static std::atomic<uint64_t> conf32{0}, conf32s{0}, conf16{0}, conf16s{0};
  MMSR_CUDA_TRY(smem_limit_once(minplus_leaf_kernel, SMEM_BYTES, conf32));
  MMSR_CUDA_TRY(smem_limit_once(minplus32_streamk_kernel, SMEM_BYTES, conf32s));
  MMSR_CUDA_TRY(smem_limit_once(minplus16_leaf_kernel, PSMEM_BYTES, conf16));
  MMSR_CUDA_TRY(smem_limit_once(minplus16_streamk_kernel, PSMEM_BYTES, conf16s));
  const bool vec = (k % 4 == 0) && (n % 4 == 0) && aligned16(A) && aligned16(B) && aligned16(C) &&
                   (W == nullptr || aligned16(W));
  int slot = -1;
  if (g_packed_mode && k > 0) {
    // the packed tile and the 32-bit tile split k into the same 32-wide blocks
    static std::atomic<unsigned> eager{0}, captured{0};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MMSR_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      slot = (int)(eager.fetch_add(1u) % (unsigned)kEagerSlots);
    } else {
      const unsigned c = captured.fetch_add(1u);
      slot = c < (unsigned)kCapturedSlots ? kEagerSlots + (int)c : -1;
    }
  }
  if (slot >= 0) {
    {
      TraceScope tr(kTrRangeScan, st);
      const bool svec = aligned16(A) && aligned16(B) && ((m * k) % 4 == 0) && ((k * n) % 4 == 0);
      int64_t blocks = ((m * k + k * n) / (svec ? 4 : 1) + 255) / 256;
      if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
      if (blocks < 1) blocks = 1;
      range_scan_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, m * k, B, k * n, slot, svec);
      MMSR_CUDA_TRY(cudaGetLastError());
    }
    const int64_t tiles_m = (m + PBM - 1) / PBM, tiles_n = (n + PBN - 1) / PBN;
    // CTAs of the packed leaf that fit on the GPU at once (the same for every
    // GB300 of the process; a racing first computation stores the same value)
    static std::atomic<int> resident_cache{0};
    int resident = resident_cache.load(std::memory_order_relaxed);
    if (!resident) {
      int per_sm = 2;
      const int sms = num_sms();
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, minplus16_streamk_kernel, PTHREADS, PSMEM_BYTES);
      resident = sms * (per_sm > 0 ? per_sm : 1);
      resident_cache.store(resident, std::memory_order_relaxed);
    }
    if (s == 1 && g_streamk_mode && tiles_m * tiles_n < 4 * (int64_t)resident) {
      TraceScope tr(kTrMinplus16Leaf, st);
      fill_inf_kernel<<<(unsigned)(num_sms() * 4), 256, 0, st>>>(C, m * n, slot);
      const int64_t nsub = (k + PBK - 1) / PBK;
      minplus16_streamk_kernel<<<(unsigned)resident, PTHREADS, PSMEM_BYTES, st>>>(
          m, n, k, A, B, C, vec, slot, tiles_m * tiles_n * nsub, nsub, tiles_n);
      MMSR_CUDA_TRY(cudaGetLastError());
    } else {
      TraceScope tr(kTrMinplus16Leaf, st);
      dim3 pgrid((unsigned)tiles_n, (unsigned)tiles_m, (unsigned)s);
      minplus16_leaf_kernel<<<pgrid, PTHREADS, PSMEM_BYTES, st>>>(m, n, k, A, B, C, W, kb_per_slice,
                                                                   vec, slot);
      MMSR_CUDA_TRY(cudaGetLastError());
    }
  }
  dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)s);
  TraceScope tr(kTrMinplusLeaf, st);
  static std::atomic<int> resident32_cache{0};
  int resident32 = resident32_cache.load(std::memory_order_relaxed);
  if (!resident32) {
    int per_sm = 2;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, minplus32_streamk_kernel, THREADS, SMEM_BYTES);
    resident32 = num_sms() * (per_sm > 0 ? per_sm : 1);
    resident32_cache.store(resident32, std::memory_order_relaxed);
  }
  const int64_t tiles32 = (int64_t)grid.x * grid.y;
  const int64_t nkb = (k + BK - 1) / BK;
  if (s == 1 && g_streamk_mode && k > 0 && tiles32 < 4 * (int64_t)resident32) {
    // the zero-workspace k-parallel form for the 32-bit leaf (its kernels
    // exit at once when the packed leaf ran)
    fill_inf32_kernel<<<(unsigned)(num_sms() * 4), 256, 0, st>>>(C, m * n, slot);
    const int64_t units = tiles32 * nkb;
    const int64_t G = std::min<int64_t>(resident32, units);
    minplus32_streamk_kernel<<<(unsigned)G, THREADS, SMEM_BYTES, st>>>(m, n, k, A, B, C, vec, slot, units, nkb,
                                                                       (int64_t)grid.x);
    return cudaGetLastError();
  }
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
  const int64_t cap = (int64_t)num_sms() * 8;
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
