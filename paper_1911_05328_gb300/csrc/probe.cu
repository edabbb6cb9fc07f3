// probe.cu -- instruction-throughput probes for the roofline denominators
// of the CUDA-core kernels (see include/mmsr_probe.h).
#include <cuda_fp16.h>

#include "../../include/mmsr_probe.h"
#include "common.cuh"
#include "tcgen05.cuh"

namespace mmsr {
namespace {

constexpr int kChains = 16;

// Result sink: keeps the chains live; written only if a chain lands on an
// unlikely value, and always a valid device address.
__device__ uint64_t g_probe_sink;

// Each thread runs kChains interleaved chains; chain i reads chain i+1, so
// the compiler can neither collapse the loop nor serialise it.
template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(int iters, uint32_t seed) {
  if (KIND == 0 || KIND == 1) {
    uint32_t acc[kChains], b[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      acc[i] = seed * (i + 3) + threadIdx.x;
      b[i] = (seed ^ (i * 0x9E3779B9u)) & 0x3FFF3FFFu;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if (KIND == 0)
          acc[i] = __viaddmin_u32(acc[(i + 1) % kChains], b[i], acc[i]);
        else
          acc[i] = __viaddmin_u16x2(acc[(i + 1) % kChains], b[i], acc[i]);
      }
    }
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) r ^= acc[i];
    if (r == 0x12345678u) g_probe_sink = r;
  } else if (KIND == 2) {
    double acc[kChains], b[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      acc[i] = 1e-3 * (i + threadIdx.x);
      b[i] = 0.5 + 1e-9 * (seed + i);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[(i + 1) % kChains], b[i], acc[i]);
    }
    double r = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) r += acc[i];
    if (r == 1.2345) g_probe_sink = __double_as_longlong(r);
  } else {
    // independent chains, loop unrolled: the loop's own instructions would
    // otherwise take a sixth of the issue slots the FMA pipe needs
    float acc[kChains], b[kChains], c[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      acc[i] = 1e-3f * (i + threadIdx.x);
      b[i] = 0.5f + 1e-6f * (seed + i);
      c[i] = 1e-5f * i;
    }
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = fmaf(acc[i], b[i], c[i]);
    }
    float r = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) r += acc[i];
    if (r == 1.2345f) g_probe_sink = __float_as_uint(r);
  }
}

// Tensor-core issue probe: one CTA per SM, seven A and seven B operand tiles
// (zeros) resident in shared memory in the 64-byte-swizzled K-major layout
// of the FP64-accuracy leaf, and one thread issuing `iters` rounds of 56
// bf16 products of shape 128 x N x 16 -- two 16-deep k-steps, each the 28
// slice pairs in digit-order groups, into min(7, 512 / N) TMEM
// accumulators.  No TMA traffic: the rate is that of the tensor core fed
// from shared memory alone.
__device__ int g_probe_status;
template <int N>
__global__ void __launch_bounds__(128, 1) probe_mma_kernel(int iters) {
  constexpr uint32_t A_TILE = 128 * 64, B_TILE = N * 64, BYTES = 7 * (A_TILE + B_TILE);
  constexpr int NACC = (512 / N) < 7 ? (512 / N) : 7;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + BYTES);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  int* abort_flag = reinterpret_cast<int*>(slot + 1);
  for (uint32_t i = threadIdx.x; i < BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tc::mbar_init(bar, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(slot, 512);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros, to the tensor core's view
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = tc::idesc_f16(128, N, 1);
    constexpr uint32_t dhi = tc::desc_hi_sw64();
    const uint32_t a_lo = tc::desc_lo(smem_u32(smem)), b_lo = tc::desc_lo(smem_u32(smem) + 7 * A_TILE);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int g = 0; g < 7; ++g)
#pragma unroll
          for (int sa = 0; sa <= g; ++sa)
            tc::mma_f16(tmem + (uint32_t)((g % NACC) * N), tc::desc_join(a_lo + ((sa * A_TILE + kk * 32) >> 4), dhi),
                        tc::desc_join(b_lo + (((g - sa) * B_TILE + kk * 32) >> 4), dhi), idesc, 1u);
    }
    tc::mma_commit(bar);
    tc::mbar_wait(bar, 0, abort_flag, &g_probe_status);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 512);
  }
}

template <int N>
cudaError_t launch_probe_mma(int sms, int iters, cudaStream_t st) {
  constexpr size_t smem = 1024 + 7 * (128 * 64 + N * 64) + 64;
  static std::atomic<uint64_t> done{0};
  MMSR_CUDA_TRY(smem_limit_once(probe_mma_kernel<N>, smem, done));
  probe_mma_kernel<N><<<sms, 128, smem, st>>>(iters);
  return cudaGetLastError();
}

}  // namespace
}  // namespace mmsr

using namespace mmsr;

extern "C" int mm_probe_peak(int kind, int iters, void* stream, double* ops_per_s, double* ms) {
  if (kind < 0 || kind > 5 || iters <= 0 || !ops_per_s || !ms) return MM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MM_ERR_CUDA;
  const int blocks = sms * 8;  // 8 x 256 threads = 2048 threads per SM
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return MM_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) return MM_ERR_CUDA;
  cudaEventRecord(a, st);
  cudaError_t e = cudaSuccess;
  switch (kind) {
    case 0: probe_kernel<0><<<blocks, 256, 0, st>>>(iters, 12345u); break;
    case 1: probe_kernel<1><<<blocks, 256, 0, st>>>(iters, 12345u); break;
    case 2: probe_kernel<2><<<blocks, 256, 0, st>>>(iters, 12345u); break;
    case 3: probe_kernel<3><<<blocks, 256, 0, st>>>(iters, 12345u); break;
    case 4: e = launch_probe_mma<64>(sms, iters, st); break;
    default: e = launch_probe_mma<128>(sms, iters, st); break;
  }
  cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return MM_ERR_CUDA;
  const double per_instr = (kind == 1) ? 4.0 : 2.0;
  double ops = (double)blocks * 256.0 * (double)iters * kChains * per_instr;
  if (kind >= 4) ops = (double)sms * iters * 56.0 * 2.0 * 128 * (kind == 4 ? 64 : 128) * 16;
  *ms = t;
  *ops_per_s = t > 0 ? ops / (t * 1e-3) : 0.0;
  return MM_OK;
}
