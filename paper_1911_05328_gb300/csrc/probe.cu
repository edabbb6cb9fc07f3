// probe.cu -- instruction-throughput probes for the roofline denominators
// of the CUDA-core kernels (see include/mmsr_probe.h).
#include <cuda_fp16.h>

#include "../../include/mmsr_probe.h"
#include "common.cuh"

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

}  // namespace
}  // namespace mmsr

using namespace mmsr;

extern "C" int mm_probe_peak(int kind, int iters, void* stream, double* ops_per_s, double* ms) {
  if (kind < 0 || kind > 3 || iters <= 0 || !ops_per_s || !ms) return MM_ERR_ARG;
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
  switch (kind) {
    case 0: probe_kernel<0><<<blocks, 256, 0, st>>>(iters, 12345u); break;
    case 1: probe_kernel<1><<<blocks, 256, 0, st>>>(iters, 12345u); break;
    case 2: probe_kernel<2><<<blocks, 256, 0, st>>>(iters, 12345u); break;
    default: probe_kernel<3><<<blocks, 256, 0, st>>>(iters, 12345u); break;
  }
  cudaEventRecord(b, st);
  cudaError_t e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return MM_ERR_CUDA;
  const double per_instr = (kind == 1) ? 4.0 : 2.0;
  const double ops = (double)blocks * 256.0 * (double)iters * kChains * per_instr;
  *ms = t;
  *ops_per_s = t > 0 ? ops / (t * 1e-3) : 0.0;
  return MM_OK;
}
