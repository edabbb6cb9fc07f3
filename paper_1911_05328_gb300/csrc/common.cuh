// common.cuh -- internal helpers shared by the CUDA sources of libmmsr.
// Nothing here is part of the C ABI (see include/mmsr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/mmsr.h"

namespace mmsr {

constexpr int kInf = 1 << 30;  // +infinity of the (min,+) semiring on [0, 2^30]
constexpr int64_t kMaxGridY = 65535;  // grid y / z extent limit; larger extents loop in-kernel
// Streaming multiprocessors of the current device, queried once per device
// and cached; grid sizes are multiples of it.  Returns 1 when no device
// answers (a launch would then fail on its own).
int num_sms();

#define MMSR_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t err_ = (expr);                                \
    if (err_ != cudaSuccess) return err_;                     \
  } while (0)

// Report a failed CUDA call on stderr (where it failed and why) and map it to
// MM_ERR_CUDA.
int report_cuda(cudaError_t e, const char* where);
#define MMSR_TRY_STATUS(expr)                                            \
  do {                                                                   \
    cudaError_t err_ = (expr);                                           \
    if (err_ != cudaSuccess) return ::mmsr::report_cuda(err_, #expr);    \
  } while (0)

// Raises a kernel's dynamic shared-memory limit once per device (the
// attribute belongs to the device's context); concurrent first calls from
// several threads only repeat an idempotent call.
template <typename F>
inline cudaError_t smem_limit_once(F* func, size_t bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  MMSR_CUDA_TRY(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  MMSR_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done.fetch_or(bit, std::memory_order_release);
  return cudaSuccess;
}

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__host__ __device__ inline bool aligned16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// ------------------------------------------------------------------ tracing
// Kernel ids of the optional event trace (names in trace.cu).
enum TraceKernel {
  kTrMinplusLeaf = 0, kTrMinReduce, kTrDfmaLeaf, kTrSumReduceF64, kTrSplitBf16, kTrTcBf16x3,
  kTrSumReduceF32, kTrSplitF64Slices, kTrTcF64Acc, kTrStrassenCombine, kTrStrassenPost,
  kTrBatched, kTrOrAndLeaf, kTrOrReduce, kTrMinplus16Leaf, kTrRangeScan, kTrOrPack, kTrClosureAux,
  kTraceKernels
};
// RAII: records a start event now and an end event at scope exit, on `st`,
// when tracing is enabled; otherwise does nothing.
class TraceScope {
 public:
  TraceScope(int id, cudaStream_t st);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  int id_;
  cudaStream_t st_;
  void* a_;
};

// ------------------------------------------------------- internal launchers
// Each returns the cudaError_t of its launch; all are asynchronous on `st`.

// (min,+) leaf over k-slices: slice z of `s` writes C (z == 0) or
// W + (z-1)*m*n; kb_per_slice k-blocks of the leaf's BK each.
cudaError_t launch_minplus_leaf(int64_t m, int64_t n, int64_t k, const int32_t* A,
                                const int32_t* B, int32_t* C, int32_t* W, int s,
                                int kb_per_slice, cudaStream_t st);
// C[i] = min(C[i], W_0[i], ..., W_{parts-1}[i]) for i < count.
cudaError_t launch_min_reduce(int64_t count, int32_t* C, const int32_t* W, int parts,
                              cudaStream_t st);
int minplus_tile_k();
extern int g_packed_mode;  // mm_set_option(MM_OPT_MINPLUS_PACKED, ...)
extern int g_streamk_mode;  // mm_set_option(MM_OPT_MINPLUS_STREAMK, ...)
extern int g_strassen_top_f64;  // mm_set_option(MM_OPT_STRASSEN_TOP_F64, ...)

// FP64 DFMA leaf, same slicing contract with FP64 partials.
cudaError_t launch_dfma_leaf(int64_t m, int64_t n, int64_t k, const double* A, const double* B,
                             double* C, double* W, int s, int kb_per_slice, cudaStream_t st);
// C[i] = C[i] + W_0[i] + ... + W_{parts-1}[i] (fixed order) for i < count.
cudaError_t launch_sum_reduce_f64(int64_t count, double* C, const double* W, int parts,
                                  cudaStream_t st);
int dfma_tile_k();
// Stream-K form of the FP64 leaf (Fig. tar-mm): workspace it needs (per-CTA
// partial slots and per-tile counters), whether the product is small enough
// to want it, and its launch (asynchronous on `st`, `ws` 16-byte aligned).
size_t dfma_streamk_bytes(int64_t m, int64_t n, int64_t k);
bool dfma_streamk_wanted(int64_t m, int64_t n, int64_t k);
cudaError_t launch_dfma_streamk(int64_t m, int64_t n, int64_t k, const double* A, const double* B, double* C,
                                void* ws, cudaStream_t st);

}  // namespace mmsr
