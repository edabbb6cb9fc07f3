// dispatch.cu -- routes mm_semiring's plan and run to the engines of the
// tensor-core semirings (FP32 bf16x3, FP64-accuracy) and the boolean
// semiring, and gathers the device status words of the bounded waits.
#include <string.h>

#include "internal.h"

namespace mmsr {

int plan_extended(int sr, int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  switch (sr) {
    case MM_SR_PLUS_TIMES_F32: return plan_f32(m, n, k, budget, p);
    case MM_SR_PLUS_TIMES_F64ACC: return plan_f64acc(m, n, k, budget, p);
    case MM_SR_OR_AND_U8: return plan_orand(m, n, k, budget, p);
    default: memset(p, 0, sizeof(*p)); return MM_ERR_UNSUPPORTED;
  }
}

int run_extended(int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B, void* C,
                 void* ws, size_t ws_bytes, cudaStream_t st, const mm_plan_t&) {
  switch (sr) {
    case MM_SR_PLUS_TIMES_F32:
      return run_f32(m, n, k, static_cast<const float*>(A), static_cast<const float*>(B),
                     static_cast<float*>(C), ws, ws_bytes, st);
    case MM_SR_OR_AND_U8:
      return run_orand(m, n, k, static_cast<const uint8_t*>(A), static_cast<const uint8_t*>(B),
                       static_cast<uint8_t*>(C), ws, ws_bytes, st);
    case MM_SR_PLUS_TIMES_F64ACC:
      return run_f64acc(m, n, k, static_cast<const double*>(A), static_cast<const double*>(B),
                        static_cast<double*>(C), ws, ws_bytes, st);
    default: return MM_ERR_UNSUPPORTED;
  }
}


int read_device_status(cudaStream_t st, int* status) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return MM_ERR_CUDA;
  int v[4] = {MM_OK, MM_OK, MM_OK, MM_OK};
  if (read_tc_status(&v[0]) != MM_OK) return MM_ERR_CUDA;
  if (read_f64acc_status(&v[1]) != MM_OK) return MM_ERR_CUDA;
  if (read_batched_status(&v[2]) != MM_OK) return MM_ERR_CUDA;
  if (read_fused_status(&v[3]) != MM_OK) return MM_ERR_CUDA;
  *status = MM_OK;
  for (int i = 3; i >= 0; --i)
    if (v[i] != MM_OK) *status = v[i];
  return MM_OK;
}

}  // namespace mmsr

