// stubs.cu -- dispatch of the semirings served by the tensor-core and
// boolean engines, plus engines not built yet (MM_ERR_UNSUPPORTED).
#include <string.h>

#include "internal.h"

namespace mmsr {

int plan_extended(int sr, int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  switch (sr) {
    case MM_SR_PLUS_TIMES_F32: return plan_f32(m, n, k, budget, p);
    default: memset(p, 0, sizeof(*p)); return MM_ERR_UNSUPPORTED;
  }
}

int run_extended(int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B, void* C,
                 void* ws, size_t ws_bytes, cudaStream_t st, const mm_plan_t&) {
  switch (sr) {
    case MM_SR_PLUS_TIMES_F32:
      return run_f32(m, n, k, static_cast<const float*>(A), static_cast<const float*>(B),
                     static_cast<float*>(C), ws, ws_bytes, st);
    default: return MM_ERR_UNSUPPORTED;
  }
}


int read_device_status(cudaStream_t st, int* status) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return MM_ERR_CUDA;
  int v = MM_OK;
  if (read_tc_status(&v) != MM_OK) return MM_ERR_CUDA;
  *status = v;
  return MM_OK;
}

}  // namespace mmsr

extern "C" {
int mm_batched(int, const mm_problem_t*, void*, size_t, void*) { return MM_ERR_UNSUPPORTED; }
size_t mm_batched_query(int, const mm_problem_t*) { return 0; }
}
