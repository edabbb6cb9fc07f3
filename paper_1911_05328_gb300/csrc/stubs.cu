// stubs.cu -- engines not built yet report MM_ERR_UNSUPPORTED.
#include "internal.h"

namespace mmsr {

int plan_extended(int, int64_t, int64_t, int64_t, size_t, mm_plan_t*) { return MM_ERR_UNSUPPORTED; }
int run_extended(int, int64_t, int64_t, int64_t, const void*, const void*, void*, void*, size_t,
                 cudaStream_t, const mm_plan_t&) {
  return MM_ERR_UNSUPPORTED;
}
int plan_strassen(int, int, int64_t, int64_t, int64_t, size_t, mm_plan_t*) { return MM_ERR_UNSUPPORTED; }
int run_strassen(int, int, int, int64_t, int64_t, int64_t, const void*, const void*, void*, void*,
                 size_t, cudaStream_t) {
  return MM_ERR_UNSUPPORTED;
}
int read_device_status(cudaStream_t st, int* status) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return MM_ERR_CUDA;
  *status = MM_OK;
  return MM_OK;
}

}  // namespace mmsr

extern "C" {
int mm_batched(int, const mm_problem_t*, void*, size_t, void*) { return MM_ERR_UNSUPPORTED; }
size_t mm_batched_query(int, const mm_problem_t*) { return 0; }
}
