// api.cu -- the C ABI of libmmsr: argument validation, the budget planner
// and dispatch to the leaf / reduction kernels.
//
// Planner (Sections 3-4 as split-K): the paper trades span against
// temporary space -- CO2 keeps all k-work in place and serial (Fig. mm-n2),
// CO3 runs the k-halves in parallel with a temporary D and a final madd
// (Fig. mm-n3), and SAR/STAR bound the number of temporaries by what the
// space budget allows (Theorems sar-mm, star-mm; "min{p, 4^d} copies per
// depth").  Here the budget decides s, the number of k-slices: slice 0
// accumulates in C (the lock winner of hlp, Fig. wrapper-sar-mm, which
// works on its parent's storage) and each further slice owns one m x n
// temporary; a fixed-order (+)-reduction (madd) folds them into C.
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace mmsr {

int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);  // racing stores write the same value
  return sms;
}

static int acc_bytes(int sr) {
  switch (sr) {
    case MM_SR_PLUS_TIMES_F64: return 8;
    case MM_SR_PLUS_TIMES_F32: return 4;
    case MM_SR_PLUS_TIMES_F64ACC: return 8;
    case MM_SR_MIN_PLUS_I32: return 4;
    case MM_SR_OR_AND_U8: return 4;
    default: return 0;
  }
}

int elem_bytes(int sr) {
  switch (sr) {
    case MM_SR_PLUS_TIMES_F64: return 8;
    case MM_SR_PLUS_TIMES_F32: return 4;
    case MM_SR_PLUS_TIMES_F64ACC: return 8;
    case MM_SR_MIN_PLUS_I32: return 4;
    case MM_SR_OR_AND_U8: return 1;
    default: return 0;
  }
}

// Split factor for a budget: as many k-slices as the budget can hold
// partial buffers for, clamped so each slice has at least one k-block.
static void split_for_budget(int64_t m, int64_t n, int64_t k, int tile_k, int accb,
                             size_t budget, int* s_out, int* kbs_out, int64_t* used) {
  const int64_t kb_total = (k + tile_k - 1) / tile_k;
  const uint64_t slice = (uint64_t)m * (uint64_t)n * (uint64_t)accb;
  uint64_t s = 1;
  if (slice > 0) s = 1 + (uint64_t)budget / slice;
  if (s > (uint64_t)kMaxSplit) s = kMaxSplit;
  if (kb_total > 0 && s > (uint64_t)kb_total) s = (uint64_t)kb_total;
  if (kb_total == 0) s = 1;
  int64_t kbs = kb_total > 0 ? (kb_total + (int64_t)s - 1) / (int64_t)s : 0;
  if (kbs > 0) s = (uint64_t)((kb_total + kbs - 1) / kbs);  // drop empty tail slices
  *s_out = (int)s;
  *kbs_out = (int)kbs;
  *used = (int64_t)((s - 1) * slice);
}

int plan_semiring(int sr, int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  int tile_k = 0;
  switch (sr) {
    case MM_SR_MIN_PLUS_I32:
      tile_k = minplus_tile_k();
      p->tile_m = 128; p->tile_n = 128; p->kernel = 1;
      break;
    case MM_SR_PLUS_TIMES_F64:
      tile_k = dfma_tile_k();
      p->tile_m = 64; p->tile_n = 64; p->kernel = 0;
      break;
    case MM_SR_PLUS_TIMES_F32:
    case MM_SR_PLUS_TIMES_F64ACC:
    case MM_SR_OR_AND_U8:
      return plan_extended(sr, m, n, k, budget, p);
    default:
      return MM_ERR_ARG;
  }
  p->tile_k = tile_k;
  if (sr == MM_SR_PLUS_TIMES_F64 && dfma_streamk_wanted(m, n, k) && budget >= dfma_streamk_bytes(m, n, k)) {
    // few tiles and room for the per-CTA partial tiles: the stream-K form
    p->tile_m = 32; p->tile_n = 32; p->tile_k = 8; p->kernel = 6;
    p->split_k = 1;
    p->workspace_used = (int64_t)dfma_streamk_bytes(m, n, k);
    return MM_OK;
  }
  int s = 1, kbs = 0;
  int64_t used = 0;
  split_for_budget(m, n, k, tile_k, acc_bytes(sr), budget, &s, &kbs, &used);
  p->split_k = s;
  p->workspace_used = used;
  p->workspace_min = 0;
  p->levels = 0;
  return MM_OK;
}

int split_plan(int64_t m, int64_t n, int64_t k, int tile_k, int accb, size_t budget, int* s,
               int* kbs, int64_t* used) {
  split_for_budget(m, n, k, tile_k, accb, budget, s, kbs, used);
  return MM_OK;
}

static int validate_common(int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                           const void* C, const void* ws, size_t ws_bytes) {
  if (acc_bytes(sr) == 0) return MM_ERR_ARG;
  if (m < 0 || n < 0 || k < 0) return MM_ERR_ARG;
  if (m > kMaxDim || n > kMaxDim || k > kMaxDim) return MM_ERR_SHAPE;
  if (m == 0 || n == 0) return MM_OK;
  if (!C || (k > 0 && (!A || !B))) return MM_ERR_ARG;
  if (ws_bytes > 0 && !ws) return MM_ERR_ARG;
  if (!aligned16(C) || (k > 0 && (!aligned16(A) || !aligned16(B)))) return MM_ERR_ALIGN;
  if (ws && !aligned16(ws)) return MM_ERR_ALIGN;
  return MM_OK;
}

int report_cuda(cudaError_t e, const char* where) {
  fprintf(stderr, "libmmsr: %s failed: CUDA error %d (%s)\n", where, (int)e, cudaGetErrorString(e));
  return MM_ERR_CUDA;
}

static int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MM_OK;
  fprintf(stderr, "libmmsr: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
  return MM_ERR_CUDA;
}

int run_semiring(int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B, void* C,
                 void* ws, size_t ws_bytes, cudaStream_t st) {
  mm_plan_t p;
  int rc = plan_semiring(sr, m, n, k, ws_bytes, &p);
  if (rc != MM_OK) return rc;
  if ((size_t)p.workspace_min > ws_bytes) return MM_ERR_WORKSPACE;
  const int s = p.split_k;
  const int64_t kb_total = (k + p.tile_k - 1) / p.tile_k;
  const int kbs = kb_total > 0 ? (int)((kb_total + s - 1) / s) : 0;
  cudaError_t e = cudaSuccess;
  switch (sr) {
    case MM_SR_MIN_PLUS_I32: {
      int32_t* W = s > 1 ? static_cast<int32_t*>(ws) : nullptr;
      e = launch_minplus_leaf(m, n, k, static_cast<const int32_t*>(A),
                              static_cast<const int32_t*>(B), static_cast<int32_t*>(C), W, s, kbs,
                              st);
      if (e == cudaSuccess && s > 1)
        e = launch_min_reduce(m * n, static_cast<int32_t*>(C), W, s - 1, st);
      break;
    }
    case MM_SR_PLUS_TIMES_F64: {
      if (p.kernel == 6) {
        e = launch_dfma_streamk(m, n, k, static_cast<const double*>(A), static_cast<const double*>(B),
                                static_cast<double*>(C), ws, st);
        break;
      }
      double* W = s > 1 ? static_cast<double*>(ws) : nullptr;
      e = launch_dfma_leaf(m, n, k, static_cast<const double*>(A), static_cast<const double*>(B),
                           static_cast<double*>(C), W, s, kbs, st);
      if (e == cudaSuccess && s > 1)
        e = launch_sum_reduce_f64(m * n, static_cast<double*>(C), W, s - 1, st);
      break;
    }
    default:
      return run_extended(sr, m, n, k, A, B, C, ws, ws_bytes, st, p);
  }
  return cuda_status(e);
}

}  // namespace mmsr

using namespace mmsr;

extern "C" {

int mm_semiring(int semiring, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                void* C, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = validate_common(semiring, m, n, k, A, B, C, workspace, workspace_bytes);
  if (rc != MM_OK || m == 0 || n == 0) return rc;
  return run_semiring(semiring, m, n, k, A, B, C, workspace, workspace_bytes,
                      static_cast<cudaStream_t>(stream));
}

int mm_strassen(int levels, int variant, int semiring, int64_t m, int64_t n, int64_t k,
                const void* A, const void* B, void* C, void* workspace, size_t workspace_bytes,
                void* stream) {
  int rc = validate_common(semiring, m, n, k, A, B, C, workspace, workspace_bytes);
  if (rc != MM_OK) return rc;
  if (variant != MM_STRASSEN_PAPER && variant != MM_STRASSEN_WINOGRAD) return MM_ERR_ARG;
  // Strassen-like recursions need the inverse of (+) (Section 5): only the
  // (+, x) semirings qualify.
  if (semiring == MM_SR_MIN_PLUS_I32 || semiring == MM_SR_OR_AND_U8) return MM_ERR_UNSUPPORTED;
  if (levels == MM_LEVELS_AUTO) levels = choose_strassen_levels(semiring, m, n, k, workspace_bytes);
  if (levels < 0 || levels > kMaxLevels) return MM_ERR_ARG;
  const int64_t mask = ((int64_t)1 << levels) - 1;
  if ((m & mask) || (n & mask) || (k & mask)) return MM_ERR_SHAPE;
  if (m == 0 || n == 0) return MM_OK;
  if (levels == 0)
    return run_semiring(semiring, m, n, k, A, B, C, workspace, workspace_bytes,
                        static_cast<cudaStream_t>(stream));
  return run_strassen(levels, variant, semiring, m, n, k, A, B, C, workspace, workspace_bytes,
                      static_cast<cudaStream_t>(stream));
}

// Shared checks of the mixed (STAR-Strassen-1) plan entry points.
static int check_star(int classic, int levels, int semiring, int64_t m, int64_t n, int64_t k) {
  if (acc_bytes(semiring) == 0 || m < 0 || n < 0 || k < 0) return MM_ERR_ARG;
  if (m > kMaxDim || n > kMaxDim || k > kMaxDim) return MM_ERR_SHAPE;
  if (classic < 0 || classic > kMaxLevels || levels < 0 || levels > kMaxLevels) return MM_ERR_ARG;
  if (semiring == MM_SR_MIN_PLUS_I32 || semiring == MM_SR_OR_AND_U8) return MM_ERR_UNSUPPORTED;
  const int64_t mask = ((int64_t)1 << (classic + levels)) - 1;
  if ((m & mask) || (n & mask) || (k & mask)) return MM_ERR_SHAPE;
  return MM_OK;
}

int mm_star_strassen(int classic_levels, int levels, int variant, int semiring, int64_t m, int64_t n,
                     int64_t k, const void* A, const void* B, void* C, void* workspace,
                     size_t workspace_bytes, void* stream) {
  int rc = validate_common(semiring, m, n, k, A, B, C, workspace, workspace_bytes);
  if (rc != MM_OK) return rc;
  if (variant != MM_STRASSEN_PAPER && variant != MM_STRASSEN_WINOGRAD) return MM_ERR_ARG;
  rc = check_star(classic_levels, levels, semiring, m, n, k);
  if (rc != MM_OK || m == 0 || n == 0) return rc;
  return run_star_strassen(classic_levels, levels, variant, semiring, m, n, k, A, B, C, workspace,
                           workspace_bytes, static_cast<cudaStream_t>(stream));
}

int mm_star_strassen_query(int classic_levels, int levels, int semiring, int64_t m, int64_t n,
                           int64_t k, size_t workspace_bytes, mm_plan_t* plan) {
  if (!plan) return MM_ERR_ARG;
  const int rc = check_star(classic_levels, levels, semiring, m, n, k);
  if (rc != MM_OK) return rc;
  return plan_star_strassen(classic_levels, levels, semiring, m, n, k, workspace_bytes, plan);
}

int mm_strassen_tar(int levels, int variant, int semiring, int64_t m, int64_t n, int64_t k, const void* A,
                    const void* B, void* C, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = validate_common(semiring, m, n, k, A, B, C, workspace, workspace_bytes);
  if (rc != MM_OK) return rc;
  if (variant != MM_STRASSEN_PAPER && variant != MM_STRASSEN_WINOGRAD) return MM_ERR_ARG;
  if (levels < 1 || levels > 2) return MM_ERR_ARG;
  if (semiring != MM_SR_PLUS_TIMES_F32 && semiring != MM_SR_PLUS_TIMES_F64ACC) return MM_ERR_UNSUPPORTED;
  const int64_t mask = (1 << levels) - 1;
  if ((m & mask) || (n & mask) || (k & mask)) return MM_ERR_SHAPE;
  if (m == 0 || n == 0) return MM_OK;
  return run_strassen_tar(levels, variant, semiring, m, n, k, A, B, C, workspace, workspace_bytes,
                          static_cast<cudaStream_t>(stream));
}

int mm_strassen_tar_query(int levels, int semiring, int64_t m, int64_t n, int64_t k, mm_plan_t* plan) {
  if (!plan) return MM_ERR_ARG;
  if (acc_bytes(semiring) == 0 || m < 0 || n < 0 || k < 0 || levels < 1 || levels > 2) return MM_ERR_ARG;
  if (m > kMaxDim || n > kMaxDim || k > kMaxDim) return MM_ERR_SHAPE;
  if (semiring != MM_SR_PLUS_TIMES_F32 && semiring != MM_SR_PLUS_TIMES_F64ACC) return MM_ERR_UNSUPPORTED;
  const int64_t mask = (1 << levels) - 1;
  if ((m & mask) || (n & mask) || (k & mask)) return MM_ERR_SHAPE;
  return plan_strassen_tar(levels, semiring, m, n, k, plan);
}

int mm_strassen_tar_waves(int levels, int variant, int* wave_of_product) {
  if (!wave_of_product) return MM_ERR_ARG;
  if (variant != MM_STRASSEN_PAPER && variant != MM_STRASSEN_WINOGRAD) return MM_ERR_ARG;
  if (levels < 1 || levels > 2) return MM_ERR_ARG;
  return strassen_tar_waves(levels, variant, wave_of_product);
}

int mm_plan_query(int semiring, int levels, int64_t m, int64_t n, int64_t k,
                  size_t workspace_bytes, mm_plan_t* plan) {
  if (!plan) return MM_ERR_ARG;
  if (acc_bytes(semiring) == 0 || m < 0 || n < 0 || k < 0) return MM_ERR_ARG;
  if (m > kMaxDim || n > kMaxDim || k > kMaxDim) return MM_ERR_SHAPE;
  if (levels < 0) return plan_semiring(semiring, m, n, k, workspace_bytes, plan);
  if (levels != MM_LEVELS_AUTO && levels > kMaxLevels) return MM_ERR_ARG;
  if (semiring == MM_SR_MIN_PLUS_I32 || semiring == MM_SR_OR_AND_U8) return MM_ERR_UNSUPPORTED;
  if (levels == MM_LEVELS_AUTO) levels = choose_strassen_levels(semiring, m, n, k, workspace_bytes);
  const int64_t mask = ((int64_t)1 << levels) - 1;
  if ((m & mask) || (n & mask) || (k & mask)) return MM_ERR_SHAPE;
  if (levels == 0) return plan_semiring(semiring, m, n, k, workspace_bytes, plan);
  return plan_strassen(levels, semiring, m, n, k, workspace_bytes, plan);
}

int mm_last_device_status(void* stream, int* status) {
  if (!status) return MM_ERR_ARG;
  return read_device_status(static_cast<cudaStream_t>(stream), status);
}

const char* mm_status_string(int status) {
  switch (status) {
    case MM_OK: return "MM_OK";
    case MM_ERR_ARG: return "MM_ERR_ARG: invalid argument";
    case MM_ERR_UNSUPPORTED: return "MM_ERR_UNSUPPORTED: operation not defined for this semiring";
    case MM_ERR_WORKSPACE: return "MM_ERR_WORKSPACE: workspace budget below the plan's minimum";
    case MM_ERR_SHAPE: return "MM_ERR_SHAPE: shape not allowed by the operation";
    case MM_ERR_CUDA: return "MM_ERR_CUDA: a CUDA runtime call failed";
    case MM_ERR_TIMEOUT: return "MM_ERR_TIMEOUT: a bounded device-side wait gave up";
    case MM_ERR_ALIGN: return "MM_ERR_ALIGN: pointer not 16-byte aligned";
    default: return "unknown mm_status_t";
  }
}

int mm_version(void) { return 100; }

int mm_set_option(int option, int value) {
  switch (option) {
    case MM_OPT_MINPLUS_PACKED:
      if (value != 0 && value != 1) return MM_ERR_ARG;
      g_packed_mode = value;
      return MM_OK;
    case MM_OPT_MINPLUS_STREAMK:
      if (value != 0 && value != 1) return MM_ERR_ARG;
      g_streamk_mode = value;
      return MM_OK;
    case MM_OPT_STRASSEN_FUSED:
      if (value != 0 && value != 1) return MM_ERR_ARG;
      g_strassen_fused = value;
      return MM_OK;
    case MM_OPT_F32_STREAMK:
      if (value < 0 || value > 3) return MM_ERR_ARG;
      g_f32_streamk = value;
      return MM_OK;
    case MM_OPT_F64_STREAMK:
      if (value < 0 || value > 2) return MM_ERR_ARG;
      g_f64_streamk = value;
      return MM_OK;
    case MM_OPT_F64ACC_SLICES:
      if (value != 0 && value != 6 && value != 7) return MM_ERR_ARG;
      g_f64acc_slices = value;
      return MM_OK;
    case MM_OPT_STRASSEN_TOP_F64:
      if (value != 0 && value != 1) return MM_ERR_ARG;
      g_strassen_top_f64 = value;
      return MM_OK;
    case MM_OPT_TEST_SKIP_SIGNAL: {
      if (value < 0 || value > 3) return MM_ERR_ARG;
      int r = arm_tc_skip_signal(value == 1);
      if (r == MM_OK) r = arm_f64acc_skip_signal(value == 2);
      if (r == MM_OK) r = arm_batched_skip_signal(value == 3);
      return r;
    }
    default:
      return MM_ERR_ARG;
  }
}

}  // extern "C"
