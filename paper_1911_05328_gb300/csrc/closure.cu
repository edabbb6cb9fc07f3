// closure.cu -- C := A* = 1 (+) A (+) A^2 (+) ... of a square matrix on an
// idempotent semiring: (min,+) gives all-pairs shortest paths, (or, and)
// reflexive-transitive reachability.  Section 2 poses MM on a closed
// semiring, whose defining extra operation is this closure; shortest paths
// are the dynamic-programming use of semiring MM the paper points to.
//
// Method: repeated squaring.  X_0 = 1 (+) A (the semiring's 1 folded into
// the diagonal) and X_{t+1} = X_t (x) X_t.  Because (+) is idempotent, X_t
// is the (+)-sum over all paths of at most 2^t arcs, and a best path needs
// at most n-1 arcs (no cycle has negative weight on [0, 2^30]), so X_T = A*
// once 2^T >= n-1.  Each squaring is one budgeted semiring product: the
// split-K budget of Sections 3-4 applies to every squaring, and the packed
// 16-bit (min,+) leaf is chosen per squaring by its own range scan (early,
// short distances) until the distances outgrow it.
//
// Optional early exit: X_{t+1} == X_t means the fixed point is reached
// (every later square equals it), so the remaining squarings are skipped.
// That test reads one device word per squaring and therefore synchronises
// the stream.
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace mmsr {
namespace {

constexpr int64_t kFlagBytes = 16;  // device word of the early-exit test (padded)

int64_t round16(int64_t x) { return (x + 15) / 16 * 16; }

// X = 1 (+) A for (min,+): A copied, diagonal min(A_ii, 0).  Each thread
// handles four consecutive elements (one 16-byte vector) when they exist.
__global__ void __launch_bounds__(256) closure_init_minplus_kernel(const int32_t* __restrict__ A,
                                                                   int32_t* __restrict__ X,
                                                                   int64_t n) {
  const int64_t total = n * n;
  const int64_t nvec = total / 4;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec;
       v += (int64_t)gridDim.x * blockDim.x) {
    int4 a = reinterpret_cast<const int4*>(A)[v];
    int32_t* e = reinterpret_cast<int32_t*>(&a);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t idx = v * 4 + q, i = idx / n;
      if (idx - i * n == i && e[q] > 0) e[q] = 0;
    }
    reinterpret_cast<int4*>(X)[v] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x < total - nvec * 4) {
    const int64_t idx = nvec * 4 + threadIdx.x, i = idx / n;
    int32_t x = A[idx];
    if (idx - i * n == i && x > 0) x = 0;
    X[idx] = x;
  }
}

// X = 1 (+) A for (or, and): nonzero -> 1, diagonal 1.  Sixteen bytes per
// thread.
__global__ void __launch_bounds__(256) closure_init_orand_kernel(const uint8_t* __restrict__ A,
                                                                 uint8_t* __restrict__ X,
                                                                 int64_t n) {
  const int64_t total = n * n;
  const int64_t nvec = total / 16;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec;
       v += (int64_t)gridDim.x * blockDim.x) {
    uint4 a = reinterpret_cast<const uint4*>(A)[v];
    uint8_t* e = reinterpret_cast<uint8_t*>(&a);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int64_t idx = v * 16 + q, i = idx / n;
      e[q] = (e[q] != 0 || idx - i * n == i) ? 1 : 0;
    }
    reinterpret_cast<uint4*>(X)[v] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x < total - nvec * 16) {
    const int64_t idx = nvec * 16 + threadIdx.x, i = idx / n;
    X[idx] = (A[idx] != 0 || idx - i * n == i) ? 1 : 0;
  }
}

// *flag |= (X != Y) over `bytes` bytes (both 16-byte aligned).
__global__ void __launch_bounds__(256) closure_diff_kernel(const uint8_t* __restrict__ X,
                                                           const uint8_t* __restrict__ Y,
                                                           int64_t bytes, int* flag) {
  const int64_t nvec = bytes / 16;
  int diff = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint4 a = reinterpret_cast<const uint4*>(X)[v];
    const uint4 b = reinterpret_cast<const uint4*>(Y)[v];
    diff |= (a.x != b.x) | (a.y != b.y) | (a.z != b.z) | (a.w != b.w);
  }
  if (blockIdx.x == 0 && threadIdx.x < bytes - nvec * 16) {
    const int64_t idx = nvec * 16 + threadIdx.x;
    diff |= X[idx] != Y[idx];
  }
  if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(flag, 1);
}

unsigned stream_grid(int64_t work) {
  int64_t b = (work + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

int closure_elem_bytes(int sr) {
  return sr == MM_SR_MIN_PLUS_I32 ? 4 : (sr == MM_SR_OR_AND_U8 ? 1 : 0);
}

}  // namespace

int closure_squarings(int64_t n) {
  int t = 0;
  while (((int64_t)1 << t) < n - 1) ++t;
  return t;
}

// Workspace: [flag word][ping buffer of n x n][the squaring's own workspace].
int plan_closure(int sr, int64_t n, size_t budget, mm_plan_t* p) {
  memset(p, 0, sizeof(*p));
  const int eb = closure_elem_bytes(sr);
  if (eb == 0) return MM_ERR_UNSUPPORTED;
  const int64_t prefix = kFlagBytes + round16(n * n * eb);
  mm_plan_t sq;
  const size_t rest = budget > (size_t)prefix ? budget - (size_t)prefix : 0;
  int rc = plan_semiring(sr, n, n, n, rest, &sq);
  if (rc != MM_OK) return rc;
  *p = sq;
  p->levels = closure_squarings(n);
  p->workspace_min = prefix + sq.workspace_min;
  p->workspace_used = prefix + sq.workspace_used;
  return MM_OK;
}

int run_closure(int sr, int64_t n, const void* A, void* C, void* ws, size_t ws_bytes, int flags,
                int* squarings, cudaStream_t st) {
  mm_plan_t p;
  int rc = plan_closure(sr, n, ws_bytes, &p);
  if (rc != MM_OK) return rc;
  if ((size_t)p.workspace_min > ws_bytes) return MM_ERR_WORKSPACE;
  const bool early = (flags & MM_CLOSURE_EARLY_EXIT) != 0;
  if (early) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MMSR_TRY_STATUS(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return MM_ERR_ARG;  // needs a host read per squaring
  }
  const int eb = closure_elem_bytes(sr);
  const int64_t bytes = n * n * eb;
  uint8_t* w = static_cast<uint8_t*>(ws);
  int* flag = reinterpret_cast<int*>(w);
  uint8_t* ping = w + kFlagBytes;
  uint8_t* sq_ws = ping + round16(bytes);
  const size_t sq_budget = ws_bytes - (size_t)(kFlagBytes + round16(bytes));
  const int T = p.levels;
  // X_t lives in buf[t % 2]; the parity puts X_T in C.
  uint8_t* buf[2];
  buf[T & 1] = static_cast<uint8_t*>(C);
  buf[(T & 1) ^ 1] = ping;
  {
    TraceScope tr(kTrClosureAux, st);
    if (sr == MM_SR_MIN_PLUS_I32)
      closure_init_minplus_kernel<<<stream_grid((n * n + 3) / 4), 256, 0, st>>>(
          static_cast<const int32_t*>(A), reinterpret_cast<int32_t*>(buf[0]), n);
    else
      closure_init_orand_kernel<<<stream_grid((n * n + 15) / 16), 256, 0, st>>>(
          static_cast<const uint8_t*>(A), buf[0], n);
    MMSR_TRY_STATUS(cudaGetLastError());
  }
  int done = 0;
  for (int t = 0; t < T; ++t) {
    rc = run_semiring(sr, n, n, n, buf[t & 1], buf[t & 1], buf[(t + 1) & 1], sq_ws, sq_budget, st);
    if (rc != MM_OK) return rc;
    done = t + 1;
    if (early && t + 1 < T) {
      {
        TraceScope tr(kTrClosureAux, st);
        MMSR_TRY_STATUS(cudaMemsetAsync(flag, 0, sizeof(int), st));
        closure_diff_kernel<<<stream_grid((bytes + 15) / 16), 256, 0, st>>>(
            buf[t & 1], buf[(t + 1) & 1], bytes, flag);
        MMSR_TRY_STATUS(cudaGetLastError());
      }
      int changed = 1;
      MMSR_TRY_STATUS(cudaMemcpyAsync(&changed, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      MMSR_TRY_STATUS(cudaStreamSynchronize(st));
      if (!changed) break;
    }
  }
  if (buf[done & 1] != static_cast<uint8_t*>(C))
    MMSR_TRY_STATUS(cudaMemcpyAsync(C, buf[done & 1], bytes, cudaMemcpyDeviceToDevice, st));
  if (squarings) *squarings = done;
  return MM_OK;
}

}  // namespace mmsr

using namespace mmsr;

extern "C" {

int mm_closure(int semiring, int64_t n, const void* A, void* C, void* workspace,
               size_t workspace_bytes, int flags, int* squarings, void* stream) {
  if (squarings) *squarings = 0;
  if (semiring != MM_SR_MIN_PLUS_I32 && semiring != MM_SR_OR_AND_U8) {
    if (semiring >= MM_SR_PLUS_TIMES_F64 && semiring <= MM_SR_PLUS_TIMES_F64ACC)
      return MM_ERR_UNSUPPORTED;
    return MM_ERR_ARG;
  }
  if (n < 0 || (flags & ~MM_CLOSURE_EARLY_EXIT) != 0) return MM_ERR_ARG;
  if (n > kMaxDim) return MM_ERR_SHAPE;
  if (n == 0) return MM_OK;
  if (!A || !C || (workspace_bytes > 0 && !workspace)) return MM_ERR_ARG;
  if (!aligned16(A) || !aligned16(C) || (workspace && !aligned16(workspace))) return MM_ERR_ALIGN;
  return run_closure(semiring, n, A, C, workspace, workspace_bytes, flags, squarings,
                     static_cast<cudaStream_t>(stream));
}

int mm_closure_query(int semiring, int64_t n, size_t workspace_bytes, mm_plan_t* plan) {
  if (!plan) return MM_ERR_ARG;
  if (semiring != MM_SR_MIN_PLUS_I32 && semiring != MM_SR_OR_AND_U8) {
    if (semiring >= MM_SR_PLUS_TIMES_F64 && semiring <= MM_SR_PLUS_TIMES_F64ACC)
      return MM_ERR_UNSUPPORTED;
    return MM_ERR_ARG;
  }
  if (n < 0) return MM_ERR_ARG;
  if (n > kMaxDim) return MM_ERR_SHAPE;
  return plan_closure(semiring, n, workspace_bytes, plan);
}

}  // extern "C"
