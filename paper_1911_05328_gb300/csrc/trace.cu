// trace.cu -- optional per-kernel CUDA-event tracing (diagnostics only).
// When enabled, every launcher brackets its kernel with two events on the
// launching stream; mm_trace_summary resolves them into per-kernel launch
// counts and summed device time.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace mmsr {
namespace {

const char* const kNames[kTraceKernels] = {
    "minplus_leaf", "min_reduce",   "dfma_leaf",   "sum_reduce_f64", "split_bf16x2",
    "tc_bf16x3",    "sum_reduce_f32", "split_f64_slices", "tc_f64acc", "strassen_combine",
    "strassen_post", "batched",     "orand_leaf",  "or_reduce",      "minplus16_leaf",
    "range_scan",   "orand_pack", "closure_aux"};

struct Rec {
  int id;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void recycle_all() {
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

}  // namespace

TraceScope::TraceScope(int id, cudaStream_t st) : id_(id), st_(st), a_(nullptr) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  a_ = get_event();
  if (a_) cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

TraceScope::~TraceScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  if (!b) {
    g_pool.push_back(static_cast<cudaEvent_t>(a_));
    return;
  }
  cudaEventRecord(b, st_);
  g_recs.push_back(Rec{id_, static_cast<cudaEvent_t>(a_), b});
}

}  // namespace mmsr

using namespace mmsr;

extern "C" {

int mm_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (on) recycle_all();
  g_on = on != 0;
  return MM_OK;
}

int mm_trace_kernel_count(void) { return kTraceKernels; }

const char* mm_trace_kernel_name(int id) {
  if (id < 0 || id >= kTraceKernels) return "unknown";
  return kNames[id];
}

int mm_trace_summary(int id, int64_t* launches, double* total_ms) {
  if (id < 0 || id >= kTraceKernels || !launches || !total_ms) return MM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t cnt = 0;
  double tot = 0.0;
  for (auto& r : g_recs) {
    if (r.id != id) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return MM_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return MM_ERR_CUDA;
    ++cnt;
    tot += ms;
  }
  *launches = cnt;
  *total_ms = tot;
  return MM_OK;
}

}  // extern "C"
