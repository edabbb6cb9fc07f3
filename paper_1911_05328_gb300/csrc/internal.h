// internal.h -- host-side interfaces between the ABI layer and the engines
// (tensor-core modes, Strassen, batched).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include <cuda_bf16.h>

#include "../../include/mmsr.h"

namespace mmsr {

constexpr int kMaxSplit = 64;          // largest split-K factor the planner uses
constexpr int64_t kMaxDim = 1 << 22;   // per-dimension cap (grid limits)
constexpr int kMaxLevels = 4;          // Strassen levels accepted

int elem_bytes(int sr);
int plan_semiring(int sr, int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p);
int run_semiring(int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B, void* C,
                 void* ws, size_t ws_bytes, cudaStream_t st);
int split_plan(int64_t m, int64_t n, int64_t k, int tile_k, int accb, size_t budget, int* s,
               int* kbs, int64_t* used);

// tensor-core and boolean semirings (plan + run)
int plan_extended(int sr, int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p);
int run_extended(int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B, void* C,
                 void* ws, size_t ws_bytes, cudaStream_t st, const mm_plan_t& p);

// FP32 mode: bf16x3 split products on tcgen05 tensor cores
int plan_f32(int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p);
int run_f32(int64_t m, int64_t n, int64_t k, const float* A, const float* B, float* C, void* ws,
            size_t ws_bytes, cudaStream_t st);
int read_tc_status(int* status);

// boolean (or, and) semiring on bit-packed operands
int plan_orand(int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p);
int run_orand(int64_t m, int64_t n, int64_t k, const uint8_t* A, const uint8_t* B, uint8_t* C,
              void* ws, size_t ws_bytes, cudaStream_t st);

// FP64-accuracy mode: digit slices per operand on tcgen05 -- six 8-bit
// slices (21 products) or seven 7-bit slices (28 products); the number of
// Strassen levels above the leaves picks the scheme (f64acc_slices_for_levels)
extern int g_f64acc_slices;  // mm_set_option(MM_OPT_F64ACC_SLICES, ...)
extern int g_f32_streamk;    // mm_set_option(MM_OPT_F32_STREAMK, ...)
extern int g_f64_streamk;    // mm_set_option(MM_OPT_F64_STREAMK, ...)
int f64acc_slices_for_levels(int levels);
int plan_f64acc(int64_t m, int64_t n, int64_t k, size_t budget, mm_plan_t* p);
int run_f64acc(int64_t m, int64_t n, int64_t k, const double* A, const double* B, double* C,
               void* ws, size_t ws_bytes, cudaStream_t st);
int read_f64acc_status(int* status);
// `batches` stacked FP64-accuracy products (Strassen leaves): A is batches x
// m x k, B batches x k x n, C batches x m x n, all contiguous.
size_t f64acc_batched_bytes(int64_t m, int64_t n, int64_t k, int batches, int slices);
// maxima_ready: the row exponents E and column maxima Fmax of A and B
// (f64acc_maxima_buffers) were already written by the pass that produced
// them, so the split skips its own passes over A's rows and B's columns.
int run_f64acc_batched(const double* A, const double* B, double* C, int64_t m, int64_t n, int64_t k,
                       int batches, int slices, void* ws, cudaStream_t st, bool maxima_ready = false);
// Where the split of those stacked products keeps, inside ws, the row
// exponents E (int, batches x m: frexp's exponent of each row's max |a|)
// and the column maxima Fmax (|b| bit patterns, batches x n, to be folded
// in with atomicMax from zero).
void f64acc_maxima_buffers(int64_t m, int64_t n, int64_t k, int batches, int slices, void* ws, int** E,
                           unsigned long long** Fmax);
int read_batched_status(int* status);
// Test switches (one-shot): the first CTA of the next launch of the FP32
// GEMM / FP64-accuracy GEMM / batched FP32 kernel skips its first ring
// stage's arrival, so a bounded wait runs out.  on = 0 disarms.
int arm_tc_skip_signal(int on);
int arm_f64acc_skip_signal(int on);
int arm_batched_skip_signal(int on);

// Leaf epilogue that adds each product into blocks of C instead of writing
// it out (TAR-Strassen): batch entry b computes the product of stacked leaf
// operands leaf[b] and adds sign[b][d] x product into dst[b][d] (d < 4,
// nullptr = unused; row pitch ld), overwriting where add[b][d] == 0.
// entries == 0 selects the ordinary output.
constexpr int kQuadEntries = 16;
template <typename T>
struct QuadOutT {
  T* dst[kQuadEntries][4];
  int8_t sign[kQuadEntries][4];
  int8_t add[kQuadEntries][4];
  int16_t leaf[kQuadEntries];
  int64_t ld;
  int entries;
};
using QuadOut = QuadOutT<float>;
using QuadOut64 = QuadOutT<double>;

// TAR-Strassen leaves in FP64-accuracy mode: exponents and digit slices of
// `batches` stacked products once, then launches whose entries add their
// products into blocks of C (QuadOut64); `ws` as for run_f64acc_batched
int f64acc_prepare_batched(const double* A, const double* B, int64_t m, int64_t n, int64_t k, int batches,
                           int slices, void* ws, cudaStream_t st, bool maxima_ready = false);
int f64acc_gemm_quad(int64_t m, int64_t n, int64_t k, int batches, int slices, void* ws, const QuadOut64& quad,
                     cudaStream_t st);

// batched leaves (independent products on stacked operands); with `quad`,
// the entries' leaves index a stack of `map_batches` operands
cudaError_t launch_bf16x3_batched(const __nv_bfloat16* ahi, const __nv_bfloat16* alo,
                                  const __nv_bfloat16* bhi, const __nv_bfloat16* blo, float* P,
                                  int64_t m, int64_t n, int64_t Kp, int batches, cudaStream_t st,
                                  const QuadOut* quad = nullptr, int map_batches = 0);
cudaError_t launch_dfma_batched(const double* A, const double* B, double* C, int64_t m, int64_t n,
                                int64_t k, int batches, cudaStream_t st);

// Strassen engine
// One FP32-mode Strassen level with the operand sums formed in the leaf's
// staging (MM_OPT_STRASSEN_FUSED): shapes it takes, the launch of its seven
// leaf products into a stack of (m/2) x (n/2) FP32 matrices, and its device
// status word.
extern int g_strassen_fused;
bool strassen_fused_shape_ok(int64_t m, int64_t n, int64_t k);
cudaError_t launch_strassen_fused_leaves(int variant, const float* A, const float* B, float* P, int64_t m, int64_t n,
                                         int64_t k, int64_t lda, int64_t ldb, cudaStream_t st);
int read_fused_status(int* status);
// Strassen depth picked for MM_LEVELS_AUTO under a workspace budget.
int choose_strassen_levels(int sr, int64_t m, int64_t n, int64_t k, size_t budget);
int plan_strassen(int levels, int sr, int64_t m, int64_t n, int64_t k, size_t budget,
                  mm_plan_t* p);
int run_strassen(int levels, int variant, int sr, int64_t m, int64_t n, int64_t k, const void* A,
                 const void* B, void* C, void* ws, size_t ws_bytes, cudaStream_t st);

// STAR-Strassen-1 mixed plans: `classic` in-place classic levels over
// `levels` Strassen levels
int plan_star_strassen(int classic, int levels, int sr, int64_t m, int64_t n, int64_t k,
                       size_t budget, mm_plan_t* p);
int run_star_strassen(int classic, int levels, int variant, int sr, int64_t m, int64_t n, int64_t k,
                      const void* A, const void* B, void* C, void* ws, size_t ws_bytes,
                      cudaStream_t st);

// TAR-Strassen, one or two levels: leaf products added straight into the
// blocks of C in conflict-free waves (FP32 and FP64-accuracy modes)
int plan_strassen_tar(int L, int sr, int64_t m, int64_t n, int64_t k, mm_plan_t* p);
int run_strassen_tar(int L, int variant, int sr, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                     void* C, void* ws, size_t ws_bytes, cudaStream_t st);
int strassen_tar_waves(int L, int variant, int* wave_of_product);

// closure by repeated squaring
int closure_squarings(int64_t n);
int plan_closure(int sr, int64_t n, size_t budget, mm_plan_t* p);
int run_closure(int sr, int64_t n, const void* A, void* C, void* ws, size_t ws_bytes, int flags,
                int* squarings, cudaStream_t st);

// device status word (bounded waits of the batched kernel)
int read_device_status(cudaStream_t st, int* status);

}  // namespace mmsr
