/*
 * mmsr.h -- C ABI of the GB300 semiring / Strassen-Winograd matrix
 * multiplication library (libmmsr.so).
 *
 * Problem (Section 2, "General MM C = A (x) B on a closed semiring
 * SR = (S, (+), (x), 0, 1)", and the quadrant recursion of Eq. (mm-dac)):
 *
 *     C[i][j] = (+)_{t=0}^{k-1} A[i][t] (x) B[t][j]
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Layout: dense row-major, no leading dimensions.  A is m x k, B is k x n,
 *    C is m x n.  A, B, C and the workspace must not overlap.
 *  - Pointers A, B, C and `workspace` are DEVICE pointers (cudaMalloc'd or
 *    torch-allocated memory on the current device).  The caller owns all of
 *    them; the library never allocates device memory on these paths.
 *  - C is OVERWRITTEN with A (x) B (it is not accumulated into).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call is asynchronous on that stream.
 *  - `workspace_bytes` is a hard cap: the plan never touches more than that
 *    many bytes of `workspace`, and never touches memory past it.  The
 *    paper's space/time trade-off (CO2 in-place k-serial vs. CO3/SAR/STAR
 *    k-parallel with temporaries, Sections 3-4) is realised as split-K:
 *    k is divided into s slices, slice 0 is accumulated in C itself and
 *    slices 1..s-1 in workspace buffers of m*n accumulators, followed by a
 *    fixed-order (+)-reduction ("madd"/"atomic-madd", Figs. mm-n3, tar-mm).
 *    s = 1 + floor(workspace_bytes / (m*n*sizeof(accumulator))), clamped so
 *    that every slice holds at least one k-block.
 *  - Errors detectable on the host return immediately, before any launch,
 *    with one of the negative mm_status_t codes; nothing is written.
 *  - Thread safety: calls are re-entrant as long as concurrent calls use
 *    different C and workspace buffers.
 */
#ifndef MMSR_H_
#define MMSR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Semirings.  Element types of A, B and C follow the name. */
typedef enum {
  /* (+, x) over FP64, plain FP64 CUDA-core (DFMA) path.  Accumulator FP64. */
  MM_SR_PLUS_TIMES_F64 = 0,
  /* (+, x) over FP32 in/out: each operand split into a bf16 (hi, lo) pair,
   * products hi*hi + hi*lo + lo*hi on tcgen05 tensor cores, FP32 accumulate.
   * Needs 4*(m*k + k*n) bytes of workspace for the split operands. */
  MM_SR_PLUS_TIMES_F32 = 1,
  /* (+, x) over FP64 in/out at FP64 accuracy: every row of A / column of B
   * is scaled by a power of two and cut into integer digit slices (bf16):
   * six 8-bit slices (21 slice products of digit order <= 5) for a plain
   * product, seven 7-bit slices (28 products) under three or four Strassen
   * levels (see MM_OPT_F64ACC_SLICES).  The products run on tcgen05 tensor
   * cores with exact chunked integer accumulation, combined once in FP64.
   * Needs 2*S*(m+n)*Kp + 4*(m+n) + 8*n bytes of workspace for S slices
   * (Kp = k rounded up to 32); mm_plan_query reports it. */
  MM_SR_PLUS_TIMES_F64ACC = 2,
  /* (min, +) tropical semiring over int32 in [0, 2^30]; 2^30 is +infinity
   * (the semiring's 0).  Sums saturate at 2^30 (never wrap).  Inputs outside
   * [0, 2^30] are a precondition violation (not checked on the device). */
  MM_SR_MIN_PLUS_I32 = 3,
  /* Boolean (or, and) over uint8; nonzero = true, output is 0 or 1.
   * Operands are bit-packed along k in the workspace (4*(m+n)*ceil(k/32)
   * bytes); split-K partials are one byte per output. */
  MM_SR_OR_AND_U8 = 4
} mm_semiring_t;

typedef enum {
  MM_OK = 0,
  MM_ERR_ARG = -1,         /* null pointer, negative size, bad enum value     */
  MM_ERR_UNSUPPORTED = -2, /* semiring/operation pair not defined (e.g.
                              Strassen needs the inverse of (+), Section 5)  */
  MM_ERR_WORKSPACE = -3,   /* workspace_bytes below the plan's minimum       */
  MM_ERR_SHAPE = -4,       /* shape not allowed by the operation             */
  MM_ERR_CUDA = -5,        /* a CUDA runtime call failed                     */
  MM_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up             */
  MM_ERR_ALIGN = -7        /* a pointer is not 16-byte aligned               */
} mm_status_t;

/* What a call would do for a given budget (filled by mm_plan_query). */
typedef struct {
  int32_t split_k;          /* s: number of k slices (1 = k-serial, CO2-like) */
  int32_t levels;           /* Strassen levels (0 for mm_semiring)            */
  int32_t tile_m, tile_n, tile_k; /* CTA tile of the leaf kernel              */
  int32_t kernel;           /* leaf kernel: 0 FP64 DFMA, 1 (min,+), 2 FP32
                               bf16x3, 3 FP64-accuracy (7 slices), 4 boolean,
                               5 FP32 stream-K, 6 FP64 stream-K, 7 FP64-
                               accuracy (6 slices)                            */
  int64_t workspace_used;   /* bytes of workspace the call touches            */
  int64_t workspace_min;    /* smallest budget for which the call is valid    */
} mm_plan_t;

/*
 * mm_semiring -- C := A (x) B on `semiring` with classic (8-way, Eq. mm-dac)
 * blocking and budgeted split-K.
 *   semiring         one of mm_semiring_t
 *   m, n, k          sizes, m, n >= 1, k >= 0 (k = 0 writes the semiring 0)
 *   A, B, C          device pointers, 16-byte aligned
 *   workspace        device pointer (may be NULL iff workspace_bytes == 0)
 *   workspace_bytes  budget, see the conventions above
 *   stream           cudaStream_t
 * Returns MM_OK or a negative mm_status_t.
 * (min,+) calls keep a small verdict record (whether the inputs fit the
 * exact 16-bit path) in library device memory.  Calls made outside stream
 * capture reuse 4096 records round-robin; each captured call owns a record
 * of its own, so a graph's replays never share one with other calls, but
 * two replays of one graph (like any two calls given one workspace) must
 * not overlap on the GPU.  After 4096 captured (min,+) calls in a process,
 * later captures run the 32-bit leaf (same results, about half the rate).
 */
int mm_semiring(int semiring, int64_t m, int64_t n, int64_t k, const void* A, const void* B,
                void* C, void* workspace, size_t workspace_bytes, void* stream);

/*
 * mm_minplus_noalloc -- (min,+) product with split-K whose partial buffers
 * live in a static device array inside the library instead of a caller
 * workspace.  The paper has no counterpart; this exists for callers that
 * cannot allocate device memory at the call site: code hosted by a
 * framework whose memory pool owns the GPU (a raw cudaMalloc bypasses its
 * accounting and can synchronise the device), or programs whose device
 * footprint is fixed at start-up.
 *   m, n, k, A, B, C  as in mm_semiring with MM_SR_MIN_PLUS_I32
 *   split_k           requested k-slices (>= 1; clamped to the k-blocks)
 *   stream            cudaStream_t
 * Scratch limit: (s-1)*m*n*4 bytes must fit in 64 MiB (67,108,864 bytes),
 * else MM_ERR_WORKSPACE and nothing is launched.  Every GPU that loads the
 * library holds the 64 MiB array until the process exits.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress),
 * so make that first call before any stream capture.  All calls share the
 * one array: calls whose executions overlap on the GPU (different streams,
 * no ordering between them) race on it.  Nothing in it needs clearing: each
 * call overwrites every partial it later reads.  Allocates nothing.
 */
int mm_minplus_noalloc(int64_t m, int64_t n, int64_t k, const void* A, const void* B, void* C,
                       int split_k, void* stream);

/* Strassen variants (Section 5 and the bilinear generalisation). */
typedef enum {
  MM_STRASSEN_PAPER = 0,   /* the paper's printed S/T/P/C formulas          */
  MM_STRASSEN_WINOGRAD = 1 /* Strassen-Winograd: 7 products, 15 additions    */
} mm_strassen_variant_t;

/*
 * mm_strassen -- C := A (x) B with `levels` levels of a Strassen-like
 * recursion (Section 5, Lemma par-strassen, Theorem star-strassen-2) over
 * classic leaves.  Requires a (+) with an inverse: only the (+, x) semirings
 * are accepted (MM_ERR_UNSUPPORTED otherwise).  m, n and k must be
 * divisible by 2^levels (MM_ERR_SHAPE otherwise); 0 <= levels <= 4.
 * levels = 0 is mm_semiring.  The temporaries (operand sums S_r, T_r and
 * products P_r of each level) are carved from `workspace`; the plan's
 * workspace_min is O(n^2) and is reported by mm_plan_query.
 * levels = MM_LEVELS_AUTO lets the library pick the depth: the fastest
 * measured depth of the semiring (2 for FP32 mode, 2 for FP64-accuracy
 * mode, 4 for plain FP64), lowered until every leaf dimension stays at
 * least 1024 (512 for plain FP64), the shape divides by 2^levels and the
 * plan fits workspace_bytes (0 levels: mm_semiring).  mm_plan_query with
 * the same value reports the depth it picks in plan->levels.
 */
#define MM_LEVELS_AUTO 16
int mm_strassen(int levels, int variant, int semiring, int64_t m, int64_t n, int64_t k,
                const void* A, const void* B, void* C, void* workspace, size_t workspace_bytes,
                void* stream);

/*
 * mm_star_strassen -- C := A (x) B as STAR-Strassen-1 (Theorem
 * star-strassen-1): the top `classic_levels` levels are the classic 8-way
 * recursion of Eq. mm-dac done in place (each of the 2^c x 2^c blocks of C
 * accumulates its 2^c block products one after the other, c =
 * classic_levels, with no temporaries), and every block product runs
 * `levels` Strassen levels of `variant`.  The Strassen temporaries are those
 * of ONE block product, (m/2^c) x (n/2^c) x (k/2^c), reused by the next, so
 * the workspace is 4^c times smaller than that of mm_strassen at the same
 * block size while the arithmetic is (8/7)^c times that of Strassen on all
 * c + levels levels.
 *   classic_levels   0 .. 4 (0 is mm_strassen)
 *   levels           0 .. 4 (0 is mm_semiring on the whole product)
 *   variant, semiring, m, n, k, A, B, C, workspace, workspace_bytes, stream
 *                    as in mm_strassen; m, n, k divisible by
 *                    2^(classic_levels + levels), else MM_ERR_SHAPE
 * In FP32 mode the block products after the first add into C with the same
 * top-level summation as mm_strassen (double-float when levels >= 3).
 * Returns MM_OK or a negative mm_status_t.
 */
int mm_star_strassen(int classic_levels, int levels, int variant, int semiring, int64_t m, int64_t n,
                     int64_t k, const void* A, const void* B, void* C, void* workspace,
                     size_t workspace_bytes, void* stream);

/* The plan (workspace_min / workspace_used, leaf tiles, levels) of
 * mm_star_strassen for these arguments.  Host-only. */
int mm_star_strassen_query(int classic_levels, int levels, int semiring, int64_t m, int64_t n,
                           int64_t k, size_t workspace_bytes, mm_plan_t* plan);

/*
 * mm_strassen_tar -- C := A (x) B with one or two Strassen levels in the
 * paper's zero-temporary schedule (TAR-Strassen, Section 5): the leaf
 * products are not stored; the leaf epilogue adds each one (times its +-1
 * coefficient) straight into the blocks of C it contributes to -- leaf
 * product 7 r1 + r2 into block (q1, q2) with coefficient gamma[q1][r1]
 * gamma[q2][r2].  Products run in waves in which no two touch the same block
 * -- a greedy colouring of the coefficients in product order, for one level
 * of the paper's formulas P1; P2 || P5; P3 || P4; P6 || P7 -- so the
 * read-modify-writes of a wave never collide; a block's first writer
 * overwrites it.
 *   levels            1 or 2 (MM_ERR_ARG otherwise)
 *   variant           MM_STRASSEN_PAPER or MM_STRASSEN_WINOGRAD; a product
 *                     may reach at most four blocks, so two Winograd levels
 *                     (its P1 reaches all four quadrants) are
 *                     MM_ERR_UNSUPPORTED
 *   semiring          MM_SR_PLUS_TIMES_F32 or MM_SR_PLUS_TIMES_F64ACC
 *                     (MM_ERR_UNSUPPORTED otherwise: the block epilogue lives
 *                     in the bf16x3 and digit-slice leaves)
 *   m, n, k           divisible by 2^levels (MM_ERR_SHAPE otherwise)
 *   A, B, C, workspace, workspace_bytes, stream   as in mm_strassen
 * Workspace (mm_strassen_tar_query): the leaf operand sums (FP32 mode: bf16
 * hi/lo; FP64-accuracy mode: FP64 sums and their digit slices) -- in FP32
 * mode the product stack of mm_strassen (7^L (m/2^L)(n/2^L) values) is not
 * needed; in FP64-accuracy mode mm_strassen already overlays it on the FP64
 * operand stack, so both need the same.
 * Returns MM_OK or a negative mm_status_t.
 */
int mm_strassen_tar(int levels, int variant, int semiring, int64_t m, int64_t n, int64_t k, const void* A,
                    const void* B, void* C, void* workspace, size_t workspace_bytes, void* stream);

/* Plan (workspace_min / workspace_used) of mm_strassen_tar.  Host-only. */
int mm_strassen_tar_query(int levels, int semiring, int64_t m, int64_t n, int64_t k, mm_plan_t* plan);

/* The wave schedule of mm_strassen_tar: writes, for leaf products p = 0 ..
 * 7^levels - 1 (p = 7 r1 + r2 at two levels, r in the order of
 * mm_strassen_tables), the wave each one runs in, and returns the number of
 * waves, MM_ERR_UNSUPPORTED when a product would reach more than four blocks
 * (the waves are still written), or MM_ERR_ARG.  Host-only. */
int mm_strassen_tar_waves(int levels, int variant, int* wave_of_product);

/*
 * mm_strassen_tables -- the bilinear coefficients one level of `variant`
 * uses (host copy of the device tables): alpha[7][4] (S_r = sum_q
 * alpha[r][q] A_q), beta[7][4] (T_r = sum_q beta[r][q] B_q) and gamma[4][7]
 * (C_q = sum_r gamma[q][r] P_r), quadrants ordered 00, 01, 10, 11, row-major
 * int8 arrays of 28 entries each, written by the call.  Section 5 prints the
 * MM_STRASSEN_PAPER table.  Returns MM_OK or MM_ERR_ARG.
 */
int mm_strassen_tables(int variant, int8_t* alpha, int8_t* beta, int8_t* gamma);

/* One problem of a batch (host-side descriptor; pointers are device). */
typedef struct {
  int32_t semiring; /* MM_SR_PLUS_TIMES_F32 or MM_SR_MIN_PLUS_I32 */
  int32_t levels;   /* Strassen-Winograd levels: 0, or 1 for an FP32 problem with
                     * even m, n, k (its seven leaf products join the batch's tile
                     * queue, their operand sums are formed by the pre-pass and a
                     * post pass folds them into C); (min,+): 0 */
  int64_t m, n, k;
  const void* A;
  const void* B;
  void* C;
  /* FP32 problems: k-slices per 128 x 128 output tile (Section 3's k-split
   * inside the batch).  0: the library's rule -- a tile whose k-blocks exceed
   * an eighth of one SM's share of the batch's FP32 work is cut into slices
   * of that size (at least 8 k-blocks, at most 16 slices); 1: never; s > 1:
   * s slices (at most 64 and the tile's 64-wide k-blocks).  Must be 0 for
   * (min,+) problems. */
  int32_t split_k;
  int32_t reserved; /* must be 0 */
} mm_problem_t;

/*
 * mm_batched -- C_p := A_p (x) B_p for `count` independent problems of
 * mixed shapes and semirings in one call (the dynamic load balance of
 * Section 6): FP32 (+, x) tiles run in a persistent tensor-core kernel that
 * pops a cost-sorted tile queue, (min,+) tiles in a CUDA-core launch over a
 * cost-sorted tile list.  Asynchronous and capturable in a CUDA graph.
 * `problems` is a HOST array read during the call; 0 <= count <= 2^20.  The
 * call copies its cost-sorted problem table into the workspace (as kernel
 * parameters of a few small launches, so a captured graph replays the same
 * table).  Workspace holds the tile counter, the per-problem range verdicts,
 * the table, the split FP32 operands and, for FP32 tiles cut into k-slices,
 * one 64 KB partial tile per slice and a counter per tile: the last slice to
 * finish folds the partials in slice order (a fixed order: results repeat
 * exactly) and writes C; for problems with a Strassen level, the seven leaf
 * products ((m/2)(n/2) FP32 values each).  mm_batched_query reports the
 * minimum.  Errors: MM_ERR_ARG (levels outside 0..1, split_k < 0, a
 * nonzero split_k on a (min,+) problem), MM_ERR_UNSUPPORTED (another
 * semiring, levels on (min,+), reserved != 0), MM_ERR_SHAPE (odd m, n or k
 * with levels = 1).
 */
int mm_batched(int count, const mm_problem_t* problems, void* workspace, size_t workspace_bytes,
               void* stream);

/* Workspace the batched call needs for these problems (0 on bad input). */
size_t mm_batched_query(int count, const mm_problem_t* problems);

/* Flags of mm_closure. */
#define MM_CLOSURE_EARLY_EXIT 1

/*
 * mm_closure -- C := A* = 1 (+) A (+) A^2 (+) ... for a square n x n matrix
 * on a semiring whose (+) is idempotent (Section 2 poses MM on a closed
 * semiring; the closure is that structure's extra operation).
 *   MM_SR_MIN_PLUS_I32: A[i][j] is the length of arc i -> j in [0, 2^30]
 *     (2^30 = no arc); C is the all-pairs shortest-path matrix (diagonal 0,
 *     2^30 = unreachable; path lengths saturate at 2^30).
 *   MM_SR_OR_AND_U8: A[i][j] nonzero = arc; C is reflexive-transitive
 *     reachability as 0/1.
 *   Other semirings: MM_ERR_UNSUPPORTED ((+, x) has no idempotent (+)).
 * Computed by repeated squaring of X_0 = 1 (+) A: T = ceil(log2(n-1))
 * squarings (0 for n <= 2), each a mm_semiring product with the budget left
 * after the closure's own buffers (so every squaring runs budgeted split-K).
 *   n                  order, n >= 0 (n = 0: nothing is done)
 *   A, C               device pointers, 16-byte aligned; A may equal C
 *   workspace(_bytes)  as in mm_semiring; at least mm_closure_query's
 *                      workspace_min (16 + n*n*elem rounded up to 16 + the
 *                      squaring's minimum), else MM_ERR_WORKSPACE
 *   flags              0: all T squarings, asynchronous and capturable;
 *                      MM_CLOSURE_EARLY_EXIT: after each squaring compare
 *                      X_{t+1} with X_t on the device and stop at the fixed
 *                      point; SYNCHRONISES the stream once per squaring and
 *                      returns MM_ERR_ARG if the stream is being captured
 *   squarings          host pointer or NULL; receives the squarings run
 * Returns MM_OK or a negative mm_status_t.
 */
int mm_closure(int semiring, int64_t n, const void* A, void* C, void* workspace,
               size_t workspace_bytes, int flags, int* squarings, void* stream);

/* Plan of mm_closure for a budget: split_k and tiles of each squaring,
 * levels = T (the number of squarings without early exit), workspace_min /
 * workspace_used of the whole call.  Host-only. */
int mm_closure_query(int semiring, int64_t n, size_t workspace_bytes, mm_plan_t* plan);

/*
 * mm_plan_query -- the plan mm_semiring (levels < 0) or mm_strassen
 * (levels >= 0, variant ignored for the budget) would run for this budget.
 * Host-only; launches nothing.  Returns MM_OK or the status the call
 * itself would return.
 */
int mm_plan_query(int semiring, int levels, int64_t m, int64_t n, int64_t k,
                  size_t workspace_bytes, mm_plan_t* plan);

/*
 * mm_last_device_status -- synchronises `stream` and returns, in *status,
 * the device-side status word written by kernels that can fail on the
 * device: the tensor-core pipelines (FP32 mode, FP64-accuracy mode, the
 * batched kernel) bound every mbarrier wait (2 s) and, on expiry, record
 * MM_ERR_TIMEOUT and stop their CTA cleanly: the CTA lets its own TMA loads
 * and tensor-core products in flight land (bounded waits), frees its TMEM
 * and writes zeros for the output tile it was working on.  After a timeout
 * the outputs of the call are not valid (other tiles and split-K sums may
 * be partial).  The words of all three are read and cleared; MM_OK when
 * none was set.  Returns MM_OK or MM_ERR_CUDA.
 */
int mm_last_device_status(void* stream, int* status);

/*
 * Tracing (diagnostics, no counterpart in the paper).  While enabled, the
 * library brackets every kernel it launches with a pair of CUDA events on
 * the launching stream.  mm_trace_enable(1) clears the record and turns
 * tracing on, mm_trace_enable(0) turns it off (the record is kept).
 * mm_trace_summary synchronises on the recorded events and returns, for one
 * kernel id (0 <= id < mm_trace_kernel_count()), the number of launches and
 * their summed device time in milliseconds.  Returns MM_OK, MM_ERR_ARG or
 * MM_ERR_CUDA.
 */
int mm_trace_enable(int on);
int mm_trace_kernel_count(void);
const char* mm_trace_kernel_name(int kernel_id);
int mm_trace_summary(int kernel_id, int64_t* launches, double* total_ms);

/*
 * mm_set_option -- process-wide tuning switches (not part of the method).
 *   MM_OPT_MINPLUS_PACKED: 1 (default) lets (min,+) products run the exact
 *   packed 2 x 16-bit leaf when a device-side range scan finds every finite
 *   input <= 16383; 0 always runs the 32-bit leaf.  Results are identical.
 *   MM_OPT_MINPLUS_STREAMK: 1 (default) lets an unsplit packed (min,+)
 *   product whose tiles fill fewer than four waves run in the zero-workspace
 *   k-parallel form (TAR-MM, Fig. tar-mm: register tiles merged into C by an
 *   atomic min); 0 disables it.  Results are identical.
 *   Option 3 is retired (it selected a CTA-pair variant of the FP32-mode
 *   leaf that is no longer built) and returns MM_ERR_ARG.
 *   MM_OPT_STRASSEN_TOP_F64: FP32-mode Strassen with levels >= 3 sums its
 *   top-level post-additions wider than FP32.  0 (default): an error-free
 *   double-float sum on the FP32 units (Sum2 of Ogita, Rump and Oishi); 1:
 *   FP64 arithmetic.  Both round the exact sum once to FP32 in all but rare
 *   tie cases; the FP64 units of this GPU are far slower.
 *   MM_OPT_TEST_SKIP_SIGNAL (testing the timeout path): 1, 2 or 3 arms a
 *   one-shot switch for the next launch of the FP32-mode GEMM kernel, the
 *   FP64-accuracy GEMM kernel or the batched FP32 kernel: that launch's first
 *   CTA skips the arrival and loads of its first pipeline stage, so its MMA
 *   wait runs out after 2 s and the call records MM_ERR_TIMEOUT (read with
 *   mm_last_device_status).  No fault is raised; the CTA quiesces and exits.
 *   0 disarms all three.  Needs a device (writes a device word).
 *   MM_OPT_F64ACC_SLICES: digit scheme of the FP64-accuracy semiring.  0
 *   (default) chooses by the Strassen levels above the leaves: six 8-bit
 *   slices (21 bf16 products; scaled rounding to 2^-47) for plain products and
 *   up to two levels, seven 7-bit slices (28 products; 2^-49) for three or
 *   four levels, whose post-additions amplify leaf errors more.  6 or 7
 *   forces a scheme.  Plans (and workspace sizes) follow the setting.
 *   MM_OPT_STRASSEN_FUSED: 1 runs one-level FP32-mode Strassen products
 *   (m, n multiples of 256, k of 64) with the operand sums formed inside the
 *   leaf kernel's staging: converter warps read the source quadrants, add and
 *   split them into the tensor core's operand ring, so the workspace is the
 *   product stack alone (1.75 m n x 4 B instead of 5.25).  Results are
 *   identical; 0 (default) keeps the materialised operand passes, which are
 *   faster on this GPU.
 *   MM_OPT_F32_STREAMK: when the FP32 mode (+,x) product may run the
 *   stream-K form (kernel id 5, Fig. tar-mm: persistent CTAs, partial tiles
 *   in per-CTA slots folded in k order by the last contributor).  1
 *   (default): the planner's rule; 0: never (classic grid or split-K); 2:
 *   whenever the budget holds its slots and the tiles fill one to four
 *   waves, every tile split into equal ranges of (tile, k-block) units; 3:
 *   as 2, but the whole waves of tiles run as plain tiles first and only the
 *   tiles left over are split.  Results agree to rounding (the k order of a
 *   split tile's sum differs).
 *   MM_OPT_F64_STREAMK: the same for the plain FP64 product's stream-K
 *   form (kernel id 6; 32 x 32 register tiles, two slots per CTA): 1
 *   (default) the planner's rule, 0 never, 2 whenever the budget holds its
 *   slots and the 64 x 64 grid fills under four waves of two CTAs per SM.
 * Returns MM_OK, MM_ERR_ARG, or MM_ERR_CUDA (arming the switch failed).
 */
typedef enum {
  MM_OPT_MINPLUS_PACKED = 1,
  MM_OPT_MINPLUS_STREAMK = 2,
  MM_OPT_STRASSEN_TOP_F64 = 4,
  MM_OPT_TEST_SKIP_SIGNAL = 5,
  MM_OPT_F64ACC_SLICES = 6,
  MM_OPT_STRASSEN_FUSED = 7,
  MM_OPT_F32_STREAMK = 8,
  MM_OPT_F64_STREAMK = 9
} mm_option_t;
int mm_set_option(int option, int value);

/* Static string for a status code. */
const char* mm_status_string(int status);

/* Library version (major*10000 + minor*100 + patch). */
int mm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MMSR_H_ */
