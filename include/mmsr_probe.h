/*
 * mmsr_probe.h -- throughput probes that measure the roofline denominators
 * of the CUDA-core kernels on the running GPU (no counterpart in the paper;
 * the paper's base-kernel runs on a CPU).
 *
 * mm_probe_peak runs one synthetic kernel that keeps every SM busy with
 * independent chains of a single instruction and reports the achieved rate.
 *   kind 0: fused add-min on uint32 (__viaddmin_u32), 2 ops per lane-instruction
 *   kind 1: fused add-min on packed 2 x uint16 (__viaddmin_u16x2), 4 ops
 *   kind 2: FP64 fused multiply-add, 2 FLOPs
 *   kind 3: FP32 fused multiply-add, 2 FLOPs
 *   kind 4: tcgen05 bf16 products 128 x 64 x 16 issued by one thread per SM
 *           from operands resident in shared memory (the FP64-accuracy
 *           leaf's product shape and order, no TMA traffic), 2 FLOPs per MAC
 *   kind 5: the same with 128 x 128 x 16 products
 * iters: inner-loop trip count per thread (work scales linearly; for kinds
 * 4 and 5, rounds of 56 products).
 * stream: cudaStream_t as void*.  The call synchronises the stream.
 * Outputs: *ops_per_s (ops as counted above per second), *ms (device time,
 * CUDA events on `stream`).  Returns MM_OK, MM_ERR_ARG or MM_ERR_CUDA.
 */
#ifndef MMSR_PROBE_H_
#define MMSR_PROBE_H_

#ifdef __cplusplus
extern "C" {
#endif

int mm_probe_peak(int kind, int iters, void* stream, double* ops_per_s, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* MMSR_PROBE_H_ */
