/*
 * xengine_peaks.h -- microbenchmarks that measure the integer roofline
 * denominators of the X-engine on the current GPU (the paper quotes its own
 * GPU's nominal peak, Sec. IV footnote; here the peaks are measured).
 *
 * Each function runs a register-resident kernel over every SM, times it
 * with CUDA events on `stream` (a cudaStream_t as void*, NULL = default),
 * and returns operations per second counting a multiply-add as 2
 * operations, or a negative CORR_* code on failure. `iters` scales the run
 * time (about 1 ms per 1000 iterations on GB300); it must be >= 1.
 * The work buffers are allocated and freed inside each call.
 */
#ifndef XENGINE_PEAKS_H
#define XENGINE_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* mma.sync m16n8k32 s8 x s8 -> s32 (the integer tensor-core form of sm_103a). */
double xe_peak_imma_s8(int iters, void* stream);

/* dp4a (4-way int8 dot product + int32 add) on the integer ALU pipe. */
double xe_peak_dp4a(int iters, void* stream);

/*
 * Both at once, in the same warps: `dp4a_per_mma` dp4a instructions per
 * mma.sync. Returns the combined operation rate; *imma_ops and *dp4a_ops
 * (may be NULL) receive each pipe's share.
 */
double xe_peak_imma_dp4a(int iters, int dp4a_per_mma, void* stream, double* imma_ops, double* dp4a_ops);

#ifdef __cplusplus
}
#endif

#endif /* XENGINE_PEAKS_H */
