/*
 * mirres_peaks.h -- measured denominators for the roofline fractions of the path's kernels.
 *
 * The path tracer is not a dense contraction: its traversal stages are bound by dependent
 * loads that hit in L2, its shading stage by FP32 arithmetic. The two peaks those stages are
 * compared against are measured here, on the device that runs them, rather than taken from a
 * data sheet: the FP32 FMA rate of the SMs (the non-tensor pipe) and the bandwidth of loads
 * that hit in L2. The paper has no counterpart (it reports no throughput figures).
 *
 * Both calls run on the calling thread's current device, allocate and free their own buffers,
 * synchronise the device and time with CUDA events after a warm-up launch; results are
 * written to the out pointers (host memory). Returns 0 on success, a cudaError_t otherwise.
 */
#ifndef MIRRES_PEAKS_H
#define MIRRES_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* FP32 fused multiply-add throughput: every resident thread runs `iters` rounds of 16
 * independent FMA chains (enough independent work to fill the pipe); FLOP/s = 2 * FMAs / time.
 * out_flops: FLOP/s; out_ms: device time of the timed launch. */
int mirres_peak_fp32(int32_t iters, double* out_flops, double* out_ms);

/* L2 load bandwidth: `passes` passes of 16-byte loads (all SMs, coalesced) over a buffer of
 * `bytes` bytes that stays resident in L2 (a few tens of MB on a 129 MB L2), after a pass that
 * brings it in. out_bytes_per_s: bytes loaded / time; out_ms: device time of the timed launch. */
int mirres_peak_l2(uint64_t bytes, int32_t passes, double* out_bytes_per_s, double* out_ms);

#ifdef __cplusplus
}
#endif
#endif /* MIRRES_PEAKS_H */
