/*
 * fsi_peaks.h - throughput probes for the rooflines of the solver's kernels
 * (libfsi_peaks.so).  Not part of the solve: the benchmark measures the FP64 and
 * FP32 fused-multiply-add rates of the GPU it runs on, so that kernels bound by an
 * arithmetic pipe (the FP64 outer SpMV, the FP32 learned-stage MLP) are reported
 * against a measured peak rather than a nominal one.  The paper has no
 * counterpart (its solver ran on CPUs).
 */
#ifndef FSI_PEAKS_H_
#define FSI_PEAKS_H_

#ifdef __cplusplus
extern "C" {
#endif

/*
 * fsi_probe_fma_rate - fused multiply-add throughput of the current CUDA device.
 *   bits          64 (FP64 FMA) or 32 (FP32 FMA)
 *   iters         loop trips per thread (>= 1); each trip issues 8 independent FMAs
 *                 per thread on a grid of 8 CTAs of 256 threads per SM
 *   reps          timed launches (>= 1), after one untimed warm-up launch
 *   fma_per_s     receives FMAs per second (best of the timed launches)
 *   best_ms       nullable: receives the best launch time in milliseconds
 * Allocates and frees one small device buffer; runs on a stream of its own and
 * waits for it.  Returns 0, or -1 on bad arguments, -3 on a CUDA error.
 */
int fsi_probe_fma_rate(int bits, int iters, int reps, double* fma_per_s, double* best_ms);

#ifdef __cplusplus
}
#endif

#endif /* FSI_PEAKS_H_ */
