/*
 * casim_peaks.h — instruction-throughput probes of the GPU the step runs on.
 *
 * Measurement support for the rooflines of the step kernels (the mixed form
 * is bound by memory latency and its conversions, the FP64 form by the FP64
 * pipe, the rate code by the special-function unit); not part of the step.
 * Built as its own library, libcasim_peaks.so.
 *
 * casim_peak_rate times, with CUDA events on `stream`, three launches of a
 * kernel of (SM count x 8) blocks x 256 threads in which every thread runs 8
 * independent chains of `iters` dependent operations of one kind, after one
 * untimed launch, and writes the operations per second to *rate.  A fused
 * multiply-add counts as one operation (two FLOPs); a packed bf16x2
 * instruction as two.  The chains are kept on a
 * bounded orbit (x -> f(x) with a constant offset where needed; the offset's
 * addition runs on another pipe and is not counted), and each thread writes
 * its result so that no chain is removed by the compiler.
 *
 * Returns 0; CASIM_PEAK_ERR_ARG (-1) for an unknown kind, iters < 1 or a null
 * rate; CASIM_PEAK_ERR_CUDA (-2) if a CUDA call failed.  Synchronises the
 * stream.
 */
#ifndef CASIM_PEAKS_H
#define CASIM_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

#define CASIM_PEAK_FFMA 0   /* fma.rn.f32: x = x * a + b */
#define CASIM_PEAK_DFMA 1   /* fma.rn.f64: x = x * a + b */
#define CASIM_PEAK_EX2 2    /* ex2.approx.ftz.f32 (special-function unit): x = 2^-x */
#define CASIM_PEAK_LG2 3    /* lg2.approx.ftz.f32: x = log2(x) + 2 */
#define CASIM_PEAK_RCP 4    /* rcp.approx.ftz.f32: x = 1/x + 1 */
#define CASIM_PEAK_TANH 5   /* tanh.approx.f32: x = tanh(x) + 0.5 */
#define CASIM_PEAK_TANH2 6  /* tanh.approx.bf16x2 on packed pairs: two operations per instruction */
#define CASIM_PEAK_NKINDS 7

#define CASIM_PEAK_ERR_ARG (-1)
#define CASIM_PEAK_ERR_CUDA (-2)

int casim_peak_rate(int kind, long long iters, void *stream, double *rate);

#ifdef __cplusplus
}
#endif
#endif
