/*
 * semlbm_peak.h - FP64 throughput probe of the GPU (measurement utility of
 * the benchmark; no counterpart in the paper, which reports no timings).
 */
#ifndef SEMLBM_PEAK_H
#define SEMLBM_PEAK_H
#ifdef __cplusplus
extern "C" {
#endif

/* Runs 8 independent fused multiply-add chains per thread on 4 CTAs of 256
 * threads per SM for `iters` iterations, three times, and returns the best
 * FP64 rate in TFLOP/s (FMA = 2 flops) and its duration in milliseconds.
 * Allocates and frees its own small output buffer and stream on `device`.
 * Returns 0, -1 (bad argument), -2 (allocation) or -3 (CUDA error). */
int semlbm_fp64_peak(int device, int iters, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif
#endif
