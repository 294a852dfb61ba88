/*
 * reaxff_probe.h -- measurement helper exported by libreaxff.so (not part of the
 * ReaxFF method): sustained FP32 / FP64 fused multiply-add throughput of the current
 * device, used as the roofline denominator of arithmetic-bound kernels.
 */
#ifndef REAXFF_PROBE_H
#define REAXFF_PROBE_H
#ifdef __cplusplus
extern "C" {
#endif
/* GFLOP/s (2 flops per FMA) of a grid-filling FMA-chain kernel; fp64 = 1 for double.
 * iters <= 0 picks a default (~0.1-1 s). Returns a negative value on a CUDA error. */
double reaxff_probe_fma_gflops(int fp64, int iters);
#ifdef __cplusplus
}
#endif
#endif
