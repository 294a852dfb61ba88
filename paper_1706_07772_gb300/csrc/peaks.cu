// FP32 / FP64 fused multiply-add throughput probe (roofline denominators for the
// ALU-bound kernels). Each thread runs 8 independent FMA chains; the grid fills every SM.
#include "reax_internal.cuh"
#include "reaxff_probe.h"

namespace {
template <typename T>
__global__ void k_fma(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)1.2345) out[0] = s;   // keeps the chains live
}

template <typename T> double run(int iters) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return -1.0;
  const int blocks = nsm * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma<T><<<blocks, threads>>>(out, 4, (T)0.999, (T)0.001);   // warm-up
  cudaEventRecord(e0);
  k_fma<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess || ms <= 0) return -1.0;
  const double flops = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads;
  return flops / (ms * 1e-3) / 1e9;
}
}  // namespace

extern "C" double reaxff_probe_fma_gflops(int fp64, int iters) {
  if (iters <= 0) iters = fp64 ? 256 : 4096;
  return fp64 ? run<double>(iters) : run<float>(iters);
}
