// FP64 pipe throughput probe: independent DFMA chains on every SM.  Used by
// the benchmark to measure the ALU roofline denominator on the GPU it runs on
// (B300's FP64 rate is not a published dense figure one can rely on).
#include <cuda_runtime.h>

#include "semlbm_peak.h"

namespace {
__global__ void dfma_chains(double* out, int iters, double b, double c) {
  double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int k = 0; k < iters; ++k) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
}  // namespace

extern "C" int semlbm_fp64_peak(int device, int iters, double* tflops, double* ms_out) {
  if (!tflops || iters <= 0) return -1;
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -3;
  const int blocks = sms * 4, threads = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return -2;
  cudaStream_t st;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_chains<<<blocks, threads, 0, st>>>(out, 200, 1.0000001, 1e-9);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    dfma_chains<<<blocks, threads, 0, st>>>(out, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(out);
  if (err != cudaSuccess) return -3;
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return 0;
}
