// FP64 FMA throughput probe: the roofline denominator for the FP64-bound sieve kernels.
// Independent FMA chains (4 per thread) over a grid of 8 warps per SM; the count of FMAs is exact.
#include <cuda_runtime.h>

#include "../../include/lhaf.h"

namespace {

__global__ void __launch_bounds__(256) fp64_fma_probe(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
      x0 = fma(x0, a, b);
      x1 = fma(x1, a, b);
      x2 = fma(x2, a, b);
      x3 = fma(x3, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

}  // namespace

extern "C" lhaf_status lhaf_fp64_probe(int device, double* gflops) {
  if (!gflops) return LHAF_EINVAL;
  *gflops = 0.0;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return LHAF_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms, threads = 256;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * threads) != cudaSuccess) {
    cudaSetDevice(prev);
    return LHAF_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_fma_probe<<<blocks, threads>>>(d, 50, 0.999, 1e-4);  // warm-up
  const int iters = 4000;
  cudaEventRecord(e0);
  fp64_fma_probe<<<blocks, threads>>>(d, iters, 0.999, 1e-4);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  cudaSetDevice(prev);
  if (err != cudaSuccess || ms <= 0.f) return LHAF_ECUDA;
  const double fmas = (double)blocks * threads * iters * 16.0 * 4.0;
  *gflops = 2.0 * fmas / (ms * 1e-3) / 1e9;
  return LHAF_OK;
}
