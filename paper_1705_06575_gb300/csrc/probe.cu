// probe.cu — arithmetic peak probe used as the roofline denominator of the ALU-bound kernels.
// Every thread runs independent FMA chains (8 per thread) in registers; with 4 CTAs of 256
// threads per SM the FP64 pipe (or the FP32 pipe) is saturated. No memory traffic in the loop.
#include <cuda_runtime.h>

#include "sym.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *out, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = (T)(threadIdx.x * 1e-3 + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = fma(acc[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(double *gflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SYM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SYM_ERR_CUDA;
  const int grid = sms * 4, threads = 256;
  const int iters = sizeof(T) == 8 ? 8000 : 160000;
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * grid * threads) != cudaSuccess) return SYM_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_peak<T><<<grid, threads>>>(out, iters / 10, (T)1.0000001, (T)1e-9);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_peak<T><<<grid, threads>>>(out, iters, (T)1.0000001, (T)1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return SYM_ERR_CUDA;
  *gflops = 2.0 * 8.0 * iters * (double)grid * threads / (best * 1e6);
  return SYM_OK;
}

}  // namespace

extern "C" int sym_fma_peak(int32_t precision, double *gflops) {
  if (!gflops) return SYM_ERR_INVALID;
  if (precision == 64) return run<double>(gflops);
  if (precision == 32) return run<float>(gflops);
  return SYM_ERR_INVALID;
}
