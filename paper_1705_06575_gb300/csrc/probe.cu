// probe.cu — arithmetic peak probe used as the roofline denominator of the ALU-bound kernels.
// Every thread runs independent FMA chains (8 per thread) in registers; with 4 CTAs of 256
// threads per SM the FP64 pipe (or the FP32 pipe) is saturated. No memory traffic in the loop.
// Also the layout check of the tensor-core update (one tile product through tcgen05).
#include <cuda_runtime.h>

#include <vector>

#include "sym.h"
#include "tc.cuh"

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

// D (128 x 64) = A (128 x 32) B (64 x 32)^T through the operand layout, descriptors and MMA of
// the FP32 tensor-core update; *failed = 1 when the completion wait runs out.
__global__ void __launch_bounds__(128) k_tc_probe(const float *A, const float *B, float *D, uint32_t lbo, uint32_t sbo,
                                                  int *failed) {
  namespace tc = sym::tc;
  __shared__ __align__(128) uint8_t As[128 * tc::KC * 4];
  __shared__ __align__(128) uint8_t Bs[64 * tc::KC * 4];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 128 * tc::KC; i += 128)
    *reinterpret_cast<float *>(As + tc::off(i / tc::KC, i % tc::KC)) = A[i];
  for (int i = tid; i < 64 * tc::KC; i += 128)
    *reinterpret_cast<float *>(Bs + tc::off(i / tc::KC, i % tc::KC)) = B[i];
  tc::fence_smem_to_async();
  if (warp == 0) tc::tmem_alloc(&tmem_slot, 64);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs);
    for (int ks = 0; ks < tc::KC / 8; ++ks)
      tc::mma_tf32(tmem, tc::desc(a0 + ks * tc::KSTEP, lbo, sbo), tc::desc(b0 + ks * tc::KSTEP, lbo, sbo),
                   tc::idesc_tf32<128, 64>(), ks > 0);
    tc::commit(&mbar);
  }
  const bool ok = tc::mbar_wait(&mbar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) *failed = 1;
  } else {
    tc::fence_after_sync();
    float v[32];
    const int r = 32 * warp + lane;
    for (int h = 0; h < 2; ++h) {
      tc::ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * h, v);
      for (int j = 0; j < 32; ++j) D[r * 64 + 32 * h + j] = v[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, 64);
  }
}

}  // namespace

extern "C" int sym_tc_probe(const float *A, const float *B, float *D, uint32_t lbo, uint32_t sbo) {
  if (!A || !B || !D) return SYM_ERR_INVALID;
  if (!((lbo == 128 && sbo == 1024) || (lbo == 1024 && sbo == 128))) return SYM_ERR_INVALID;
  const size_t na = 128 * sym::tc::KC, nbv = 64 * sym::tc::KC, nd = 128 * 64;
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int *dflag = nullptr;
  int rc = SYM_OK;
  if (cudaMalloc(&dA, na * 4) != cudaSuccess || cudaMalloc(&dB, nbv * 4) != cudaSuccess ||
      cudaMalloc(&dD, nd * 4) != cudaSuccess || cudaMalloc(&dflag, sizeof(int)) != cudaSuccess)
    rc = SYM_ERR_OOM;
  int flag = 0;
  if (rc == SYM_OK) {
    if (cudaMemcpy(dA, A, na * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dB, B, nbv * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(dD, 0, nd * 4) != cudaSuccess || cudaMemset(dflag, 0, sizeof(int)) != cudaSuccess)
      rc = SYM_ERR_CUDA;
  }
  if (rc == SYM_OK) {
    k_tc_probe<<<1, 128>>>(dA, dB, dD, lbo, sbo, dflag);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(D, dD, nd * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = SYM_ERR_CUDA;
    else if (flag)
      rc = SYM_ERR_TIMEOUT;
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dflag);
  return rc;
}

extern "C" int sym_fma_peak(int32_t precision, double *gflops) {
  if (!gflops) return SYM_ERR_INVALID;
  if (precision == 64) return run<double>(gflops);
  if (precision == 32) return run<float>(gflops);
  return SYM_ERR_INVALID;
}
