// Arithmetic-pipe peak microbenchmark.
//
// The find and eval kernels are bound by the FP64 (plain path) or FP32
// (mixed path) FMA pipes, not by HBM or tensor cores, and no vendor figure is
// used for those pipes: this kernel measures them.  Each thread runs 8
// independent FMA chains; the grid covers every SM several times, so the
// pipe rather than latency is the limit.  Result in GFLOP/s (FMA = 2 flop).
#include <cuda_runtime.h>
#include <stdint.h>

#include "fp_common.cuh"

namespace {

template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ out, int iters, T a, T b) {
  T acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run_peak(int iters, int blocks_per_sm, double* gflops, cudaStream_t st) {
  int dev = 0, nsm = 0;
  FP_CUDA_TRY(cudaGetDevice(&dev));
  FP_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  constexpr int threads = 256, chains = 8;
  const int blocks = nsm * blocks_per_sm;
  T* out = nullptr;
  FP_CUDA_TRY(cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T, chains><<<blocks, threads, 0, st>>>(out, iters / 8 + 1, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0, st);
  k_fma_chains<T, chains><<<blocks, threads, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, st);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return FP_ELAUNCH;
  const double flop = 2.0 * 4.0 * chains * (double)iters * threads * (double)blocks;
  *gflops = flop / (ms * 1e-3) / 1e9;
  return FP_OK;
}

}  // namespace

extern "C" int fp_alu_peak(int which, int iters, double* gflops, void* stream) {
  if (!gflops || iters <= 0) return FP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (which == 0) return run_peak<double>(iters, 8, gflops, st);
  if (which == 1) return run_peak<float>(iters, 8, gflops, st);
  return FP_EINVAL;
}
