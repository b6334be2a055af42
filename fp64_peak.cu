// FMA-throughput probe of bench.py (measurement utility, not part of the library): the
// denominator of the roofline of the FP64 kernels, whose bound on this GPU is the FP64 pipe.
//
// Every thread runs 8 independent FMA chains x <- x*a + b for a fixed number of iterations
// (no data dependence between chains, so the pipe, not latency, limits the rate); the grid is
// 8 blocks of 256 threads per SM. Rate = 2 flops x 8 chains x iterations x threads / best time
// of 5 launches (CUDA events). The loop count is fixed: the kernel always ends.
#include <cuda_runtime.h>

namespace {

template <class T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <class T>
int measure(int iters, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -3;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -3;
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T><<<blocks, threads>>>(out, 100, (T)0.999, (T)0.001);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return -3;
  *tflops = 2.0 * 8 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return 0;
}

}  // namespace

// FMA throughput of the current device in TFLOP/s; fp64 != 0 for double, else float.
// Returns 0, or -2 (allocation failed) / -3 (CUDA error).
extern "C" int ovl_probe_fma_tflops(int fp64, double* tflops) {
  if (!tflops) return -1;
  return fp64 ? measure<double>(4000, tflops) : measure<float>(40000, tflops);
}
