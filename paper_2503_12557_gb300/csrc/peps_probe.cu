// FMA throughput probe: the measured CUDA-core peak that the contraction kernels' ALU roofline
// is quoted against.  Every thread runs 8 independent dependent-FMA chains in registers (enough
// independent work to cover the FMA latency on every scheduler), the grid fills every SM with
// several resident blocks, and the elapsed time comes from CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "peps_gb300.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, T* sink) {
  T x0 = (T)threadIdx.x, x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == T(-12345.678)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
peps_status run_probe(double* tflops, cudaStream_t s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PEPS_E_CUDA;
  const int blocks = nsm * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 64 : 2048;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return PEPS_E_WORKSPACE;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = T(0.999999), b = T(1e-7);
  k_fma_probe<T><<<blocks, threads, 0, s>>>(iters, a, b, sink);  // warm-up
  cudaEventRecord(e0, s);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) k_fma_probe<T><<<blocks, threads, 0, s>>>(iters, a, b, sink);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess || ms <= 0.f) return PEPS_E_CUDA;
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return PEPS_OK;
}

}  // namespace

extern "C" peps_status peps_probe_fma(int fp64, double* tflops_host, void* stream) {
  if (!tflops_host) return PEPS_E_ARG;
  return fp64 ? run_probe<double>(tflops_host, (cudaStream_t)stream) : run_probe<float>(tflops_host, (cudaStream_t)stream);
}
