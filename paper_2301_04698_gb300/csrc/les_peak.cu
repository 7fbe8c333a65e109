// les_peak.cu -- measured FP32 and FP64 FMA rates: the ALU bounds against
// which the issue-bound stencil kernels (the predictors) and the FP64
// configurations are set.  Not part of the method; a measurement of the
// device, like the copy bandwidth and the BF16 GEMM rate the roofline of the
// HBM- and tensor-bound kernels uses.
//
// Every thread runs kChains independent FMA chains (x = x * a + b), kUnroll
// steps per loop trip, so the FMA pipes never wait on a dependency; the
// blocks fill every SM.  The rate counts 2 flops per FMA.
#include <algorithm>
#include <string>

#include "les_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(T* sink, int trips, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * T(1e-3);
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  // a store the compiler cannot prove dead, taken by no thread in practice
  if (s == T(-1.2345e30)) sink[blockIdx.x] = s;
}

template <typename T>
int measure_fma(cudaStream_t st, int trips, double* tflops, double* ms) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T>, kThreads, 0)) != cudaSuccess)
    return LES_ERR_CUDA;
  // four waves of resident blocks: the ramp at either end is a small part
  const int blocks = std::max(1, nsm * std::max(1, per_sm) * 4);
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LES_OK;
  if ((e = cudaMallocAsync((void**)&sink, (size_t)blocks * sizeof(T), st)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    rc = LES_ERR_CUDA;
  } else {
    // one warm-up launch, then the timed one
    k_fma_rate<T><<<blocks, kThreads, 0, st>>>(sink, trips, T(0.999), T(1e-3));
    cudaEventRecord(e0, st);
    k_fma_rate<T><<<blocks, kThreads, 0, st>>>(sink, trips, T(0.999), T(1e-3));
    cudaEventRecord(e1, st);
    float t = 0.f;
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) {
      rc = LES_ERR_CUDA;
    } else {
      const double fmas = (double)blocks * kThreads * trips * kUnroll * kChains;
      *ms = t;
      *tflops = 2.0 * fmas / (t * 1e-3) / 1e12;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFreeAsync(sink, st);
  return rc;
}

}  // namespace

extern "C" int les_measure_fma(void* stream, int32_t precision, int32_t trips, double* tflops, double* ms) {
  if (trips <= 0 || !tflops || !ms || (precision != 32 && precision != 64)) return LES_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == 64 ? measure_fma<double>(st, trips, tflops, ms) : measure_fma<float>(st, trips, tflops, ms);
}
