// les_peak.cu -- a measured FP32 FMA rate: the ALU bound against which the
// issue-bound stencil kernels (the predictors) are judged.  Not part of the
// method; a measurement of the device, like the copy bandwidth and the BF16
// GEMM rate the roofline of the HBM- and tensor-bound kernels uses.
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

__global__ void __launch_bounds__(kThreads) k_fma_rate(float* sink, int trips, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  // a store the compiler cannot prove dead, taken by no thread in practice
  if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int les_measure_fp32_fma(void* stream, int32_t trips, double* tflops, double* ms) {
  if (trips <= 0 || !tflops || !ms) return LES_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate, kThreads, 0)) != cudaSuccess)
    return LES_ERR_CUDA;
  // four waves of resident blocks: the ramp at either end is a small part
  const int blocks = std::max(1, nsm * std::max(1, per_sm) * 4);
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LES_OK;
  if ((e = cudaMallocAsync((void**)&sink, (size_t)blocks * sizeof(float), st)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    rc = LES_ERR_CUDA;
  } else {
    // one warm-up launch, then the timed one
    k_fma_rate<<<blocks, kThreads, 0, st>>>(sink, trips, 0.999f, 1e-3f);
    cudaEventRecord(e0, st);
    k_fma_rate<<<blocks, kThreads, 0, st>>>(sink, trips, 0.999f, 1e-3f);
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
