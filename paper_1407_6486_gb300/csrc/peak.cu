// peak.cu -- measured FP64 FMA throughput of the device, the denominator of the roofline
// of the library's FP64-bound kernels (the end-of-iteration pass of the fine level).
//
// Every thread runs kChains independent FMA chains x <- x * a + b (a slightly below 1,
// so every chain converges to b / (1 - a) and stays normal); the grid holds 8 CTAs of
// 256 threads per SM, enough warps to cover the FMA latency.  FLOPs per launch =
// 2 * kChains * kUnroll * iters * threads; the rate is the best of several launches
// timed with CUDA events on the caller's stream.
#include <cstdio>

#include "pfasst_mg.h"
#include "pmg_internal.cuh"

namespace {

constexpr int kChains = 8, kUnroll = 16, kThreads = 256, kCtasPerSm = 8;

__global__ void __launch_bounds__(kThreads) fp64_fma_probe_kernel(double *out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (threadIdx.x + 1) * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) out[blockIdx.x] = s;  // never true (every chain stays positive): keeps the chains live
}

}  // namespace

extern "C" int pfasst_mg_fp64_peak(void *stream, int launches, double *gflops) {
  if (!gflops || launches < 1 || launches > 100) return PMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return PMG_ERR_CUDA;
  }
  const int blocks = sms * kCtasPerSm, iters = 1000;
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kThreads;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return PMG_ERR_CUDA;
  }
  double best = 0.0;
  int rc = PMG_OK;
  for (int k = 0; k <= launches && rc == PMG_OK; ++k) {  // k = 0: warm-up
    float ms = 0.f;
    if (cudaEventRecord(e0, st) != cudaSuccess) { rc = PMG_ERR_CUDA; break; }
    fp64_fma_probe_kernel<<<blocks, kThreads, 0, st>>>(nullptr, iters, 0.99999999, 1e-8);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = PMG_ERR_CUDA;
      break;
    }
    if (k > 0 && ms > 0.f) {
      const double r = flops / (ms * 1e-3) / 1e9;
      if (r > best) best = r;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PMG_OK) {
    cudaGetLastError();
    return rc;
  }
  *gflops = best;
  return PMG_OK;
}
