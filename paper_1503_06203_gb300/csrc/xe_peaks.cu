// Integer-pipe microbenchmarks (declared in include/xengine_peaks.h).
#include <cuda_runtime.h>

#include <cstdint>

#include "xengine.h"
#include "xengine_peaks.h"
#include "xe_ptx.cuh"

namespace {

constexpr int kIlp = 8;

template <int kDp4aPerMma, bool kMma>
__global__ void __launch_bounds__(256) peak_kernel(int iters, int32_t* sink) {
  uint32_t a0 = threadIdx.x * 0x01010101u, a1 = a0 ^ 0x5a5a5a5au, a2 = a0 + 3, a3 = a0 - 7;
  uint32_t b0 = blockIdx.x * 0x01030507u, b1 = b0 ^ 0x33u;
  int32_t acc[kIlp][4];
  int32_t d[kIlp];
#pragma unroll
  for (int j = 0; j < kIlp; ++j) {
    acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = j;
    d[j] = j;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kIlp; ++j) {
      if (kMma) xe::mma_s8_16832(acc[j], a0, a1, a2, a3, b0, b1);
#pragma unroll
      for (int x = 0; x < kDp4aPerMma; ++x)
        asm volatile("dp4a.s32.s32 %0, %1, %2, %0;\n" : "+r"(d[(j + x) % kIlp]) : "r"(a0 ^ x), "r"(b0));
    }
  }
  int32_t s = 0;
#pragma unroll
  for (int j = 0; j < kIlp; ++j) s += acc[j][0] + acc[j][1] + acc[j][2] + acc[j][3] + d[j];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int kD, bool kM>
double run_peak(int iters, void* stream, double* mma_ops_s, double* dp4a_ops_s) {
  if (iters < 1) return CORR_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CORR_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CORR_ECUDA;
  const int blocks = sms * 2, threads = 256;
  int32_t* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(int32_t) * blocks * threads) != cudaSuccess) return CORR_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  peak_kernel<kD, kM><<<blocks, threads, 0, st>>>(iters / 8 + 1, sink);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    peak_kernel<kD, kM><<<blocks, threads, 0, st>>>(iters, sink);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return CORR_ECUDA;
  const double warps = static_cast<double>(blocks) * threads / 32.0;
  const double steps = warps * iters * kIlp;
  const double sec = best * 1e-3;
  const double mma = kM ? steps * (2.0 * 16 * 8 * 32) / sec : 0.0;
  const double dp = steps * kD * 32.0 * 8.0 / sec;
  if (mma_ops_s) *mma_ops_s = mma;
  if (dp4a_ops_s) *dp4a_ops_s = dp;
  return mma + dp;
}

}  // namespace

extern "C" {

double xe_peak_imma_s8(int iters, void* stream) { return run_peak<0, true>(iters, stream, nullptr, nullptr); }

double xe_peak_dp4a(int iters, void* stream) { return run_peak<8, false>(iters, stream, nullptr, nullptr); }

double xe_peak_imma_dp4a(int iters, int dp4a_per_mma, void* stream, double* imma_ops, double* dp4a_ops) {
  switch (dp4a_per_mma) {
    case 8: return run_peak<8, true>(iters, stream, imma_ops, dp4a_ops);
    case 16: return run_peak<16, true>(iters, stream, imma_ops, dp4a_ops);
    case 24: return run_peak<24, true>(iters, stream, imma_ops, dp4a_ops);
    case 32: return run_peak<32, true>(iters, stream, imma_ops, dp4a_ops);
    default: return CORR_EINVAL;
  }
}

}  // extern "C"
