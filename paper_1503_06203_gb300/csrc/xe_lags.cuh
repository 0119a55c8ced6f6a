// Per-element integer time shift of a frame before correlation (Sec. IV: a
// kernel that shifts individual elements by integer time steps, to create or
// compensate lags, e.g. for unequal cable lengths).
//
//   out[t][f][i] = in[t - lag_i][f][i]   if 0 <= t - lag_i < T
//                = 0x88 (= 0 + 0i)       otherwise
//
// HBM-bound. A CTA shifts one band's block of 64 elements over kLagTB output
// samples: it stages the source rows those elements need (the time block
// widened by the block's lag span) in shared memory with coalesced 16-byte
// loads, then writes each output row of 64 bytes as 32-bit words. A block
// whose lags span more than kLagHalo samples gathers bytes from global memory
// instead.
#pragma once
#include <cstdint>

namespace xe {

constexpr int kLagTB = 256;    // output samples per CTA
constexpr int kLagHalo = 256;  // largest lag span staged in shared memory
constexpr int kLagThreads = 256;

__global__ void __launch_bounds__(kLagThreads) shift_lags_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                                 int32_t N, int32_t F, int32_t T,
                                                                 const int32_t* __restrict__ lags) {
  __shared__ __align__(16) uint8_t stage[(kLagTB + kLagHalo) * 64];
  __shared__ int32_t lag_s[64];
  __shared__ int32_t span[2];
  const int nblk = (N + 63) / 64;
  const int64_t cta = blockIdx.x;
  const int eb = static_cast<int>(cta % nblk);
  const int64_t rest = cta / nblk;
  const int f = static_cast<int>(rest % F);
  const int64_t t0 = (rest / F) * kLagTB;
  const int i0 = eb * 64;
  const int ne = min(64, N - i0);
  if (threadIdx.x == 0) {
    span[0] = INT32_MAX;
    span[1] = INT32_MIN;
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int32_t l = threadIdx.x < ne ? lags[i0 + threadIdx.x] : 0;
    lag_s[threadIdx.x] = l;
    if (threadIdx.x < ne) {
      atomicMin(&span[0], l);
      atomicMax(&span[1], l);
    }
  }
  __syncthreads();
  const int32_t lmin = span[0], lmax = span[1];
  const int64_t tb = min(static_cast<int64_t>(kLagTB), T - t0);  // output rows of this CTA
  const int64_t row_stride = static_cast<int64_t>(F) * N;
  const bool staged = static_cast<int64_t>(lmax) - lmin <= kLagHalo;
  // source rows t0 - lmax .. t0 + tb - 1 - lmin, clipped to the frame
  const int64_t s_lo = max(int64_t(0), t0 - lmax);
  const int64_t s_hi = min(static_cast<int64_t>(T), t0 + tb - lmin);  // exclusive
  if (staged && s_hi > s_lo) {
    const bool vec = (N % 16 == 0) && ne == 64 && ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
    const int64_t rows = s_hi - s_lo;
    if (vec) {
      for (int64_t k = threadIdx.x; k < rows * 4; k += kLagThreads) {
        const int64_t r = k >> 2;
        const int q = static_cast<int>(k & 3);
        const uint4 v = *reinterpret_cast<const uint4*>(in + (s_lo + r) * row_stride + static_cast<int64_t>(f) * N + i0 + 16 * q);
        *reinterpret_cast<uint4*>(stage + r * 64 + 16 * q) = v;
      }
    } else {
      for (int64_t k = threadIdx.x; k < rows * 64; k += kLagThreads) {
        const int64_t r = k >> 6;
        const int e = static_cast<int>(k & 63);
        stage[r * 64 + e] = e < ne ? in[(s_lo + r) * row_stride + static_cast<int64_t>(f) * N + i0 + e] : 0x88;
      }
    }
  }
  __syncthreads();
  const bool word_ok = (N % 4) == 0;
  // each thread writes 4 consecutive elements of an output row
  for (int k = threadIdx.x; k < tb * 16; k += kLagThreads) {
    const int r = k >> 4;
    const int e0 = (k & 15) * 4;
    if (e0 >= ne) continue;
    const int64_t t = t0 + r;
    uint32_t word = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u;
      uint32_t b = 0x88u;
      if (e < ne) {
        const int64_t src = t - lag_s[e];
        if (src >= 0 && src < T) {
          b = staged ? stage[(src - s_lo) * 64 + e] : in[src * row_stride + static_cast<int64_t>(f) * N + i0 + e];
        }
      }
      word |= b << (8 * u);
    }
    uint8_t* dst = out + t * row_stride + static_cast<int64_t>(f) * N + i0 + e0;
    if (word_ok) {
      *reinterpret_cast<uint32_t*>(dst) = word;
    } else {
      for (int u = 0; u < 4 && e0 + u < ne; ++u) dst[u] = static_cast<uint8_t>(word >> (8 * u));
    }
  }
}

}  // namespace xe
