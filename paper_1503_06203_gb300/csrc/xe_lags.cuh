// Per-element integer time shift of a frame before correlation (Sec. IV: a
// kernel that shifts individual elements by integer time steps, to create or
// compensate lags, e.g. for unequal cable lengths).
//
//   out[t][f][i] = in[t - lag_i][f][i]   if 0 <= t - lag_i < T
//                = 0x88 (= 0 + 0i)       otherwise
//
// HBM-bound: every output byte is written once and every input byte read at
// most once. A thread writes 4 consecutive elements of one (time, band) row
// as one 32-bit word (warps write 128 contiguous bytes); it gathers the four
// source bytes, which are contiguous when the lags are equal.
#pragma once
#include <cstdint>

namespace xe {

__global__ void shift_lags_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int32_t N, int32_t F,
                                  int32_t T, const int32_t* __restrict__ lags) {
  const int64_t rows = static_cast<int64_t>(T) * F;  // (t, f) rows of N bytes
  const int32_t quads = (N + 3) / 4;
  const int64_t total = rows * quads;
  const bool word_ok = (N % 4) == 0;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = k / quads;
    const int32_t i0 = static_cast<int32_t>(k - row * quads) * 4;
    const int64_t t = row / F;
    const int64_t f = row - t * F;
    uint32_t word = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int32_t i = i0 + u;
      uint32_t b = 0x88u;
      if (i < N) {
        const int64_t src = t - lags[i];
        if (src >= 0 && src < T) b = in[(src * F + f) * N + i];
      }
      word |= b << (8 * u);
    }
    uint8_t* dst = out + row * N + i0;
    if (word_ok) {
      *reinterpret_cast<uint32_t*>(dst) = word;
    } else {
      for (int u = 0; u < 4 && i0 + u < N; ++u) dst[u] = static_cast<uint8_t>(word >> (8 * u));
    }
  }
}

}  // namespace xe
