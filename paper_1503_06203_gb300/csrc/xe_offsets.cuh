// The offset-encoded operand route (Eq. 3; the paper's running-sum and
// pre-seed kernels, restated for the three-product form).
//
// The correlator may multiply the encoded nibbles Xr = xr + 8, Xi = xi + 8
// directly (unsigned operands) and remove the bias afterwards. With, over the
// frame's T samples, E1 = sum Xr_i Xr_j, E2 = sum Xi_i Xi_j,
// E3 = sum (Xr_i + Xi_i)(Xr_j - Xi_j + 15), and the per-element sums
// R_i = sum Xr_i, I_i = sum Xi_i, expanding xr = Xr - 8, xi = Xi - 8 gives
//   Re V_ij = E1 + E2 - 8 (R_i + R_j + I_i + I_j) + 128 T
//   Im V_ij = (E3 - E1 + E2) - 7 R_i - 23 I_i - 8 R_j + 8 I_j
// The kernel folds E1 + E2 and E3 - E1 + E2 exactly as it folds the signed
// products, so pre-seeding the output with the offset terms (the second
// kernel) and letting the correlator add onto them yields V. The first kernel
// computes R and I (Eq. 3's sums over time of the encoded values).
//
// All of it is modular int32 arithmetic: intermediate values may wrap, the
// final sums are exact whenever the true result fits (as in the signed path).
#pragma once
#include <cstdint>

namespace xe {

constexpr int kSumRows = 2048;    // time rows per block of the running-sum kernel
constexpr int kSumThreads = 256;

// sums[f][i] = {sum_t Xr[t][f][i], sum_t Xi[t][f][i]} over rows [0, T), added
// atomically (the caller zeroes sums). Time row t starts row_bytes * t bytes
// after `frame` and holds F bands of Np bytes (Np % 4 == 0, row_bytes % 4 ==
// 0, 4-byte aligned); elements i >= N are skipped. Thread x reads word x of
// every row of its block's time range.
__global__ void __launch_bounds__(kSumThreads) nibble_sums_kernel(const uint8_t* __restrict__ frame, int32_t N,
                                                                  int32_t Np, int32_t F, int32_t T,
                                                                  int64_t row_bytes, int32_t* __restrict__ sums) {
  const int64_t Wr = static_cast<int64_t>(F) * (Np / 4);  // words per row read
  const int64_t W = row_bytes / 4;                        // words between time rows
  const int64_t x = static_cast<int64_t>(blockIdx.x) * kSumThreads + threadIdx.x;
  if (x >= Wr) return;
  const int32_t t0 = static_cast<int32_t>(blockIdx.y) * kSumRows;
  const int32_t t1 = min(T, t0 + kSumRows);
  const uint32_t* col = reinterpret_cast<const uint32_t*>(frame) + x;
  uint32_t sr[4] = {0, 0, 0, 0}, si[4] = {0, 0, 0, 0};
  for (int32_t t = t0; t < t1; t += 16) {
    // byte-lane partial sums of at most 16 rows (16 x 15 = 240 < 256)
    uint32_t ar = 0, ai = 0;
    if (t + 16 <= t1) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const uint32_t w = __ldg(col + static_cast<int64_t>(t + k) * W);
        ar += (w >> 4) & 0x0F0F0F0Fu;
        ai += w & 0x0F0F0F0Fu;
      }
    } else {
      for (int32_t k = t; k < t1; ++k) {
        const uint32_t w = __ldg(col + static_cast<int64_t>(k) * W);
        ar += (w >> 4) & 0x0F0F0F0Fu;
        ai += w & 0x0F0F0F0Fu;
      }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      sr[b] += (ar >> (8 * b)) & 0xFFu;
      si[b] += (ai >> (8 * b)) & 0xFFu;
    }
  }
  const int64_t e0 = 4 * x;  // first byte of the word within the row
  const int32_t f = static_cast<int32_t>(e0 / Np);
  const int32_t i0 = static_cast<int32_t>(e0 % Np);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (i0 + b >= N) break;
    int32_t* s = sums + (static_cast<int64_t>(f) * N + i0 + b) * 2;
    atomicAdd(s, static_cast<int32_t>(sr[b]));
    atomicAdd(s + 1, static_cast<int32_t>(si[b]));
  }
}

// Offset terms of every packed entry (band f, i <= j), stored (add == 0) or
// added (add == 1) into vis [F][N(N+1)/2][2]. One block per (band, row i).
__global__ void offset_seed_kernel(const int32_t* __restrict__ sums, int32_t N, int64_t B, int32_t T, int add,
                                   int32_t* __restrict__ vis) {
  const int32_t i = static_cast<int32_t>(blockIdx.x % N);
  const int32_t f = static_cast<int32_t>(blockIdx.x / N);
  const int32_t* s = sums + static_cast<int64_t>(f) * N * 2;
  const int64_t Ri = s[2 * i], Ii = s[2 * i + 1];
  const int64_t row = static_cast<int64_t>(i) * N - static_cast<int64_t>(i) * (i - 1) / 2;  // p(i, i)
  int32_t* out = vis + (static_cast<int64_t>(f) * B + row) * 2;
  const int64_t re_i = -8 * (Ri + Ii) + 128 * static_cast<int64_t>(T);
  const int64_t im_i = -7 * Ri - 23 * Ii;
  for (int32_t j = i + threadIdx.x; j < N; j += blockDim.x) {
    const int64_t Rj = s[2 * j], Ij = s[2 * j + 1];
    const uint32_t re = static_cast<uint32_t>(re_i - 8 * (Rj + Ij));
    const uint32_t im = static_cast<uint32_t>(im_i - 8 * Rj + 8 * Ij);
    int32_t* o = out + 2 * static_cast<int64_t>(j - i);
    if (add) {
      o[0] = static_cast<int32_t>(static_cast<uint32_t>(o[0]) + re);
      o[1] = static_cast<int32_t>(static_cast<uint32_t>(o[1]) + im);
    } else {
      o[0] = static_cast<int32_t>(re);
      o[1] = static_cast<int32_t>(im);
    }
  }
}

}  // namespace xe
