// Work list of a batched launch, built on the device from per-frame
// descriptors (Sec. II.C: the tiles of every frame and band are independent
// units of work; Sec. I: bands are independent).
//
// Frame k contributes ranges_k x F_k x tiles_k items: its time axis is cut
// into ranges_k ranges of per_k chunks, and each range covers every tile of
// every band (band-major, each band's upper triangle row by row). The host
// orders the frames by the chunks per item, longest first, and passes the
// prefix sums of their item counts in that order; item i of the list so
// formed goes to CTA slot i mod grid in snake order (rows of `grid` items
// run alternately forward and backward, a ragged last row forward), so each
// CTA's share of the longest items is nearly equal.
#pragma once
#include <cstdint>

#include "xe_corr.cuh"

namespace xe {

// Row-major upper-triangle tile u of an nb x nb block grid -> (bi, bj), bi <= bj.
__device__ __forceinline__ void triangle_tile(int64_t u, int32_t nb, int32_t& bi, int32_t& bj) {
  // row r starts at s(r) = r nb - r (r - 1) / 2; solve s(r) <= u for the largest r
  const double b = 2.0 * nb + 1.0;
  int64_t r = static_cast<int64_t>((b - sqrt(b * b - 8.0 * static_cast<double>(u))) * 0.5);
  r = r < 0 ? 0 : (r >= nb ? nb - 1 : r);
  auto start = [nb](int64_t q) { return q * nb - q * (q - 1) / 2; };
  while (r + 1 < nb && start(r + 1) <= u) ++r;
  while (r > 0 && start(r) > u) --r;
  bi = static_cast<int32_t>(r);
  bj = static_cast<int32_t>(r + (u - start(r)));
}

// first[s] = items before the s-th frame in cost order (first[n] = nitems),
// order[s] = that frame's index. Items: {band | frame << 20, bi | bj << 16, c0, c1}.
__global__ void batch_plan_kernel(const FrameDesc* __restrict__ frames, const int64_t* __restrict__ first,
                                  const int32_t* __restrict__ order, int32_t nframes, int4* __restrict__ items,
                                  int64_t nitems, int64_t grid) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < nitems;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t lo = 0, hi = nframes - 1;  // the s with first[s] <= i < first[s + 1]
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (first[mid] <= i)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int32_t k = order[lo];
    const FrameDesc& d = frames[k];
    const int64_t tb = static_cast<int64_t>(d.nb) * (d.nb + 1) / 2;  // tiles per band
    const int64_t local = i - first[lo];
    const int64_t per_range = tb * d.F;
    const int64_t r = local / per_range, rem = local - r * per_range;
    const int32_t f = static_cast<int32_t>(rem / tb);
    int32_t bi, bj;
    triangle_tile(rem - static_cast<int64_t>(f) * tb, d.nb, bi, bj);
    const int32_t c0 = static_cast<int32_t>(r * d.per);
    const int32_t c1 = static_cast<int32_t>(min(static_cast<int64_t>(d.nch), (r + 1) * d.per));
    const int64_t row = i / grid, c = i - row * grid;
    const bool partial = (row + 1) * grid > nitems;
    const int64_t col = ((row & 1) && !partial) ? grid - 1 - c : c;
    items[row * grid + col] = make_int4(f | (k << 20), bi | (bj << 16), c0, c1);
  }
}

}  // namespace xe
