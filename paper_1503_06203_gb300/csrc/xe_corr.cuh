// The correlator kernel: TMA-staged 4-bit input, in-register excess-8
// unpack, integer tensor-core Hermitian product, packed upper-triangle
// writer. One CTA computes one 64x64 tile (block row bi <= block column bj)
// of one band over a time range; tiles below the diagonal are never
// scheduled (Sec. II.C, Fig. 1 of the paper).
//
// Arithmetic (Eq. 1): with each sample's parts interleaved along the
// reduction axis, k = 2t + {0: re, 1: im},
//   Re V[i,j] = sum_k A[i,k] * Bre[j,k],  A = Bre = (re, im) per sample
//   Im V[i,j] = sum_k A[i,k] * Bim[j,k],  Bim = (-im, re) per sample
// so both are int8 x int8 -> int32 dot products on the tensor cores.
// Every product is exact; sums are exact in int32 up to the sample cap
// enforced on the host.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "xe_ptx.cuh"

namespace xe {

constexpr int kTile = 64;                 // tile edge (elements)
constexpr int kTC = 64;                   // time samples per pipeline stage
constexpr int kStages = 4;                // TMA ring depth
constexpr int kConsumerWarps = 4;         // 2 x 2 warps, 32 x 32 warp tiles
constexpr int kThreads = (kConsumerWarps + 1) * 32;  // + one TMA producer warp
constexpr int kBoxBytes = kTile * kTC;    // one operand box per stage
constexpr uint32_t kSpinLimit = 1u << 24; // bounded mbarrier polls

// Writer modes
enum : int { kStore = 0, kAdd = 1, kRed = 2 };

// Device fault codes (OR-ed into the error word)
enum : int { kErrTimeoutFull = 1, kErrTimeoutEmpty = 2 };

// One work item: band f, tile (bi, bj), time range [t0, t1).
// Packed as int4 {f, bi | bj << 16, t0, t1}.
struct CorrArgs {
  const int4* items;
  int32_t num_items;
  int32_t N;
  int64_t B;        // N(N+1)/2
  int32_t* vis;     // [F][B][2] accumulators
  int32_t mode;     // kStore / kAdd / kRed
  int32_t* err;     // device error word
};

struct __align__(128) CorrSmem {
  uint8_t box[kStages][2][kBoxBytes];  // [stage][A|B][time][element]
  uint64_t full[kStages];
  uint64_t empty[kStages];
  int abort_flag;
};

// Unpack one packed word (4 time samples of one element, byte u = sample u)
// into the two mma fragment registers of the (re, im) operand.
__device__ __forceinline__ void unpack_reim(uint32_t pk, uint32_t& r0, uint32_t& r1, uint32_t& re_out,
                                            uint32_t& lo_out) {
  const uint32_t hi = (pk >> 4) & 0x0F0F0F0Fu;
  const uint32_t lo = pk & 0x0F0F0F0Fu;
  // nibble - 8 per byte: (v + 0x78) ^ 0x80 has no carry between bytes for v <= 15
  const uint32_t re = (hi + 0x78787878u) ^ 0x80808080u;
  const uint32_t im = (lo + 0x78787878u) ^ 0x80808080u;
  r0 = prmt(re, im, 0x5140);  // re0 im0 re1 im1
  r1 = prmt(re, im, 0x7362);  // re2 im2 re3 im3
  re_out = re;
  lo_out = lo;
}

// The (-im, re) operand from the pieces unpack_reim produced.
__device__ __forceinline__ void unpack_negim_re(uint32_t re, uint32_t lo, uint32_t& r0, uint32_t& r1) {
  // 8 - v per byte: (0x88 - v) ^ 0x80, no borrow between bytes for v <= 15
  const uint32_t nim = (0x88888888u - lo) ^ 0x80808080u;
  r0 = prmt(nim, re, 0x5140);  // -im0 re0 -im1 re1
  r1 = prmt(nim, re, 0x7362);
}

// Gather element e's bytes at time rows row0 + 4u (u = 0..3) of a [time][element]
// box into one word; rows at or past `nvalid` read as 0x88 (= 0 + 0i).
template <bool kMasked>
__device__ __forceinline__ uint32_t gather4(const uint8_t* box, int row0, int e, int nvalid) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(box);
  const int col = e >> 2;
  const uint32_t bsel = static_cast<uint32_t>(e & 3);
  uint32_t v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int row = row0 + 4 * u;
    v[u] = w[row * (kTile / 4) + col];
    if (kMasked) v[u] = row < nvalid ? v[u] : 0x88888888u;
  }
  const uint32_t s = bsel | ((bsel + 4) << 4);
  const uint32_t x01 = prmt(v[0], v[1], s);
  const uint32_t x23 = prmt(v[2], v[3], s);
  return prmt(x01, x23, 0x5410);
}

// One pipeline stage (kTC samples) of a warp's 32x32 piece of the tile.
// skip: 0 = full warp tile, 1 = on the diagonal (skip sub-tiles strictly
// below it), 2 = entirely below the diagonal (no work).
template <bool kMasked>
__device__ __forceinline__ void stage_mma(const uint8_t* boxA, const uint8_t* boxB, int wm, int wn, int lane,
                                          int skip, int nvalid, int32_t (&acc_re)[2][4][4],
                                          int32_t (&acc_im)[2][4][4]) {
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int ks = 0; ks < kTC / 16; ++ks) {
    const int row0 = ks * 16 + q;
    if (kMasked && ks * 16 >= nvalid) break;
    // A operand: rows wm*32 + mi*16 + g (+8)
    uint32_t a[2][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t pk = gather4<kMasked>(boxA, row0, wm * 32 + mi * 16 + g + 8 * h, nvalid);
        uint32_t r0, r1, re, lo;
        unpack_reim(pk, r0, r1, re, lo);
        a[mi][h] = r0;      // a0 / a1: k = 4q..4q+3 of rows g / g+8
        a[mi][2 + h] = r1;  // a2 / a3: k = 4q+16..4q+19
      }
    }
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const uint32_t pk = gather4<kMasked>(boxB, row0, wn * 32 + ni * 8 + g, nvalid);
      uint32_t b0, b1, re, lo, c0, c1;
      unpack_reim(pk, b0, b1, re, lo);
      unpack_negim_re(re, lo, c0, c1);
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        if (skip == 1 && mi == 1 && ni < 2) continue;  // sub-tile strictly below the diagonal
        mma_s8_16832(acc_re[mi][ni], a[mi][0], a[mi][1], a[mi][2], a[mi][3], b0, b1);
        mma_s8_16832(acc_im[mi][ni], a[mi][0], a[mi][1], a[mi][2], a[mi][3], c0, c1);
      }
    }
  }
}

__device__ __forceinline__ void put_vis(int32_t* p, int32_t re, int32_t im, int mode) {
  if (mode == kStore) {
    *reinterpret_cast<int2*>(p) = make_int2(re, im);
  } else if (mode == kAdd) {
    int2 v = *reinterpret_cast<int2*>(p);
    v.x += re;
    v.y += im;
    *reinterpret_cast<int2*>(p) = v;
  } else {
    atomicAdd(p, re);
    atomicAdd(p + 1, im);
  }
}

// Packed-triangle writer: drop entries with i > j (diagonal tiles) or
// outside the N x N matrix; entry (i, j) goes to (f*B + p(i,j))*2.
__device__ __forceinline__ void write_tile(const CorrArgs& a, int f, int i0, int j0, int wm, int wn, int lane,
                                           const int32_t (&acc_re)[2][4][4], const int32_t (&acc_im)[2][4][4]) {
  const int g = lane >> 2, q = lane & 3;
  const int64_t N = a.N;
  int32_t* base = a.vis + static_cast<int64_t>(f) * a.B * 2;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = i0 + wm * 32 + mi * 16 + g + 8 * h;
      if (i >= N) continue;
      const int64_t prow = i * N - i * (i - 1) / 2 - i;  // p(i, j) = prow + j
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int64_t j = j0 + wn * 32 + ni * 8 + 2 * q + c;
          if (j < i || j >= N) continue;
          put_vis(base + (prow + j) * 2, acc_re[mi][ni][2 * h + c], acc_im[mi][ni][2 * h + c], a.mode);
        }
    }
}

__global__ void __launch_bounds__(kThreads) corr_tile_kernel(const __grid_constant__ CUtensorMap tmap, CorrArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  CorrSmem& sm = *reinterpret_cast<CorrSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], kConsumerWarps);
    }
    sm.abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == kConsumerWarps) {
    // ---------------- TMA producer (one thread) ----------------
    if (lane == 0) {
      tma_prefetch_desc(&tmap);
      uint32_t it = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < args.num_items && ok; item += gridDim.x) {
        const int4 w = args.items[item];
        const int f = w.x, bi = w.y & 0xFFFF, bj = w.y >> 16, t0 = w.z, t1 = w.w;
        const bool diag = bi == bj;
        for (int t = t0; t < t1; t += kTC, ++it) {
          const int s = it % kStages;
          if (it >= kStages && !mbar_wait_bounded(&sm.empty[s], ((it / kStages) - 1) & 1, kSpinLimit)) {
            atomicOr(args.err, kErrTimeoutEmpty);
            sm.abort_flag = 1;
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&sm.full[s], diag ? kBoxBytes : 2 * kBoxBytes);
          tma_load_3d(sm.box[s][0], &tmap, &sm.full[s], bi * kTile, f, t);
          if (!diag) tma_load_3d(sm.box[s][1], &tmap, &sm.full[s], bj * kTile, f, t);
        }
      }
      // Drain: never leave with copies in flight (bounded).
      const uint32_t first = it > kStages ? it - kStages : 0;
      for (uint32_t k = first; k < it; ++k) mbar_wait_bounded(&sm.full[k % kStages], (k / kStages) & 1, kSpinLimit);
    }
    return;
  }

  // ---------------- consumers: 4 warps, 2 x 2 warp grid ----------------
  const int wm = warp >> 1, wn = warp & 1;
  int32_t acc_re[2][4][4], acc_im[2][4][4];
  uint32_t it = 0;
  for (int item = blockIdx.x; item < args.num_items; item += gridDim.x) {
    const int4 w = args.items[item];
    const int f = w.x, bi = w.y & 0xFFFF, bj = w.y >> 16, t0 = w.z, t1 = w.w;
    const bool diag = bi == bj;
    const int skip = !diag ? 0 : (wm > wn ? 2 : (wm == wn ? 1 : 0));
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc_re[mi][ni][c] = acc_im[mi][ni][c] = 0;

    bool ok = true;
    for (int t = t0; t < t1; t += kTC, ++it) {
      const int s = it % kStages;
      if (!mbar_wait_bounded(&sm.full[s], (it / kStages) & 1, kSpinLimit)) {
        if (lane == 0) atomicOr(args.err, kErrTimeoutFull);
        ok = false;
        break;
      }
      const uint8_t* bA = sm.box[s][0];
      const uint8_t* bB = diag ? sm.box[s][0] : sm.box[s][1];
      const int nvalid = t1 - t;
      if (skip != 2) {
        if (nvalid >= kTC)
          stage_mma<false>(bA, bB, wm, wn, lane, skip, kTC, acc_re, acc_im);
        else
          stage_mma<true>(bA, bB, wm, wn, lane, skip, nvalid, acc_re, acc_im);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.empty[s]);
    }
    if (!ok) return;
    if (skip != 2) write_tile(args, f, bi * kTile, bj * kTile, wm, wn, lane, acc_re, acc_im);
  }
}

// Copy frames whose rows are not 16-byte aligned into an aligned staging
// buffer [T][F][Np] (Np = N rounded up to 16); padding bytes are 0x88.
__global__ void repack_rows_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, int64_t rows,
                                   int32_t N, int32_t Np) {
  const int64_t total = rows * Np;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = k / Np;
    const int32_t e = static_cast<int32_t>(k - r * Np);
    dst[k] = e < N ? src[r * N + e] : static_cast<uint8_t>(0x88);
  }
}

}  // namespace xe
