// The correlator kernel: TMA-staged 4-bit input, excess-8 unpack into
// K-major int8 planes in shared memory, integer tensor-core Hermitian
// product in the three-product form, packed upper-triangle writer.
//
// A CTA walks a contiguous range of (tile, time-chunk) units of one frame.
// Tiles are 64x64 blocks (block row bi <= block column bj) of one band;
// tiles below the diagonal are never scheduled (Sec. II.C, Fig. 1).
//
// Arithmetic. Eq. 1 gives Re = sum xr_i xr_j + xi_i xi_j and
// Im = sum xi_i xr_j - xr_i xi_j. With three real products per pair,
//   P1 = sum_t xr_i xr_j,   P2 = sum_t xi_i xi_j,
//   Q  = sum_t (xr_i + xi_i)(xr_j - xi_j)  (= P1 - P2 + Im),
// Re = P1 + P2 and Im = Q - P1 + P2. Each is an int8 x int8 -> int32 dot
// product over time (xr, xi in [-8, 7]; xr+xi in [-16, 14]; xr-xi in
// [-15, 15]), so every product is exact. The int32 sums wrap modulo 2^32;
// Re and Im themselves stay inside int32 under the host's sample cap, so
// the wrapped arithmetic gives them exactly.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "xe_ptx.cuh"

namespace xe {

constexpr int kTile = 64;                  // tile edge (elements)
constexpr int kTC = 128;                   // time samples per chunk (pipeline stage)
#ifndef XE_STAGES
#define XE_STAGES 4
#endif
#ifndef XE_PLANE_BUFS
#define XE_PLANE_BUFS 3
#endif
constexpr int kStages = XE_STAGES;         // TMA ring depth
constexpr int kPlaneBufs = XE_PLANE_BUFS;  // unpacked-plane buffers between the unpack and product warps
constexpr int kMmaWarps = 16;              // product warps: 4 x 4 warps of 16 x 16
constexpr int kUnpackThreads = 128;        // unpack warpgroup
constexpr int kThreads = kMmaWarps * 32 + kUnpackThreads;
constexpr int kBoxBytes = kTile * kTC;     // packed box: [time][element] bytes
constexpr int kPlaneBytes = kTile * kTC;   // plane: [element][time] int8, swizzled
constexpr uint32_t kSpinLimit = 1u << 24;  // bounded mbarrier polls

// Device fault codes (OR-ed into the error word)
enum : int { kErrTimeoutFull = 1, kErrTimeoutEmpty = 2 };

// Plane slots. A side (rows i): xr, xi, s = xr + xi. B side (columns j): xr, xi, d = xr - xi.
enum : int { kPxr = 0, kPxi = 1, kPsd = 2 };

// One frame of a batched launch (device memory; the TMA descriptor first, 64-byte aligned).
struct FrameDesc {  // (aligned as its CUtensorMap)
  CUtensorMap map;   // [T][F][Np] bytes of the frame
  int32_t N, T, nch, fresh;
  int64_t B;         // N(N+1)/2
  int32_t* vis;      // [F][B][2] accumulators of the frame's handle
  int32_t t0;        // samples before t0 count as zero (gated segments); 0 for whole frames
  int32_t atomic;    // 1: add atomically (several segments feed the same accumulators)
  // for the device-side work list of batched launches (xe_batch.cuh)
  int32_t F;         // bands
  int32_t nb;        // tile rows: ceil(N / kTile)
  int32_t per;       // chunks per time range of the frame's items
  // gated launches with gate windows by arithmetic (kGateArith): this
  // descriptor is gate `gate` of G; sample t is in it when
  // floor(((t + phase) mod period) * G / period) == gate (period >= kTC)
  int32_t period, phase, G, gate;
};

struct CorrArgs {
  // {band f (| frame << 20 in a batch), bi | bj << 16 (| 1 << 31: hold the sums
  //  for this CTA's next item instead of writing them), first chunk, end chunk};
  //  CTA k takes items k, k + grid, ...
  const int4* items;
  const FrameDesc* frames = nullptr;  // batch: per-frame descriptors; nullptr: the one frame described below
  int32_t nitems;
  int32_t nch;          // chunks per tile: ceil(T / kTC)
  int32_t T;            // samples in the frame
  int32_t N;
  int64_t B;            // N(N+1)/2
  int32_t* vis;         // [F][B][2] accumulators
  int32_t fresh;        // 1: accumulators hold no integration yet (whole tiles store)
  int32_t hybrid;       // split of each chunk's 128 samples between tensor cores and dp4a (kSplit*)
  int32_t* err;         // device error word
};

// What a chunk's consumers need to know (batched and gated launches): the
// TMA issuer writes it beside the chunk's box, the unpack warps pass it on
// beside the planes, so no consumer loads work items or frame descriptors
// from global memory on its critical path.
struct ChunkMeta {
  int32_t f;        // band
  int32_t bij;      // bi | bj << 16
  int32_t lo, hi;   // valid rows of the chunk: [lo, hi) and [lo2, hi2)
  int32_t lo2, hi2;
  int32_t flags;    // kMetaValid | kMetaEnd | write mode << 4 (kMetaEnd unset while a gated group holds)
  int32_t N;
  int64_t B;
  int32_t* vis;
};
enum : int { kMetaValid = 1, kMetaEnd = 2 };

struct __align__(128) CorrSmem {
  uint8_t box[kStages][2][kBoxBytes];          // TMA ring: [stage][A|B][time][element]
  uint8_t plane[kPlaneBufs][2][3][kPlaneBytes];  // [buffer][A|B][slot][element][time]
  uint64_t full[kStages];   // box landed (TMA transaction count)
  uint64_t bempty[kStages]; // box read by all 128 unpack threads
  uint64_t pfull[kPlaneBufs];   // plane buffer written (128 unpack threads)
  uint64_t pempty[kPlaneBufs];  // plane buffer read (16 product warps)
  ChunkMeta meta[kStages];      // per box slot (batched and gated launches)
  ChunkMeta pmeta[kPlaneBufs];  // per plane buffer (batched and gated launches)
};

// Swizzle of a plane (rows of kTC = 128 bytes, 8 chunks of 16): chunk c of
// row e sits at chunk c ^ f(e), f(e) = (e ^ (e >> 3)) & 7. Eight consecutive
// rows then hit eight different 16-byte bank groups (ldmatrix, the dp4a
// operand loads), and so do the unpack stores below (rows 4eg + slot across a
// quarter-warp).
__device__ __forceinline__ uint32_t plane_off(int e, int chunk) {
  const int f = (e ^ (e >> 3)) & 7;
  return static_cast<uint32_t>(e * kTC + ((chunk ^ f) << 4));
}

// ---- unpack: packed box [time][element] -> planes [element][time] --------------
//
// A call handles 4 elements (4eg..4eg+3) x 16 samples (16tg..16tg+15) of one
// block. It loads 16 row words, transposes 4x4 byte blocks with prmt, then
// turns each 4-sample word into the plane bytes with carry-free byte
// arithmetic (v = nibble in [0, 15]):
//   v - 8      = (v + 0x78) ^ 0x80
//   hi + lo - 16 = (hi + lo + 0x70) ^ 0x80      (xr + xi)
//   hi - lo    = ((hi | 0x80) - lo) ^ 0x80       (xr - xi)
// Lanes 16..31 load their rows in the order k ^ 1 and odd element quads
// store their elements in the order slot ^ 1, so that loads and stores are
// free of bank conflicts; runtime prmt selectors undo both reorderings.
//
// kEnc (offset-encoded operands, the Eq. 3 route): the planes keep the
// encoded nibbles, all unsigned: Xr = hi, Xi = lo, Xr + Xi = hi + lo (row
// side) and Xr - Xi + 15 = (hi + 15) - lo (column side), each in [0, 30];
// masked rows are 0x00, which zeroes every product they enter (each product
// has a row-side factor Xr, Xi or Xr + Xi).
template <bool kMasked, bool kEnc>
__device__ __forceinline__ void unpack_unit(const uint8_t* box, uint32_t pl0, uint32_t pl1, uint32_t pl2,
                                            bool side_b, int eg, int tg, int p, int lo, int hi, int lo2 = 0,
                                            int hi2 = 0) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(box);
  uint32_t r[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int t = 16 * tg + (k ^ p);
    r[k] = w[t * (kTile / 4) + eg];
    // rows outside [lo, hi) and [lo2, hi2): no products
    if (kMasked) r[k] = ((t >= lo && t < hi) || (t >= lo2 && t < hi2)) ? r[k] : (kEnc ? 0u : 0x88888888u);
  }
  const int s = eg & 1;
  const uint32_t selA = p ? 0x1504u : 0x5140u;  // interleave two rows, bytes 0-1
  const uint32_t selB = p ? 0x3726u : 0x7362u;  // bytes 2-3
  const uint32_t lo16 = s ? 0x7632u : 0x5410u;  // slots 0 / 2: element (slot ^ s)
  const uint32_t hi16 = s ? 0x5410u : 0x7632u;  // slots 1 / 3
  uint32_t wd[4][4];  // [slot][time quad]
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t x0 = prmt(r[4 * j], r[4 * j + 1], selA);
    const uint32_t x1 = prmt(r[4 * j], r[4 * j + 1], selB);
    const uint32_t y0 = prmt(r[4 * j + 2], r[4 * j + 3], selA);
    const uint32_t y1 = prmt(r[4 * j + 2], r[4 * j + 3], selB);
    wd[0][j] = prmt(x0, y0, lo16);
    wd[1][j] = prmt(x0, y0, hi16);
    wd[2][j] = prmt(x1, y1, lo16);
    wd[3][j] = prmt(x1, y1, hi16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = 4 * eg + (k ^ s);
    uint32_t xr[4], xi[4], sd[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t hi = (wd[k][j] >> 4) & 0x0F0F0F0Fu;
      const uint32_t lo = wd[k][j] & 0x0F0F0F0Fu;
      if (kEnc) {
        xr[j] = hi;
        xi[j] = lo;
        sd[j] = side_b ? ((hi + 0x0F0F0F0Fu) - lo) : (hi + lo);
      } else {
        xr[j] = (hi + 0x78787878u) ^ 0x80808080u;
        xi[j] = (lo + 0x78787878u) ^ 0x80808080u;
        sd[j] = side_b ? (((hi | 0x80808080u) - lo) ^ 0x80808080u) : ((hi + lo + 0x70707070u) ^ 0x80808080u);
      }
    }
    const uint32_t off = plane_off(e, tg);
    if (pl0) sts128(pl0 + off, xr[0], xr[1], xr[2], xr[3]);  // (0 = plane not wanted)
    if (pl1) sts128(pl1 + off, xi[0], xi[1], xi[2], xi[3]);
    sts128(pl2 + off, sd[0], sd[1], sd[2], sd[3]);
  }
}

// ---- product: one 128-sample chunk of a warp's 16 x 16 piece of the tile --------
// acc[0] = P1, acc[1] = P2, acc[2] = Q, each over the piece's two 16 x 8
// sub-tiles (ni = 0, 1). Planes are addressed as shared-memory offsets: A side
// slot p at a_base + p*kPlaneBytes; B side slots 0-1 at b01_base +
// p*kPlaneBytes and slot 2 at b2_base (on a diagonal tile the B side's xr, xi
// planes are the A side's). Sub-tile selection: kSelAll = both sub-tiles,
// kSelN0 / kSelN1 = only sub-tile 0 / 1 (used on diagonal tiles, see the kernel).
enum : int { kSelAll = 0, kSelN0 = 1, kSelN1 = 2, kSelIdle = 3 };

__device__ __forceinline__ constexpr bool sub_on(int sel, int ni) { return sel == kSelAll || ni == sel - 1; }

__device__ __forceinline__ void zero_acc(int32_t (&acc)[3][2][4]) {
#pragma unroll
  for (int pl = 0; pl < 3; ++pl)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[pl][ni][r] = 0;
}

// Tensor cores only, k-steps [0, ksteps) of the chunk.
template <int sel, bool kEnc>
__device__ __forceinline__ void chunk_mma(uint32_t a_base, uint32_t b01_base, uint32_t b2_base, int pr, int pc,
                                          int lane, int ksteps, int32_t (&acc)[3][2][4]) {
  const int arow = pr * 16 + (lane & 15);
  const int brow = pc * 16 + (lane & 7) + ((lane >> 4) << 3);
  const int ahalf = lane >> 4, bhalf = (lane >> 3) & 1;
#pragma unroll
  for (int ks = 0; ks < kTC / 32; ++ks) {
    if (ks >= ksteps) break;
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
      const uint32_t pa = a_base + pl * kPlaneBytes;
      const uint32_t pb = pl < 2 ? b01_base + pl * kPlaneBytes : b2_base;
      uint32_t a[4], b[2][2];
      ldsm_x4(pa + plane_off(arow, 2 * ks + ahalf), a[0], a[1], a[2], a[3]);
      ldsm_x4(pb + plane_off(brow, 2 * ks + bhalf), b[0][0], b[0][1], b[1][0], b[1][1]);
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
        if (sub_on(sel, ni)) mma_8bit<kEnc>(acc[pl][ni], a[0], a[1], a[2], a[3], b[ni][0], b[ni][1]);
    }
  }
}

// ---- product, hybrid: tensor cores and the integer ALU side by side -----------
// The tensor pipe and the dp4a pipe of an SM sub-partition run concurrently
// and at about the same rate on this GPU. A warp runs the three products for
// the chunk's first kMmaK k-steps (32 samples each) on the tensor cores and
// for the remaining samples with dp4a (4 samples per instruction),
// accumulating both into the same registers: thread (g, q) owns, per
// sub-tile ni, the entries (row g + 8h, column ni*8 + 2q + c) of the MMA
// accumulator layout, so its dp4a work is those entries' dot products. The
// dp4a work comes in blocks of 8 samples of one plane; the MMAs are spread
// evenly over the blocks.
// The dp4a block order: block k of a chunk with kMmaK tensor-core k-steps
// works on plane (e & 3), samples group (e >> 2), e = 5 bits of the table.
// The order keeps each block off the accumulators of the MMAs issued in it
// (and mostly in the block before), whose results are still in flight, and
// changes plane between consecutive blocks where it can (dp4a_order.py
// beside this file states the criterion and regenerates the table).
__device__ __forceinline__ constexpr uint32_t dp4a_block(int mk, int k) {
  return static_cast<uint32_t>(((k < 12 ? (mk == 3 ? 0x6b1c94114501841ull : 0x8258e4288628022ull)
                                        : 0xef338f569a8da4dull) >> (5 * (k % 12))) & 31u);
}

template <int sel, int kMmaK, bool kEnc>
__device__ __forceinline__ void chunk_hybrid(uint32_t a_base, uint32_t b01_base, uint32_t b2_base, int pr, int pc,
                                             int lane, int32_t (&acc)[3][2][4]) {
  constexpr int kNi0 = sel == kSelN1 ? 1 : 0;  // first column sub-tile
  constexpr int kNi = sel == kSelAll ? 2 : 1;   // column sub-tiles
  constexpr int kMmas = kMmaK * 6;              // (k-step, plane, sub-tile)
  constexpr int kBlocks = (kTC - 32 * kMmaK) / 8 * 3;  // (8 samples, plane)
  const int g = lane >> 2, q = lane & 3;
  const int arow = pr * 16 + (lane & 15);
  const int brow = pc * 16 + (lane & 7) + ((lane >> 4) << 3);
  const int ahalf = lane >> 4, bhalf = (lane >> 3) & 1;
  uint32_t fa[4], fb[2][2];
#pragma unroll
  for (int k = 0; k < kBlocks; ++k) {
    // ---- tensor cores: this block's share of the MMAs ----
#pragma unroll
    for (int m = k * kMmas / kBlocks; m < (k + 1) * kMmas / kBlocks; ++m) {
      const int mks = m / 6, mpl = (m / 2) % 3, mni = m & 1;
      if (mni == 0) {
        const uint32_t pa = a_base + mpl * kPlaneBytes;
        const uint32_t pb = mpl < 2 ? b01_base + mpl * kPlaneBytes : b2_base;
        ldsm_x4(pa + plane_off(arow, 2 * mks + ahalf), fa[0], fa[1], fa[2], fa[3]);
        ldsm_x4(pb + plane_off(brow, 2 * mks + bhalf), fb[0][0], fb[0][1], fb[1][0], fb[1][1]);
      }
      if (sub_on(sel, mni)) mma_8bit<kEnc>(acc[mpl][mni], fa[0], fa[1], fa[2], fa[3], fb[mni][0], fb[mni][1]);
    }
    // ---- integer ALU: samples 32*kMmaK + 8*grp .. +7 of plane dpl ----
    const uint32_t ord = dp4a_block(kMmaK, k);
    const int grp = static_cast<int>(ord >> 2), dpl = static_cast<int>(ord & 3);
    const int s0 = 32 * kMmaK + 8 * grp, chunk = s0 >> 4, inner = s0 & 15;
    const uint32_t pa = a_base + dpl * kPlaneBytes;
    const uint32_t pb = dpl < 2 ? b01_base + dpl * kPlaneBytes : b2_base;
    uint32_t av[2][2], bv[2][2][2];  // [h][word], [n][c][word]
#pragma unroll
    for (int h = 0; h < 2; ++h) lds64(pa + plane_off(pr * 16 + g + 8 * h, chunk) + inner, av[h][0], av[h][1]);
#pragma unroll
    for (int n = 0; n < kNi; ++n)
#pragma unroll
      for (int c = 0; c < 2; ++c)
        lds64(pb + plane_off(pc * 16 + (kNi0 + n) * 8 + 2 * q + c, chunk) + inner, bv[n][c][0], bv[n][c][1]);
#pragma unroll
    for (int wd = 0; wd < 2; ++wd)
#pragma unroll
      for (int n = 0; n < kNi; ++n)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int c = 0; c < 2; ++c) dp4a_8bit<kEnc>(acc[dpl][kNi0 + n][2 * h + c], av[h][wd], bv[n][c][wd]);
  }
}

// ---- writer: tile piece -> packed upper triangle ---------------------------------
// mode 0: store (whole tile, fresh integration); 1: add (whole tile onto
// resident accumulators); 2: atomic add (part of the time range of a tile
// whose other parts other CTAs add). Entries with i > j, outside the N x N
// matrix, or in sub-tiles the warp did not compute are dropped; entry (i, j)
// of band f lives at (f*B + p(i,j))*2, p(i,j) = i*N - i(i-1)/2 + j - i.
__device__ __forceinline__ void write_piece(int N, int64_t B, int32_t* vis, int f, int i0, int j0, int pr, int pc,
                                            int lane, int mode, int sel, int32_t (&acc)[3][2][4]) {
  // fold in place: Re = P1 + P2 into acc[0], Im = Q - P1 + P2 into acc[2] (modulo 2^32;
  // exact for in-range Re, Im)
#pragma unroll
  for (int ni = 0; ni < 2; ++ni)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t p1 = static_cast<uint32_t>(acc[0][ni][r]), p2 = static_cast<uint32_t>(acc[1][ni][r]);
      acc[0][ni][r] = static_cast<int32_t>(p1 + p2);
      acc[2][ni][r] = static_cast<int32_t>(static_cast<uint32_t>(acc[2][ni][r]) - p1 + p2);
    }
  const int g = lane >> 2, q = lane & 3;
  int32_t* base = vis + static_cast<int64_t>(f) * B * 2;
  const int jw = j0 + pc * 16 + 2 * q;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = i0 + pr * 16 + g + 8 * h;
    if (i >= N) continue;
    const int64_t ii = i;
    int32_t* rowp = base + (ii * N - ii * (ii - 1) / 2 - ii) * 2;  // entry (i, j) at rowp + 2j
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int j = jw + ni * 8 + c;
        if (j < i || j >= N || !sub_on(sel, ni)) continue;
        const int32_t re = acc[0][ni][2 * h + c], im = acc[2][ni][2 * h + c];
        int32_t* dst = rowp + 2 * j;
        if (mode == 0) {
          *reinterpret_cast<int2*>(dst) = make_int2(re, im);
        } else if (mode == 1) {
          int2 v = *reinterpret_cast<int2*>(dst);
          v.x = static_cast<int32_t>(static_cast<uint32_t>(v.x) + static_cast<uint32_t>(re));
          v.y = static_cast<int32_t>(static_cast<uint32_t>(v.y) + static_cast<uint32_t>(im));
          *reinterpret_cast<int2*>(dst) = v;
        } else {
          atomicAdd(dst, re);
          atomicAdd(dst + 1, im);
        }
      }
  }
}

// ---- the kernel ------------------------------------------------------------------
// Work items are (band, tile, chunk range); CTA k takes items k, k + grid,
// k + 2 grid, ... in list order. The list is band-major, so the CTAs that run
// at the same time work on the tiles of one band over the same time chunks
// and share that band's input in L2.
//
// Warp roles. Warps 0-15 (warpgroups 0-3): product and writer, 4 x 4 warps
// of 16 x 16 pieces (three int32 accumulator sets, 24 registers a thread);
// four of them share each SM sub-partition. Warps 16-19 (warpgroup 4):
// unpack; lane 0 of warp 16 also issues the TMA loads. One CTA per SM.

// ---- gate arithmetic (kGateArith launches) --------------------------------------
// Gate g of G holds the positions [a, b) of a period P, a = ceil(g P / G),
// b = ceil((g + 1) P / G): floor(pos G / P) == g exactly there. Sample t has
// position (t + phase) mod P. Chunks are kTC samples; P >= kTC, so a chunk's
// positions wrap at most once and the gate meets a chunk in at most two runs.
// 32-bit unsigned arithmetic is exact: sample indices are below 2^31 and the
// host takes this route only for P <= 2^29, so sample + phase and
// sample + 2P stay below 2^32.

// The first sample >= s whose position lies in [a, b) (a < b <= P).
__device__ __forceinline__ uint32_t gate_next_sample(uint32_t s, uint32_t P, uint32_t phase, uint32_t a, uint32_t b) {
  const uint32_t pos = (s + phase) % P;
  if (pos >= a && pos < b) return s;
  return s + (pos < a ? a - pos : P - pos + a);
}

// The first chunk >= c holding a sample t < T of the gate; nch if none.
__device__ __forceinline__ int32_t gate_chunk(int32_t c, int32_t nch, int32_t T, int32_t P, int32_t phase, int32_t a,
                                              int32_t b) {
  if (c >= nch || a >= b) return nch;
  const uint32_t s = gate_next_sample(static_cast<uint32_t>(c) * kTC, static_cast<uint32_t>(P),
                                      static_cast<uint32_t>(phase), static_cast<uint32_t>(a), static_cast<uint32_t>(b));
  return s >= static_cast<uint32_t>(T) ? nch : static_cast<int32_t>(s / kTC);
}

// The gate's rows of chunk c (relative to its first sample), as two windows
// [lo, hi) and [lo2, hi2): the run before the chunk's positions wrap past P
// and the run after it; both clipped to the frame's T samples.
__device__ __forceinline__ void gate_windows(int32_t c, int32_t T, int32_t P, int32_t phase, int32_t a, int32_t b,
                                             ChunkMeta& m) {
  const uint32_t s0 = static_cast<uint32_t>(c) * kTC;
  const int32_t p0 = static_cast<int32_t>((s0 + static_cast<uint32_t>(phase)) % static_cast<uint32_t>(P));
  const int32_t tmax = min(kTC, T - static_cast<int32_t>(s0));
  m.lo = max(0, a - p0);
  m.hi = min(tmax, b - p0);
  m.lo2 = max(0, a - p0 + P);
  m.hi2 = min(tmax, b - p0 + P);
}

// Walks (item, chunk) pairs of this CTA in order. T and nch are the current
// item's frame's (from its descriptor in a batch, else from args); the writer
// reads the rest when it needs it. kArith: the item is one (band, tile, gate)
// over the frame, and its chunks are those that hold samples of the gate
// (the current one c, the next one cn).
template <bool kFrames, bool kHold, bool kArith = false>
struct Walk {
  int item, c, f, bi, bj, c1, frame, T, nch, T0;
  const int4* items;
  const FrameDesc* frames;
  int nitems, stride;
  // batched and gated launches (the TMA issuer's walk): the current item's
  // write mode and hold bit, the current frame's output
  int mode, hold, fN, fresh, atomic;
  int64_t fB;
  int32_t* fvis;
  // kArith: the gate of the current descriptor, and the item's next chunk
  int gP, gphase, ga, gb, cn;
  __device__ __forceinline__ void load() {
    for (; item < nitems; item += stride) {
      const int4 w = items[item];
      bi = w.y & 0xFFFF;
      c = w.z;
      c1 = w.w;
      if (kFrames) {
        bj = kHold ? (w.y >> 16) & 0x7FFF : w.y >> 16;  // (bit 31: hold, read by the writer)
        f = w.x & 0xFFFFF;
        const int fr = w.x >> 20;
        if (fr != frame) {
          frame = fr;
          T = frames[fr].T;
          nch = frames[fr].nch;
          T0 = frames[fr].t0;
          fN = frames[fr].N;
          fB = frames[fr].B;
          fvis = frames[fr].vis;
          fresh = frames[fr].fresh;
          atomic = frames[fr].atomic;
          if (kArith) {
            gP = frames[fr].period;
            gphase = frames[fr].phase;
            const int64_t G = frames[fr].G, g = frames[fr].gate;
            ga = static_cast<int>((g * gP + G - 1) / G);
            gb = static_cast<int>(((g + 1) * gP + G - 1) / G);
          }
        }
        hold = kHold && w.y < 0;
        // a gated group covers all of its gate's samples in the frame, like a whole tile
        const bool whole = kHold || kArith || (w.z == 0 && w.w == nch);
        mode = atomic ? 2 : (whole ? (fresh ? 0 : 1) : 2);
        if (kArith) {
          c = gate_chunk(c, c1, T, gP, gphase, ga, gb);
          if (c >= c1) continue;  // the gate has no samples here: nothing to do or write
          cn = gate_chunk(c + 1, c1, T, gP, gphase, ga, gb);
        }
      } else {
        bj = w.y >> 16;
        f = w.x;
      }
      return;
    }
  }
  __device__ __forceinline__ void start(const CorrArgs& a) {
    items = a.items;
    frames = a.frames;
    nitems = a.nitems;
    stride = gridDim.x;
    item = blockIdx.x;
    frame = -1;
    T = a.T;
    nch = a.nch;
    T0 = 0;
    load();
  }
  __device__ __forceinline__ bool valid() const { return item < nitems; }
  // the current chunk is the item's last
  __device__ __forceinline__ bool last() const { return kArith ? cn >= c1 : c + 1 == c1; }
  __device__ __forceinline__ void next() {
    if (kArith) {
      if (cn < c1) {
        c = cn;
        cn = gate_chunk(c + 1, c1, T, gP, gphase, ga, gb);
        return;
      }
    } else if (++c != c1) {
      return;
    }
    item += stride;
    load();
  }
  __device__ __forceinline__ const CUtensorMap* map(const CUtensorMap* single) const {
    return kFrames ? &frames[frame].map : single;
  }
};

// Off-diagonal tile: warp w takes piece (w / 4, w % 4); warps w, w+4, w+8,
// w+12 share SM sub-partition w % 4.
// Diagonal tile: the 10 pieces on or above the diagonal hold its 20 needed
// 16 x 8 sub-tiles. Eight pieces go whole to warps 0-7; pieces (2,2) and
// (3,3) are split into single sub-tiles for warps 8-11; warps 12-15 idle.
// Each sub-partition then runs 5 sub-tiles (8 on a full tile).
// (2 bits per warp: piece row, piece column, selection)
constexpr uint32_t kDiagR = 0xfa9050u, kDiagC = 0xfaedd8u, kDiagSel = 0xff990000u;

// Split of a chunk's 128 samples between the tensor cores (k-steps of 32)
// and dp4a (the rest), chosen per launch: the same split for every chunk, or
// two splits alternating between consecutive chunks of a CTA, which gives the
// finer average shares in between. Shares 5 and 4 apply to off-diagonal
// tiles; diagonal tiles keep 6. Every split gives the same exact sums.
// Tensor-core k-steps per pair of chunks:
enum : int {
  kSplitMma = 0,   // 8 of 8: tensor cores only
  kSplit6 = 1,     // 6 of 8 (96 / 32 per chunk)
  kSplit7 = 2,     // 7 of 8 (alternating 128 / 0 and 96 / 32)
  kSplit5 = 3,     // 5 of 8 (alternating 64 / 64 and 96 / 32)
  kSplit4 = 4      // 4 of 8 (64 / 64 per chunk)
};

// Tensor-core k-steps of a chunk under split `hybrid`; odd = the CTA's chunk count is odd.
__device__ __forceinline__ int mma_ksteps(int hybrid, int odd) {
  switch (hybrid) {
    case kSplit6: return 3;
    case kSplit7: return odd ? 4 : 3;
    case kSplit5: return odd ? 2 : 3;
    case kSplit4: return 2;
    default: return 4;
  }
}

template <int sel, bool kEnc>
__device__ __forceinline__ void chunk_split(int mk, uint32_t a_base, uint32_t b01, uint32_t b2, int pr, int pc,
                                            int lane, int32_t (&acc)[3][2][4]) {
  if (mk == 3)
    chunk_hybrid<sel, 3, kEnc>(a_base, b01, b2, pr, pc, lane, acc);
  else if (mk == 2)
    chunk_hybrid<sel, 2, kEnc>(a_base, b01, b2, pr, pc, lane, acc);
  else
    chunk_mma<sel, kEnc>(a_base, b01, b2, pr, pc, lane, kTC / 32, acc);
}

// One product warp's share of one chunk in plane buffer `buf`; nvalid = valid
// rows of the chunk; it = the CTA's chunk count. kSplitT < 0: the split is
// args.hybrid, kSplitMma or kSplit6, chosen at run time; else the split is
// kSplitT, fixed at compile time (one instantiation per split keeps the hot
// loop to two code paths and within the register budget). Returns the warp's
// piece (pr, pc) and selection.
template <bool kEnc, int kSplitT>
__device__ __forceinline__ void product_chunk(CorrSmem& sm, int buf, int warp, int lane, bool diag, int nvalid,
                                              int hybrid, uint32_t it, int& pr, int& pc, int& sel,
                                              int32_t (&acc)[3][2][4]) {
  pr = diag ? static_cast<int>((kDiagR >> (2 * warp)) & 3) : warp >> 2;
  pc = diag ? static_cast<int>((kDiagC >> (2 * warp)) & 3) : warp & 3;
  sel = diag ? static_cast<int>((kDiagSel >> (2 * warp)) & 3) : kSelAll;
  if (sel == kSelIdle) return;
  const uint32_t a_base = smem_u32(sm.plane[buf][0][0]);
  const uint32_t b_side = smem_u32(sm.plane[buf][1][0]);
  const uint32_t b01 = diag ? a_base : b_side, b2 = b_side + kPsd * kPlaneBytes;
  const int ksteps = nvalid >= kTC ? kTC / 32 : (nvalid + 31) / 32;
  // shares below 6 apply to off-diagonal tiles: a diagonal tile, with a quarter of its product warps
  // idle and a quarter on single sub-tiles, runs best at 6 (measured)
  const int split0 = kSplitT < 0 ? (hybrid == kSplitMma ? kSplitMma : kSplit6) : kSplitT;
  const int split = diag && (split0 == kSplit5 || split0 == kSplit4) ? kSplit6 : split0;
  if (split != kSplitMma && ksteps == kTC / 32) {  // (a ragged last chunk takes the tensor-core path)
    const int mk = mma_ksteps(split, static_cast<int>(it & 1));
    if (sel == kSelAll)
      chunk_split<kSelAll, kEnc>(mk, a_base, b01, b2, pr, pc, lane, acc);
    else if (sel == kSelN0)
      chunk_split<kSelN0, kEnc>(mk, a_base, b01, b2, pr, pc, lane, acc);
    else
      chunk_split<kSelN1, kEnc>(mk, a_base, b01, b2, pr, pc, lane, acc);
  } else if (sel == kSelAll) {
    chunk_mma<kSelAll, kEnc>(a_base, b01, b2, pr, pc, lane, ksteps, acc);
  } else if (sel == kSelN0) {
    chunk_mma<kSelN0, kEnc>(a_base, b01, b2, pr, pc, lane, ksteps, acc);
  } else {
    chunk_mma<kSelN1, kEnc>(a_base, b01, b2, pr, pc, lane, ksteps, acc);
  }
}

// kMode: kSingle = one frame (args), kBatch = per-frame descriptors, kGated =
// descriptors plus hold bits (a gated (tile, gate) group's segments),
// kGateArith = one descriptor per gate, each item a (band, tile, gate) whose
// chunks and rows follow from the gate arithmetic above.
enum : int { kSingle = 0, kBatch = 1, kGated = 2, kGateArith = 3 };

template <int kMode, bool kEnc, int kSplitT = -1>
__global__ void __launch_bounds__(kThreads, 1) corr_tile_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                CorrArgs args) {
  constexpr bool kFrames = kMode != kSingle;
  constexpr bool kHold = kMode == kGated;
  constexpr bool kArith = kMode == kGateArith;
  extern __shared__ uint8_t smem_raw[];
  CorrSmem& sm = *reinterpret_cast<CorrSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                              ~static_cast<uintptr_t>(127));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.bempty[s], kUnpackThreads);
    }
    for (int b = 0; b < kPlaneBufs; ++b) {
      mbar_init(&sm.pfull[b], kUnpackThreads);
      mbar_init(&sm.pempty[b], kMmaWarps);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (warp >= kMmaWarps) {
    // ================= unpack warps (+ TMA issue) =================
    const int uw = warp - kMmaWarps;  // 0..3
    const bool producer = uw == 0 && lane == 0;
    const int eg = lane & 15, p = lane >> 4, tg = 2 * uw + p;  // samples 16tg..16tg+15 of each chunk
    Walk<kFrames, kHold, kArith> ld;  // the TMA issuer walks the same units, kStages ahead
    ld.start(args);
    uint32_t issued = 0;
    const CUtensorMap* fenced = nullptr;
    auto issue = [&](void) {
      const int s = issued % kStages;
      const bool diag = ld.bi == ld.bj;
      const CUtensorMap* map = ld.map(&tmap);
      if (kFrames && map != fenced) {  // a frame descriptor copied in before the launch
        tensormap_acquire(map);
        fenced = map;
      }
      if constexpr (kFrames) {  // the chunk's consumers read this instead of the work list
        ChunkMeta& m = sm.meta[s];
        m.f = ld.f;
        m.bij = ld.bi | (ld.bj << 16);
        if (kArith) {
          gate_windows(ld.c, ld.T, ld.gP, ld.gphase, ld.ga, ld.gb, m);
        } else {
          m.lo = ld.T0 - ld.c * kTC;
          m.hi = ld.T - ld.c * kTC;
          m.lo2 = m.hi2 = 0;
        }
        m.flags = kMetaValid | ((ld.last() && !ld.hold) ? kMetaEnd : 0) | (ld.mode << 4);
        m.N = ld.fN;
        m.B = ld.fB;
        m.vis = ld.fvis;
      }
      // (the arrive releases the stores above to the slot's waiters)
      mbar_arrive_expect_tx(&sm.full[s], diag ? kBoxBytes : 2 * kBoxBytes);
      tma_load_3d(sm.box[s][0], map, &sm.full[s], ld.bi * kTile, ld.f, ld.c * kTC);
      if (!diag) tma_load_3d(sm.box[s][1], map, &sm.full[s], ld.bj * kTile, ld.f, ld.c * kTC);
      ++issued;
      ld.next();
    };
    // batched and gated launches end the chunk stream with an entry without
    // kMetaValid (no copy; a plain arrive completes its phase)
    bool ended = false;
    auto issue_end = [&](void) {
      const int s = issued % kStages;
      sm.meta[s].flags = 0;
      mbar_arrive(&sm.full[s]);
      ++issued;
      ended = true;
    };
    if (producer) {
      if (!kFrames) tma_prefetch_desc(&tmap);
      for (int k = 0; k < kStages; ++k) {
        if (ld.valid()) {
          issue();
        } else {
          if (kFrames) issue_end();
          break;
        }
      }
    }
    uint32_t it = 0;
    bool ok = true;
    if constexpr (kFrames) {
      for (;; ++it) {
        const int s = it % kStages, buf = it % kPlaneBufs;
        if ((it >= kPlaneBufs && !mbar_wait_bounded(&sm.pempty[buf], ((it / kPlaneBufs) - 1) & 1, kSpinLimit)) ||
            !mbar_wait_bounded(&sm.full[s], (it / kStages) & 1, kSpinLimit)) {
          if (lane == 0) atomicOr(args.err, kErrTimeoutFull);
          ok = false;
          break;
        }
        const ChunkMeta& m = sm.meta[s];
        const int flags = m.flags, bij = m.bij, lo = m.lo, hi = m.hi, lo2 = m.lo2, hi2 = m.hi2;
        if (threadIdx.x == kMmaWarps * 32) sm.pmeta[buf] = m;  // passed on with the planes
        if (!(flags & kMetaValid)) {
          mbar_arrive(&sm.pfull[buf]);
          break;
        }
        const bool diag = (bij & 0xFFFF) == (bij >> 16);
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
          const uint8_t* box = sm.box[s][diag ? 0 : j];
          uint32_t pl0 = smem_u32(sm.plane[buf][j][kPxr]);
          uint32_t pl1 = smem_u32(sm.plane[buf][j][kPxi]);
          const uint32_t pl2 = smem_u32(sm.plane[buf][j][kPsd]);
          if (diag && j == 1) pl0 = pl1 = 0;
          if (lo <= 0 && hi >= kTC)
            unpack_unit<false, kEnc>(box, pl0, pl1, pl2, j == 1, eg, tg, p, 0, kTC);
          else
            unpack_unit<true, kEnc>(box, pl0, pl1, pl2, j == 1, eg, tg, p, lo, hi, lo2, hi2);
        }
        mbar_arrive(&sm.pfull[buf]);
        mbar_arrive(&sm.bempty[s]);
        if (producer && !ended) {  // refill slot s once every unpack thread is done with it
          if (!mbar_wait_bounded(&sm.bempty[s], (it / kStages) & 1, kSpinLimit)) {
            atomicOr(args.err, kErrTimeoutEmpty);
            ok = false;
            break;
          }
          if (ld.valid())
            issue();
          else
            issue_end();
        }
      }
    } else {
    Walk<kFrames, kHold> x;
    for (x.start(args); x.valid(); x.next(), ++it) {
      const bool diag = x.bi == x.bj;
      const int s = it % kStages, buf = it % kPlaneBufs;
      // the plane buffer must be free (its previous chunk's products issued) and the box landed
      if ((it >= kPlaneBufs && !mbar_wait_bounded(&sm.pempty[buf], ((it / kPlaneBufs) - 1) & 1, kSpinLimit)) ||
          !mbar_wait_bounded(&sm.full[s], (it / kStages) & 1, kSpinLimit)) {
        if (lane == 0) atomicOr(args.err, kErrTimeoutFull);
        ok = false;
        break;
      }
      const int lo = x.T0 - x.c * kTC, hi = x.T - x.c * kTC;  // valid rows of this chunk
      // two units per thread: the row side (j = 0) and the column side (j = 1); a
      // diagonal tile's column side is only its xr - xi plane, from the same box
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        const uint8_t* box = sm.box[s][diag ? 0 : j];
        uint32_t pl0 = smem_u32(sm.plane[buf][j][kPxr]);
        uint32_t pl1 = smem_u32(sm.plane[buf][j][kPxi]);
        const uint32_t pl2 = smem_u32(sm.plane[buf][j][kPsd]);
        if (diag && j == 1) pl0 = pl1 = 0;
        if (lo <= 0 && hi >= kTC)
          unpack_unit<false, kEnc>(box, pl0, pl1, pl2, j == 1, eg, tg, p, 0, kTC);
        else
          unpack_unit<true, kEnc>(box, pl0, pl1, pl2, j == 1, eg, tg, p, lo, hi);
      }
      mbar_arrive(&sm.pfull[buf]);   // release this thread's plane stores
      mbar_arrive(&sm.bempty[s]);    // this thread is done reading box slot s
      if (producer && ld.valid()) {  // refill slot s once every unpack thread is done with it
        if (!mbar_wait_bounded(&sm.bempty[s], (it / kStages) & 1, kSpinLimit)) {
          atomicOr(args.err, kErrTimeoutEmpty);
          ok = false;
          break;
        }
        issue();
      }
    }
    }
    if (producer) {
      // Never leave with copies in flight: a bulk copy writes this CTA's shared
      // memory, and the CTA lives until this thread returns, so waiting here
      // for each armed barrier keeps every copy inside the CTA's lifetime. A
      // copy in flight completes on its own; the wait is bounded all the same
      // (also after a fault, when it may be the stuck barrier itself).
      const uint32_t first = issued > kStages ? issued - kStages : 0;
      for (uint32_t k = first; k < issued; ++k)
        mbar_wait_bounded(&sm.full[k % kStages], (k / kStages) & 1, kSpinLimit);
    }
    (void)ok;
    return;
  }

  // ================= product warps =================
  int32_t acc[3][2][4];
  zero_acc(acc);
  uint32_t it = 0;
  if constexpr (kFrames) {
    for (;; ++it) {
      const int buf = it % kPlaneBufs;
      if (!mbar_wait_bounded(&sm.pfull[buf], (it / kPlaneBufs) & 1, kSpinLimit)) {
        if (lane == 0) atomicOr(args.err, kErrTimeoutFull);
        return;
      }
      const ChunkMeta& m = sm.pmeta[buf];
      const int flags = m.flags;
      if (!(flags & kMetaValid)) return;  // end of this CTA's chunks
      const int bi = m.bij & 0xFFFF, bj = m.bij >> 16;
      // rows past the last valid one are masked to zero: their k-steps can be skipped
      const int nvalid = m.hi2 > m.lo2 ? max(m.hi, m.hi2) : m.hi;
      int pr, pc, sel;
      product_chunk<kEnc, kSplitT>(sm, buf, warp, lane, bi == bj, nvalid, args.hybrid, it, pr, pc, sel, acc);
      // the writer's fields, read before the buffer (and its metadata) is released
      const int f = m.f, N = m.N;
      const int64_t B = m.B;
      int32_t* const vis = m.vis;
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.pempty[buf]);
      if (flags & kMetaEnd) {  // end of the item (a gated group's last segment): write it
        if (sel != kSelIdle) write_piece(N, B, vis, f, bi * kTile, bj * kTile, pr, pc, lane, (flags >> 4) & 3, sel, acc);
        zero_acc(acc);
      }
    }
  } else {
  Walk<kFrames, kHold> x;
  for (x.start(args); x.valid(); ++it) {
    const bool diag = x.bi == x.bj;
    const int buf = it % kPlaneBufs;
    if (!mbar_wait_bounded(&sm.pfull[buf], (it / kPlaneBufs) & 1, kSpinLimit)) {
      if (lane == 0) atomicOr(args.err, kErrTimeoutFull);
      return;
    }
    int pr, pc, sel;
    product_chunk<kEnc, kSplitT>(sm, buf, warp, lane, diag, x.T - x.c * kTC, args.hybrid, it, pr, pc, sel, acc);
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.pempty[buf]);
    if (x.c + 1 == x.c1) {  // end of the item: write it
      const int4 w = args.items[x.item];
      const bool whole = w.z == 0 && w.w == x.nch;
      const int mode = whole ? (args.fresh ? 0 : 1) : 2;
      if (sel != kSelIdle)
        write_piece(args.N, args.B, args.vis, x.f, x.bi * kTile, x.bj * kTile, pr, pc, lane, mode, sel, acc);
      zero_acc(acc);
    }
    x.next();
  }
  }
}

// Copy the bands [f0, f0 + F) of a frame [T][F_in][N] whose rows are not
// 16-byte aligned into an aligned staging buffer [T][F][Np] (Np = N rounded
// up to 16); padding bytes are 0x88. rows = T * F.
__global__ void repack_rows_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, int64_t rows,
                                   int32_t N, int32_t Np, int32_t F, int32_t F_in, int32_t f0) {
  const int64_t total = rows * Np;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = k / Np;
    const int32_t e = static_cast<int32_t>(k - r * Np);
    const int64_t t = r / F, f = r - t * F;
    dst[k] = e < N ? src[(t * F_in + f0 + f) * N + e] : static_cast<uint8_t>(0x88);
  }
}

}  // namespace xe
