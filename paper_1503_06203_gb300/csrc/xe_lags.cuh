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

namespace xe {

// ---- streaming form: a TMA ring along time ----------------------------------
// A CTA owns one band's block of 64 elements over a segment of `tseg` output
// samples and walks it in blocks of 128 samples. Source rows arrive by TMA in
// boxes of 64 elements x 128 samples (box b = rows 128b .. 128b+127) into a
// ring of kLagRing boxes, where row s sits at ((s mod 1024) * 64). Each source
// row is read from HBM once per segment. The block at t0 needs the boxes of
// rows t0 - lmax .. t0 + 127 - lmin (lmin, lmax: the block's lag range), at
// most 6 when lmax - lmin <= kLagSpanRing; box b + kLagRing replaces box b
// once no thread reads it. Boxes are issued in order from the CTA's first
// box, so box b is use (b - first) / kLagRing of its barrier.
//
// Shared-memory banks: a warp covers 8 rows x 4 quads of 16 bytes; lane
// (quad q, row r) visits its quad's words starting at word r / 2, so that at
// every step the 32 lanes read 32 different banks (rows r, r + 1 share the
// word but their source rows differ by one, i.e. by 16 banks).
constexpr int kLagRing = 8;
constexpr int kLagRingRows = kLagRing * 128;  // 1024: row s lives at (s & 1023) * 64
constexpr int kLagSpanRing = 512;
constexpr int kLagStreamThreads = 256;
constexpr int kLagRingBytes = kLagRingRows * 64;  // 64 KiB
constexpr int kLagStreamSmem = kLagRingBytes + 128;  // dynamic shared memory (aligned to 128 inside)

struct LagStreamArgs {
  const uint8_t* in;  // the frame the map describes (for blocks with a wide lag range)
  uint8_t* out;
  const int32_t* lags;
  int32_t N, F, T;
  int32_t tseg;   // output samples per CTA (a multiple of 128)
  int32_t* err;   // set to 1 when a wait ran out (host-mapped)
};

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

// One lane's 16 output bytes of row t (see the bank note above): visiting
// step w reads word (w + rot) & 3 of the lane's quad; kInterior = every
// source row of the block lies inside the frame.
template <bool kInterior>
__device__ __forceinline__ uint4 lag_unit(const uint8_t* ring, int32_t t, const uint32_t (&c)[16],
                                          const int32_t (&lg)[16], int rot, int32_t T) {
  const uint32_t tb = static_cast<uint32_t>(t & (kLagRingRows - 1)) * 64u;
  uint32_t wv[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int k = 4 * w + b;
      uint32_t v = ring[(tb + c[k]) & (kLagRingBytes - 1u)];
      if (!kInterior) {
        const int64_t src = static_cast<int64_t>(t) - lg[k];
        if (src < 0 || src >= T) v = 0x88u;
      }
      word |= v << (8 * b);
    }
    wv[w] = word;
  }
  // undo the rotation: output word j was read at step (j - rot) & 3
  uint4 o;
  o.x = rot == 0 ? wv[0] : rot == 1 ? wv[3] : rot == 2 ? wv[2] : wv[1];
  o.y = rot == 0 ? wv[1] : rot == 1 ? wv[0] : rot == 2 ? wv[3] : wv[2];
  o.z = rot == 0 ? wv[2] : rot == 1 ? wv[1] : rot == 2 ? wv[0] : wv[3];
  o.w = rot == 0 ? wv[3] : rot == 1 ? wv[2] : rot == 2 ? wv[1] : wv[0];
  return o;
}

__global__ void __launch_bounds__(kLagStreamThreads, 3) shift_lags_stream_kernel(const __grid_constant__ CUtensorMap map,
                                                                              const LagStreamArgs a) {
  extern __shared__ __align__(16) uint8_t dyn_smem[];
  // 128-byte aligned ring, addressed from dyn_smem so the compiler keeps shared-space loads
  uint8_t* const ring = dyn_smem + ((128u - (smem_u32(dyn_smem) & 127u)) & 127u);
  __shared__ __align__(8) uint64_t full[kLagRing];
  __shared__ int32_t lag_s[64];
  __shared__ int32_t span[2];
  const int tid = threadIdx.x;
  const int nblk = (a.N + 63) / 64;
  const int eb = static_cast<int>(blockIdx.x % nblk);
  const int rest = static_cast<int>(blockIdx.x / nblk);
  const int f = rest % a.F;
  const int64_t t_begin = static_cast<int64_t>(rest / a.F) * a.tseg;
  const int64_t t_end = min(static_cast<int64_t>(a.T), t_begin + a.tseg);
  const int i0 = eb * 64;
  const int ne = min(64, a.N - i0);  // a multiple of 16 (N % 16 == 0)
  if (tid == 0) {
    span[0] = INT32_MAX;
    span[1] = INT32_MIN;
    for (int k = 0; k < kLagRing; ++k) mbar_init(&full[k], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid < 64) {
    const int32_t l = tid < ne ? a.lags[i0 + tid] : 0;
    lag_s[tid] = l;
    if (tid < ne) {
      atomicMin(&span[0], l);
      atomicMax(&span[1], l);
    }
  }
  __syncthreads();
  const int64_t lmin = span[0], lmax = span[1];
  const int64_t row_stride = static_cast<int64_t>(a.F) * a.N;
  if (lmax - lmin > kLagSpanRing) {  // too wide for the ring: gather bytes from global memory
    for (int64_t k = tid; k < (t_end - t_begin) * 16; k += kLagStreamThreads) {
      const int64_t t = t_begin + (k >> 4);
      const int e0 = static_cast<int>(k & 15) * 4;
      if (e0 >= ne) continue;
      uint32_t word = 0;
      for (int u = 0; u < 4; ++u) {
        const int64_t src = t - lag_s[e0 + u];
        const uint32_t v = (src >= 0 && src < a.T) ? a.in[src * row_stride + static_cast<int64_t>(f) * a.N + i0 + e0 + u] : 0x88u;
        word |= v << (8 * u);
      }
      *reinterpret_cast<uint32_t*>(a.out + t * row_stride + static_cast<int64_t>(f) * a.N + i0 + e0) = word;
    }
    return;
  }
  // every source row this CTA needs, clipped to the frame
  const int64_t s_lo = max(int64_t(0), t_begin - lmax);
  const int64_t s_hi = min(static_cast<int64_t>(a.T) - 1, t_end - 1 - lmin);
  const bool any = s_lo <= s_hi;
  const int64_t first = s_lo >> 7, last = s_hi >> 7;

  // this lane's quad, rows and rotated word order
  const int lane = tid & 31, warp = tid >> 5;
  const int q = lane & 3, rr = lane >> 2;  // rows rr and rr + 8 of each warp's 16
  const int rot = rr >> 1;
  uint32_t c[16];  // (e - 64 * lag) mod 2^32 for the lane's 16 elements in visiting order
  int32_t lg[16];
#pragma unroll
  for (int w = 0; w < 4; ++w)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int e = 16 * q + 4 * ((w + rot) & 3) + b;
      lg[4 * w + b] = lag_s[e];
      c[4 * w + b] = static_cast<uint32_t>(e) - 64u * static_cast<uint32_t>(lag_s[e]);
    }
  const bool quad_live = 16 * q < ne;
  uint8_t* out_base = a.out + static_cast<int64_t>(f) * a.N + i0 + 16 * q;

  int64_t next = first;  // next box to issue (thread 0)
  auto issue_upto = [&](int64_t lim) {
    lim = min(lim, last);
    for (; next <= lim; ++next) {
      uint64_t* bar = &full[next % kLagRing];
      mbar_arrive_expect_tx(bar, 64u * 128u);
      tma_load_3d(ring + (next % kLagRing) * (128 * 64), &map, bar, i0, f, static_cast<int32_t>(next * 128));
    }
  };
  if (tid == 0 && any) {
    tma_prefetch_desc(&map);
    issue_upto(first + kLagRing - 1);
  }
  bool fault = false;
  for (int64_t t0 = t_begin; t0 < t_end; t0 += 128) {
    int64_t lo = 0;
    bool ok = true;
    if (any) {
      lo = clamp64((t0 - lmax) >> 7, first, last);
      const int64_t hi = clamp64((t0 + 127 - lmin) >> 7, first, last);
      for (int64_t b = lo; b <= hi && ok; ++b)
        ok = mbar_wait_bounded(&full[b % kLagRing], static_cast<uint32_t>(((b - first) / kLagRing) & 1), kSpinLimit);
    }
    if (!__syncthreads_and(ok)) {  // uniform: every thread leaves together
      fault = true;
      break;
    }
    // every thread is past the previous block: boxes below lo are free
    if (tid == 0 && any) issue_upto(lo + kLagRing - 1);
    const bool interior = t0 - lmax >= 0 && t0 + 127 - lmin < a.T;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int32_t tt = static_cast<int32_t>(t0) + warp * 16 + rr + 8 * h;
      if (tt >= t_end || !quad_live) continue;
      const uint4 o = interior ? lag_unit<true>(ring, tt, c, lg, rot, a.T) : lag_unit<false>(ring, tt, c, lg, rot, a.T);
      *reinterpret_cast<uint4*>(out_base + static_cast<int64_t>(tt) * row_stride) = o;
    }
  }
  if (fault && tid == 0) {
    atomicOr(a.err, 1);
    // never leave with copies in flight (bounded)
    const int64_t from = max(first, next - kLagRing);
    for (int64_t b = from; b < next; ++b)
      mbar_wait_bounded(&full[b % kLagRing], static_cast<uint32_t>(((b - first) / kLagRing) & 1), kSpinLimit);
  }
}

}  // namespace xe
