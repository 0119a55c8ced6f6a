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
// A CTA owns one band's block of kW elements (kW = 128, or 64 for narrow
// frames) over a segment of `tseg` output samples and walks it in blocks of
// kBR = 8192 / kW samples. Source rows arrive by TMA in boxes of kW elements x
// kBR samples (box b = rows kBR b .. kBR b + kBR - 1) into a 64 KiB ring of
// kLagRing boxes, where row s sits at (s mod kRR) * kW, kRR = kLagRing kBR.
// Each source row is read from HBM once per segment. The block at t0 needs
// the boxes of rows t0 - lmax .. t0 + kBR - 1 - lmin (lmin, lmax: the block's
// lag range), at most 6 when lmax - lmin <= 4 kBR; box b + kLagRing replaces
// box b once no thread reads it. Boxes are issued in order from the CTA's
// first box, so box b is use (b - first) / kLagRing of its barrier. Wider
// blocks make every TMA row request and every store a whole 128-byte line.
//
// Shared-memory banks: a warp covers kR = 32 / kQ rows x kQ = kW / 16 quads of
// 16 bytes; lane (quad q, row r) visits its quad's words starting at word
// 4 r / kR, so that at every step the 32 lanes read 32 different banks. With
// kW = 128 rows are 32 words apart and the 4 rows start at 4 different words;
// with kW = 64 rows are 16 words apart, and rows r, r + 1 share the start
// word but their source rows differ by one, i.e. by 16 banks.
constexpr int kLagRing = 8;
constexpr int kLagRingBytes = 64 * 1024;
constexpr int kLagStreamThreads = 256;
constexpr int kLagStreamSmem = kLagRingBytes + 128;  // dynamic shared memory (aligned to 128 inside)

template <int kW>
struct LagGeom {
  static constexpr int kBR = 8192 / kW;         // rows per box and per block
  static constexpr int kBRLog = kW == 64 ? 7 : 6;
  static constexpr int kRR = kLagRing * kBR;    // ring rows
  static constexpr int kSpan = 4 * kBR;         // largest lag range the ring serves
  static constexpr int kQ = kW / 16;            // quads per row
  static constexpr int kR = 32 / kQ;            // rows per warp step
  static constexpr int kPassRows = 8 * kR;      // rows per pass of the 8 warps
  static_assert((1 << kBRLog) == kBR && kBR == 2 * kPassRows, "two passes per block");
};

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
template <int kW, bool kInterior>
__device__ __forceinline__ uint4 lag_unit(const uint8_t* ring, int32_t t, const uint32_t (&c)[16],
                                          const int32_t (&lg)[16], int rot, int32_t T) {
  const uint32_t tb = static_cast<uint32_t>(t & (LagGeom<kW>::kRR - 1)) * kW;
  uint32_t wv[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    uint32_t v[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int k = 4 * w + b;
      v[b] = ring[(tb + c[k]) & (kLagRingBytes - 1u)];
      if (!kInterior) {
        const int64_t src = static_cast<int64_t>(t) - lg[k];
        if (src < 0 || src >= T) v[b] = 0x88u;
      }
    }
    wv[w] = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
  }
  // undo the rotation: output word j was read at step (j - rot) & 3
  uint4 o;
  o.x = rot == 0 ? wv[0] : rot == 1 ? wv[3] : rot == 2 ? wv[2] : wv[1];
  o.y = rot == 0 ? wv[1] : rot == 1 ? wv[0] : rot == 2 ? wv[3] : wv[2];
  o.z = rot == 0 ? wv[2] : rot == 1 ? wv[1] : rot == 2 ? wv[0] : wv[3];
  o.w = rot == 0 ? wv[3] : rot == 1 ? wv[2] : rot == 2 ? wv[1] : wv[0];
  return o;
}

template <int kW>
__global__ void __launch_bounds__(kLagStreamThreads, 3) shift_lags_stream_kernel(const __grid_constant__ CUtensorMap map,
                                                                              const LagStreamArgs a) {
  using G = LagGeom<kW>;
  extern __shared__ __align__(16) uint8_t dyn_smem[];
  // 128-byte aligned ring, addressed from dyn_smem so the compiler keeps shared-space loads
  uint8_t* const ring = dyn_smem + ((128u - (smem_u32(dyn_smem) & 127u)) & 127u);
  __shared__ __align__(8) uint64_t full[kLagRing];
  __shared__ int32_t lag_s[kW];
  __shared__ int32_t span[2];
  const int tid = threadIdx.x;
  const int nblk = (a.N + kW - 1) / kW;
  const int eb = static_cast<int>(blockIdx.x % nblk);
  const int rest = static_cast<int>(blockIdx.x / nblk);
  const int f = rest % a.F;
  const int64_t t_begin = static_cast<int64_t>(rest / a.F) * a.tseg;
  const int64_t t_end = min(static_cast<int64_t>(a.T), t_begin + a.tseg);
  const int i0 = eb * kW;
  const int ne = min(kW, a.N - i0);  // a multiple of 16 (N % 16 == 0)
  if (tid == 0) {
    span[0] = INT32_MAX;
    span[1] = INT32_MIN;
    for (int k = 0; k < kLagRing; ++k) mbar_init(&full[k], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid < kW) {
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
  if (lmax - lmin > G::kSpan) {  // too wide for the ring: gather bytes from global memory
    for (int64_t k = tid; k < (t_end - t_begin) * (kW / 4); k += kLagStreamThreads) {
      const int64_t t = t_begin + k / (kW / 4);
      const int e0 = static_cast<int>(k % (kW / 4)) * 4;
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
  const int64_t first = s_lo >> G::kBRLog, last = s_hi >> G::kBRLog;

  // this lane's quad, rows and rotated word order
  const int lane = tid & 31, warp = tid >> 5;
  const int q = lane % G::kQ, rr = lane / G::kQ;  // rows warp kR + rr and that + kPassRows of each block
  const int rot = rr * 4 / G::kR;
  uint32_t c[16];  // (e - kW lag) mod 2^32 for the lane's 16 elements in visiting order
  int32_t lg[16];
#pragma unroll
  for (int w = 0; w < 4; ++w)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int e = 16 * q + 4 * ((w + rot) & 3) + b;
      lg[4 * w + b] = lag_s[e];
      c[4 * w + b] = static_cast<uint32_t>(e) - static_cast<uint32_t>(kW) * static_cast<uint32_t>(lag_s[e]);
    }
  const bool quad_live = 16 * q < ne;
  uint8_t* out_base = a.out + static_cast<int64_t>(f) * a.N + i0 + 16 * q;

  int64_t next = first;  // next box to issue (thread 0)
  auto issue_upto = [&](int64_t lim) {
    lim = min(lim, last);
    for (; next <= lim; ++next) {
      uint64_t* bar = &full[next % kLagRing];
      mbar_arrive_expect_tx(bar, static_cast<uint32_t>(kW * G::kBR));
      tma_load_3d(ring + (next % kLagRing) * (kW * G::kBR), &map, bar, i0, f, static_cast<int32_t>(next * G::kBR));
    }
  };
  if (tid == 0 && any) {
    tma_prefetch_desc(&map);
    issue_upto(first + kLagRing - 1);
  }
  bool fault = false;
  for (int64_t t0 = t_begin; t0 < t_end; t0 += G::kBR) {
    int64_t lo = 0;
    bool ok = true;
    if (any) {
      lo = clamp64((t0 - lmax) >> G::kBRLog, first, last);
      const int64_t hi = clamp64((t0 + G::kBR - 1 - lmin) >> G::kBRLog, first, last);
      for (int64_t b = lo; b <= hi && ok; ++b)
        ok = mbar_wait_bounded(&full[b % kLagRing], static_cast<uint32_t>(((b - first) / kLagRing) & 1), kSpinLimit);
    }
    if (!__syncthreads_and(ok)) {  // uniform: every thread leaves together
      fault = true;
      break;
    }
    // every thread is past the previous block: boxes below lo are free
    if (tid == 0 && any) issue_upto(lo + kLagRing - 1);
    const bool interior = t0 - lmax >= 0 && t0 + G::kBR - 1 - lmin < a.T;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int32_t tt = static_cast<int32_t>(t0) + h * G::kPassRows + warp * G::kR + rr;
      if (tt >= t_end || !quad_live) continue;
      const uint4 o = interior ? lag_unit<kW, true>(ring, tt, c, lg, rot, a.T)
                               : lag_unit<kW, false>(ring, tt, c, lg, rot, a.T);
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
