// Host side of the C ABI declared in include/xengine.h: handles, the
// upper-triangle tile scheduler, TMA descriptors, launches and ordering.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "xengine.h"
#include "xe_batch.cuh"
#include "xe_corr.cuh"
#include "xe_lags.cuh"
#include "xe_offsets.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

// ---- cuTensorMapEncodeTiled through the runtime's driver entry point --------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;

EncodeTiledFn encode_fn() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  });
  return g_encode;
}

// ---- per-device kernel set-up ---------------------------------------------------
constexpr size_t kSmemBytes = sizeof(xe::CorrSmem) + 128;  // + alignment slack
std::mutex g_dev_mu;
int g_blocks_per_sm[64];
int g_sms[64];
bool g_dev_ready[64];

int device_setup(int dev) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (dev < 0 || dev >= 64) return fail(CORR_EINVAL, "device ordinal %d out of range", dev);
  if (g_dev_ready[dev]) return CORR_OK;
  cudaError_t e = cudaSuccess;
  for (const void* k : {reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kSingle, false>),
                        reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kSingle, false, xe::kSplit7>),
                        reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kSingle, false, xe::kSplit5>),
                        reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kSingle, false, xe::kSplit4>),
                        reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kBatch, false>),
                        reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kGated, false>),
                        reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kGateArith, false>),
                        reinterpret_cast<const void*>(xe::corr_tile_kernel<xe::kSingle, true>)})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemBytes));
  if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, xe::corr_tile_kernel<xe::kSingle, false>, xe::kThreads,
                                                    kSmemBytes);
  if (e != cudaSuccess || bps < 1)
    return fail(CORR_ECUDA, "occupancy query: %s (blocks/SM %d)", cudaGetErrorString(e), bps);
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "SM count: %s", cudaGetErrorString(e));
  g_blocks_per_sm[dev] = bps;
  g_sms[dev] = sms;
  g_dev_ready[dev] = true;
  return CORR_OK;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// A failed allocation leaves the runtime's last-error slot set; clear it so a
// later launch check does not report it as the launch's own error.
int alloc_failed(const char* what, size_t bytes, cudaError_t e) {
  cudaGetLastError();
  return fail(CORR_ENOMEM, "%s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
}

// Product path: 1 = tensor cores + dp4a (chunk_hybrid), 0 = tensor cores only,
// 2 = as 1 on offset-encoded operands with the Eq. 3 corrections (xe_offsets.cuh).
// XE_PRODUCT=mma in the environment makes the tensor-core-only path the default.
int product_hybrid() {
  const char* v = getenv("XE_PRODUCT");
  return (v && strcmp(v, "mma") == 0) ? 0 : 1;
}
const int g_hybrid = product_hybrid();

int effective_product(int product) { return product < 0 ? g_hybrid : product; }
// The kernel's split of each chunk (xe::kSplit*): tensor cores only for
// product 0, else `mma_steps` of every 8 k-steps of 32 samples on the tensor
// cores (CORR_OPT_MMA_STEPS) and the rest on dp4a.
int chunk_hybrid_flag(int product, int mma_steps) {
  if (effective_product(product) == 0) return xe::kSplitMma;
  switch (mma_steps) {
    case 8: return xe::kSplitMma;
    case 7: return xe::kSplit7;
    case 5: return xe::kSplit5;
    case 4: return xe::kSplit4;
    default: return xe::kSplit6;
  }
}

// Upper-triangle tile order: block rows bi <= block columns bj, row-major (Fig. 1).
void triangle_tiles(int32_t N, int32_t tile, std::vector<int32_t>& bi, std::vector<int32_t>& bj) {
  const int32_t nb = static_cast<int32_t>(ceil_div(N, tile));
  bi.clear();
  bj.clear();
  for (int32_t r = 0; r < nb; ++r)
    for (int32_t c = r; c < nb; ++c) {
      bi.push_back(r);
      bj.push_back(c);
    }
}

}  // namespace

// A launch schedule: work items (band, tile, chunk range) taken round-robin
// by the CTAs of one persistent launch.
struct Plan {
  int4* d_items = nullptr;  // {f, bi | bj << 16, c0, c1}
  int32_t nitems = 0, nch = 0, grid = 0, T = 0, split = 1;
};

// ---- the handle ----------------------------------------------------------------
struct corr_handle {
  int32_t N = 0, F = 0, T = 0;
  // input frames hold F_in bands; the handle correlates bands [f0, f0 + F) of them
  int32_t F_in = 0, f0 = 0;
  int64_t B = 0;
  int device = 0;
  int32_t* acc = nullptr;  // [F][B][2]
  bool own_acc = false;
  bool fresh = true;       // accumulators logically zero (memory may hold anything)
  int64_t samples = 0;
  int64_t launches = 0;    // kernels launched by this handle
  int product = -1;        // CORR_OPT_PRODUCT (-1: library default)
  int split_opt = 0;       // CORR_OPT_SPLIT (0: automatic)
  int mma_steps = 5;       // CORR_OPT_MMA_STEPS: tensor-core k-steps per 8 (the rest on dp4a)
  int sticky = CORR_OK;
  int32_t* d_err = nullptr;
  cudaEvent_t last = nullptr;
  cudaStream_t last_stream = nullptr;
  bool has_last = false;
  // schedules (tile list + per-CTA unit ranges) for full frames and the host path's chunks
  Plan plan, plan_chunk, plan_tail;
  // aligned staging for frames whose rows are not 16-byte aligned
  uint8_t* stage = nullptr;
  size_t stage_bytes = 0;
  // host-input path: two device chunk buffers, two streams
  uint8_t* hchunk[2] = {nullptr, nullptr};
  int32_t hchunk_T = 0, tail_T = 0;
  uint32_t hseq = 0;  // chunks copied so far: chunk buffers alternate across calls
  cudaStream_t s_copy = nullptr, s_comp = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr}, ev_in = nullptr;
  // offset-encoded route: per-element nibble sums [F][N][2] of the current launch
  int32_t* d_sums = nullptr;
  // a time piece's work list (batched calls that run a piece alone), grown on demand
  int4* d_piece = nullptr;
  int64_t piece_cap = 0;
  // corr_status: a private stream and a pinned word to read the fault word
  // after the handle's last call only (not after unrelated work)
  cudaStream_t s_status = nullptr;
  int32_t* h_status = nullptr;
  // overlapped readouts (corr_readout_async): a second accumulator set; the
  // event after the copy out of each set; whether the active set must wait
  // for its copy out before the next write into it
  int32_t* acc_alt = nullptr;
  cudaEvent_t ev_copied_out[2] = {nullptr, nullptr};
  int active_set = 0;         // which of {the handle's own set, acc_alt} is acc (0: acc_own)
  int32_t* acc_own = nullptr; // the set the handle was created with
  bool acc_wait = false;      // the active set still has a copy out in flight
};

namespace {

int cuda_fail(corr_handle* h, cudaError_t e, const char* what) {
  if (h) h->sticky = CORR_ECUDA;
  return fail(CORR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define XE_CHECK(h, call)                                          \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);       \
  } while (0)

// Relative cost of one chunk of a diagonal tile: its 20 needed 16 x 8
// sub-tiles run 5 per SM sub-partition (8 on a full tile), a little slower
// per sub-tile than a full tile's.
constexpr double kDiagCost = 0.7;

// Tiles of a frame: band-major, row-major over the upper triangle of each band.
void frame_tiles(int32_t N, int32_t F, std::vector<int2>& tiles, std::vector<double>& cost) {
  std::vector<int32_t> bi, bj;
  triangle_tiles(N, xe::kTile, bi, bj);
  const size_t per_band = bi.size();
  tiles.resize(per_band * static_cast<size_t>(F));
  cost.resize(tiles.size());
  for (size_t u = 0; u < tiles.size(); ++u) {
    const size_t k = u % per_band;
    tiles[u] = make_int2(static_cast<int32_t>(u / per_band), bi[k] | (bj[k] << 16));
    cost[u] = bi[k] == bj[k] ? kDiagCost : 1.0;
  }
}

// Items of a frame: the time axis cut into `split` ranges of whole chunks
// (split-major), each range over every tile in frame order. CTA k of P takes
// items k, k+P, ... so the CTAs running together work on neighbouring tiles
// of one band over the same time range and share its input in L2.
void make_items(const std::vector<int2>& tiles, int64_t nch, int64_t split, std::vector<int4>& items) {
  items.clear();
  const int64_t per = ceil_div(nch, split);
  for (int64_t k = 0; k < split; ++k) {
    const int64_t c0 = k * per, c1 = std::min<int64_t>(nch, (k + 1) * per);
    if (c0 >= c1) continue;
    for (const int2& t : tiles)
      items.push_back(make_int4(t.x, t.y, static_cast<int32_t>(c0), static_cast<int32_t>(c1)));
  }
}

// Largest per-CTA cost over the mean under round-robin assignment.
double imbalance(const std::vector<int4>& items, const std::vector<double>& cost_of_tile, int64_t ntiles, int64_t P) {
  std::vector<double> load(static_cast<size_t>(P), 0.0);
  double total = 0.0;
  for (size_t k = 0; k < items.size(); ++k) {
    const double c = cost_of_tile[k % ntiles] * (items[k].w - items[k].z);
    load[k % P] += c;
    total += c;
  }
  const double mean = total / static_cast<double>(P);
  return *std::max_element(load.begin(), load.end()) / mean;
}

// Pick the time split: the smallest that keeps the busiest CTA within 3% of
// the mean (whole tiles need no atomics), else the best of the candidates.
void plan_items(int32_t N, int32_t F, int32_t T, int64_t slots, std::vector<int4>& items, int64_t* split_out,
                int64_t* grid_out, int64_t forced_split = 0) {
  std::vector<int2> tiles;
  std::vector<double> cost;
  frame_tiles(N, F, tiles, cost);
  const int64_t ntiles = static_cast<int64_t>(tiles.size());
  const int64_t nch = ceil_div(T, xe::kTC);
  int64_t best_split = 1;
  double best = 1e30;
  if (forced_split > 0) best_split = std::min<int64_t>(forced_split, nch);
  for (int64_t split : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64}) {
    if (forced_split > 0) break;
    if (split > nch) break;
    std::vector<int4> cand;
    make_items(tiles, nch, split, cand);
    const int64_t P = std::min<int64_t>(slots, static_cast<int64_t>(cand.size()));
    // a launch narrower than the GPU runs at P/slots of its speed
    const double eff = imbalance(cand, cost, ntiles, P) * static_cast<double>(slots) / static_cast<double>(P);
    if (eff < best - 1e-9) {
      best = eff;
      best_split = split;
    }
    if (eff <= 1.03) break;
  }
  make_items(tiles, nch, best_split, items);
  *split_out = best_split;
  *grid_out = std::min<int64_t>(slots, static_cast<int64_t>(items.size()));
}

// Schedule a frame of T samples for the resident CTAs of this device.
int build_plan(corr_handle* h, int32_t T, Plan* pl) {
  const int64_t slots = static_cast<int64_t>(g_sms[h->device]) * g_blocks_per_sm[h->device];
  std::vector<int4> items;
  int64_t split = 1, grid = 1;
  plan_items(h->N, h->F, T, slots, items, &split, &grid, h->split_opt);
  if (items.size() > static_cast<size_t>(INT32_MAX)) return fail(CORR_EINVAL, "schedule too large");
  cudaError_t ae = cudaMalloc(&pl->d_items, items.size() * sizeof(int4));
  if (ae != cudaSuccess) {
    pl->d_items = nullptr;
    return alloc_failed("work list", items.size() * sizeof(int4), ae);
  }
  XE_CHECK(h, cudaMemcpy(pl->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  pl->nitems = static_cast<int32_t>(items.size());
  pl->nch = static_cast<int32_t>(ceil_div(T, xe::kTC));
  pl->grid = static_cast<int32_t>(grid);
  pl->T = T;
  pl->split = static_cast<int32_t>(split);
  return CORR_OK;
}

void free_plan(Plan* pl) {
  if (pl->d_items) cudaFree(pl->d_items);
  *pl = Plan();
}

// 3-D map (elements, bands, time) of F bands of Np bytes starting at `base`;
// consecutive time samples are row_bytes apart (0: F * Np, a frame of exactly
// these bands). Elements past Np and samples past T read as zero bytes.
int make_tmap(CUtensorMap* m, const uint8_t* base, int32_t Np, int32_t F, int32_t T, uint32_t box_n = xe::kTile,
              uint32_t box_t = xe::kTC, int64_t row_bytes = 0) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(CORR_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (row_bytes == 0) row_bytes = static_cast<int64_t>(Np) * F;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(Np), static_cast<cuuint64_t>(F), static_cast<cuuint64_t>(T)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(Np), static_cast<cuuint64_t>(row_bytes)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(box_n), 1u, static_cast<cuuint32_t>(box_t)};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CORR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return CORR_OK;
}

// Order this call after the handle's previous call if that ran on another
// stream, and after the copy out of the active accumulator set if an
// overlapped readout of that set is still in flight.
int order_after_last(corr_handle* h, cudaStream_t st) {
  if (h->has_last && h->last_stream != st) XE_CHECK(h, cudaStreamWaitEvent(st, h->last, 0));
  if (h->acc_wait) {
    XE_CHECK(h, cudaStreamWaitEvent(st, h->ev_copied_out[h->active_set], 0));
    h->acc_wait = false;
  }
  return CORR_OK;
}

int record_last(corr_handle* h, cudaStream_t st) {
  XE_CHECK(h, cudaEventRecord(h->last, st));
  h->last_stream = st;
  h->has_last = true;
  return CORR_OK;
}

int check_handle(corr_handle* h) {
  if (!h) return fail(CORR_EINVAL, "NULL handle");
  if (h->sticky != CORR_OK) return fail(h->sticky, "handle has a sticky error (%d)", h->sticky);
  return CORR_OK;
}

// Launch the correlator over the handle's F bands of Np bytes (16-byte
// aligned rows) at `frame`, time samples row_bytes apart.
int launch_frame(corr_handle* h, const uint8_t* frame, int32_t Np, int64_t row_bytes, const Plan& pl,
                 cudaStream_t st) {
  CUtensorMap tm;
  int rc = make_tmap(&tm, frame, Np, h->F, pl.T, xe::kTile, xe::kTC, row_bytes);
  if (rc) return rc;
  const bool enc = effective_product(h->product) == 2;
  if (enc) {
    // Eq. 3 route: nibble sums over this launch's samples, then the offset
    // terms stored (fresh) or added into the accumulators; the correlator
    // then adds the encoded products onto them
    const size_t sbytes = static_cast<size_t>(h->F) * h->N * 2 * sizeof(int32_t);
    if (!h->d_sums) {
      cudaError_t e = cudaMalloc(&h->d_sums, sbytes);
      if (e != cudaSuccess) {
        h->d_sums = nullptr;
        return alloc_failed("nibble sums", sbytes, e);
      }
    }
    XE_CHECK(h, cudaMemsetAsync(h->d_sums, 0, sbytes, st));
    const int64_t words = static_cast<int64_t>(h->F) * (Np / 4);
    const dim3 sg(static_cast<unsigned>(ceil_div(words, xe::kSumThreads)), static_cast<unsigned>(ceil_div(pl.T, xe::kSumRows)));
    xe::nibble_sums_kernel<<<sg, xe::kSumThreads, 0, st>>>(frame, h->N, Np, h->F, pl.T, row_bytes, h->d_sums);
    XE_CHECK(h, cudaGetLastError());
    xe::offset_seed_kernel<<<static_cast<unsigned>(static_cast<int64_t>(h->F) * h->N), 256, 0, st>>>(
        h->d_sums, h->N, h->B, pl.T, h->fresh ? 0 : 1, h->acc);
    XE_CHECK(h, cudaGetLastError());
    h->launches += 2;
    h->fresh = false;  // the correlator adds onto the seeded terms
  } else if (h->fresh && pl.split > 1) {  // time-split items add atomically onto zeros
    XE_CHECK(h, cudaMemsetAsync(h->acc, 0, static_cast<size_t>(h->F) * h->B * 2 * sizeof(int32_t), st));
  }
  xe::CorrArgs a;
  a.items = pl.d_items;
  a.nitems = pl.nitems;
  a.nch = pl.nch;
  a.T = pl.T;
  a.N = h->N;
  a.B = h->B;
  a.vis = h->acc;
  a.fresh = h->fresh ? 1 : 0;
  a.hybrid = chunk_hybrid_flag(h->product, h->mma_steps);
  a.err = h->d_err;
  if (enc)  // (the offset-encoded route splits 96 / 32 or runs tensor cores only)
    xe::corr_tile_kernel<xe::kSingle, true><<<pl.grid, xe::kThreads, kSmemBytes, st>>>(tm, a);
  else if (a.hybrid == xe::kSplit7)
    xe::corr_tile_kernel<xe::kSingle, false, xe::kSplit7><<<pl.grid, xe::kThreads, kSmemBytes, st>>>(tm, a);
  else if (a.hybrid == xe::kSplit5)
    xe::corr_tile_kernel<xe::kSingle, false, xe::kSplit5><<<pl.grid, xe::kThreads, kSmemBytes, st>>>(tm, a);
  else if (a.hybrid == xe::kSplit4)
    xe::corr_tile_kernel<xe::kSingle, false, xe::kSplit4><<<pl.grid, xe::kThreads, kSmemBytes, st>>>(tm, a);
  else
    xe::corr_tile_kernel<xe::kSingle, false><<<pl.grid, xe::kThreads, kSmemBytes, st>>>(tm, a);
  XE_CHECK(h, cudaGetLastError());
  ++h->launches;
  h->fresh = false;
  return CORR_OK;
}

// A handle for bands [f0, f0 + F) of frames with F_in bands.
corr_handle_t* create_impl(int32_t N, int32_t F, int32_t T, int32_t* acc_dev, int32_t F_in, int32_t f0) {
  if (N < 1 || N > CORR_MAX_N) return fail(CORR_EINVAL, "N=%d outside [1, %d]", N, CORR_MAX_N), nullptr;
  if (F < 1) return fail(CORR_EINVAL, "F=%d must be >= 1", F), nullptr;
  if (f0 < 0 || F_in < 1 || static_cast<int64_t>(f0) + F > F_in)
    return fail(CORR_EINVAL, "bands [%d, %lld) do not lie within a frame of %d bands", f0,
                static_cast<long long>(f0) + F, F_in), nullptr;
  if (T < 1 || T > CORR_MAX_SAMPLES) return fail(CORR_EINVAL, "T=%d outside [1, %d]", T, CORR_MAX_SAMPLES), nullptr;
  const int64_t B = static_cast<int64_t>(N) * (N + 1) / 2;
  const int64_t nb = static_cast<int64_t>(ceil_div(N, xe::kTile));
  if (static_cast<int64_t>(F) * B * 2 > (int64_t(1) << 40)) return fail(CORR_EINVAL, "accumulators too large"), nullptr;
  if (static_cast<int64_t>(F) * nb * (nb + 1) / 2 > (int64_t(1) << 28))
    return fail(CORR_EINVAL, "too many tiles"), nullptr;
  if (acc_dev && (reinterpret_cast<uintptr_t>(acc_dev) & 15))
    return fail(CORR_EINVAL, "acc_dev must be 16-byte aligned"), nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e)), nullptr;
  if (device_setup(dev) != CORR_OK) return nullptr;
  corr_handle* h = new (std::nothrow) corr_handle;
  if (!h) return fail(CORR_ENOMEM, "host allocation failed"), nullptr;
  h->N = N;
  h->F = F;
  h->T = T;
  h->F_in = F_in;
  h->f0 = f0;
  h->B = B;
  h->device = dev;
  const size_t acc_bytes = static_cast<size_t>(F) * B * 2 * sizeof(int32_t);
  bool ok = true;
  if (acc_dev) {
    h->acc = acc_dev;
  } else {
    e = cudaMalloc(&h->acc, acc_bytes);
    if (e != cudaSuccess) {
      alloc_failed("cudaMalloc for accumulators", acc_bytes, e);
      h->acc = nullptr;
      ok = false;
    }
    h->own_acc = ok;
  }
  if (ok && (e = cudaMalloc(&h->d_err, sizeof(int32_t))) != cudaSuccess) {
    alloc_failed("cudaMalloc for the error word", sizeof(int32_t), e);
    ok = false;
  }
  if (ok && cudaMemset(h->d_err, 0, sizeof(int32_t)) != cudaSuccess) ok = !fail(CORR_ECUDA, "memset error word");
  if (ok && cudaEventCreateWithFlags(&h->last, cudaEventDisableTiming) != cudaSuccess)
    ok = !fail(CORR_ECUDA, "cudaEventCreate failed");
  if (ok && build_plan(h, T, &h->plan) != CORR_OK) ok = false;
  if (!ok) {
    std::string msg = g_last_error;
    corr_destroy(h);
    g_last_error = msg;
    return nullptr;
  }
  return h;
}

// The handle's bands of an input frame [T][F_in][N]: in place when its rows
// are 16-byte aligned (*frame = the first of the handle's bands, time samples
// *row_bytes apart), else copied into the staging buffer [T][F][Np].
int stage_if_needed(corr_handle* h, const uint8_t* in, int32_t T, cudaStream_t st, const uint8_t** frame,
                    int32_t* Np, int64_t* row_bytes) {
  const bool aligned = (h->N % 16 == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
  if (aligned) {
    *frame = in + static_cast<size_t>(h->f0) * h->N;
    *Np = h->N;
    *row_bytes = static_cast<int64_t>(h->F_in) * h->N;
    return CORR_OK;
  }
  const int32_t np = static_cast<int32_t>(ceil_div(h->N, 16) * 16);
  const size_t need = static_cast<size_t>(np) * h->F * static_cast<size_t>(T);
  if (need > h->stage_bytes) {
    if (h->stage) {
      XE_CHECK(h, cudaStreamSynchronize(st));
      XE_CHECK(h, cudaFree(h->stage));
      h->stage = nullptr;
      h->stage_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&h->stage, need);
    if (e != cudaSuccess) {
      h->stage = nullptr;
      return alloc_failed("staging buffer", need, e);
    }
    h->stage_bytes = need;
  }
  const int64_t rows = static_cast<int64_t>(T) * h->F;
  const int64_t total = rows * np;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>(ceil_div(total, threads), int64_t(g_sms[h->device]) * 8);
  xe::repack_rows_kernel<<<static_cast<int>(std::max<int64_t>(blocks, 1)), threads, 0, st>>>(
      in, h->stage, rows, h->N, np, h->F, h->F_in, h->f0);
  XE_CHECK(h, cudaGetLastError());
  ++h->launches;
  *frame = h->stage;
  *Np = np;
  *row_bytes = static_cast<int64_t>(np) * h->F;
  return CORR_OK;
}

}  // namespace

// ---- batched launch: many frames, one persistent kernel, replayed as a CUDA graph ----
//
// The frames' tiles form one work list (Sec. II.C: tiles are independent;
// Sec. I: bands are independent). Items are whole tiles, sorted by cost
// (longest integration first, a stable sort so one band's tiles stay
// together) and laid out in snake order over the CTAs, so each CTA gets a
// near-equal share. A graph of {descriptor copy, item copy, kernel} is built
// for a batch's sizes and replayed while the sizes repeat; the copies read
// pinned host buffers, so each replay carries the new frames. Two buffer sets
// alternate, so a batch can be prepared while the previous one runs.
namespace {

constexpr int kMaxBatchFrames = 2047;  // frame index lives in bits 20..30 of an item

struct BatchSet {
  xe::FrameDesc* h_desc = nullptr;  // pinned
  int4* h_items = nullptr;          // pinned
  xe::FrameDesc* d_desc = nullptr;
  int4* d_items = nullptr;
  size_t cap_frames = 0, cap_items = 0;
  cudaEvent_t done = nullptr;  // after the last graph launch that read this set
  bool pending = false;
  cudaGraphExec_t exec = nullptr;
  int64_t key_frames = -1, key_items = -1, key_grid = -1, key_hybrid = -1, key_gated = -1;
  int32_t* key_err = nullptr;
};

struct BatchCtx {
  BatchSet set[2];
  int next = 0;
};

std::mutex g_batch_mu;
BatchCtx* g_batch[64];  // per device, kept for the life of the process

int grow_set(BatchSet& b, size_t frames, size_t items) {
  if (frames > b.cap_frames) {
    if (b.h_desc) cudaFreeHost(b.h_desc);
    if (b.d_desc) cudaFree(b.d_desc);
    b.h_desc = nullptr;
    b.d_desc = nullptr;
    const size_t cap = std::max<size_t>(frames, 64);
    cudaError_t e = cudaMallocHost(&b.h_desc, cap * sizeof(xe::FrameDesc));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_desc, cap * sizeof(xe::FrameDesc));
    if (e != cudaSuccess) return alloc_failed("batch descriptor buffers", cap * sizeof(xe::FrameDesc), e);
    b.cap_frames = cap;
    if (b.exec) {
      cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
    }
  }
  if (items > b.cap_items) {
    if (b.h_items) cudaFreeHost(b.h_items);
    if (b.d_items) cudaFree(b.d_items);
    b.h_items = nullptr;
    b.d_items = nullptr;
    const size_t cap = std::max<size_t>(items + items / 4, 4096);
    cudaError_t e = cudaMallocHost(&b.h_items, cap * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_items, cap * sizeof(int4));
    if (e != cudaSuccess) return alloc_failed("batch work-list buffers", cap * sizeof(int4), e);
    b.cap_items = cap;
    if (b.exec) {
      cudaGraphExecDestroy(b.exec);
      b.exec = nullptr;
    }
  }
  if (!b.done && cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess)
    return fail(CORR_ECUDA, "batch event");
  return CORR_OK;
}

// kind: 1 = gate segments (corr_tile_kernel<kGated>), 2 = gate arithmetic (<kGateArith>).
int build_graph(BatchSet& b, int64_t nframes, int64_t nitems, int64_t grid, int32_t* err, int hybrid, int kind) {
  if (b.exec) {
    cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaGraphCreate: %s", cudaGetErrorString(e));
  cudaGraphNode_t cp[2], kn;
  e = cudaGraphAddMemcpyNode1D(&cp[0], g, nullptr, 0, b.d_desc, b.h_desc, nframes * sizeof(xe::FrameDesc),
                               cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaGraphAddMemcpyNode1D(&cp[1], g, nullptr, 0, b.d_items, b.h_items, nitems * sizeof(int4),
                                 cudaMemcpyHostToDevice);
  CUtensorMap unused;  // batch frames carry their own descriptors
  memset(&unused, 0, sizeof unused);
  xe::CorrArgs a;
  a.items = b.d_items;
  a.frames = b.d_desc;
  a.nitems = static_cast<int32_t>(nitems);
  a.nch = 0;
  a.T = 0;
  a.N = 0;
  a.B = 0;
  a.vis = nullptr;
  a.fresh = 0;
  a.hybrid = hybrid;
  a.err = err;
  void* params[2] = {&unused, &a};
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof kp);
  kp.func = kind == 1 ? reinterpret_cast<void*>(xe::corr_tile_kernel<xe::kGated, false>)
                      : reinterpret_cast<void*>(xe::corr_tile_kernel<xe::kGateArith, false>);
  kp.gridDim = dim3(static_cast<unsigned>(grid));
  kp.blockDim = dim3(xe::kThreads);
  kp.sharedMemBytes = static_cast<unsigned>(kSmemBytes);
  kp.kernelParams = params;
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&kn, g, cp, 2, &kp);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b.exec = nullptr;
    return fail(CORR_ECUDA, "building the batch graph: %s", cudaGetErrorString(e));
  }
  b.key_frames = nframes;
  b.key_items = nitems;
  b.key_grid = grid;
  b.key_hybrid = hybrid;
  b.key_gated = kind;
  b.key_err = err;
  return CORR_OK;
}

// ---- batched launches: a ring of launch sets, each a graph instantiated once ----
// A set holds one launch's frame descriptors and frame order (pinned host
// block, copied by the graph's first node), its work list (device, written
// by the plan kernel, the second node) and the correlator (third node).
// Launches update the nodes' parameters; the graph is never rebuilt. The
// host writes a set only after the launch that last read it has finished,
// and waits for that only when every set of the ring is in flight.
constexpr int kBatchSets = 4;
constexpr size_t kDescBytes = sizeof(xe::FrameDesc) * kMaxBatchFrames;
constexpr size_t kFirstOff = (kDescBytes + 255) / 256 * 256;                   // int64 first[n + 1]
constexpr size_t kOrderOff = kFirstOff + sizeof(int64_t) * (kMaxBatchFrames + 1);  // int32 order[n]
constexpr size_t kBlockBytes = (kOrderOff + sizeof(int32_t) * kMaxBatchFrames + 255) / 256 * 256;

struct RingSet {
  uint8_t* h_blk = nullptr;  // pinned
  uint8_t* d_blk = nullptr;
  int4* d_items = nullptr;   // stream-ordered allocation
  size_t cap_items = 0;
  cudaEvent_t done = nullptr;
  bool pending = false;
  cudaGraph_t graph = nullptr;  // kept: its node handles address the nodes of `exec` in updates
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t n_copy = nullptr, n_plan = nullptr, n_corr = nullptr;
  int key_hybrid = -1;
  // kernel arguments (the graph's kernel nodes read them when their parameters are set)
  const xe::FrameDesc* p_frames = nullptr;
  const int64_t* p_first = nullptr;
  const int32_t* p_order = nullptr;
  int32_t p_nframes = 0;
  int4* p_items = nullptr;
  int64_t p_nitems = 0, p_grid = 0;
  CUtensorMap p_unused;
  xe::CorrArgs p_args;
};

struct BatchRing {
  RingSet set[kBatchSets];
  int next = 0;
};

BatchRing* g_ring[64];  // per device, kept for the life of the process (guarded by g_batch_mu)

int ring_set_init(RingSet& r) {
  if (r.h_blk) return CORR_OK;
  cudaError_t e = cudaMallocHost(&r.h_blk, kBlockBytes);
  if (e != cudaSuccess) {
    r.h_blk = nullptr;
    return alloc_failed("batch descriptor block (pinned)", kBlockBytes, e);
  }
  e = cudaMalloc(&r.d_blk, kBlockBytes);
  if (e != cudaSuccess) {
    r.d_blk = nullptr;
    return alloc_failed("batch descriptor block", kBlockBytes, e);
  }
  if (cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess) return fail(CORR_ECUDA, "batch event");
  memset(&r.p_unused, 0, sizeof r.p_unused);
  return CORR_OK;
}

// Work-list capacity, grown by doubling with stream-ordered allocation (no
// device-wide synchronisation). The old list is freed after the set's last launch.
int ring_set_items(RingSet& r, int64_t nitems, cudaStream_t st) {
  if (static_cast<size_t>(nitems) <= r.cap_items) return CORR_OK;
  size_t cap = std::max<size_t>(r.cap_items * 2, 1 << 16);
  while (cap < static_cast<size_t>(nitems)) cap *= 2;
  cudaError_t e;
  if (r.d_items) {
    if ((e = cudaStreamWaitEvent(st, r.done, 0)) != cudaSuccess) return fail(CORR_ECUDA, "batch: %s", cudaGetErrorString(e));
    if ((e = cudaFreeAsync(r.d_items, st)) != cudaSuccess) return fail(CORR_ECUDA, "batch: %s", cudaGetErrorString(e));
    r.d_items = nullptr;
    r.cap_items = 0;
  }
  e = cudaMallocAsync(reinterpret_cast<void**>(&r.d_items), cap * sizeof(int4), st);
  if (e != cudaSuccess) {
    r.d_items = nullptr;
    return alloc_failed("batch work list", cap * sizeof(int4), e);
  }
  r.cap_items = cap;
  return CORR_OK;
}

// Batched launches run kSplitMma or kSplit6, chosen at run time (other shares run as 6: a share-5
// instantiation of the batch kernel spilled and measured slower than share 6).
void* corr_kernel_fn(int hybrid) {
  (void)hybrid;
  return reinterpret_cast<void*>(xe::corr_tile_kernel<xe::kBatch, false>);
}

// Set the three nodes' parameters from r.p_* (and build the graph the first time).
int ring_set_launch(RingSet& r, int hybrid, cudaStream_t st) {
  const unsigned plan_blocks = static_cast<unsigned>(std::min<int64_t>(ceil_div(r.p_nitems, 256), 4096));
  void* plan_params[7] = {&r.p_frames, &r.p_first, &r.p_order, &r.p_nframes, &r.p_items, &r.p_nitems, &r.p_grid};
  void* corr_params[2] = {&r.p_unused, &r.p_args};
  cudaKernelNodeParams kp_plan, kp_corr;
  memset(&kp_plan, 0, sizeof kp_plan);
  kp_plan.func = reinterpret_cast<void*>(xe::batch_plan_kernel);
  kp_plan.gridDim = dim3(plan_blocks);
  kp_plan.blockDim = dim3(256);
  kp_plan.kernelParams = plan_params;
  memset(&kp_corr, 0, sizeof kp_corr);
  kp_corr.func = corr_kernel_fn(hybrid);
  kp_corr.gridDim = dim3(static_cast<unsigned>(r.p_grid));
  kp_corr.blockDim = dim3(xe::kThreads);
  kp_corr.sharedMemBytes = static_cast<unsigned>(kSmemBytes);
  kp_corr.kernelParams = corr_params;
  cudaError_t e = cudaSuccess;
  if (r.exec) {  // update the instantiated graph in place; rebuild it if the update is refused
    e = cudaGraphExecKernelNodeSetParams(r.exec, r.n_plan, &kp_plan);
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(r.exec, r.n_corr, &kp_corr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(r.exec);
      cudaGraphDestroy(r.graph);
      r.exec = nullptr;
      r.graph = nullptr;
    }
  }
  if (!r.exec) {
    cudaGraph_t g = nullptr;
    e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&r.n_copy, g, nullptr, 0, r.d_blk, r.h_blk, kBlockBytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&r.n_plan, g, &r.n_copy, 1, &kp_plan);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&r.n_corr, g, &r.n_plan, 1, &kp_corr);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&r.exec, g, 0);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      r.exec = nullptr;
      return fail(CORR_ECUDA, "building the batch graph: %s", cudaGetErrorString(e));
    }
    r.graph = g;
  }
  r.key_hybrid = hybrid;
  if ((e = cudaGraphLaunch(r.exec, st)) != cudaSuccess) return fail(CORR_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  if ((e = cudaEventRecord(r.done, st)) != cudaSuccess) return fail(CORR_ECUDA, "batch event record");
  r.pending = true;
  return CORR_OK;
}

static int batch_shared(corr_handle_t* const* hs, const uint8_t* const* inputs, const int32_t* Ts, int n,
                        cudaStream_t st);

// A time piece's work list: the items of a schedule that keeps tiles whole
// (every item starts at chunk 0), each ending at the piece's last chunk.
__global__ void piece_items_kernel(const int4* __restrict__ src, int4* __restrict__ dst, int64_t n, int32_t nch) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int4 w = src[k];
    w.w = nch;
    dst[k] = w;
  }
}

// One frame of T samples (at most the handle's T; fewer only where the
// handle's schedule keeps its tiles whole) through the single-frame kernel:
// the body of corr_accumulate, its checks done by the caller. A shorter frame
// runs the handle's schedule with each item cut to its own chunks (a copy of
// the work list rewritten on the device, after the handle's last call).
static int accumulate_alone(corr_handle_t* h, const uint8_t* packed_dev, int32_t T, cudaStream_t st) {
  int rc = order_after_last(h, st);
  if (rc) return rc;
  const uint8_t* frame;
  int32_t np;
  int64_t row_bytes;
  if ((rc = stage_if_needed(h, packed_dev, T, st, &frame, &np, &row_bytes))) return rc;
  Plan pl = h->plan;
  if (T != h->T) {
    const int64_t n = pl.nitems;
    if (h->piece_cap < n) {
      if (h->d_piece) XE_CHECK(h, cudaFreeAsync(h->d_piece, st));
      h->d_piece = nullptr;
      h->piece_cap = 0;
      cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&h->d_piece), static_cast<size_t>(n) * sizeof(int4), st);
      if (e != cudaSuccess) {
        h->d_piece = nullptr;
        return alloc_failed("time-piece work list", static_cast<size_t>(n) * sizeof(int4), e);
      }
      h->piece_cap = n;
    }
    pl.T = T;
    pl.nch = static_cast<int32_t>(ceil_div(T, xe::kTC));
    const int blocks = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), 4 * g_sms[h->device]));
    piece_items_kernel<<<blocks, 256, 0, st>>>(h->plan.d_items, h->d_piece, n, pl.nch);
    XE_CHECK(h, cudaGetLastError());
    ++h->launches;
    pl.d_items = h->d_piece;
  }
  if ((rc = launch_frame(h, frame, np, row_bytes, pl, st))) return rc;
  h->samples += T;
  return record_last(h, st);
}

// Whole tiles per CTA slot from which a frame runs alone: its tiles then fill
// every SM four times over, so it gains nothing from sharing a launch, and the
// single-frame kernel (no frame descriptors or chunk metadata, tensor-core
// share 5 built) runs it faster than the batched one. A frame of fewer
// samples than its handle's T (a time piece) runs alone only where the
// handle's schedule keeps tiles whole, so that every item stays balanced.
constexpr int64_t kAloneWaves = CORR_BATCH_ALONE_WAVES;

int batch_impl(corr_handle_t* const* hs, const uint8_t* const* inputs, const int32_t* Ts, int n, void* stream) {
  if (n < 0 || (n > 0 && (!hs || !inputs))) return fail(CORR_EINVAL, "bad batch arguments");
  if (n == 0) return CORR_OK;
  if (n > kMaxBatchFrames) return fail(CORR_EINVAL, "batch of %d frames exceeds %d", n, kMaxBatchFrames);
  const int dev = hs[0] ? hs[0]->device : 0;
  for (int k = 0; k < n; ++k) {
    int rc = check_handle(hs[k]);
    if (rc) return rc;
    if (!inputs[k]) return fail(CORR_EINVAL, "batch input %d is NULL", k);
    if (hs[k]->device != dev) return fail(CORR_EINVAL, "batch handles live on different devices");
    if (hs[k]->F >= (1 << 20)) return fail(CORR_EINVAL, "batch frames need F < 2^20");
    const int32_t Tk = Ts ? Ts[k] : hs[k]->T;
    if (Tk < 1 || Tk > CORR_MAX_SAMPLES) return fail(CORR_EINVAL, "batch frame %d: T=%d out of range", k, Tk);
    if (hs[k]->samples + Tk > CORR_MAX_SAMPLES)
      return fail(CORR_EOVERFLOW, "batch frame %d would exceed %d samples since its handle's reset", k,
                  CORR_MAX_SAMPLES);
    for (int j = 0; j < k; ++j)
      if (hs[j] == hs[k]) return fail(CORR_EINVAL, "batch handles must be distinct (frames %d and %d)", j, k);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // frames that fill the GPU on their own run alone, in order, on the stream;
  // the rest share one batched launch after them
  const int64_t slots = static_cast<int64_t>(g_sms[dev]) * g_blocks_per_sm[dev];
  std::vector<corr_handle_t*> sh;
  std::vector<const uint8_t*> si;
  std::vector<int32_t> sT;
  for (int k = 0; k < n; ++k) {
    corr_handle* h = hs[k];
    const int32_t Tk = Ts ? Ts[k] : h->T;
    const int64_t nb = ceil_div(h->N, xe::kTile);
    if (Tk <= h->T && (Tk == h->T || h->plan.split == 1) && nb * (nb + 1) / 2 * h->F >= kAloneWaves * slots) {
      int rc = accumulate_alone(h, inputs[k], Tk, st);
      if (rc) return rc;
    } else {
      sh.push_back(h);
      si.push_back(inputs[k]);
      sT.push_back(Tk);
    }
  }
  if (sh.empty()) return CORR_OK;
  return batch_shared(sh.data(), si.data(), sT.data(), static_cast<int>(sh.size()), st);
}

// The batched launch: one work list over every frame's items, built on the
// device, one correlator launch (checks done by batch_impl).
static int batch_shared(corr_handle_t* const* hs, const uint8_t* const* inputs, const int32_t* Ts, int n,
                        cudaStream_t st) {
  const int dev = hs[0]->device;
  const int64_t slots = static_cast<int64_t>(g_sms[dev]) * g_blocks_per_sm[dev];
  // Per frame: tiles, chunks, and a time split that keeps its items short
  // against a CTA's share of the whole batch (a frame with few tiles and a
  // long time axis is cut into ranges, written with atomic adds), so the
  // launch's tail is not set by one long tile.
  std::vector<int64_t> tiles(n), nch(n), per(n), ranges(n);
  double work = 0.0;
  for (int k = 0; k < n; ++k) {
    const int64_t nb = ceil_div(hs[k]->N, xe::kTile);
    tiles[k] = nb * (nb + 1) / 2 * hs[k]->F;
    nch[k] = ceil_div(Ts ? Ts[k] : hs[k]->T, xe::kTC);
    work += static_cast<double>(hs[k]->F) * (nb * (nb - 1) / 2 + kDiagCost * nb) * nch[k];
  }
  const double share = work / static_cast<double>(slots);  // chunks per CTA, evenly spread
  int64_t nitems = 0;
  for (int k = 0; k < n; ++k) {
    int64_t s = static_cast<int64_t>(std::ceil(static_cast<double>(nch[k]) / std::max(1.0, share / 4.0)));
    s = std::max<int64_t>(1, std::min<int64_t>({s, nch[k], 64}));
    per[k] = ceil_div(nch[k], s);
    ranges[k] = ceil_div(nch[k], per[k]);
    nitems += tiles[k] * ranges[k];
  }
  if (nitems > INT32_MAX) return fail(CORR_EINVAL, "batch work list too long");
  const int64_t grid = std::min<int64_t>(slots, nitems);
  // frames by the chunks of their items, longest first (stable: frame order breaks ties)
  std::vector<int32_t> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return per[a] > per[b]; });

  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (!g_ring[dev]) g_ring[dev] = new (std::nothrow) BatchRing;
  if (!g_ring[dev]) return fail(CORR_ENOMEM, "batch ring");
  BatchRing& ring = *g_ring[dev];
  RingSet& r = ring.set[ring.next];
  int rc = ring_set_init(r);
  if (rc) return rc;
  if (r.pending) {  // the launch that last read this set's pinned block must be done
    cudaError_t e = cudaEventSynchronize(r.done);
    if (e != cudaSuccess) return fail(CORR_ECUDA, "waiting for a previous batch: %s", cudaGetErrorString(e));
    r.pending = false;
  }
  if ((rc = ring_set_items(r, nitems, st))) return rc;
  xe::FrameDesc* desc = reinterpret_cast<xe::FrameDesc*>(r.h_blk);
  int64_t* first = reinterpret_cast<int64_t*>(r.h_blk + kFirstOff);
  int32_t* ord = reinterpret_cast<int32_t*>(r.h_blk + kOrderOff);
  int64_t acc_items = 0;
  for (int s = 0; s < n; ++s) {
    first[s] = acc_items;
    ord[s] = order[s];
    acc_items += tiles[order[s]] * ranges[order[s]];
  }
  first[n] = acc_items;
  for (int k = 0; k < n; ++k) {
    corr_handle* h = hs[k];
    const int32_t Tk = Ts ? Ts[k] : h->T;
    if ((rc = order_after_last(h, st))) return rc;
    const uint8_t* frame;
    int32_t np;
    int64_t row_bytes;
    if ((rc = stage_if_needed(h, inputs[k], Tk, st, &frame, &np, &row_bytes))) return rc;
    xe::FrameDesc& d = desc[k];
    if ((rc = make_tmap(&d.map, frame, np, h->F, Tk, xe::kTile, xe::kTC, row_bytes))) return rc;
    if (ranges[k] > 1 && h->fresh) {  // time-split items add atomically onto zeros
      XE_CHECK(h, cudaMemsetAsync(h->acc, 0, static_cast<size_t>(h->F) * h->B * 2 * sizeof(int32_t), st));
      h->fresh = false;
    }
    d.N = h->N;
    d.T = Tk;
    d.nch = static_cast<int32_t>(nch[k]);
    d.fresh = h->fresh ? 1 : 0;
    d.B = h->B;
    d.vis = h->acc;
    d.t0 = 0;
    d.atomic = 0;
    d.F = h->F;
    d.nb = static_cast<int32_t>(ceil_div(h->N, xe::kTile));
    d.per = static_cast<int32_t>(per[k]);
  }
  const int hybrid = chunk_hybrid_flag(hs[0]->product, hs[0]->mma_steps);
  r.p_frames = reinterpret_cast<const xe::FrameDesc*>(r.d_blk);
  r.p_first = reinterpret_cast<const int64_t*>(r.d_blk + kFirstOff);
  r.p_order = reinterpret_cast<const int32_t*>(r.d_blk + kOrderOff);
  r.p_nframes = n;
  r.p_items = r.d_items;
  r.p_nitems = nitems;
  r.p_grid = grid;
  xe::CorrArgs& a = r.p_args;
  a.items = r.d_items;
  a.frames = r.p_frames;
  a.nitems = static_cast<int32_t>(nitems);
  a.nch = 0;
  a.T = 0;
  a.N = 0;
  a.B = 0;
  a.vis = nullptr;
  a.fresh = 0;
  a.hybrid = hybrid == xe::kSplitMma ? xe::kSplitMma : xe::kSplit6;  // (the runtime-split instantiation's choice)
  a.err = hs[0]->d_err;
  if ((rc = ring_set_launch(r, hybrid, st))) return rc;
  ring.next = (ring.next + 1) % kBatchSets;
  for (int k = 0; k < n; ++k) {
    hs[k]->fresh = false;
    hs[k]->samples += Ts ? Ts[k] : hs[k]->T;
    hs[k]->launches += 2;  // the handle's frame ran in one (shared) plan and correlator launch
    if ((rc = record_last(hs[k], st))) return rc;
  }
  return CORR_OK;
}

// ---- gated correlation, gate windows by arithmetic ---------------------------------
// One descriptor per gate (the same frame map, the gate's accumulators and
// fresh flag, the gate arithmetic), one item per (band, tile, gate) over the
// whole frame; the kernel visits only the chunks that hold samples of the
// item's gate and masks the other rows. Items are dealt round-robin in
// (gate, band, tile) order.
int gated_arith_launch(corr_handle_t* const* gates, int G, const CUtensorMap& map, int32_t T, int32_t period,
                       int32_t phase, const std::vector<int64_t>& per_gate, const std::vector<int32_t>& gate_fresh,
                       cudaStream_t st) {
  corr_handle* h0 = gates[0];
  if (G >= kMaxBatchFrames) return fail(CORR_EINVAL, "gated: at most %d gates", kMaxBatchFrames - 1);
  std::vector<int32_t> bi, bj;
  triangle_tiles(h0->N, xe::kTile, bi, bj);
  const int32_t nch = static_cast<int32_t>(ceil_div(T, xe::kTC));
  int live = 0;
  for (int g = 0; g < G; ++g) live += per_gate[g] > 0;
  const int64_t nitems = static_cast<int64_t>(h0->F) * live * static_cast<int64_t>(bi.size());
  if (nitems == 0) return CORR_OK;
  if (nitems > INT32_MAX || h0->F >= (1 << 20)) return fail(CORR_EINVAL, "gated: work list too large");
  const int dev = h0->device;
  const int64_t slots = static_cast<int64_t>(g_sms[dev]) * g_blocks_per_sm[dev];
  const int64_t grid = std::min<int64_t>(slots, nitems);

  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (!g_batch[dev]) g_batch[dev] = new (std::nothrow) BatchCtx;
  if (!g_batch[dev]) return fail(CORR_ENOMEM, "batch context");
  BatchCtx& ctx = *g_batch[dev];
  BatchSet& b = ctx.set[ctx.next];
  if (b.pending) {
    cudaError_t e = cudaEventSynchronize(b.done);
    if (e != cudaSuccess) return fail(CORR_ECUDA, "waiting for a previous batch: %s", cudaGetErrorString(e));
    b.pending = false;
  }
  int rc = grow_set(b, static_cast<size_t>(G), static_cast<size_t>(nitems));
  if (rc) return rc;
  // gate-major: a CTA's consecutive items (grid apart) mostly share a gate, so
  // its descriptor rarely changes; the CTAs running together still take the
  // tiles of a few bands of one gate and share those bands' input in L2
  int64_t k = 0;
  for (int g = 0; g < G; ++g) {
    if (per_gate[g] == 0) continue;
    for (int32_t f = 0; f < h0->F; ++f)
      for (size_t u = 0; u < bi.size(); ++u)
        b.h_items[k++] = make_int4(f | (g << 20), bi[u] | (bj[u] << 16), 0, nch);
  }
  for (int g = 0; g < G; ++g) {
    xe::FrameDesc& d = b.h_desc[g];
    d.map = map;
    d.N = h0->N;
    d.T = T;
    d.nch = nch;
    d.fresh = gate_fresh[g];
    d.B = h0->B;
    d.vis = gates[g]->acc;
    d.t0 = 0;
    d.atomic = 0;
    d.F = h0->F;
    d.nb = static_cast<int32_t>(ceil_div(h0->N, xe::kTile));
    d.per = nch;
    d.period = period;
    d.phase = phase;
    d.G = G;
    d.gate = g;
  }
  const int hybrid = chunk_hybrid_flag(h0->product, h0->mma_steps) == xe::kSplitMma ? xe::kSplitMma : xe::kSplit6;
  if (!b.exec || b.key_frames != G || b.key_items != nitems || b.key_grid != grid || b.key_hybrid != hybrid ||
      b.key_gated != 2 || b.key_err != h0->d_err)
    if ((rc = build_graph(b, G, nitems, grid, h0->d_err, hybrid, 2))) return rc;
  cudaError_t e = cudaGraphLaunch(b.exec, st);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  if ((e = cudaEventRecord(b.done, st)) != cudaSuccess) return fail(CORR_ECUDA, "batch event record");
  b.pending = true;
  ctx.next ^= 1;
  for (int g = 0; g < G; ++g) {
    gates[g]->samples += per_gate[g];
    ++gates[g]->launches;
    if ((rc = record_last(gates[g], st))) return rc;
  }
  return CORR_OK;
}

// ---- gated correlation: the samples of each gate add into that gate's handle ----
// gate(t) = floor(((t + phase) mod period) * G / period) (Sec. IV: products
// binned by time, for periodic signals). Every maximal run of samples in one
// gate is a segment; a segment is a frame descriptor over the same input
// whose samples outside [t0, t1) read as zero, adding atomically into its
// gate's accumulators. The segments' tiles form one batched launch.
int gated_impl(corr_handle_t* const* gates, int G, const uint8_t* in, int32_t T, int32_t period, int32_t phase,
               void* stream) {
  if (G < 1 || !gates || !in) return fail(CORR_EINVAL, "gated: bad arguments");
  if (T < 1 || period < 1 || phase < 0 || phase >= period)
    return fail(CORR_EINVAL, "gated: need T >= 1, period >= 1, 0 <= phase < period");
  for (int g = 0; g < G; ++g) {
    int rc = check_handle(gates[g]);
    if (rc) return rc;
    if (gates[g]->N != gates[0]->N || gates[g]->F != gates[0]->F || gates[g]->F_in != gates[0]->F_in ||
        gates[g]->f0 != gates[0]->f0 || gates[g]->device != gates[0]->device)
      return fail(CORR_EINVAL, "gated: gate handles must share N, the bands and the device");
    for (int j = 0; j < g; ++j)
      if (gates[j] == gates[g]) return fail(CORR_EINVAL, "gated: gate handles must be distinct");
  }
  corr_handle* h0 = gates[0];
  // periods of at least one chunk (and small enough for 32-bit gate positions)
  // take the gate-arithmetic kernel: one item per (band, tile, gate)
  const bool arith = period >= xe::kTC && period <= (1 << 29);
  // segments, found from the gate boundaries within a period
  struct Seg {
    int32_t t0, t1, g;
  };
  std::vector<Seg> segs;
  std::vector<int64_t> per_gate(G, 0);
  for (int64_t t = 0; t < T;) {
    const int64_t pos = (t + phase) % period;
    const int64_t g = pos * G / period;
    const int64_t next = std::min<int64_t>(period, ceil_div((g + 1) * period, G));  // first position of gate g+1
    const int64_t t1 = std::min<int64_t>(T, t + (next - pos));
    if (!arith) segs.push_back({static_cast<int32_t>(t), static_cast<int32_t>(t1), static_cast<int32_t>(g)});
    per_gate[g] += t1 - t;
    t = t1;
    if (static_cast<int64_t>(segs.size()) >= kMaxBatchFrames)  // (one descriptor is kept for padding)
      return fail(CORR_EINVAL, "gated: more than %d gate segments in one frame (shorten T or lengthen the period)",
                  kMaxBatchFrames);
  }
  for (int g = 0; g < G; ++g)
    if (gates[g]->samples + per_gate[g] > CORR_MAX_SAMPLES)
      return fail(CORR_EOVERFLOW, "gated: gate %d would exceed %d samples since its reset", g, CORR_MAX_SAMPLES);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  for (int g = 0; g < G; ++g)
    if ((rc = order_after_last(gates[g], st))) return rc;
  const uint8_t* frame;
  int32_t np;
  int64_t row_bytes;
  if ((rc = stage_if_needed(h0, in, T, st, &frame, &np, &row_bytes))) return rc;
  CUtensorMap map;
  if ((rc = make_tmap(&map, frame, np, h0->F, T, xe::kTile, xe::kTC, row_bytes))) return rc;
  // Each (band, tile, gate) group is written once, by one CTA, with every
  // sample of its gate in this frame: stored into a fresh gate, added into
  // one that holds sums; no atomics. A gate with no samples here stays as it is.
  std::vector<int32_t> gate_fresh(G);
  for (int g = 0; g < G; ++g) {
    gate_fresh[g] = gates[g]->fresh ? 1 : 0;
    if (per_gate[g] > 0) gates[g]->fresh = false;
  }
  if (arith) return gated_arith_launch(gates, G, map, T, period, phase, per_gate, gate_fresh, st);
  // groups: one (band, tile, gate) with all its segments in time order, run by
  // one CTA back to back ("hold" between them) and written once. Groups are
  // dealt in (band, gate, tile) order, each onto the least-loaded CTA: CTAs
  // running at the same time then hold the tiles of one band and gate, walk
  // the same chunks and share their input in L2 (with many groups per CTA the
  // greedy deal stays within one group of balance)
  std::vector<int32_t> bi, bj;
  triangle_tiles(h0->N, xe::kTile, bi, bj);
  std::vector<std::vector<int32_t>> gate_segs(G);
  for (size_t s = 0; s < segs.size(); ++s) gate_segs[segs[s].g].push_back(static_cast<int32_t>(s));
  struct Group {
    int32_t f, tile, g;
    double cost;
  };
  std::vector<Group> groups;
  for (int32_t f = 0; f < h0->F; ++f)
    for (int g = 0; g < G; ++g) {
      if (gate_segs[g].empty()) continue;
      double c = 0.0;
      for (int32_t s : gate_segs[g]) c += ceil_div(segs[s].t1, xe::kTC) - segs[s].t0 / xe::kTC;
      for (size_t u = 0; u < bi.size(); ++u)
        groups.push_back({f, static_cast<int32_t>(u), g, c * (bi[u] == bj[u] ? kDiagCost : 1.0)});
    }
  const int dev = h0->device;
  const int64_t slots = static_cast<int64_t>(g_sms[dev]) * g_blocks_per_sm[dev];
  const int64_t grid = std::min<int64_t>(slots, static_cast<int64_t>(groups.size()));
  std::vector<std::vector<int4>> column(static_cast<size_t>(grid));
  {
    std::vector<std::pair<double, int64_t>> heap;  // (load, cta), min-heap
    for (int64_t c = 0; c < grid; ++c) heap.push_back({0.0, c});
    auto cmp = [](const std::pair<double, int64_t>& a, const std::pair<double, int64_t>& b) { return a.first > b.first; };
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (const Group& gr : groups) {
      std::pop_heap(heap.begin(), heap.end(), cmp);
      auto& slot = heap.back();
      const auto& ss = gate_segs[gr.g];
      for (size_t k = 0; k < ss.size(); ++k) {
        const Seg& sg = segs[ss[k]];
        const int32_t hold = k + 1 < ss.size() ? static_cast<int32_t>(0x80000000u) : 0;
        column[slot.second].push_back(make_int4(gr.f | (ss[k] << 20), bi[gr.tile] | (bj[gr.tile] << 16) | hold,
                                                sg.t0 / xe::kTC, static_cast<int32_t>(ceil_div(sg.t1, xe::kTC))));
      }
      slot.first += gr.cost;
      std::push_heap(heap.begin(), heap.end(), cmp);
    }
  }
  size_t rows = 0;
  for (const auto& col : column) rows = std::max(rows, col.size());
  // CTA c's r-th item sits at r*grid + c. Shorter columns are padded with one-chunk
  // items over an extra, empty segment (every sample masked) that hold (never write).
  const int64_t nitems = static_cast<int64_t>(rows) * grid;
  const int64_t nseg = static_cast<int64_t>(segs.size()) + 1;
  const int4 pad = make_int4(static_cast<int32_t>(segs.size()) << 20, static_cast<int32_t>(0x80000000u), 0, 1);
  if (nitems > INT32_MAX || h0->F >= (1 << 20)) return fail(CORR_EINVAL, "gated: work list too large");

  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (!g_batch[dev]) g_batch[dev] = new (std::nothrow) BatchCtx;
  if (!g_batch[dev]) return fail(CORR_ENOMEM, "batch context");
  BatchCtx& ctx = *g_batch[dev];
  BatchSet& b = ctx.set[ctx.next];
  if (b.pending) {
    cudaError_t e = cudaEventSynchronize(b.done);
    if (e != cudaSuccess) return fail(CORR_ECUDA, "waiting for a previous batch: %s", cudaGetErrorString(e));
    b.pending = false;
  }
  if ((rc = grow_set(b, static_cast<size_t>(nseg), static_cast<size_t>(nitems)))) return rc;
  for (int64_t c = 0; c < grid; ++c)
    for (size_t r = 0; r < rows; ++r) b.h_items[r * grid + c] = r < column[c].size() ? column[c][r] : pad;
  for (int64_t s = 0; s < nseg; ++s) {
    const bool empty = s == nseg - 1;
    xe::FrameDesc& d = b.h_desc[s];
    d.map = map;
    d.N = h0->N;
    d.T = empty ? 0 : segs[s].t1;
    d.nch = static_cast<int32_t>(ceil_div(T, xe::kTC));
    d.fresh = empty ? 0 : gate_fresh[segs[s].g];
    d.B = h0->B;
    d.vis = gates[empty ? 0 : segs[s].g]->acc;
    d.t0 = empty ? 1 : segs[s].t0;  // t0 > T: nothing is valid
    d.atomic = 0;
  }
  const int hybrid = chunk_hybrid_flag(h0->product, h0->mma_steps) == xe::kSplitMma ? xe::kSplitMma : xe::kSplit6;
  if (!b.exec || b.key_frames != nseg || b.key_items != nitems || b.key_grid != grid || b.key_hybrid != hybrid ||
      b.key_gated != 1 || b.key_err != h0->d_err)
    if ((rc = build_graph(b, nseg, nitems, grid, h0->d_err, hybrid, 1))) return rc;
  cudaError_t e = cudaGraphLaunch(b.exec, st);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  if ((e = cudaEventRecord(b.done, st)) != cudaSuccess) return fail(CORR_ECUDA, "batch event record");
  b.pending = true;
  ctx.next ^= 1;
  for (int g = 0; g < G; ++g) {
    gates[g]->samples += per_gate[g];
    ++gates[g]->launches;
    if ((rc = record_last(gates[g], st))) return rc;
  }
  return CORR_OK;
}

}  // namespace

// =================================== C ABI ===================================
extern "C" {

corr_handle_t* corr_create(int32_t N, int32_t F, int32_t T) { return create_impl(N, F, T, nullptr, F, 0); }

corr_handle_t* corr_create_ex(int32_t N, int32_t F, int32_t T, int32_t* acc_dev) {
  if (!acc_dev) return fail(CORR_EINVAL, "acc_dev is NULL"), nullptr;
  return create_impl(N, F, T, acc_dev, F, 0);
}

corr_handle_t* corr_create_bands(int32_t N, int32_t F_in, int32_t f0, int32_t f1, int32_t T) {
  if (f1 <= f0) return fail(CORR_EINVAL, "empty band range [%d, %d)", f0, f1), nullptr;
  return create_impl(N, f1 - f0, T, nullptr, F_in, f0);
}

int corr_bands(const corr_handle_t* h, int32_t* F_in, int32_t* f0, int32_t* f1) {
  if (!h) return fail(CORR_EINVAL, "NULL handle");
  if (F_in) *F_in = h->F_in;
  if (f0) *f0 = h->f0;
  if (f1) *f1 = h->f0 + h->F;
  return CORR_OK;
}

int corr_accumulate(corr_handle_t* h, const uint8_t* packed_dev, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!packed_dev) return fail(CORR_EINVAL, "packed_dev is NULL");
  if (h->samples + h->T > CORR_MAX_SAMPLES)
    return fail(CORR_EOVERFLOW, "accumulating %d more samples would exceed %d since the last reset", h->T,
                CORR_MAX_SAMPLES);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((rc = order_after_last(h, st))) return rc;
  const uint8_t* frame;
  int32_t np;
  int64_t row_bytes;
  if ((rc = stage_if_needed(h, packed_dev, h->T, st, &frame, &np, &row_bytes))) return rc;
  if ((rc = launch_frame(h, frame, np, row_bytes, h->plan, st))) return rc;
  h->samples += h->T;
  return record_last(h, st);
}

int corr_accumulate_host(corr_handle_t* h, const uint8_t* packed_host, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!packed_host) return fail(CORR_EINVAL, "packed_host is NULL");
  if (h->samples + h->T > CORR_MAX_SAMPLES)
    return fail(CORR_EOVERFLOW, "accumulating %d more samples would exceed %d since the last reset", h->T,
                CORR_MAX_SAMPLES);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int32_t Np = static_cast<int32_t>(ceil_div(h->N, 16) * 16);
  const size_t row = static_cast<size_t>(h->F_in) * h->N;  // bytes per time sample (host layout)
  const size_t band0 = static_cast<size_t>(h->f0) * h->N;  // the handle's first band within a time sample
  if (!h->s_copy) {
    // Time chunks of at most 1 GiB per buffer (a stage multiple). Each chunk
    // after the first adds onto the output once more, so the frame is split
    // in two (the copy of one half overlapping the correlation of the other)
    // only where its input outweighs its output; otherwise it is one chunk,
    // and the next call's copy (into the other buffer) overlaps this call's
    // correlation.
    const int64_t in_bytes = int64_t(h->T) * h->F * Np, out_bytes = int64_t(h->F) * h->B * 2 * 4;
    int64_t cT = in_bytes > out_bytes ? ceil_div(ceil_div(h->T, 2), xe::kTC) * xe::kTC : h->T;
    const int64_t cap = std::max<int64_t>(xe::kTC, ((int64_t(1) << 30) / (int64_t(h->F) * Np)) / xe::kTC * xe::kTC);
    cT = std::max<int64_t>(xe::kTC, std::min<int64_t>(cT, cap));
    cT = std::min<int64_t>(cT, ceil_div(h->T, xe::kTC) * xe::kTC);
    h->hchunk_T = static_cast<int32_t>(cT);
    const size_t bytes = static_cast<size_t>(cT) * h->F * Np;
    for (int k = 0; k < 2; ++k) {
      cudaError_t e = cudaMalloc(&h->hchunk[k], bytes);
      if (e != cudaSuccess) {
        h->hchunk[k] = nullptr;
        return alloc_failed("host-path chunk buffer", bytes, e);
      }
      XE_CHECK(h, cudaEventCreateWithFlags(&h->ev_copied[k], cudaEventDisableTiming));
      XE_CHECK(h, cudaEventCreateWithFlags(&h->ev_used[k], cudaEventDisableTiming));
    }
    XE_CHECK(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    XE_CHECK(h, cudaStreamCreateWithFlags(&h->s_copy, cudaStreamNonBlocking));
    XE_CHECK(h, cudaStreamCreateWithFlags(&h->s_comp, cudaStreamNonBlocking));
    if ((rc = build_plan(h, h->hchunk_T, &h->plan_chunk))) return rc;
    h->tail_T = h->T % h->hchunk_T;
    if (h->tail_T && (rc = build_plan(h, h->tail_T, &h->plan_tail))) return rc;
  }
  // the correlation starts after everything already queued on `st` (and the
  // handle's last call); the copies wait only for their chunk buffer to be
  // free, so they overlap the previous frame's correlation and readout
  if ((rc = order_after_last(h, st))) return rc;
  XE_CHECK(h, cudaEventRecord(h->ev_in, st));
  XE_CHECK(h, cudaStreamWaitEvent(h->s_comp, h->ev_in, 0));
  const int32_t nchunks = static_cast<int32_t>(ceil_div(h->T, h->hchunk_T));
  for (int32_t c = 0; c < nchunks; ++c) {
    const int b = static_cast<int>((h->hseq + static_cast<uint32_t>(c)) & 1);
    const int32_t t0 = c * h->hchunk_T;
    const int32_t cT = std::min(h->hchunk_T, h->T - t0);
    // buffer b's last reader: the chunk two before this one, in this call or
    // an earlier one (an event never recorded is passed at once)
    XE_CHECK(h, cudaStreamWaitEvent(h->s_copy, h->ev_used[b], 0));
    // into the chunk buffer [cT][F][Np]: the handle's bands of each time sample
    const uint8_t* src = packed_host + static_cast<size_t>(t0) * row + band0;
    const size_t wide = static_cast<size_t>(h->F) * h->N;  // the handle's bytes per time sample
    if (Np == h->N && h->F == h->F_in) {
      XE_CHECK(h, cudaMemcpyAsync(h->hchunk[b], src, static_cast<size_t>(cT) * row, cudaMemcpyHostToDevice,
                                  h->s_copy));
    } else if (Np == h->N) {  // a band range: one row of F*N bytes per time sample
      XE_CHECK(h, cudaMemcpy2DAsync(h->hchunk[b], wide, src, row, wide, static_cast<size_t>(cT),
                                    cudaMemcpyHostToDevice, h->s_copy));
    } else if (h->F == h->F_in) {  // rows of N bytes into rows of Np
      XE_CHECK(h, cudaMemcpy2DAsync(h->hchunk[b], Np, src, h->N, h->N, static_cast<size_t>(cT) * h->F,
                                    cudaMemcpyHostToDevice, h->s_copy));
    } else {  // both: one 2-D copy per band
      for (int32_t f = 0; f < h->F; ++f)
        XE_CHECK(h, cudaMemcpy2DAsync(h->hchunk[b] + static_cast<size_t>(f) * Np, static_cast<size_t>(h->F) * Np,
                                      src + static_cast<size_t>(f) * h->N, row, h->N, static_cast<size_t>(cT),
                                      cudaMemcpyHostToDevice, h->s_copy));
    }
    XE_CHECK(h, cudaEventRecord(h->ev_copied[b], h->s_copy));
    XE_CHECK(h, cudaStreamWaitEvent(h->s_comp, h->ev_copied[b], 0));
    const bool tail = cT != h->hchunk_T;
    if ((rc = launch_frame(h, h->hchunk[b], Np, static_cast<int64_t>(Np) * h->F, tail ? h->plan_tail : h->plan_chunk,
                           h->s_comp)))
      return rc;
    XE_CHECK(h, cudaEventRecord(h->ev_used[b], h->s_comp));
  }
  h->hseq += static_cast<uint32_t>(nchunks);
  // the caller's stream continues after the last chunk
  XE_CHECK(h, cudaEventRecord(h->last, h->s_comp));
  XE_CHECK(h, cudaStreamWaitEvent(st, h->last, 0));
  h->samples += h->T;
  return record_last(h, st);
}

static int readout_impl(corr_handle_t* h, int32_t* vis, int reset, void* stream, cudaMemcpyKind kind) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!vis) return fail(CORR_EINVAL, "output pointer is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((rc = order_after_last(h, st))) return rc;
  const size_t bytes = static_cast<size_t>(h->F) * h->B * 2 * sizeof(int32_t);
  if (h->fresh) {  // logically zero: make it so, then copy
    XE_CHECK(h, cudaMemsetAsync(h->acc, 0, bytes, st));
    h->fresh = false;
  }
  XE_CHECK(h, cudaMemcpyAsync(vis, h->acc, bytes, kind, st));
  if (reset) {
    h->fresh = true;
    h->samples = 0;
  }
  return record_last(h, st);
}

// Overlapped readout: the finished integration is copied out of the active
// set on copy_stream while the handle continues in the other set.
static int readout_async_impl(corr_handle_t* h, int32_t* vis, void* copy_stream, cudaMemcpyKind kind) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!vis) return fail(CORR_EINVAL, "output pointer is NULL");
  cudaStream_t cs = static_cast<cudaStream_t>(copy_stream);
  const size_t bytes = static_cast<size_t>(h->F) * h->B * 2 * sizeof(int32_t);
  if (!h->acc_alt) {
    cudaError_t e = cudaMalloc(&h->acc_alt, bytes);
    if (e != cudaSuccess) {
      h->acc_alt = nullptr;
      return alloc_failed("second accumulator set", bytes, e);
    }
    for (int k = 0; k < 2; ++k) XE_CHECK(h, cudaEventCreateWithFlags(&h->ev_copied_out[k], cudaEventDisableTiming));
    h->acc_own = h->acc;
  }
  // the copy follows the handle's last call (and a pending copy out of this set)
  if ((rc = order_after_last(h, cs))) return rc;
  if (h->fresh) XE_CHECK(h, cudaMemsetAsync(h->acc, 0, bytes, cs));  // an empty integration reads as zeros
  XE_CHECK(h, cudaMemcpyAsync(vis, h->acc, bytes, kind, cs));
  XE_CHECK(h, cudaEventRecord(h->ev_copied_out[h->active_set], cs));
  // continue in the other set, fresh; before its first write, wait for its own copy out, if one was made
  const int next = h->active_set ^ 1;
  h->acc = next ? h->acc_alt : h->acc_own;
  h->active_set = next;
  h->acc_wait = true;  // (an event never recorded is passed at once)
  h->fresh = true;
  h->samples = 0;
  // the handle's next call orders itself after its last compute, not after this copy
  return CORR_OK;
}

int corr_readout_async(corr_handle_t* h, int32_t* vis_dev, void* copy_stream) {
  return readout_async_impl(h, vis_dev, copy_stream, cudaMemcpyDeviceToDevice);
}

int corr_readout_host_async(corr_handle_t* h, int32_t* vis_host, void* copy_stream) {
  return readout_async_impl(h, vis_host, copy_stream, cudaMemcpyDeviceToHost);
}

int corr_readout(corr_handle_t* h, int32_t* vis_dev, int reset, void* stream) {
  return readout_impl(h, vis_dev, reset, stream, cudaMemcpyDeviceToDevice);
}

int corr_readout_host(corr_handle_t* h, int32_t* vis_host, int reset, void* stream) {
  return readout_impl(h, vis_host, reset, stream, cudaMemcpyDeviceToHost);
}

int corr_reset(corr_handle_t* h, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  (void)stream;
  h->fresh = true;
  h->samples = 0;
  return CORR_OK;
}

int corr_accumulate_batch(corr_handle_t* const* hs, const uint8_t* const* inputs, int n, void* stream) {
  return batch_impl(hs, inputs, nullptr, n, stream);
}

int corr_accumulate_batch_ex(corr_handle_t* const* hs, const uint8_t* const* inputs, const int32_t* Ts, int n,
                             void* stream) {
  return batch_impl(hs, inputs, Ts, n, stream);
}

int corr_accumulate_gated(corr_handle_t* const* gates, int G, const uint8_t* packed_dev, int32_t T, int32_t period,
                          int32_t phase, void* stream) {
  return gated_impl(gates, G, packed_dev, T, period, phase, stream);
}

// Fault word of the streaming lag kernel: host-mapped, so the next call reads
// it without a device synchronisation.
std::mutex g_lag_mu;
int32_t* g_lag_err_host = nullptr;
int32_t* g_lag_err_dev = nullptr;
int g_lag_ctas_per_sm[64] = {};

int lag_stream_setup(int dev) {
  std::lock_guard<std::mutex> lk(g_lag_mu);
  if (!g_lag_err_host) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&g_lag_err_host), sizeof(int32_t), cudaHostAllocMapped);
    if (e != cudaSuccess) {
      g_lag_err_host = nullptr;
      return alloc_failed("shift_lags fault word", sizeof(int32_t), e);
    }
    *g_lag_err_host = 0;
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&g_lag_err_dev), g_lag_err_host, 0);
    if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaHostGetDevicePointer: %s", cudaGetErrorString(e));
  }
  if (!g_lag_ctas_per_sm[dev]) {
    int bps = 1 << 30;
    for (const void* k : {reinterpret_cast<const void*>(xe::shift_lags_stream_kernel<64>),
                          reinterpret_cast<const void*>(xe::shift_lags_stream_kernel<128>)}) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, xe::kLagStreamSmem);
      if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      int b = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, xe::kLagStreamThreads, xe::kLagStreamSmem);
      if (e != cudaSuccess || b < 1) return fail(CORR_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
      bps = std::min(bps, b);
    }
    g_lag_ctas_per_sm[dev] = bps;
  }
  return CORR_OK;
}

int corr_shift_lags(const uint8_t* in_dev, uint8_t* out_dev, int32_t N, int32_t F, int32_t T, const int32_t* lags_dev,
                    void* stream) {
  if (!in_dev || !out_dev || !lags_dev) return fail(CORR_EINVAL, "shift_lags: NULL pointer");
  if (in_dev == out_dev) return fail(CORR_EINVAL, "shift_lags: the output must not be the input");
  if (N < 1 || N > CORR_MAX_N || F < 1 || T < 1) return fail(CORR_EINVAL, "shift_lags: bad N, F or T");
  if (N % 4 == 0 && (reinterpret_cast<uintptr_t>(out_dev) & 3))
    return fail(CORR_EINVAL, "shift_lags: output must be 4-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  int rc = device_setup(dev);
  if (rc) return rc;
  if (g_lag_err_host && *reinterpret_cast<volatile int32_t*>(g_lag_err_host)) {
    *g_lag_err_host = 0;
    return fail(CORR_ETIMEOUT, "an earlier shift_lags launch reported a device wait that ran out");
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool streamable = N % 16 == 0 && (reinterpret_cast<uintptr_t>(in_dev) & 15) == 0 &&
                          (reinterpret_cast<uintptr_t>(out_dev) & 15) == 0;
  if (streamable) {
    rc = lag_stream_setup(dev);
    if (rc) return rc;
    // segments of the time axis: about 8 waves of CTAs, each segment at least
    // 1024 samples (its boundary re-reads the lag range once)
    const int kw = N >= 128 ? 128 : 64;  // element block width (see xe_lags.cuh)
    const int64_t units = ceil_div(N, kw) * F;
    const int64_t slots = static_cast<int64_t>(g_sms[dev]) * g_lag_ctas_per_sm[dev];
    const int64_t nseg_want = std::max<int64_t>(1, ceil_div(8 * slots, units));
    int64_t tseg = ceil_div(ceil_div(T, nseg_want), 128) * 128;
    tseg = std::max<int64_t>(tseg, std::min<int64_t>(ceil_div(T, 128) * 128, 1024));
    const int64_t ctas = units * ceil_div(T, tseg);
    if (ctas > INT32_MAX) return fail(CORR_EINVAL, "shift_lags: frame too large");
    CUtensorMap tm;
    rc = make_tmap(&tm, in_dev, N, F, T, static_cast<uint32_t>(kw), static_cast<uint32_t>(8192 / kw));
    if (rc) return rc;
    xe::LagStreamArgs la{in_dev, out_dev, lags_dev, N, F, T, static_cast<int32_t>(tseg), g_lag_err_dev};
    if (kw == 128)
      xe::shift_lags_stream_kernel<128><<<static_cast<unsigned>(ctas), xe::kLagStreamThreads, xe::kLagStreamSmem, st>>>(tm, la);
    else
      xe::shift_lags_stream_kernel<64><<<static_cast<unsigned>(ctas), xe::kLagStreamThreads, xe::kLagStreamSmem, st>>>(tm, la);
  } else {
    const int64_t ctas = ceil_div(N, 64) * F * ceil_div(T, xe::kLagTB);
    if (ctas > INT32_MAX) return fail(CORR_EINVAL, "shift_lags: frame too large");
    xe::shift_lags_kernel<<<static_cast<unsigned>(ctas), xe::kLagThreads, 0, st>>>(in_dev, out_dev, N, F, T, lags_dev);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CORR_ECUDA, "shift_lags launch: %s", cudaGetErrorString(e));
  return CORR_OK;
}

int corr_set_option(corr_handle_t* h, int option, int64_t value) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (option == CORR_OPT_PRODUCT) {
    if (value < -1 || value > 2) return fail(CORR_EINVAL, "CORR_OPT_PRODUCT must be -1, 0, 1 or 2");
    h->product = static_cast<int>(value);
    return CORR_OK;
  }
  if (option == CORR_OPT_MMA_STEPS) {
    if (value < 4 || value > 8) return fail(CORR_EINVAL, "CORR_OPT_MMA_STEPS must be in [4, 8]");
    h->mma_steps = static_cast<int>(value);
    return CORR_OK;
  }
  if (option == CORR_OPT_SPLIT) {
    if (value < 0 || value > 4096) return fail(CORR_EINVAL, "CORR_OPT_SPLIT must be in [0, 4096]");
    if (h->split_opt == value) return CORR_OK;
    // the schedule is rebuilt, so the handle's queued work must be done reading the old one
    if (h->has_last) {
      cudaError_t e = cudaEventQuery(h->last);
      if (e == cudaErrorNotReady) return fail(CORR_EBUSY, "CORR_OPT_SPLIT: the handle still has work in flight");
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventQuery");
    }
    h->split_opt = static_cast<int>(value);
    free_plan(&h->plan);
    if ((rc = build_plan(h, h->T, &h->plan))) return rc;
    if (h->plan_chunk.d_items) {
      free_plan(&h->plan_chunk);
      if ((rc = build_plan(h, h->hchunk_T, &h->plan_chunk))) return rc;
    }
    if (h->plan_tail.d_items) {
      free_plan(&h->plan_tail);
      if ((rc = build_plan(h, h->tail_T, &h->plan_tail))) return rc;
    }
    return CORR_OK;
  }
  return fail(CORR_EINVAL, "unknown option %d", option);
}

int64_t corr_get_option(const corr_handle_t* h, int option) {
  if (!h) return fail(CORR_EINVAL, "NULL handle");
  if (option == CORR_OPT_PRODUCT) return effective_product(h->product);
  if (option == CORR_OPT_SPLIT) return h->split_opt;
  if (option == CORR_OPT_MMA_STEPS) return h->mma_steps;
  return fail(CORR_EINVAL, "unknown option %d", option);
}

int corr_synchronize(corr_handle_t* h, int64_t timeout_ms) {
  if (!h) return fail(CORR_EINVAL, "NULL handle");
  if (!h->has_last) return CORR_OK;
  if (timeout_ms < 0) {
    cudaError_t e = cudaEventSynchronize(h->last);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    return corr_status(h);
  }
  // poll with a deadline
  cudaEvent_t probe = h->last;
  for (int64_t waited_us = 0;; waited_us += 50) {
    cudaError_t e = cudaEventQuery(probe);
    if (e == cudaSuccess) return corr_status(h);
    if (e != cudaErrorNotReady) return cuda_fail(h, e, "cudaEventQuery");
    if (waited_us >= timeout_ms * 1000) return fail(CORR_ETIMEOUT, "handle still busy after %lld ms", (long long)timeout_ms);
    struct timespec ts = {0, 50000};
    nanosleep(&ts, nullptr);
  }
}

int corr_status(corr_handle_t* h) {
  if (!h) return fail(CORR_EINVAL, "NULL handle");
  if (h->sticky != CORR_OK) return h->sticky;
  if (!h->s_status) {
    XE_CHECK(h, cudaStreamCreateWithFlags(&h->s_status, cudaStreamNonBlocking));
    cudaError_t ae = cudaHostAlloc(reinterpret_cast<void**>(&h->h_status), sizeof(int32_t), cudaHostAllocDefault);
    if (ae != cudaSuccess) {
      h->h_status = nullptr;
      return alloc_failed("status word", sizeof(int32_t), ae);
    }
  }
  // the fault word as it stands after the handle's last call (other streams' work is not waited for)
  if (h->has_last) XE_CHECK(h, cudaStreamWaitEvent(h->s_status, h->last, 0));
  XE_CHECK(h, cudaMemcpyAsync(h->h_status, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->s_status));
  XE_CHECK(h, cudaStreamSynchronize(h->s_status));
  const int32_t err = *h->h_status;
  if (err) {
    h->sticky = CORR_ETIMEOUT;
    return fail(CORR_ETIMEOUT, "device reported a wait that ran out (code %d)", err);
  }
  return CORR_OK;
}

int64_t corr_samples(const corr_handle_t* h) { return h ? h->samples : -1; }

int64_t corr_kernel_launches(const corr_handle_t* h) { return h ? h->launches : -1; }

int corr_dims(const corr_handle_t* h, int32_t* N, int32_t* F, int32_t* T) {
  if (!h) return fail(CORR_EINVAL, "NULL handle");
  if (N) *N = h->N;
  if (F) *F = h->F;
  if (T) *T = h->T;
  return CORR_OK;
}

const char* corr_last_error(void) { return g_last_error.c_str(); }

void corr_destroy(corr_handle_t* h) {
  if (!h) return;
  if (h->has_last) cudaEventSynchronize(h->last);
  for (int k = 0; k < 2; ++k)
    if (h->ev_copied_out[k]) {
      cudaEventSynchronize(h->ev_copied_out[k]);  // overlapped readouts still copying out
      cudaEventDestroy(h->ev_copied_out[k]);
    }
  if (h->acc_alt) {  // both sets: free the library's, leave a caller-owned one to the caller
    cudaFree(h->acc_alt);
    h->acc = h->acc_own;
  }
  if (h->own_acc && h->acc) cudaFree(h->acc);
  if (h->d_err) cudaFree(h->d_err);
  free_plan(&h->plan);
  free_plan(&h->plan_chunk);
  free_plan(&h->plan_tail);
  if (h->stage) cudaFree(h->stage);
  if (h->d_sums) cudaFree(h->d_sums);
  if (h->d_piece) cudaFree(h->d_piece);
  for (int k = 0; k < 2; ++k) {
    if (h->hchunk[k]) cudaFree(h->hchunk[k]);
    if (h->ev_copied[k]) cudaEventDestroy(h->ev_copied[k]);
    if (h->ev_used[k]) cudaEventDestroy(h->ev_used[k]);
  }
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->s_status) cudaStreamDestroy(h->s_status);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->s_copy) cudaStreamDestroy(h->s_copy);
  if (h->s_comp) cudaStreamDestroy(h->s_comp);
  if (h->last) cudaEventDestroy(h->last);
  delete h;
}

int64_t corr_plan_tiles(int32_t N, int32_t tile, int32_t* bi_out, int32_t* bj_out, int64_t cap) {
  if (N < 1 || N > CORR_MAX_N || tile < 1) return fail(CORR_EINVAL, "bad N or tile");
  std::vector<int32_t> bi, bj;
  triangle_tiles(N, tile, bi, bj);
  const int64_t n = static_cast<int64_t>(bi.size());
  for (int64_t k = 0; k < n && k < cap; ++k) {
    if (bi_out) bi_out[k] = bi[k];
    if (bj_out) bj_out[k] = bj[k];
  }
  return n;
}

int64_t corr_plan_schedule(int32_t N, int32_t F, int32_t T, int32_t ctas, int32_t* items_out, int64_t items_cap,
                           int32_t* grid_out) {
  if (N < 1 || N > CORR_MAX_N || F < 1 || T < 1 || ctas < 1) return fail(CORR_EINVAL, "bad schedule query");
  std::vector<int4> items;
  int64_t split = 1, grid = 1;
  plan_items(N, F, T, ctas, items, &split, &grid);
  if (items_out)
    for (int64_t k = 0; k < static_cast<int64_t>(items.size()) && k < items_cap; ++k) {
      items_out[4 * k] = items[k].x;
      items_out[4 * k + 1] = items[k].y;
      items_out[4 * k + 2] = items[k].z;
      items_out[4 * k + 3] = items[k].w;
    }
  if (grid_out) *grid_out = static_cast<int32_t>(grid);
  return static_cast<int64_t>(items.size());
}

double corr_effective_ops(int32_t N, int32_t F, int32_t T) {
  return 4.0 * static_cast<double>(N) * (static_cast<double>(N) + 1.0) * F * static_cast<double>(T);
}

}  // extern "C"

// =============================================================================
// Allocation-free correlation of one frame (corr_correlate_noalloc).
//
// Some callers cannot allocate device memory when they need a correlation:
// applications whose device memory belongs to their own pool allocator and
// may not be taken behind its back, and real-time hosts that reserve every
// byte up front and forbid allocations on the processing path.
// corr_correlate_noalloc serves them: the caller passes the frame and the
// output buffer, and the only other device memory the kernel needs (its work
// list and its fault word) is the fixed array below. Every GPU that loads
// this library holds that array until the process exits. Its device address
// is looked up once per device and kept, so a cudaDeviceReset while the
// library is in use is not supported.
// =============================================================================
namespace {

// Work items the fixed array can hold: 65,536 (1 MiB), enough for N = 8192 at
// F = 7 or N = 2048 at F = 124 with whole tiles. Element 0 holds the fault word.
constexpr int64_t kNoAllocMaxItems = 65536;
static __device__ __align__(256) int4 g_noalloc_scratch[1 + kNoAllocMaxItems];

std::mutex g_noalloc_mu;
int4* g_noalloc_addr[64];  // device address of g_noalloc_scratch, per device

// Writes the frame's work list: item k = split s, tile u of the frame (bands
// outermost, each band's upper triangle row by row), chunks [s*per, ...).
__global__ void noalloc_plan_kernel(int4* items, int32_t nb, int32_t F, int32_t nch, int32_t per, int64_t nitems) {
  const int64_t per_band = static_cast<int64_t>(nb) * (nb + 1) / 2;
  const int64_t ntiles = per_band * F;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nitems;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t s = k / ntiles, u = k % ntiles;
    const int32_t f = static_cast<int32_t>(u / per_band);
    int64_t q = u % per_band;
    int32_t bi = 0;
    while (q >= nb - bi) {  // row bi of the triangle holds nb - bi tiles
      q -= nb - bi;
      ++bi;
    }
    const int32_t bj = bi + static_cast<int32_t>(q);
    const int32_t c0 = static_cast<int32_t>(s * per);
    const int32_t c1 = static_cast<int32_t>(min(static_cast<int64_t>(nch), (s + 1) * per));
    items[k] = make_int4(f, bi | (bj << 16), c0, c1);
  }
}

// Once per device, with that device current: the array's device address.
int noalloc_setup(int dev, int4** addr) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<int4*>(p);
  }
  *addr = g_noalloc_addr[dev];
  return CORR_OK;
}

}  // namespace

extern "C" int corr_correlate_noalloc(const uint8_t* packed_dev, int32_t N, int32_t F, int32_t T, int32_t* vis_dev,
                                      int32_t* status_dev, void* stream) {
  if (!packed_dev || !vis_dev) return fail(CORR_EINVAL, "noalloc: NULL input or output");
  if (N < 1 || N > CORR_MAX_N || F < 1 || T < 1 || T > CORR_MAX_SAMPLES)
    return fail(CORR_EINVAL, "noalloc: N=%d F=%d T=%d out of range", N, F, T);
  if (N % 16 != 0 || (reinterpret_cast<uintptr_t>(packed_dev) & 15) != 0)
    return fail(CORR_EINVAL, "noalloc: needs N a multiple of 16 and a 16-byte aligned frame (N=%d)", N);
  const int64_t nb = ceil_div(N, xe::kTile);
  const int64_t ntiles = nb * (nb + 1) / 2 * F;
  const int64_t nch = ceil_div(T, xe::kTC);
  if (ntiles > kNoAllocMaxItems)
    return fail(CORR_EINVAL, "noalloc: %lld tiles exceed the fixed work-list size of %lld items",
                static_cast<long long>(ntiles), static_cast<long long>(kNoAllocMaxItems));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  int rc = device_setup(dev);
  if (rc) return rc;
  int4* scratch = nullptr;
  if ((rc = noalloc_setup(dev, &scratch))) return rc;
  const int64_t slots = static_cast<int64_t>(g_sms[dev]) * g_blocks_per_sm[dev];
  // time split: enough items to keep every CTA busy, within the array and the frame's chunks
  int64_t split = std::min<int64_t>({ceil_div(4 * slots, ntiles), kNoAllocMaxItems / ntiles, nch, int64_t(64)});
  split = std::max<int64_t>(split, 1);
  const int64_t per = ceil_div(nch, split);
  split = ceil_div(nch, per);  // no empty ranges
  const int64_t nitems = ntiles * split;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vis_bytes = static_cast<size_t>(F) * (static_cast<size_t>(N) * (N + 1) / 2) * 2 * sizeof(int32_t);
  // the fault word starts at zero; time-split items add atomically onto a zeroed output
  if ((e = cudaMemsetAsync(scratch, 0, sizeof(int4), st)) != cudaSuccess)
    return fail(CORR_ECUDA, "noalloc: clearing the fault word: %s", cudaGetErrorString(e));
  if (split > 1 && (e = cudaMemsetAsync(vis_dev, 0, vis_bytes, st)) != cudaSuccess)
    return fail(CORR_ECUDA, "noalloc: clearing the output: %s", cudaGetErrorString(e));
  const int pb = static_cast<int>(std::min<int64_t>(ceil_div(nitems, 256), 1024));
  noalloc_plan_kernel<<<pb, 256, 0, st>>>(scratch + 1, static_cast<int32_t>(nb), F, static_cast<int32_t>(nch),
                                          static_cast<int32_t>(per), nitems);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(CORR_ECUDA, "noalloc plan: %s", cudaGetErrorString(e));
  CUtensorMap tm;
  if ((rc = make_tmap(&tm, packed_dev, N, F, T))) return rc;
  xe::CorrArgs a;
  a.items = scratch + 1;
  a.nitems = static_cast<int32_t>(nitems);
  a.nch = static_cast<int32_t>(nch);
  a.T = T;
  a.N = N;
  a.B = static_cast<int64_t>(N) * (N + 1) / 2;
  a.vis = vis_dev;
  a.fresh = 1;
  a.hybrid = 0;
  a.err = reinterpret_cast<int32_t*>(scratch);
  const int grid = static_cast<int>(std::min<int64_t>(slots, nitems));
  xe::corr_tile_kernel<xe::kSingle, false><<<grid, xe::kThreads, kSmemBytes, st>>>(tm, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(CORR_ECUDA, "noalloc correlate: %s", cudaGetErrorString(e));
  if (status_dev && (e = cudaMemcpyAsync(status_dev, scratch, sizeof(int32_t), cudaMemcpyDeviceToDevice, st)) !=
                        cudaSuccess)
    return fail(CORR_ECUDA, "noalloc: copying the fault word: %s", cudaGetErrorString(e));
  return CORR_OK;
}

// ---- bounded-wait self test ----------------------------------------------------
namespace {

__device__ int32_t g_wait_probe_status;

// Waits (bounded) on a barrier whose phase never completes: nothing arrives.
__global__ void wait_probe_kernel(uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    xe::mbar_init(&bar, 1);
    xe::fence_barrier_init();
  }
  __syncthreads();
  const bool completed = xe::mbar_wait_bounded(&bar, 0, polls);
  if (threadIdx.x == 0) g_wait_probe_status = completed ? 0 : 1;
}

}  // namespace

int corr_selftest_wait_timeout(int32_t polls, void* stream) {
  if (polls < 1 || polls > (1 << 20)) return fail(CORR_EINVAL, "polls must be in [1, 2^20]");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int32_t unset = -1;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_wait_probe_status, &unset, sizeof unset, 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "wait probe: %s", cudaGetErrorString(e));
  wait_probe_kernel<<<1, 32, 0, st>>>(static_cast<uint32_t>(polls));
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CORR_ECUDA, "wait probe launch: %s", cudaGetErrorString(e));
  int32_t status = unset;
  e = cudaMemcpyFromSymbolAsync(&status, g_wait_probe_status, sizeof status, 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CORR_ECUDA, "wait probe: %s", cudaGetErrorString(e));
  if (status == 1) return fail(CORR_ETIMEOUT, "device wait ran out after %d polls (expected)", polls);
  if (status == 0) return CORR_OK;
  return fail(CORR_ECUDA, "wait probe recorded no status");
}
