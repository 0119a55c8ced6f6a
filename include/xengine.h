/*
 * xengine.h -- C ABI of the GB300 4-bit X-engine.
 *
 * The library computes, for every frequency band f and every pair of input
 * elements i <= j (autocorrelations included), the exact integer visibility
 *
 *     V[f,i,j] = sum_t x[t,f,i] * conj(x[t,f,j])
 *     Re = sum_t xr_i xr_j + xi_i xi_j,   Im = sum_t xi_i xr_j - xr_i xi_j
 *
 * (Eq. 1 of the paper, Sec. II.A, with X = element i and Y = element j,
 * accumulated over time samples as Sec. II.A describes; only the upper
 * triangle is formed because the matrix is Hermitian, Eq. 2).
 *
 * Input layout (Sec. III, Fig. 2): uint8 x[T][F][N], one byte per complex
 * sample, time outermost, then band, then element. Each part is an excess-8
 * 4-bit integer: value = nibble - 8 in [-8, 7]. The high nibble holds the
 * real part and the low nibble the imaginary part (the paper says only that
 * both share one byte; this is the reading the library fixes).
 *
 * Output layout (the paper leaves the final layout open; this is the
 * library's): int32 V[F][B][2] with B = N(N+1)/2, bands outermost, (Re, Im)
 * interleaved, entries row-major over the upper triangle:
 *     p(i, j) = i*N - i*(i-1)/2 + (j - i),   0 <= i <= j < N.
 *
 * Accumulation is exact in int32. One accumulated sample adds at most 128
 * in magnitude to an entry (|Re| <= 2*8*8), so a handle refuses to
 * accumulate more than CORR_MAX_SAMPLES samples between resets.
 *
 * Threading and ordering: every call that takes a stream is asynchronous on
 * that stream (a cudaStream_t passed as void*; NULL = legacy default
 * stream). The caller keeps input and output buffers alive until the work
 * on the stream has finished. A handle may be used from one host thread at
 * a time. Consecutive calls on one handle made on different streams are
 * ordered by an event the handle records after each call.
 *
 * Errors: functions return CORR_OK or a negative code and set a
 * thread-local message (corr_last_error). CUDA failures are sticky on the
 * handle (corr_status). Kernels never trap; a device-side fault report
 * (a bounded wait that ran out) is read back by corr_status.
 */
#ifndef XENGINE_H
#define XENGINE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct corr_handle corr_handle_t;

enum {
  CORR_OK = 0,
  CORR_EINVAL = -1,    /* bad argument: NULL handle, size out of range, bad pointer kind */
  CORR_ENOMEM = -2,    /* device or host allocation failed */
  CORR_ECUDA = -3,     /* a CUDA call failed; sticky on the handle */
  CORR_EOVERFLOW = -4, /* accumulating would exceed CORR_MAX_SAMPLES since the last reset */
  CORR_ETIMEOUT = -5,  /* a bounded wait ran out (host deadline or device wait) */
  CORR_EBUSY = -6      /* the handle still has work in flight where the call needs it idle */
};

#define CORR_MAX_N 16384
/* floor((2^31 - 1) / 128): samples an int32 accumulator can take without overflow */
#define CORR_MAX_SAMPLES 16777215

/*
 * corr_create -- make a handle for frames of N elements, F bands and T time
 * samples (the problem of Sec. II.A: N inputs, each band's N x N matrix
 * accumulated over time samples; 1 <= N <= CORR_MAX_N, F >= 1, T >= 1,
 * F*B(N)*2 int32 accumulators addressable). The handle allocates its own
 * device accumulators on the current CUDA device and starts in the reset
 * (all-zero) state; they stay resident until corr_destroy.
 * Returns NULL on error; corr_last_error() says why.
 */
corr_handle_t* corr_create(int32_t N, int32_t F, int32_t T);

/*
 * corr_create_ex -- as corr_create (Sec. II.A; library lifecycle), but the
 * accumulators live in a caller-owned device buffer acc_dev of
 * F*N(N+1)/2*2 int32 (e.g. a torch tensor), 16-byte aligned. The caller
 * keeps it alive until corr_destroy. Its contents on entry are ignored: the
 * handle starts in the reset state.
 */
corr_handle_t* corr_create_ex(int32_t N, int32_t F, int32_t T, int32_t* acc_dev);

/*
 * corr_create_bands -- a handle for the bands [f0, f1) of frames that hold
 * F_in bands (Sec. I and Sec. IV: frequency bands are independent, so the
 * bands of one frame can be split across GPUs with no exchange; each GPU
 * holds a handle for its own range). 0 <= f0 < f1 <= F_in. Every call that
 * takes a frame (corr_accumulate, corr_accumulate_host, the batched and
 * gated calls) then takes the whole frame uint8 x[T][F_in][N] and reads only
 * the handle's bands; corr_readout gives int32 V[f1 - f0][B][2], band f0
 * first. The visibilities of the ranges of a partition of [0, F_in),
 * concatenated in band order, equal those of one handle over all F_in bands.
 * Otherwise as corr_create (the handle's F is f1 - f0). NULL on error.
 */
corr_handle_t* corr_create_bands(int32_t N, int32_t F_in, int32_t f0, int32_t f1, int32_t T);

/*
 * corr_bands -- the handle's input band count and band range [f0, f1)
 * (F_in = f1 - f0 = F and f0 = 0 for handles from corr_create). Any pointer
 * may be NULL. CORR_EINVAL for a NULL handle.
 */
int corr_bands(const corr_handle_t* h, int32_t* F_in, int32_t* f0, int32_t* f1);

/*
 * corr_accumulate -- add one frame to the handle's accumulators
 * (Sec. III: results are added to the previous results).
 * packed_dev: device pointer to uint8 x[T][F][N] (layout above). Any
 * alignment and any N are accepted; inputs whose rows are not 16-byte
 * aligned are first copied into an aligned staging buffer on the device.
 * Asynchronous on `stream`. Returns CORR_EOVERFLOW (and launches nothing)
 * if the samples since the last reset would exceed CORR_MAX_SAMPLES.
 */
int corr_accumulate(corr_handle_t* h, const uint8_t* packed_dev, void* stream);

/*
 * corr_accumulate_host -- as corr_accumulate with packed_host in host memory
 * (pinned memory gives full copy speed; pageable memory works). The frame
 * is copied to the device in time-chunks, each chunk correlated while the
 * next one is copied. The copies wait only for the handle's chunk buffers,
 * not for work already queued on `stream`: they may overlap the previous
 * frame's correlation and readout. So the frame must be in host memory when
 * the call is made (not produced later by work queued on `stream`), and it
 * must stay unchanged until the stream has passed this call. The
 * correlation itself runs after everything queued on `stream` before.
 */
int corr_accumulate_host(corr_handle_t* h, const uint8_t* packed_host, void* stream);

/*
 * corr_readout -- copy the packed visibilities int32 V[F][B][2] to vis_dev
 * (device memory, or host memory for corr_readout_host); with reset != 0
 * the accumulators then return to the all-zero state (Sec. II.A: a new
 * integration starts). Asynchronous on `stream`.
 */
int corr_readout(corr_handle_t* h, int32_t* vis_dev, int reset, void* stream);
int corr_readout_host(corr_handle_t* h, int32_t* vis_host, int reset, void* stream);

/*
 * corr_readout_async / corr_readout_host_async -- end the integration and
 * copy its visibilities int32 V[F][B][2] to vis (device or host memory),
 * overlapped with the next integration (Sec. II.A: visibilities are read out
 * once an integration ends, while the next one accumulates). The handle keeps
 * a second accumulator set (allocated on the first call, F*B(N)*2 int32 in
 * device memory, freed by corr_destroy): the finished set is copied out on
 * copy_stream, after the handle's last call, while the handle's later calls
 * add into the other set, starting from zero. The copy is ordered on
 * copy_stream only, not on the handle's other streams: synchronise
 * copy_stream (or make a stream wait on it) before reading vis. The next
 * write into a set waits, on the device, for that set's last copy out, so
 * readouts may alternate freely with accumulates. Like corr_readout with
 * reset != 0 otherwise. CORR_ENOMEM if the second set cannot be allocated.
 */
int corr_readout_async(corr_handle_t* h, int32_t* vis_dev, void* copy_stream);
int corr_readout_host_async(corr_handle_t* h, int32_t* vis_host, void* copy_stream);

/*
 * corr_reset -- return the accumulators to the all-zero state without a
 * readout (Sec. II.A: a new integration starts). Host-side bookkeeping: the
 * handle's next call starts from zero (it stores instead of adding, after the
 * handle's last call as always); nothing is launched, and `stream` is not
 * used (NULL is fine).
 */
int corr_reset(corr_handle_t* h, void* stream);

/*
 * corr_accumulate_batch -- n frames of possibly different N, F, T in one
 * call: frame k (packed device bytes inputs[k]) is added to handle hs[k].
 * The frames' tiles share one persistent work list (Sec. II.C: tiles are
 * independent; Sec. IV: bands are independent), one correlator launch.
 * Handles must be distinct. A frame whose whole tiles (F x nb(nb+1)/2,
 * nb = ceil(N/64)) number at least CORR_BATCH_ALONE_WAVES per CTA slot of the
 * GPU (one per SM) fills the GPU on its own: it is launched alone, through the
 * single-frame kernel, before the shared launch, in frame order, on the same
 * stream. That holds for a frame of its handle's full T, and for one of fewer
 * samples (a time piece, corr_accumulate_batch_ex) where the handle's own
 * schedule keeps tiles whole (no time split). Results are the same either way.
 */
#define CORR_BATCH_ALONE_WAVES 4
int corr_accumulate_batch(corr_handle_t* const* hs, const uint8_t* const* inputs, int n, void* stream);

/*
 * corr_accumulate_batch_ex -- as corr_accumulate_batch, with frame k holding
 * Ts[k] samples (host array; 1 <= Ts[k]; NULL = each handle's T). Lets a
 * stream of frames of varying length share one handle's resident
 * accumulators (the sample cap counts the samples actually added).
 */
int corr_accumulate_batch_ex(corr_handle_t* const* hs, const uint8_t* const* inputs, const int32_t* Ts, int n,
                             void* stream);

/*
 * corr_shift_lags -- shift every element of a frame by its own integer
 * number of samples before correlation (Sec. IV: lags between elements, e.g.
 * unequal cable lengths, are created or compensated in software):
 *   out[t][f][i] = in[t - lags[i]][f][i]  when 0 <= t - lags[i] < T,
 *   out[t][f][i] = 0x88 (the code of 0 + 0i) otherwise.
 * in_dev, out_dev: distinct device frames uint8 [T][F][N]; out_dev 4-byte
 * aligned when N % 4 == 0. lags_dev: device int32 [N], any sign (a lag of T
 * or more in magnitude empties the element). Asynchronous on `stream`; the
 * caller keeps the buffers alive. Samples shifted past the frame's ends are
 * dropped (each frame is shifted on its own).
 */
int corr_shift_lags(const uint8_t* in_dev, uint8_t* out_dev, int32_t N, int32_t F, int32_t T, const int32_t* lags_dev,
                    void* stream);

/*
 * corr_set_option -- per-handle launch knobs (the autotuner's controls; the
 * results do not depend on them):
 *   CORR_OPT_PRODUCT: 0 = tensor cores for every sample, 1 = tensor cores and
 *     dp4a side by side (their shares: CORR_OPT_MMA_STEPS), 2 = as 1
 *     on the offset-encoded nibbles (unsigned operands, Sec. III.A's route):
 *     two extra kernels per call sum each element's nibbles over time and
 *     seed the output with the Eq. 3 offset terms (restated for the
 *     three-product form), and the correlator adds onto them; -1 = the
 *     library default (1 unless the XE_PRODUCT=mma environment variable is
 *     set). Batched and gated launches treat 2 as 1.
 *   CORR_OPT_SPLIT: 0 = automatic time split, k >= 1 = cut the time axis into
 *     k ranges (atomic adds when k > 1). Changing it rebuilds the handle's
 *     schedule, so the handle must be idle (its last call finished, e.g.
 *     after corr_synchronize): otherwise CORR_EBUSY and nothing changes.
 *   CORR_OPT_MMA_STEPS: for product paths 1 and 2, how many of every 8
 *     k-steps of 32 samples (two 128-sample chunks) run on the tensor cores,
 *     the rest on dp4a: 8 = tensor cores only, 7 (chunks alternate 128/0 and
 *     96/32), 6 (96/32 in every chunk), 5 (the default: alternate 64/64 and
 *     96/32), 4 (64/64). Shares 5 and 4 apply to off-diagonal tiles; diagonal
 *     tiles (bi == bj) keep 6. The two pipes run side by side on this GPU, so
 *     the share sets how the work is balanced between them. Single-frame calls
 *     (corr_accumulate, corr_accumulate_host) on product path 1 take every
 *     share; batched and gated calls and product path 2 take 8 or 6 (other
 *     values run as 6).
 * A batched launch takes its product path and share from its first handle.
 * Returns CORR_OK, CORR_EINVAL or CORR_EBUSY.
 */
#define CORR_OPT_PRODUCT 1
#define CORR_OPT_SPLIT 2
#define CORR_OPT_MMA_STEPS 3
int corr_set_option(corr_handle_t* h, int option, int64_t value);
int64_t corr_get_option(const corr_handle_t* h, int option);

/*
 * corr_accumulate_gated -- gated correlation of one frame (Sec. IV: the
 * products are binned by time into gates, for periodic signals such as
 * pulsars or calibration sources). Sample t of the frame belongs to gate
 *   g(t) = floor(((t + phase) mod period) * G / period)
 * and its products are added to gates[g]'s accumulators. gates: G distinct
 * handles with the same N and F (their T is not used); packed_dev: device
 * frame uint8 [T][F][N]; 1 <= period, 0 <= phase < period. Each maximal run
 * of samples in one gate is a segment; at most 2047 segments per call
 * (CORR_EINVAL beyond). Asynchronous on `stream`, one launch for all gates.
 */
int corr_accumulate_gated(corr_handle_t* const* gates, int G, const uint8_t* packed_dev, int32_t T, int32_t period,
                          int32_t phase, void* stream);

/* corr_synchronize -- wait (host) for the handle's last call, at most timeout_ms (<0: no limit);
 * library lifecycle, no counterpart in the paper. */
int corr_synchronize(corr_handle_t* h, int64_t timeout_ms);

/* corr_status -- CORR_OK or the handle's sticky error (CUDA failure or device fault report); library
 * lifecycle, no counterpart in the paper. Reads the device fault word with a copy ordered after the
 * handle's last call (it waits for that call to finish, but not for other work on other streams). */
int corr_status(corr_handle_t* h);

/* corr_samples -- samples accumulated since the last reset. */
int64_t corr_samples(const corr_handle_t* h);

/* corr_kernel_launches -- kernels this handle has launched so far (the library's own kernels only). */
int64_t corr_kernel_launches(const corr_handle_t* h);

/* corr_dims -- N, F, T of the handle (any pointer may be NULL). */
int corr_dims(const corr_handle_t* h, int32_t* N, int32_t* F, int32_t* T);

/* corr_last_error -- message for the calling thread's last failed call ("" if none). */
const char* corr_last_error(void);

/* corr_destroy -- wait for the handle's work, free what it owns. NULL is a no-op. Library lifecycle,
 * no counterpart in the paper. */
void corr_destroy(corr_handle_t* h);

/*
 * corr_plan_tiles -- host-only scheduler query (no CUDA calls): the number
 * of tiles covering the upper triangle of an N x N matrix with square tiles
 * of `tile` elements, nb(nb+1)/2 with nb = ceil(N / tile) (Sec. II.C,
 * Fig. 1). If bi_out/bj_out are non-NULL they receive the tile coordinates
 * in launch order (block rows bi <= block columns bj); cap bounds the
 * entries written. Returns the count, or CORR_EINVAL.
 */
int64_t corr_plan_tiles(int32_t N, int32_t tile, int32_t* bi_out, int32_t* bj_out, int64_t cap);

/*
 * corr_plan_schedule -- host-only scheduler query (no CUDA calls): the work
 * items the library launches for a frame of N, F, T on `ctas` resident CTAs.
 * Tiles are 64 x 64, band-major, row-major over each band's upper triangle
 * (Sec. II.C); time is cut into 128-sample chunks, and into `split` equal
 * ranges of chunks when whole tiles would leave the CTAs unbalanced. Item k
 * is {band f, bi | bj << 16, first chunk, end chunk} (4 int32 each in
 * items_out, at most items_cap items); CTA c runs items c, c + grid, ...
 * *grid_out (if non-NULL) receives the grid size. Returns the item count, or
 * CORR_EINVAL.
 */
int64_t corr_plan_schedule(int32_t N, int32_t F, int32_t T, int32_t ctas, int32_t* items_out, int64_t items_cap,
                           int32_t* grid_out);

/*
 * corr_effective_ops -- Eq. 2 per band and time step, times F*T:
 * 4*N*(N+1)*F*T, the "effective operations" of one frame.
 */
double corr_effective_ops(int32_t N, int32_t F, int32_t T);

/*
 * corr_correlate_noalloc -- correlate one frame without allocating anything.
 * (The paper has no counterpart.) It serves callers that cannot allocate
 * device memory at the moment they correlate: applications whose device
 * memory belongs to their own pool allocator, which must not have memory
 * taken behind its back, and real-time hosts that reserve every byte before
 * they start and forbid allocation on their processing path.
 *
 * packed_dev: device frame uint8 x[T][F][N] (layout above); N must be a
 *   multiple of 16 and the pointer 16-byte aligned (no staging copy here).
 * vis_dev: device output int32 [F][N(N+1)/2][2], overwritten with this
 *   frame's visibilities (a fresh integration: nothing is added to it).
 * status_dev: NULL, or a device int32 that receives 0, or a nonzero fault
 *   code if a bounded wait inside the kernel ran out.
 * The kernel's work list and fault word live in a fixed array of 65,536
 * work items (1 MiB) inside the library, which every GPU that loads the
 * library holds until the process exits. Frames with more than 65,536
 * tiles of 64 x 64 (N(N+1)/2-triangle tiles times F) return CORR_EINVAL
 * without launching anything. The call uses no cudaMalloc, cudaFree or other
 * allocating routine; on success it touches no allocator at all (a failure
 * records its message for corr_last_error). Asynchronous on `stream`.
 * The first call on each device, with that device current, looks up the
 * array's device address and sets the kernel's shared-memory limit; make
 * that first call before any stream capture. The address is kept for the
 * life of the process, so cudaDeviceReset must not be called while the
 * library is in use. All calls share the one array and each call rewrites
 * it (the fault word is cleared at the start of every call), so calls that
 * can overlap on the GPU (different streams, no ordering between them) race
 * and must not be issued; calls on one stream are safe.
 */
int corr_correlate_noalloc(const uint8_t* packed_dev, int32_t N, int32_t F, int32_t T, int32_t* vis_dev,
                           int32_t* status_dev, void* stream);

/*
 * corr_selftest_wait_timeout -- exercise the bounded device wait every kernel
 * of this library uses (no counterpart in the paper). One CTA waits on a
 * shared-memory barrier that nothing arrives on, polling at most `polls`
 * times (1 .. 2^20), then records that the wait ran out and returns; the
 * context stays usable. Synchronous on `stream`. Returns CORR_ETIMEOUT when
 * the wait ran out (the expected outcome), CORR_OK if it did not, CORR_EINVAL
 * for polls outside the range, CORR_ECUDA on a CUDA failure.
 */
int corr_selftest_wait_timeout(int32_t polls, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* XENGINE_H */
