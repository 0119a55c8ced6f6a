"""GB300-native 4-bit X-engine (after arXiv:1503.06203).

Python face of the C ABI in ``include/xengine.h``. Every step of the
correlation runs in the CUDA library; this module only passes pointers,
sizes and streams. PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (CORR_BATCH_ALONE_WAVES, CORR_EINVAL, CORR_EOVERFLOW, CORR_ETIMEOUT, CORR_MAX_N, CORR_MAX_SAMPLES,
                   CORR_OK, CORR_OPT_MMA_STEPS, CORR_OPT_PRODUCT, CORR_OPT_SPLIT, XEngineError, check, last_error, lib)

__all__ = ["Correlator", "accumulate_batch", "plan_tiles", "effective_ops", "baselines", "packed_index",
           "plan_schedule", "correlate_noalloc", "selftest_wait_timeout", "shift_lags", "accumulate_gated",
           "band_range", "CORR_OPT_PRODUCT", "CORR_OPT_SPLIT", "CORR_OPT_MMA_STEPS", "XEngineError", "CORR_MAX_SAMPLES", "CORR_MAX_N",
           "CORR_BATCH_ALONE_WAVES", "batch_runs_alone",
           "build", "last_error"]


def build(force: bool = False) -> str:
    from .builder import build as _b
    return _b(force=force)


def baselines(N: int) -> int:
    """Entries of the packed upper triangle, autos included: N(N+1)/2."""
    return N * (N + 1) // 2


def packed_index(N: int, i, j):
    """Row-major upper-triangle position p(i, j) = i*N - i*(i-1)/2 + (j - i), i <= j."""
    return i * N - i * (i - 1) // 2 + (j - i)


def effective_ops(N: int, F: int, T: int) -> float:
    """Eq. 2 operations per band and sample times F*T: 4 N (N+1) F T."""
    return float(lib().corr_effective_ops(N, F, T))


def plan_tiles(N: int, tile: int):
    """(bi, bj) block coordinates of the upper-triangle tiles in launch order."""
    L = lib()
    n = L.corr_plan_tiles(N, tile, None, None, 0)
    if n < 0:
        raise XEngineError(int(n), last_error())
    bi = np.empty(n, dtype=np.int32)
    bj = np.empty(n, dtype=np.int32)
    L.corr_plan_tiles(N, tile, bi.ctypes.data, bj.ctypes.data, n)
    return bi, bj


def plan_schedule(N: int, F: int, T: int, ctas: int):
    """(items int32 [K][4] = {f, bi | bj << 16, c0, c1}, grid) the library launches; CTA c runs items c, c+grid, ..."""
    L = lib()
    n = L.corr_plan_schedule(N, F, T, ctas, None, 0, None)
    if n < 0:
        raise XEngineError(int(n), last_error())
    items = np.empty((n, 4), dtype=np.int32)
    grid = ctypes.c_int32()
    L.corr_plan_schedule(N, F, T, ctas, items.ctypes.data, n, ctypes.byref(grid))
    return items, grid.value


def band_range(rank: int, world: int, F: int):
    """Bands [f0, f1) of rank `rank` of `world` when F independent bands are split across GPUs (Sec. I, Sec. IV).

    Contiguous ranges in rank order, sizes differing by at most one; every band
    belongs to exactly one rank. A rank beyond F gets an empty range (f0 == f1).
    """
    if not (0 <= rank < world) or F < 1:
        raise ValueError(f"bad partition: rank {rank} of {world}, F={F}")
    base, extra = divmod(F, world)
    f0 = rank * base + min(rank, extra)
    return f0, f0 + base + (1 if rank < extra else 0)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Correlator:
    """A handle: resident int32 accumulators for frames of N elements, F bands, T samples.

    With bands=(f0, f1) the handle correlates only bands [f0, f1) of frames that
    hold F bands (corr_create_bands): frames passed to it are [T][F][N], its
    visibilities are [f1 - f0][N(N+1)/2][2], and self.F is f1 - f0 (self.F_in = F).
    """

    def __init__(self, N: int, F: int, T: int, acc=None, bands=None):
        L = lib()
        self._acc = acc  # keep a caller-owned tensor alive
        self.F_in, self.f0 = F, 0
        if bands is not None:
            if acc is not None:
                raise ValueError("a band-range handle owns its accumulators")
            f0, f1 = bands
            h = L.corr_create_bands(N, F, f0, f1, T)
            self.F_in, self.f0, F = F, f0, f1 - f0
        elif acc is None:
            h = L.corr_create(N, F, T)
        else:
            import torch
            assert acc.is_cuda and acc.dtype == torch.int32 and acc.is_contiguous()
            assert acc.numel() == F * baselines(N) * 2
            h = L.corr_create_ex(N, F, T, ctypes.c_void_p(acc.data_ptr()))
        if not h:
            raise XEngineError(CORR_EINVAL, last_error())
        self._h = ctypes.c_void_p(h)
        self.N, self.F, self.T = N, F, T

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            lib().corr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls --
    def _check_frame(self, x):
        if tuple(x.shape) != (self.T, self.F_in, self.N):
            raise ValueError(f"frame shape {tuple(x.shape)} != (T, F, N) = {(self.T, self.F_in, self.N)}")

    def accumulate(self, x, stream=None):
        """Add a device frame (torch uint8 [T][F][N], contiguous) to the accumulators."""
        import torch
        self._check_frame(x)
        if not (x.is_cuda and x.dtype == torch.uint8 and x.is_contiguous()):
            raise ValueError("accumulate expects a contiguous CUDA uint8 tensor")
        check(lib().corr_accumulate(self._h, ctypes.c_void_p(x.data_ptr()), _stream_ptr(stream)))

    def accumulate_host(self, x, stream=None):
        """Add a host frame (numpy uint8 or a CPU torch tensor, ideally pinned): copies overlap compute."""
        self._check_frame(x)
        ptr = x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
        check(lib().corr_accumulate_host(self._h, ctypes.c_void_p(ptr), _stream_ptr(stream)))

    def readout(self, out=None, reset: bool = False, stream=None):
        """Packed visibilities int32 [F][N(N+1)/2][2] into a device tensor (allocated if None)."""
        import torch
        if out is None:
            out = torch.empty((self.F, baselines(self.N), 2), dtype=torch.int32, device="cuda")
        assert out.is_cuda and out.dtype == torch.int32 and out.is_contiguous()
        assert out.numel() == self.F * baselines(self.N) * 2
        check(lib().corr_readout(self._h, ctypes.c_void_p(out.data_ptr()), int(reset), _stream_ptr(stream)))
        return out

    def readout_host(self, out, reset: bool = False, stream=None):
        """Packed visibilities into host memory (numpy int32 or CPU torch tensor, ideally pinned)."""
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
        check(lib().corr_readout_host(self._h, ctypes.c_void_p(ptr), int(reset), _stream_ptr(stream)))
        return out

    def readout_async(self, out, copy_stream):
        """End the integration; copy it into `out` (CUDA or host int32 [F][N(N+1)/2][2]) on copy_stream,
        overlapped with the next integration (a second accumulator set). Synchronise copy_stream before
        reading `out`."""
        import torch
        assert out.dtype == torch.int32 and out.is_contiguous() and out.numel() == self.F * baselines(self.N) * 2
        fn = lib().corr_readout_async if out.is_cuda else lib().corr_readout_host_async
        check(fn(self._h, ctypes.c_void_p(out.data_ptr()), _stream_ptr(copy_stream)))
        return out

    def reset(self, stream=None):
        # (the library orders a reset by the handle's own last call; the stream is passed through as given)
        check(lib().corr_reset(self._h, None if stream is None else _stream_ptr(stream)))

    def synchronize(self, timeout_ms: int = -1):
        check(lib().corr_synchronize(self._h, timeout_ms))

    def status(self) -> int:
        return int(lib().corr_status(self._h))

    @property
    def samples(self) -> int:
        return int(lib().corr_samples(self._h))

    def set_option(self, option: int, value: int):
        """Launch knobs (results never depend on them): CORR_OPT_PRODUCT, CORR_OPT_SPLIT, CORR_OPT_MMA_STEPS."""
        check(lib().corr_set_option(self._h, option, int(value)))

    def get_option(self, option: int) -> int:
        return int(lib().corr_get_option(self._h, option))

    @property
    def kernel_launches(self) -> int:
        return int(lib().corr_kernel_launches(self._h))

    @property
    def handle(self):
        return self._h


def shift_lags(x, lags, out=None, stream=None):
    """Per-element time shift before correlation (Sec. IV): out[t,f,i] = x[t - lags[i], f, i], zero outside.

    x: CUDA uint8 [T][F][N]; lags: CUDA int32 [N]; returns `out` (allocated if None).
    """
    import torch
    if not (x.is_cuda and x.dtype == torch.uint8 and x.dim() == 3 and x.is_contiguous()):
        raise ValueError("x must be a contiguous CUDA uint8 tensor [T][F][N]")
    T, F, N = x.shape
    if out is None:
        out = torch.empty_like(x)
    if not (out.is_cuda and out.dtype == torch.uint8 and out.shape == x.shape and out.is_contiguous()):
        raise ValueError("out must be a contiguous CUDA uint8 tensor shaped like x")
    assert lags.is_cuda and lags.dtype == torch.int32 and lags.numel() == N and lags.is_contiguous()
    check(lib().corr_shift_lags(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), N, F, T,
                                ctypes.c_void_p(lags.data_ptr()), _stream_ptr(stream)))
    return out


def accumulate_gated(gates, x, period: int, phase: int = 0, stream=None):
    """Gated correlation (Sec. IV): sample t of frame x goes to gates[((t + phase) % period) * G // period]."""
    G = len(gates)
    T, F, N = x.shape
    for c in gates:
        if (c.N, c.F_in) != (N, F):
            raise ValueError("gate correlators must match the frame's N and F")
    hs = (ctypes.c_void_p * G)(*[c._h.value for c in gates])
    check(lib().corr_accumulate_gated(hs, G, ctypes.c_void_p(x.data_ptr()), T, period, phase, _stream_ptr(stream)))


def correlate_noalloc(x, out, status=None, stream=None):
    """One frame into `out` (int32 [F][N(N+1)/2][2], overwritten) with no allocation by the library.

    For callers that cannot allocate device memory at call time (an
    application's own pool allocator owns the memory, or a real-time host
    forbids allocation on its processing path): the work list lives in a
    fixed 1 MiB array inside the library. `x` is a contiguous CUDA uint8 [T][F][N]
    tensor with N a multiple of 16; `status`, if given, is a CUDA int32 tensor
    that receives the kernel's fault word (0 = no fault). Calls that may overlap
    on the GPU race on the shared array; keep them on one stream.
    """
    T, F, N = x.shape
    check(lib().corr_correlate_noalloc(ctypes.c_void_p(x.data_ptr()), N, F, T, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(status.data_ptr()) if status is not None else None,
                                       _stream_ptr(stream)))
    return out


def selftest_wait_timeout(polls: int = 4096, stream=None) -> int:
    """Run the library's bounded device wait on a barrier nothing arrives on; returns the status code
    (CORR_ETIMEOUT expected). The context stays usable afterwards."""
    return int(lib().corr_selftest_wait_timeout(int(polls), _stream_ptr(stream)))


def accumulate_batch(correlators, inputs, stream=None):
    """Several frames in one call: inputs[k] (device uint8 [T_k][F][N]) is added to correlators[k].

    The frames share one batched launch, except that a frame which fills the GPU
    on its own (batch_runs_alone) is launched alone first, through the
    single-frame kernel. T_k may differ from the correlator's T (frames of
    varying length); the correlators must be distinct.
    """
    n = len(correlators)
    assert len(inputs) == n
    shapes = [x.shape for x in inputs]
    for c, x, sh in zip(correlators, inputs, shapes):
        if len(sh) != 3 or sh[1] != c.F_in or sh[2] != c.N or not x.is_contiguous():
            raise ValueError(f"frame shape {tuple(sh)} does not fit (T, F, N) with F={c.F}, N={c.N}")
    hs = (ctypes.c_void_p * n)(*[c._h.value for c in correlators])
    xs = (ctypes.c_void_p * n)(*[x.data_ptr() for x in inputs])
    Ts = (ctypes.c_int32 * n)(*[sh[0] for sh in shapes])
    check(lib().corr_accumulate_batch_ex(hs, xs, Ts, n, _stream_ptr(stream)))


def batch_runs_alone(N: int, F: int, sms: int) -> bool:
    """Whether accumulate_batch launches a frame of its correlator's full T alone (single-frame kernel):
    its whole 64 x 64 tiles number at least CORR_BATCH_ALONE_WAVES per SM. A shorter frame (a time
    piece) of such a correlator also runs alone where the correlator's schedule keeps tiles whole."""
    nb = -(-N // 64)
    return nb * (nb + 1) // 2 * F >= CORR_BATCH_ALONE_WAVES * sms
