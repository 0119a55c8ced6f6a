"""CPU oracle for the 4-bit X-engine -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The GPU library never calls it and
shares no code with it.

What it computes is the plain definition (Eq. 1 accumulated over time, the
upper triangle of Sec. II.A, the excess-8 decoding of Sec. III), in C with
int64 accumulators: see ``xcorr_oracle.c``. Parity status: pinned (the
``tests/test_oracle_*.py`` pins: hand-worked cases, brute force with Python
complex numbers, a numpy matmul special case, Hermitian symmetry, autos,
the identical-sequence closed form, the Freivalds identity, the Eq. 3
identity, and the lag-shift pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xcorr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library with plain gcc flags."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        for name in ("oracle_visibilities", "oracle_visibilities_full"):
            fn = getattr(lib, name)
            fn.argtypes = [vp, i64, i64, i64, vp, ci]
            fn.restype = ci
        lib.oracle_entries.argtypes = [vp, i64, i64, i64, vp, i64, vp, ci]
        lib.oracle_entries.restype = ci
        lib.oracle_freivalds_rhs.argtypes = [vp, i64, i64, i64, vp, vp]
        lib.oracle_freivalds_rhs.restype = ci
        lib.oracle_offset_terms.argtypes = [vp, i64, i64, i64, vp]
        lib.oracle_offset_terms.restype = ci
        lib.oracle_shift_lags.argtypes = [vp, i64, i64, i64, vp, vp]
        lib.oracle_shift_lags.restype = ci
        lib.oracle_gated.argtypes = [vp, i64, i64, i64, i64, i64, i64, vp]
        lib.oracle_gated.restype = ci
        _lib = lib
    return _lib


def threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _check_x(x: np.ndarray):
    if x.dtype != np.uint8 or x.ndim != 3 or not x.flags.c_contiguous:
        raise ValueError("x must be a C-contiguous uint8 array [T][F][N]")
    T, F, N = x.shape
    return N, F, T


def baselines(N: int) -> int:
    """Number of upper-triangle entries, autos included (Eq. 2's N(N+1)/2)."""
    return N * (N + 1) // 2


def packed_index(N: int, i, j):
    """Row-major upper-triangle position of (i, j), i <= j."""
    return i * N - i * (i - 1) // 2 + (j - i)


def visibilities(x: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """Packed upper triangle, int64 [F][N(N+1)/2][2] (Re, Im)."""
    N, F, T = _check_x(x)
    V = np.empty((F, baselines(N), 2), dtype=np.int64)
    rc = _load().oracle_visibilities(x.ctypes.data, N, F, T, V.ctypes.data, nthreads or threads())
    if rc != 0:
        raise RuntimeError(f"oracle_visibilities failed ({rc})")
    return V


def visibilities_full(x: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """Every ordered pair, int64 [F][N][N][2] (small N only)."""
    N, F, T = _check_x(x)
    V = np.empty((F, N, N, 2), dtype=np.int64)
    rc = _load().oracle_visibilities_full(x.ctypes.data, N, F, T, V.ctypes.data, nthreads or threads())
    if rc != 0:
        raise RuntimeError(f"oracle_visibilities_full failed ({rc})")
    return V


def entries(x: np.ndarray, fij: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """Single visibilities V[f,i,j] for rows of fij (int64 [K][3]); returns int64 [K][2]."""
    N, F, T = _check_x(x)
    fij = np.ascontiguousarray(fij, dtype=np.int64).reshape(-1, 3)
    out = np.empty((fij.shape[0], 2), dtype=np.int64)
    rc = _load().oracle_entries(x.ctypes.data, N, F, T, fij.ctypes.data, fij.shape[0], out.ctypes.data,
                                nthreads or threads())
    if rc != 0:
        raise RuntimeError(f"oracle_entries failed ({rc})")
    return out


def freivalds_rhs(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_t x_i * sum_j conj(x_j) w_j per band: int64 [F][N][2] for complex weights w int64 [F][N][2]."""
    N, F, T = _check_x(x)
    w = np.ascontiguousarray(w, dtype=np.int64)
    assert w.shape == (F, N, 2)
    r = np.empty((F, N, 2), dtype=np.int64)
    rc = _load().oracle_freivalds_rhs(x.ctypes.data, N, F, T, w.ctypes.data, r.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_freivalds_rhs failed ({rc})")
    return r


def offset_terms(x: np.ndarray) -> np.ndarray:
    """Eq. 3 offsets for encoded-value products, packed like visibilities(): int64 [F][B][2]."""
    N, F, T = _check_x(x)
    out = np.empty((F, baselines(N), 2), dtype=np.int64)
    rc = _load().oracle_offset_terms(x.ctypes.data, N, F, T, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_offset_terms failed ({rc})")
    return out


def shift_lags(x: np.ndarray, lags) -> np.ndarray:
    """Per-element time shift (Sec. IV): out[t,f,i] = x[t - lag_i, f, i], zero (0x88) outside the frame."""
    N, F, T = _check_x(x)
    lags = np.ascontiguousarray(lags, dtype=np.int32)
    assert lags.shape == (N,)
    out = np.empty_like(x)
    rc = _load().oracle_shift_lags(x.ctypes.data, N, F, T, lags.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_shift_lags failed ({rc})")
    return out


def gated(x: np.ndarray, G: int, period: int, phase: int = 0) -> np.ndarray:
    """Gated visibilities (Sec. IV), int64 [G][F][B][2]; gate(t) = ((t + phase) % period) * G // period."""
    N, F, T = _check_x(x)
    V = np.empty((G, F, baselines(N), 2), dtype=np.int64)
    rc = _load().oracle_gated(x.ctypes.data, N, F, T, G, period, phase, V.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_gated failed ({rc})")
    return V


def timed_visibilities(x: np.ndarray, nthreads: int | None = None):
    """(V, seconds, threads) -- the oracle as it stands, wall-clock timed."""
    n = nthreads or threads()
    t0 = time.perf_counter()
    V = visibilities(x, n)
    return V, time.perf_counter() - t0, n
