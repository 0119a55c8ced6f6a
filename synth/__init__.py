"""Seeded synthetic inputs for the 4-bit X-engine.

This package only makes input bytes (it holds none of the correlator's
arithmetic). The CPU oracle and the GPU library both consume what it makes.

Format (Sec. III and Fig. 2 of the paper): ``uint8[T][F][N]``, one byte per
complex sample, excess-8 parts (value + 8 in [0, 15]), high nibble = real,
low nibble = imaginary.

The fast path is a small C library (``synth.c``, pthreads); ``*_np`` are
pure-numpy restatements of the same recipe used to cross-check it on small
sizes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_libsynth.so")
_lib = None

GAMMA = np.uint64(0x9E3779B97F4A7C15)


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (gcc, no -march flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_uniform.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_uint64, ctypes.c_int]
        lib.synth_uniform.restype = ctypes.c_int
        lib.synth_gauss.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
        lib.synth_gauss.restype = ctypes.c_int
        lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_draw.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _out(N, F, T, out):
    if out is None:
        out = np.empty((T, F, N), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.shape == (T, F, N) and out.flags.c_contiguous
    return out


def uniform(N: int, F: int, T: int, seed: int, nthreads: int | None = None, out=None) -> np.ndarray:
    """Uniform nibbles: byte (t,f,n) = top 8 bits of draw ((t*F+f)*N+n)."""
    out = _out(N, F, T, out)
    rc = _load().synth_uniform(out.ctypes.data, N, F, T, seed, nthreads or default_threads())
    if rc != 0:
        raise RuntimeError("synth_uniform failed")
    return out


def gauss(N: int, F: int, T: int, sigma: float, seed: int, tone_amp: float = 0.0, tone_k: float = 0.0,
          nthreads: int | None = None, out=None) -> np.ndarray:
    """Gaussian levels clip(rint(sigma*z + tone), -8, 7) per part, optional common tone."""
    out = _out(N, F, T, out)
    rc = _load().synth_gauss(out.ctypes.data, N, F, T, float(sigma), float(tone_amp), float(tone_k), seed,
                             nthreads or default_threads())
    if rc != 0:
        raise RuntimeError("synth_gauss failed")
    return out


def gauss_flat(nbytes: int, sigma: float, seed: int, nthreads: int | None = None) -> np.ndarray:
    """`nbytes` Gaussian-level bytes as one flat array, the same bytes as gauss(nbytes, 1, 1, ...).

    The generator is counter-based on the flat index, so any [T][1][N] shape of
    the same size gives the same bytes; generating many rows lets every thread
    take a share (threads split the rows).
    """
    rows = 1
    while rows < 8192 and nbytes % (2 * rows) == 0:
        rows *= 2
    return gauss(nbytes // rows, 1, rows, sigma, seed, nthreads=nthreads).reshape(-1)


def draw(seed: int, c: int) -> int:
    """Draw number c of the SplitMix64 stream seeded with `seed` (C implementation)."""
    return int(_load().synth_draw(seed, c))


# ----------------------------------------------------------------------------
# pure-numpy restatement (small sizes only; cross-checks the C library)
# ----------------------------------------------------------------------------

def draw_np(seed: int, c: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c.astype(np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_np(N: int, F: int, T: int, seed: int) -> np.ndarray:
    c = np.arange(T * F * N, dtype=np.uint64)
    return (draw_np(seed, c) >> np.uint64(56)).astype(np.uint8).reshape(T, F, N)


def gauss_np(N: int, F: int, T: int, sigma: float, seed: int, tone_amp: float = 0.0, tone_k: float = 0.0):
    c = np.arange(T * F * N, dtype=np.uint64)
    r1 = draw_np(seed, 2 * c)
    r2 = draw_np(seed, 2 * c + np.uint64(1))
    u1 = ((r1 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (r2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    zr = rad * np.cos(2 * np.pi * u2)
    zi = rad * np.sin(2 * np.pi * u2)
    t = (np.arange(T * F * N) // (F * N)).astype(np.float64)
    if tone_amp != 0.0:
        th = 2 * np.pi * tone_k * t / T
        tr, ti = tone_amp * np.cos(th), tone_amp * np.sin(th)
    else:
        tr = ti = 0.0
    re = np.clip(np.rint(sigma * zr + tr), -8, 7).astype(np.int64)
    im = np.clip(np.rint(sigma * zi + ti), -8, 7).astype(np.int64)
    return (((re + 8) << 4) | (im + 8)).astype(np.uint8).reshape(T, F, N)


# ----------------------------------------------------------------------------
# workload recipes (shapes of the paper's workloads: Pathfinder N=256, large N)
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Frame:
    """One correlation frame: N elements, F bands, T samples and its generator recipe."""
    N: int
    F: int
    T: int
    kind: str = "gauss"      # "uniform" or "gauss"
    sigma: float = 2.5
    seed: int = 0
    tone_amp: float = 0.0
    tone_k: float = 0.0

    @property
    def nbytes(self) -> int:
        return self.N * self.F * self.T

    def make(self, nthreads: int | None = None, out=None) -> np.ndarray:
        if self.kind == "uniform":
            return uniform(self.N, self.F, self.T, self.seed, nthreads, out)
        return gauss(self.N, self.F, self.T, self.sigma, self.seed, self.tone_amp, self.tone_k, nthreads, out)


TONE_K = 37  # tone bin of the large-N workload's common tone
TINY = Frame(16, 4, 256, "uniform", seed=1000)                      # tiny: uniform nibbles
PATHFINDER = Frame(256, 256, 16384, "gauss", 2.5, 1001)             # N=256 (128 dual-pol feeds)
LARGE_N = Frame(8192, 4, 2048, "gauss", 2.5, 1002, 3.0, TONE_K)     # noise + common tone
LARGE_N_TONE_ONLY = Frame(8192, 4, 2048, "gauss", 0.0, 1002, 3.0, TONE_K)

BATCH_N_CHOICES = (64, 128, 256, 512, 1024, 2048)


def batched_frames(count: int = 64, seed: int = 1003) -> list[Frame]:
    """Uneven frames: N from BATCH_N_CHOICES, F in 1..64, T in 512..8192 (multiple of 256), sigma in [1.5, 3.5].

    Frame k's parameters come from draws 4k..4k+3 of stream `seed`; its samples from stream seed*1000+k.
    """
    frames = []
    for k in range(count):
        d = [draw(seed, 4 * k + i) for i in range(4)]
        N = BATCH_N_CHOICES[d[0] % len(BATCH_N_CHOICES)]
        F = 1 + d[1] % 64
        T = 256 * (2 + d[2] % 31)
        sigma = 1.5 + 2.0 * (d[3] >> 11) * 2.0 ** -53
        frames.append(Frame(N, F, T, "gauss", sigma, seed * 1000 + k))
    return frames


SMALL_N_CHOICES = (64, 128, 256)


def small_frames(count: int = 64, seed: int = 1005) -> list[Frame]:
    """Small uneven frames: N from SMALL_N_CHOICES, F in 1..8, T in 512..1024 (multiple of 256), sigma in [1.5, 3.5].

    Each frame alone is microseconds of work, too little to fill the GPU: the case batching is for.
    Frame k's parameters come from draws 4k..4k+3 of stream `seed`; its samples from stream seed*1000+k.
    """
    frames = []
    for k in range(count):
        d = [draw(seed, 4 * k + i) for i in range(4)]
        N = SMALL_N_CHOICES[d[0] % len(SMALL_N_CHOICES)]
        F = 1 + d[1] % 8
        T = 256 * (2 + d[2] % 3)
        sigma = 1.5 + 2.0 * (d[3] >> 11) * 2.0 ** -53
        frames.append(Frame(N, F, T, "gauss", sigma, seed * 1000 + k))
    return frames
