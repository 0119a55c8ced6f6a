"""Autotuner: the launch knobs that run a frame shape fastest on this GPU.

Knobs (results never depend on them; see corr_set_option in include/xengine.h):
the product path (tensor cores + dp4a, tensor cores alone, or tensor cores +
dp4a on offset-encoded operands with the Eq. 3 corrections), the share of
each pair of 128-sample chunks that runs on the tensor cores (8, 7, 6, 5 or 4
of 8 k-steps of 32 samples, the rest on dp4a; each share is its own kernel
instantiation, built in), and the time split (automatic, or a fixed number
of ranges). For a frame shape (N, F, T)
the tuner times every candidate with CUDA events on random frames and keeps
the choice in a JSON cache keyed by the GPU and the shape, so a shape is
tuned once per GPU model. The choice is the first candidate, in preference
order (the library default first), within MARGIN of the fastest: candidates
within timing noise of each other do not flip it from one tuning run to the
next.
"""
from __future__ import annotations

import json
import os

from . import CORR_OPT_MMA_STEPS, CORR_OPT_PRODUCT, CORR_OPT_SPLIT, Correlator

CACHE_ENV = "XE_TUNE_CACHE"
# (product path, tensor-core k-steps of 8), in order of preference: tensor cores + dp4a at every share (the
# library default, 5, first), tensor cores alone, offset-encoded operands (Eq. 3)
PATHS = ((1, 5), (1, 6), (1, 7), (1, 4), (0, 8), (2, 6))
SPLITS = (0, 1, 2, 4)  # automatic, fixed
MARGIN = 0.01          # relative speed-up a candidate needs over the default


def cache_path() -> str:
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.expanduser("~"), ".cache", "xengine_tune.json")


def gpu_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm_{p.major}{p.minor}|{p.multi_processor_count}sm"


TUNER_VERSION = 2  # the candidate set and the kernels it chose among: entries of another version are not reused


def shape_key(N: int, F: int, T: int) -> str:
    return f"N{N}_F{F}_T{T}_v{TUNER_VERSION}"


def candidates(T: int):
    """(product, mma_steps, split) in trial order; the library default first."""
    nch = -(-T // 128)
    return [(p, m, s) for p, m in PATHS for s in SPLITS if s <= nch]


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def set_knobs(c: Correlator, product: int, mma_steps: int, split: int):
    c.set_option(CORR_OPT_PRODUCT, product)
    c.set_option(CORR_OPT_MMA_STEPS, mma_steps)
    c.set_option(CORR_OPT_SPLIT, split)


def time_config(c: Correlator, x, product: int, mma_steps: int, split: int, reps: int) -> float:
    """Median ms of one frame accumulate under (product, mma_steps, split)."""
    import torch
    torch.cuda.synchronize()  # the split option needs the handle idle
    set_knobs(c, product, mma_steps, split)
    for _ in range(2):
        c.reset()
        c.accumulate(x)
    torch.cuda.synchronize()
    ev = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c.reset()
        a.record()
        c.accumulate(x)
        b.record()
        ev.append((a, b))
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    return ms[len(ms) // 2]


def pick(trials: list[dict]) -> dict:
    """The first trial, in preference order (the library default first, each path's automatic time
    split before its fixed ones), within MARGIN of the fastest: candidates within timing noise of each
    other do not flip the choice from one tuning run to the next."""
    best = min(d["ms"] for d in trials)
    return next(d for d in trials if d["ms"] <= best * (1.0 + MARGIN))


def tune(N: int, F: int, T: int, reps: int = 5, path: str | None = None, force: bool = False) -> dict:
    """Time every candidate for (N, F, T) and cache the fastest; returns the cache entry."""
    import torch
    cache = load_cache(path)
    g, k = gpu_key(), shape_key(N, F, T)
    if not force and k in cache.get(g, {}):
        return cache[g][k]
    x = torch.randint(0, 256, (T, F, N), dtype=torch.uint8, device="cuda")
    trials = []
    with Correlator(N, F, T) as c:
        for product, mma_steps, split in candidates(T):
            ms = time_config(c, x, product, mma_steps, split, reps)
            trials.append({"product": product, "mma_steps": mma_steps, "split": split, "ms": round(ms, 4)})
    best = pick(trials)
    entry = {"product": best["product"], "mma_steps": best["mma_steps"], "split": best["split"], "ms": best["ms"],
             "trials": trials}
    cache = load_cache(path)  # re-read: another process may have written meanwhile
    cache.setdefault(g, {})[k] = entry
    save_cache(cache, path)
    return entry


def apply(c: Correlator, path: str | None = None, tune_if_missing: bool = True) -> dict | None:
    """Set a correlator's knobs from the cache (tuning its shape first if it is missing)."""
    cache = load_cache(path)
    entry = cache.get(gpu_key(), {}).get(shape_key(c.N, c.F, c.T))
    if entry is None and tune_if_missing:
        entry = tune(c.N, c.F, c.T, path=path)
    if entry is not None:
        set_knobs(c, entry["product"], entry.get("mma_steps", 6), entry["split"])
    return entry
