#!/usr/bin/env python
"""Benchmark of the GB300 4-bit X-engine: effective TOPS on one correlation frame, with the
other workloads of the hot path as sub-records of the same line.

One step = one pass of the whole hot path over one frame of synthetic
4-bit input already resident in HBM: TMA staging, unpack, Hermitian
product, upper-triangle scheduling and the packed-triangle write of the
visibilities (a fresh integration each step). The headline workload is the
Pathfinder shape, N=256 elements, F=256 bands, T=16384 samples per
integration (1 GiB of input, larger than L2, so no flush is needed).

Effective operations follow Eq. 2 of the paper: 4 N (N+1) F T per frame.

The default single-GPU run adds, in the same JSON line:
  large_n     the N=8192, F=4, T=2048 frame (roofline, CPU-oracle sample, e2e);
  batched     64 uneven frames: one batched launch per step vs one launch per frame;
  served      32 served streams, Poisson arrivals at 10, 40 and 80 frames/s:
              continuous batching vs one frame per launch (frames/s, p50/p99);
  lags_gates  the Sec. IV lag shift (GB/s vs HBM) and gated correlation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xengine|reference] [--split frames|bands]

Under torchrun (N > 1) there is no collective on the data path: with
--split frames (the default) every rank correlates its own frame (weak
scaling); with --split bands the ranks share one frame and each correlates
its range of bands (strong scaling; bands are independent, Sec. I and IV).
The value is all ranks' operations over the slowest rank's time.
``--impl reference`` times the CPU oracle (the plain definition) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "pathfinder": ("PATHFINDER", "Pathfinder shape N=256 F=256 T=16384, Gaussian sigma=2.5 levels, one frame per launch"),
    "large_n": ("LARGE_N", "large N: N=8192 F=4 T=2048, sigma=2.5 plus a common tone, one frame per launch"),
}
EXTRA_WORKLOADS = ("batched", "batched_small", "served", "lags_gates")
KERNEL_NAME = "corr_tile_kernel"
KERNEL_SOURCES = ["paper_1503_06203_gb300/csrc/xe_corr.cuh", "paper_1503_06203_gb300/csrc/xe_ptx.cuh"]
TRAFFIC_FILES = {"pathfinder": os.path.join(ROOT, "profiles", "corr_tile_kernel_pathfinder.md"),
                 "large_n": os.path.join(ROOT, "profiles", "corr_tile_kernel_large_n.md")}
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SERVED_RATES = "10,40,80"


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["xengine", "reference"], default="xengine")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + list(EXTRA_WORKLOADS), default="pathfinder")
    ap.add_argument("--split", choices=["frames", "bands"], default="frames",
                    help="N > 1: each rank its own frame (weak scaling) or its bands of one frame (strong scaling)")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only (no sub-records)")
    ap.add_argument("--rates", default=SERVED_RATES, help="served: Poisson arrival rates (frames/s) to sweep")
    ap.add_argument("--served-frames", type=int, default=0, help="served: frames per rate (0: about 6 s of arrivals)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default launch knobs (profiling runs)")
    ap.add_argument("--product", type=int, choices=[0, 1, 2], default=None,
                    help="force the product path (0 tensor cores, 1 tensor cores + dp4a, 2 offset-encoded operands)")
    ap.add_argument("--mma-steps", type=int, choices=[4, 5, 6, 7, 8], default=None,
                    help="force the tensor-core share: k-steps of every 8 on the tensor cores, the rest on dp4a")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the GPU works."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="xe_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [s.strip() for s in line.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ----------------------------------------------------------------------------- roofline helpers
def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def effective_split(N: int, F: int, T: int, split: int, ctas: int) -> int:
    """The time split a launch actually uses (0 = the library's automatic choice for this shape)."""
    if split > 0:
        return min(split, -(-T // 128))
    import paper_1503_06203_gb300 as xe
    items, _ = xe.plan_schedule(N, F, T, ctas)
    nb = -(-N // 64)
    return len(items) // (nb * (nb + 1) // 2 * F)


def recorded_traffic(workload: str, product: int, split: int, mma_steps: int):
    """DRAM bytes per launch from the committed ncu summary of this workload, if taken on the current
    kernel source with the same launch knobs (a time split changes the writers' traffic; `split` is the
    effective split, see effective_split)."""
    path = TRAFFIC_FILES.get(workload)
    if not path or not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_source_hash() or vals.get("workload") != workload:
        return None
    if vals.get("options") != f"product={product} split={split} mma_steps={mma_steps}":
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def hardware_ops(N: int, F: int, T: int) -> float:
    """Tensor-core operations one launch issues (2 per int8 multiply-add).

    64x64 tiles of 2x2 warps of 32x32; each warp runs 2x4 m16n8k32 MMAs per
    product per 32 samples, three products (P1, P2, Q). On diagonal tiles the
    warp below the diagonal is idle and the two on it skip 2 of 8 sub-tiles:
    20 of 32 sub-tiles run.
    """
    nb = -(-N // 64)
    off, diag = nb * (nb - 1) // 2, nb
    ksteps = -(-T // 32)
    mmas = F * (off * 32 + diag * 20) * 3 * ksteps
    return mmas * 2.0 * 16 * 8 * 32


def measured_peaks_file():
    try:
        with open(MEASURED_PEAKS) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


# ----------------------------------------------------------------------------- CPU oracle leg
def int_mm_rate(n: int = 8192, reps: int = 5) -> float:
    """int8 x int8 -> int32 GEMM rate of the vendor library (torch._int_mm, n^3), in operations/s."""
    import torch
    a = torch.randint(-8, 8, (n, n), dtype=torch.int8, device="cuda")
    b = torch.randint(-8, 8, (n, n), dtype=torch.int8, device="cuda")
    for _ in range(2):
        torch._int_mm(a, b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        torch._int_mm(a, b)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del a, b
    return 2.0 * n ** 3 / (ms * 1e-3)


def cpu_oracle_sample(frame, x, target_s: float, per_band_s: float | None = None, bands: int | None = None):
    """Time the CPU oracle as it stands on a bounded sample: the first F_s bands of the frame.

    F_s is `bands` if given, else chosen so the sample takes about target_s (from per_band_s,
    measured on up to 2 bands if None).
    Returns (effective TOPS, cores, sample description, seconds, per-band seconds).
    """
    import numpy as np

    import oracle

    n = oracle.threads()
    if bands is not None:
        F_s = int(max(1, min(frame.F, bands)))
    else:
        if per_band_s is None:
            F_cal = max(1, min(frame.F, 2))
            _, t_cal, _ = oracle.timed_visibilities(np.ascontiguousarray(x[:, :F_cal, :]), n)
            per_band_s = max(t_cal / F_cal, 1e-6)
        F_s = int(max(1, min(frame.F, round(target_s / per_band_s))))
    xs = np.ascontiguousarray(x[:, :F_s, :])
    _, t, n = oracle.timed_visibilities(xs, n)
    ops = 4.0 * frame.N * (frame.N + 1) * F_s * frame.T
    desc = f"first {F_s} of {frame.F} bands of the N={frame.N} T={frame.T} frame ({ops / 1e12:.4f}e12 effective ops)"
    return ops / t / 1e12, n, desc, t, t / F_s


def run_reference(args, wl_key):
    """The oracle arm: rank 0 times the plain CPU definition; other ranks exit without work."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import synth
    frame = getattr(synth, WORKLOADS[wl_key][0])
    x = frame.make()
    # each step: a bounded sample (a few bands) sized so warm-up + steps stay within minutes
    per_step_target = max(0.5, min(10.0, 120.0 / max(1, args.steps + args.warmup)))
    vals, tsum, cores, desc, per_band = [], 0.0, 1, "", None
    for k in range(args.warmup + args.steps):
        v, cores, desc, t, per_band = cpu_oracle_sample(frame, x, per_step_target, per_band)
        if k >= args.warmup:
            vals.append(v)
            tsum += t
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "Effective TOPS", "value": round(value, 6), "unit": "TOPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tsum / max(1, len(vals)), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64 (oracle)", "data": "synthetic (seeded, paper's shapes)",
        "config": {"workload": WORKLOADS[wl_key][1], "N": frame.N, "F": frame.F, "T": frame.T,
                   "per_step_sample": desc},
        "cpu_baseline": {"value": round(value, 6), "unit": "TOPS", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(value, 6), "unit": "TOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- the X-engine arm
def _dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(world, v: float) -> float:
    """The slowest rank's time (the only cross-rank step: no collective touches the data path)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_frame(base, rank: int):
    """Weak scaling: rank r correlates its own frame (bands are independent, Sec. I): same shape, own seed."""
    import dataclasses
    return dataclasses.replace(base, seed=base.seed + 7919 * rank)


def aggregate_tops(world: int, ops_per_frame: float, steps: int, max_ms: float) -> float:
    """Whole-job effective TOPS: every rank's frames over the slowest rank's time."""
    return world * ops_per_frame * steps / (max_ms * 1e-3) / 1e12


def measure_peaks(L, sp) -> dict:
    """Integer-pipe peaks of this GPU, measured now (the roofline denominators), in operations/s."""
    import ctypes
    imma = L.xe_peak_imma_s8(4000, sp)
    mo, do = ctypes.c_double(), ctypes.c_double()
    combo = max(L.xe_peak_imma_dp4a(4000, r, sp, ctypes.byref(mo), ctypes.byref(do)) for r in (16, 24, 32))
    dp4a = L.xe_peak_dp4a(4000, sp)
    return {"imma": imma, "combo": combo, "dp4a": dp4a, "int_mm": int_mm_rate()}


def pinned_copy(x_np):
    """A pinned host copy of a numpy array, read once by the GPU before any timing.

    The generator writes ordinary memory (byte-by-byte writes straight into pinned
    memory were measured at tens of MB/s on this machine's Grace hosts), and the copy into
    pinned memory is one bulk numpy copy. On these hosts the GPU's first read of
    host pages the CPU has just written runs at 3-20 GB/s and later reads at about
    210 GB/s, so one untimed pass gives every timed copy the steady rate.
    """
    import torch
    t = torch.empty(x_np.shape, dtype=torch.uint8).pin_memory()
    t.numpy()[...] = x_np
    flat = t.view(-1)
    step = 1 << 30
    buf = torch.empty(min(step, flat.numel()), dtype=torch.uint8, device="cuda")
    for k in range(0, flat.numel(), step):
        n = min(step, flat.numel() - k)
        buf[:n].copy_(flat[k:k + n], non_blocking=True)
    torch.cuda.synchronize()
    del buf
    return t


def h2d_rate(x_host, x_dev) -> float:
    """This machine's host-to-device copy rate from pinned memory, GB/s (context for the e2e figure)."""
    import torch
    x_dev.copy_(x_host, non_blocking=True)
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record()
    for _ in range(3):
        x_dev.copy_(x_host, non_blocking=True)
    h1.record()
    torch.cuda.synchronize()
    return 3 * x_host.numel() / (h0.elapsed_time(h1) * 1e-3) / 1e9


def single_frame_record(args, wl_key, frame, peaks, rank=0, world=1, bands=None, local=0, cpu=True,
                        cpu_bands=None, job_ops=None):
    """Time one frame per launch on resident input (the K timed steps), then end to end through the
    public API with host buffers; check sampled visibilities against the oracle; roofline and CPU leg.

    bands=(f0, f1): this rank correlates only those bands of the frame (corr_create_bands).
    job_ops: operations of one step of the whole job (all ranks), for the e2e figure (default world x ours).
    Returns (record dict, max over ranks of the timed region in ms, timed-region ops of this rank).
    """
    import numpy as np
    import torch

    import oracle
    import paper_1503_06203_gb300 as xe
    from paper_1503_06203_gb300 import autotune

    N, F, T = frame.N, frame.F, frame.T
    f0, f1 = bands if bands is not None else (0, F)
    Fb = f1 - f0
    ops = 4.0 * N * (N + 1) * Fb * T
    in_bytes = N * Fb * T
    out_bytes = Fb * xe.baselines(N) * 2 * 4
    stream = torch.cuda.current_stream()
    x_host = pinned_copy(frame.make())
    x_dev = torch.empty((T, F, N), dtype=torch.uint8, device="cuda")
    h2d_gbs = h2d_rate(x_host, x_dev)

    c = xe.Correlator(N, F, T, bands=bands)
    # knobs for this shape on this GPU (tuned once, outside the timed region)
    tuned = {"note": "library defaults"} if args.no_tune else autotune.apply(c)
    if args.product is not None:
        c.set_option(xe.CORR_OPT_PRODUCT, args.product)
        tuned = dict(tuned or {}, product=args.product, forced=True)
    if args.mma_steps is not None:
        c.set_option(xe.CORR_OPT_MMA_STEPS, args.mma_steps)
        tuned = dict(tuned or {}, mma_steps=args.mma_steps, forced=True)
    sampler = ClockSampler(local).start()
    for _ in range(args.warmup):
        c.reset()
        c.accumulate(x_dev)
    torch.cuda.synchronize()
    _barrier(world)
    torch.cuda.synchronize()
    launches0 = c.kernel_launches
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        c.reset()
        ev[k][0].record(stream)
        c.accumulate(x_dev)
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = c.kernel_launches - launches0
    if c.status() != 0:
        raise RuntimeError(f"device status {c.status()}: {xe.last_error()}")
    max_ms = _max_over_ranks(world, t_start.elapsed_time(t_end))
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    avg_kernel_ms = sum(kernel_ms) / len(kernel_ms)

    # spot-check the last device result against the oracle: entries at tile edges and at random
    V = c.readout().cpu().numpy()
    rng = np.random.default_rng(rank)
    K = 64
    fi = rng.integers(0, Fb, K)
    ii = np.concatenate([rng.integers(0, N, K - 2), [0, N - 1]])
    jj = np.concatenate([rng.integers(0, N, K - 2), [N - 1, N - 1]])
    ii, jj = np.minimum(ii, jj), np.maximum(ii, jj)
    ref = oracle.entries(x_host.numpy(), np.stack([fi + f0, ii, jj], 1))
    if not np.array_equal(V[fi, xe.packed_index(N, ii, jj)].astype(np.int64), ref):
        raise RuntimeError(f"{wl_key}: result differs from the oracle")

    # end to end through the public API: host frame in (pinned, copied in time chunks that overlap the
    # correlation), visibilities out (pinned) by overlapped readouts: each integration is copied out on
    # a copy stream while the next one runs; the timed region ends after the last copy out
    out_host = torch.empty((Fb, xe.baselines(N), 2), dtype=torch.int32).pin_memory()
    copy_stream = torch.cuda.Stream()
    for _ in range(2):
        c.accumulate_host(x_host)
        c.readout_async(out_host, copy_stream)
    torch.cuda.synchronize()
    # three timed regions of e2e_steps steps each; the median is reported (a one-off host hiccup of
    # tens of ms inside one region would otherwise set the figure), all three are in the record
    e2e_runs = []
    for _ in range(3):
        _barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            c.accumulate_host(x_host)
            c.readout_async(out_host, copy_stream)
        stream.wait_stream(copy_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_runs.append(_max_over_ranks(world, e0.elapsed_time(e1)))
    e2e_ms = sorted(e2e_runs)[1]
    if not np.array_equal(out_host.numpy()[fi, xe.packed_index(N, ii, jj)].astype(np.int64), ref):
        raise RuntimeError(f"{wl_key}: end-to-end result differs from the oracle")

    cpu_rec = None
    if cpu and rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc, _, _ = cpu_oracle_sample(frame, x_host.numpy(), args.cpu_seconds, bands=cpu_bands)
        cpu_rec = {"value": round(v, 6), "unit": "TOPS", "cores": cores, "kind": "oracle", "sample": desc}
        if wl_key == "pathfinder":  # and on one core, one band (the oracle as it stands, single-threaded)
            _, t1, _ = oracle.timed_visibilities(np.ascontiguousarray(x_host.numpy()[:, :1, :]), 1)
            cpu_rec["single_thread"] = {"value": round(4.0 * N * (N + 1) * T / t1 / 1e12, 6), "cores": 1,
                                        "sample": f"band 0 of the N={N} T={T} frame"}

    achieved = ops / (avg_kernel_ms * 1e-3) / 1e12
    product = c.get_option(xe.CORR_OPT_PRODUCT)
    mma_steps = c.get_option(xe.CORR_OPT_MMA_STEPS)
    split = c.get_option(xe.CORR_OPT_SPLIT)
    hybrid = product != 0 and mma_steps < 8  # tensor cores and dp4a side by side
    peak = (peaks["combo"] if hybrid else peaks["imma"]) / 1e12
    hw_ops = hardware_ops(N, Fb, T)
    hw_tops = hw_ops / (avg_kernel_ms * 1e-3) / 1e12
    ctas = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    traffic = (recorded_traffic(wl_key, product, effective_split(N, Fb, T, split, ctas), mma_steps)
               if bands is None or Fb == F else None)
    hbm = (measured_peaks_file() or {}).get("hbm_gbs", 6699.8)
    rec = {
        "value": None, "ms_per_step": round(max_ms / args.steps, 4),
        "config": {"workload": WORKLOADS[wl_key][1], "N": N, "F": F, "T": T, "bands": [f0, f1],
                   "frames_per_step": 1, "input_bytes": in_bytes, "output_bytes": out_bytes,
                   "l2": ("inputs larger than L2, no flush" if in_bytes > 129e6 else
                          "input smaller than L2: output writes larger than L2 dominate, no flush"),
                   "tuned": {k: v for k, v in (tuned or {}).items() if k != "trials"}},
        "roofline": {"bound": "tensor", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TOPS",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": ("measured in this run, all SMs, register-resident operands: "
                                     + ("mma.sync m16n8k32 s8 and dp4a issued together (best of 16/24/32 dp4a per MMA)"
                                        if hybrid else "mma.sync m16n8k32 s8")),
                     "product_path": {0: "tensor cores", 1: "tensor cores + dp4a",
                                      2: "tensor cores + dp4a on offset-encoded operands (Eq. 3 route)"}[product],
                     "mma_steps_of_8": mma_steps if product != 0 else 8,
                     "note": "achieved counts Eq. 2 operations (8 per complex MAC); the kernel's three-product form "
                             "executes 6 integer operations per complex MAC, so achieved/peak can reach 4/3; "
                             "hw_frac compares the executed operations with the peak",
                     "hw_ops_per_launch": hw_ops, "hw_tops": round(hw_tops, 3), "hw_frac": round(hw_tops / peak, 4),
                     "kernel": KERNEL_NAME, "avg_launch_ms": round(avg_kernel_ms, 4),
                     "algorithmic_bytes": in_bytes + out_bytes,
                     "hbm_frac": round((in_bytes + out_bytes) / (avg_kernel_ms * 1e-3) / 1e9 / hbm, 4)},
        "e2e": {"value": round((job_ops or world * ops) * args.e2e_steps / (e2e_ms * 1e-3) / 1e12, 3), "unit": "TOPS",
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes,
                "h2d_gbs_measured": round(h2d_gbs, 1),
                "ms_per_step": round(e2e_ms / args.e2e_steps, 4),
                "timing": f"median of 3 timed regions of {args.e2e_steps} steps",
                "runs_ms_per_step": [round(r / args.e2e_steps, 4) for r in e2e_runs]},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu_rec,
    }
    c.close()
    del x_dev, x_host, out_host
    torch.cuda.empty_cache()
    return rec, max_ms, ops


def run_xengine(args, wl_key):
    import ctypes

    import torch

    import paper_1503_06203_gb300 as xe
    import synth
    from paper_1503_06203_gb300._lib import lib

    rank, world, local = _dist_setup()
    torch.cuda.set_device(local)
    xe.build()
    L = lib()
    base = getattr(synth, WORKLOADS[wl_key][0])
    bands = None
    if args.split == "bands":
        frame = base  # one frame shared by every rank
        bands = xe.band_range(rank, world, base.F)
    else:
        frame = rank_frame(base, rank)
    stream = torch.cuda.current_stream()
    peaks = measure_peaks(L, ctypes.c_void_p(stream.cuda_stream))
    frame_ops = 4.0 * frame.N * (frame.N + 1) * frame.F * frame.T
    job_ops = frame_ops if args.split == "bands" else world * frame_ops
    rec, max_ms, _ = single_frame_record(args, wl_key, frame, peaks, rank, world, bands, local, job_ops=job_ops)
    if args.split == "bands":  # strong scaling: the one frame's operations over the slowest rank's time
        value = frame_ops * args.steps / (max_ms * 1e-3) / 1e12
        parallelism = f"bands of one frame split over {world} ranks" if world > 1 else "single GPU"
    else:
        value = aggregate_tops(world, frame_ops, args.steps, max_ms)
        parallelism = f"one frame per rank, dp{world}" if world > 1 else "single GPU"
    rec["config"]["parallelism"] = parallelism
    line = {
        "metric": "Effective TOPS", "value": round(value, 3), "unit": "TOPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
        "higher_is_better": True, "scaling": "strong" if args.split == "bands" else "weak", "vs_baseline": None,
        "dtype": "s8 x s8 -> s32", "data": "synthetic (seeded generator, paper's shapes)",
        "config": rec["config"], "roofline": rec["roofline"],
        "peaks_tops": {"imma_s8": round(peaks["imma"] / 1e12, 2), "dp4a": round(peaks["dp4a"] / 1e12, 2),
                       "imma_plus_dp4a": round(peaks["combo"] / 1e12, 2),
                       "cublaslt_int8_gemm_8192": round(peaks["int_mm"] / 1e12, 2)},
        "e2e": rec["e2e"], "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"],
        "cpu_baseline": rec["cpu_baseline"],
        "paper_context": "5.6 effective TOPS on an AMD R9 280X at N=2048 (context only)",
    }
    if wl_key == "pathfinder" and world == 1 and not args.no_extras:
        # the other workloads of the hot path, each timed on its own after the headline's timed region
        ln, ln_ms, ln_ops = single_frame_record(args, "large_n", synth.LARGE_N, peaks, cpu_bands=1)
        ln["value"] = round(ln_ops * args.steps / (ln_ms * 1e-3) / 1e12, 3)
        ln["e2e"]["note"] = ("each step copies in the 67 MB frame in one piece, overlapping the previous "
                             "frame's correlation, and reads out the 1.07 GB packed triangle (16x the input) "
                             "to pinned host memory, overlapped with the next integration "
                             "(corr_readout_host_async)")
        line["large_n"] = ln
        line["batched"] = batched_record(args)
        line["batched_small"] = batched_record(args, small=True)
        line["served"] = served_record(args)
        line["lags_gates"] = lags_gates_record(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- batched / served
def batched_record(args, small: bool = False) -> dict:
    """64 uneven frames: one launch per frame (back to back, no host waits) vs one batched
    (graph-replayed) launch per step. Both modes run the same frames into the same handles.
    small: the small-frame recipe (each frame microseconds of work) instead of the uneven-frame one."""
    import numpy as np
    import torch

    import oracle
    import paper_1503_06203_gb300 as xe
    import synth
    frames = synth.small_frames() if small else synth.batched_frames()
    cors = [xe.Correlator(f.N, f.F, f.T) for f in frames]
    xs_host = [f.make() for f in frames]
    xs = [torch.from_numpy(x).cuda() for x in xs_host]
    ops = sum(4.0 * f.N * (f.N + 1) * f.F * f.T for f in frames)
    stream = torch.cuda.current_stream()
    # frames that fill the GPU on their own run alone inside the batched call (the library's rule)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    alone = sum(1 for f in frames if xe.batch_runs_alone(f.N, f.F, sms))

    def step(batched):
        for c in cors:
            c.reset()
        if batched:
            xe.accumulate_batch(cors, xs)
        else:
            for c, x in zip(cors, xs):
                c.accumulate(x)

    res = {}
    sampler = ClockSampler(0).start()
    for mode in (False, True):
        for _ in range(args.warmup):
            step(mode)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(mode)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res["batched" if mode else "plain"] = {"ms_per_step": round(ms, 4),
                                               "frames_per_s": round(len(frames) / ms * 1e3, 2),
                                               "effective_tops": round(ops / ms / 1e9, 3),
                                               "launches_per_step": (alone + (alone < len(frames))) if mode
                                               else len(frames)}
    clocks = sampler.stop()
    # the batched result of the last step against the oracle: sampled entries of every frame
    rng = np.random.default_rng(5)
    for fr, c, x in zip(frames, cors, xs_host):
        V = c.readout().cpu().numpy()
        K = 16
        f = rng.integers(0, fr.F, K)
        i = rng.integers(0, fr.N, K)
        j = rng.integers(0, fr.N, K)
        i, j = np.minimum(i, j), np.maximum(i, j)
        if not np.array_equal(V[f, xe.packed_index(fr.N, i, j)].astype(np.int64),
                              oracle.entries(x, np.stack([f, i, j], 1))):
            raise RuntimeError("batched: result differs from the oracle")
    for c in cors:
        c.close()
    del xs
    torch.cuda.empty_cache()
    workload = ("64 small frames (N 64..256, F 1..8, T 512..1024, sigma 1.5..3.5) per step" if small else
                "64 uneven frames (N 64..2048, F 1..64, T 512..8192, sigma 1.5..3.5) per step")
    in_bytes = sum(f.nbytes for f in frames)
    return {"metric": "Effective TOPS", "value": res["batched"]["effective_tops"], "unit": "TOPS",
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": workload, "frames": len(frames), "effective_ops_per_step": ops,
                       "input_bytes_per_step": in_bytes,
                       "l2": ("inputs larger than L2, no flush" if in_bytes > 129e6 else
                              "inputs smaller than L2 (resident across steps, as in a real stream of small frames)")},
            "batched": dict(res["batched"], frames_alone=alone), "plain": res["plain"],
            "speedup_batched_over_plain": round(res["plain"]["ms_per_step"] / res["batched"]["ms_per_step"], 3),
            "clocks": clocks}


def served_specs():
    import numpy as np

    from paper_1503_06203_gb300 import serve
    rng = np.random.default_rng(1004)
    return [serve.StreamSpec(int(rng.choice([256, 1024, 2048])), int(rng.choice([16, 64, 256]))) for _ in range(32)]


def served_record(args) -> dict:
    """32 served streams with Poisson arrivals at each rate: continuous batching vs one frame per launch,
    the same arrivals (seeded by the rate) for both."""
    import torch

    import synth
    from paper_1503_06203_gb300 import serve
    specs = served_specs()
    t_min, t_max = 1024, 8192
    pool_bytes = max(s.N * s.F for s in specs) * t_max
    pool = pinned_copy(synth.gauss_flat(pool_bytes, 2.5, 1004))
    budget = 24 << 30
    srv = serve.Server(specs, t_max, pool, budget_bytes=budget, readout_every=16)
    h2d = srv.measure_copy_rate()  # sets the piece counts of large frames (copy hidden behind correlation)
    sweeps = []
    sampler = ClockSampler(0).start()
    for rate in (float(r) for r in args.rates.split(",")):
        # about 12 s of arrivals at low rates, 6 s at 40 frames/s, at most 240 frames
        count = args.served_frames or int(min(240, max(120, 6 * rate)))
        arr = serve.poisson_arrivals(rate, count, len(specs), t_min, t_max, pool_bytes, specs,
                                     1004000 + int(round(10 * rate)))
        out = {"rate_hz": rate, "frames": count}
        for mode in ("served", "plain"):
            srv.reset()
            st = srv.run_served(arr) if mode == "served" else srv.run_plain(arr)
            out[mode] = st.summary()
        out["served_beats_plain"] = {
            "frames_per_s": out["served"]["frames_per_s"] >= out["plain"]["frames_per_s"],
            "p99": out["served"]["p99_ms"] <= out["plain"]["p99_ms"],
            # served / plain; at low offered rates both launch every frame on arrival and tie
            "frames_per_s_ratio": round(out["served"]["frames_per_s"] / out["plain"]["frames_per_s"], 4),
            "p99_ratio": round(out["served"]["p99_ms"] / out["plain"]["p99_ms"], 4)}
        sweeps.append(out)
    clocks = sampler.stop()
    acc_gb = sum(s.F * s.N * (s.N + 1) * 4 for s in specs) / 1e9
    srv.close()
    del pool
    torch.cuda.empty_cache()
    return {"metric": "served frames/s and p50/p99 frame latency (continuous batching vs one frame per launch)",
            "unit": "frames/s",
            "config": {"workload": "32 streams, N in {256,1024,2048}, F in {16,64,256} per stream, T 1024..8192 "
                                   "per frame, Poisson arrivals, readout every 16 frames",
                       "streams": [[s.N, s.F] for s in specs], "resident_accumulators_gb": round(acc_gb, 2),
                       "input_budget_gb": budget / 2 ** 30, "h2d_gbs_measured": round(h2d, 1)},
            "sweep": sweeps, "clocks": clocks}


def lags_gates_record(args) -> dict:
    """Sec. IV extensions on the Pathfinder frame: lag-shift bandwidth, gated vs plain correlation."""
    import numpy as np
    import torch

    import oracle
    import paper_1503_06203_gb300 as xe
    import synth
    fr = synth.PATHFINDER
    N, F, T = fr.N, fr.F, fr.T
    x_np = fr.make()
    x = torch.from_numpy(x_np).cuda()
    lags_np = np.random.default_rng(7).integers(-64, 64, N).astype(np.int32)
    lags = torch.from_numpy(lags_np).cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_shift = timed(lambda: xe.shift_lags(x, lags, out=y), 20)
    # two bands of the shifted frame against the oracle's shift
    if not np.array_equal(y[:, :2, :].cpu().numpy(), oracle.shift_lags(np.ascontiguousarray(x_np[:, :2, :]), lags_np)):
        raise RuntimeError("lag shift differs from the oracle")
    gbs = 2.0 * N * F * T / ms_shift / 1e6
    hbm = (measured_peaks_file() or {}).get("hbm_gbs", 6699.8)
    G, period = 8, 1024
    gates = [xe.Correlator(N, F, T) for _ in range(G)]
    plain = xe.Correlator(N, F, T)

    def gated_step():
        for c in gates:
            c.reset()
        xe.accumulate_gated(gates, x, period, 0)

    def plain_step():
        plain.reset()
        plain.accumulate(x)

    ms_gated = timed(gated_step, 10)
    ms_plain = timed(plain_step, 10)
    ops = 4.0 * N * (N + 1) * F * T
    for c in gates + [plain]:
        c.close()
    del x, y
    torch.cuda.empty_cache()
    return {"config": {"workload": "Pathfinder frame N=256 F=256 T=16384; lags uniform in [-64, 64); "
                                   f"{G} gates of a {period}-sample period"},
            "lag_shift": {"kernel": "shift_lags_stream_kernel", "ms": round(ms_shift, 4), "gbs": round(gbs, 1),
                          "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                                       "frac": round(gbs / hbm, 4), "algorithmic_bytes": 2 * N * F * T}},
            "gated": {"ms": round(ms_gated, 4), "effective_tops": round(ops / ms_gated / 1e9, 3), "gates": G,
                      "segments": T // (period // G)},
            "plain": {"ms": round(ms_plain, 4), "effective_tops": round(ops / ms_plain / 1e9, 3)}}


def _standalone(args, metric, unit, rec):
    import paper_1503_06203_gb300 as xe  # noqa: F401
    line = {"metric": metric, "unit": unit, "n_gpus": 1, "higher_is_better": True, "dtype": "s8 x s8 -> s32",
            "data": "synthetic (seeded generator, paper's shapes)", **rec}
    print(json.dumps(line), flush=True)


def run_batched(args):
    import paper_1503_06203_gb300 as xe
    xe.build()
    rec = batched_record(args, small=args.workload == "batched_small")
    _standalone(args, rec.pop("metric"), rec.pop("unit"), rec)


def run_served(args):
    import paper_1503_06203_gb300 as xe
    xe.build()
    rec = served_record(args)
    rec["value"] = max(d["served"]["frames_per_s"] for d in rec["sweep"])
    _standalone(args, rec.pop("metric"), rec.pop("unit"), rec)


def run_lags_gates(args):
    import paper_1503_06203_gb300 as xe
    xe.build()
    rec = lags_gates_record(args)
    rec["value"] = rec["gated"]["effective_tops"]
    _standalone(args, "lag shift GB/s and gated-correlation effective TOPS", "TOPS", rec)


def main():
    args = parse_args()
    if args.workload == "lags_gates":
        run_lags_gates(args)
    elif args.workload in ("batched", "batched_small"):
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_xengine(args, args.workload)


if __name__ == "__main__":
    main()
