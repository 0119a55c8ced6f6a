"""Served correlation streams: continuous batching over the C ABI.

A correlation stream is one instrument's data flow: N elements and F bands,
fixed for the stream, arriving as frames of T samples (Sec. III: time
steps of all bands of all elements). Each stream keeps its int32
visibilities resident on the device (one Correlator handle) and reads them
out every `readout_every` frames, which starts the next integration
(Sec. II.A: products are accumulated over many samples).

The server admits arriving frames while their input bytes fit a device-
memory budget (first-fit blocks inside one preallocated slab), copies each
admitted frame to the device on a copy stream (a large frame in up to four
time pieces, each launched as soon as it has landed), and launches copied
pieces together in one batched launch: at most one piece per stream per
launch, each stream's frames in arrival order (a stream's frames add into
the same accumulators). A piece larger than the launch's work so far starts
the next launch, so older work never waits for a larger, younger piece.
Frames keep arriving and copying while launches run; up to three launches
are in flight (the library keeps four launch sets, so the host never waits
for the GPU to launch). The plain mode is the reference: one whole frame per
launch, copied and then correlated, each waited for before the next starts.

PyTorch provides device memory, pinned host memory and streams; every
correlation runs in the CUDA library.
"""
from __future__ import annotations

import bisect
import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import Correlator, accumulate_batch, baselines

import torch


@dataclass
class StreamSpec:
    N: int
    F: int


@dataclass
class Arrival:
    t: float          # seconds after the start of the run
    stream: int
    T: int
    offset: int       # byte offset of the frame's data in the host pool


@dataclass
class FrameRecord:
    """Host-clock times (seconds after the start of the run) of one frame's steps."""
    arrival: float
    admitted: float = float("nan")   # input space granted, copy issued
    copied: float = float("nan")     # copy (of its first piece) seen complete
    launched: float = float("nan")   # (its first piece) in a launch
    done: float = float("nan")       # its launch seen complete


@dataclass
class RunStats:
    mode: str
    frames: int
    seconds: float
    latencies_ms: list = field(default_factory=list)
    ops: float = 0.0
    records: list = field(default_factory=list)  # FrameRecord per frame (served mode)
    launches: int = 0
    gpu_trace: dict = field(default_factory=dict)  # served with trace_gpu: GPU-clock times of copies and launches

    def breakdown(self) -> dict:
        """p50 / p99 of each step's share of the latency (served mode), in ms."""
        if not self.records:
            return {}
        r = self.records
        parts = {"wait_for_space": [x.admitted - x.arrival for x in r], "copy": [x.copied - x.admitted for x in r],
                 "wait_for_launch": [x.launched - x.copied for x in r], "gpu": [x.done - x.launched for x in r]}
        return {k: {"p50": round(1e3 * float(np.percentile(v, 50)), 3), "p99": round(1e3 * float(np.percentile(v, 99)), 3)}
                for k, v in parts.items()}

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms)
        out = {"mode": self.mode, "frames": self.frames, "seconds": round(self.seconds, 4),
               "frames_per_s": round(self.frames / self.seconds, 3),
               "effective_tops": round(self.ops / self.seconds / 1e12, 3),
               "p50_ms": round(float(np.percentile(lat, 50)), 3) if lat.size else None,
               "p99_ms": round(float(np.percentile(lat, 99)), 3) if lat.size else None,
               "launches": self.launches}
        if self.records:
            out["latency_parts_ms"] = self.breakdown()
        return out


def poisson_arrivals(rate_hz: float, count: int, streams: int, t_min: int, t_max: int, pool_bytes: int,
                     specs, seed: int) -> list[Arrival]:
    """Poisson arrivals at `rate_hz`; stream uniform; T uniform in [t_min, t_max], a multiple of 256."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, count))
    out = []
    for k in range(count):
        s = int(rng.integers(0, streams))
        T = 256 * int(rng.integers(t_min // 256, t_max // 256 + 1))
        nbytes = T * specs[s].F * specs[s].N
        off = int(rng.integers(0, max(1, (pool_bytes - nbytes) // 256 + 1))) * 256
        out.append(Arrival(float(t[k]), s, T, off))
    return out


class SlabAllocator:
    """First-fit allocator inside one device buffer: the in-flight input budget.

    Frames may finish in any order (a stream's next frame waits for the
    stream's current one). A freed block is merged with its free neighbours
    at once, so a frame still waiting behind its stream's earlier frames does
    not hold up the space of frames that already finished.
    """

    def __init__(self, nbytes: int, device: str | None = "cuda"):
        # device=None keeps only the bookkeeping (host-side tests)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device) if device else None
        self.size = nbytes
        self.free_blocks = [[0, nbytes]]  # [start, end), sorted by start, never adjacent
        self.live = {}                    # start -> end
        self.used = 0

    def alloc(self, nbytes: int):
        nbytes = (nbytes + 255) // 256 * 256
        if nbytes > self.size:
            raise ValueError("frame larger than the device-memory budget")
        for k, (s, e) in enumerate(self.free_blocks):
            if e - s >= nbytes:
                if e - s == nbytes:
                    del self.free_blocks[k]
                else:
                    self.free_blocks[k][0] = s + nbytes
                self.live[s] = s + nbytes
                self.used += nbytes
                return s
        return None

    def free(self, start: int):
        end = self.live.pop(start)  # KeyError for a block that is not live
        self.used -= end - start
        starts = [b[0] for b in self.free_blocks]
        k = bisect.bisect_left(starts, start)
        self.free_blocks.insert(k, [start, end])
        if k + 1 < len(self.free_blocks) and self.free_blocks[k + 1][0] == end:  # merge right
            self.free_blocks[k][1] = self.free_blocks[k + 1][1]
            del self.free_blocks[k + 1]
        if k > 0 and self.free_blocks[k - 1][1] == start:  # merge left
            self.free_blocks[k - 1][1] = self.free_blocks[k][1]
            del self.free_blocks[k]


class Server:
    """Streams with resident accumulators, served by continuous batching or one frame per launch."""

    def __init__(self, specs: list[StreamSpec], t_max: int, pool: torch.Tensor, budget_bytes: int,
                 readout_every: int = 16):
        self.specs = specs
        self.t_max = t_max
        self.pool = pool  # pinned host bytes the frames are cut from
        self.readout_every = readout_every
        self.cors = [Correlator(s.N, s.F, t_max) for s in specs]
        self.outs = [torch.empty((s.F, baselines(s.N), 2), dtype=torch.int32, device="cuda") for s in specs]
        self.readouts = [[] for _ in specs]  # host copies of every readout (for checks), optional
        self.keep_readouts = False
        self.counts = [0] * len(specs)
        self.ring = SlabAllocator(budget_bytes)
        self.rate_tops = 200.0  # effective TOPS assumed when estimating a frame's GPU time
        self.piece_bytes = 0     # 0: piece counts from the cost model (piece_count); else pieces of this many bytes
        self.max_pieces = 4
        self.piece_cost_ms = 4.0
        self.h2d_gbs = 200.0     # host-to-device copy rate (measure_copy_rate sets it)
        self.hbm_gbs = 6000.0    # device memory rate for the accumulators' extra passes
        self.copy_stream = torch.cuda.Stream()
        self.compute_stream = torch.cuda.Stream()

    def _frame_view(self, a: Arrival) -> torch.Tensor:
        s = self.specs[a.stream]
        n = a.T * s.F * s.N
        return self.pool[a.offset:a.offset + n].view(a.T, s.F, s.N)

    def _after_frame(self, stream_id: int):
        """Readout every `readout_every` frames of a stream (on the compute stream)."""
        self.counts[stream_id] += 1
        if self.counts[stream_id] % self.readout_every == 0:
            self.cors[stream_id].readout(self.outs[stream_id], reset=True, stream=self.compute_stream)
            if self.keep_readouts:  # (a synchronous copy after the readout, for checks only)
                with torch.cuda.stream(self.compute_stream):
                    self.readouts[stream_id].append(self.outs[stream_id].cpu())

    def close(self):
        for c in self.cors:
            c.close()
        self.cors = []
        self.outs = []
        self.ring.buf = None

    def reset(self):
        for c in self.cors:
            c.reset()
        self.counts = [0] * len(self.specs)
        self.readouts = [[] for _ in self.specs]

    def ops(self, arrivals) -> float:
        return sum(4.0 * self.specs[a.stream].N * (self.specs[a.stream].N + 1) * self.specs[a.stream].F * a.T
                   for a in arrivals)

    # ---------------------------------------------------------------- served
    def measure_copy_rate(self, nbytes: int = 256 << 20) -> float:
        """This host link's copy rate from the pinned pool into the input slab, GB/s (sets h2d_gbs)."""
        n = min(nbytes, self.pool.numel(), self.ring.size)
        self.ring.buf[:n].copy_(self.pool[:n], non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        self.ring.buf[:n].copy_(self.pool[:n], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        self.h2d_gbs = n / (e0.elapsed_time(e1) * 1e-3) / 1e9
        return self.h2d_gbs

    def frame_ms(self, a: Arrival) -> float:
        """Estimated GPU time of a frame: its Eq. 2 operations at rate_tops."""
        s = self.specs[a.stream]
        return 4.0 * s.N * (s.N + 1) * s.F * a.T / (self.rate_tops * 1e9)

    def piece_count(self, a: Arrival) -> int:
        """How many time pieces a frame is copied and correlated in.

        Pieces hide all but the first piece's copy behind the correlation; each
        extra piece costs one more read and write of the stream's accumulators
        and a launch's fill and drain (piece_cost_ms; traces on 2048 x 256
        frames put the whole cost near 2.5 ms, and the default keeps a margin).
        The count maximises copy_ms (1 - 1/n) - (n - 1) cost, with copy_ms from
        the copy rate this server measured (h2d_gbs). piece_bytes, if set,
        instead cuts pieces of at least that many bytes (tests use it).
        """
        s = self.specs[a.stream]
        nbytes = a.T * s.F * s.N
        limit = max(1, min(self.max_pieces, a.T // 256))
        if self.piece_bytes:
            return int(max(1, min(limit, nbytes // self.piece_bytes)))
        copy_ms = nbytes / (self.h2d_gbs * 1e6)
        cost_ms = self.piece_cost_ms + 2.0 * s.F * s.N * (s.N + 1) * 4 / (self.hbm_gbs * 1e6)
        gain = [copy_ms * (1.0 - 1.0 / n) - (n - 1) * cost_ms for n in range(1, limit + 1)]
        return 1 + int(np.argmax(gain))

    def pieces(self, a: Arrival) -> list[tuple[int, int]]:
        """Sample ranges [t0, t1) a frame is copied and correlated in (piece_count of them, whole
        256-sample blocks). The visibilities are the same (integer sums over the frame's samples, in
        any grouping)."""
        n = self.piece_count(a)
        bounds = [256 * ((a.T // 256) * k // n) for k in range(n)] + [a.T]
        return [(bounds[k], bounds[k + 1]) for k in range(n)]

    def run_served(self, arrivals: list[Arrival], max_inflight: int = 3, small_ms: float = 2.0,
                   trace_gpu: bool = False, join_frac: float = 0.25) -> RunStats:
        recs = [FrameRecord(a.t) for a in arrivals]
        pending = collections.deque(range(len(arrivals)))  # not yet arrived
        waiting = collections.deque()   # arrived, waiting for budget
        copying = collections.deque()   # (frame, piece, copy event), in copy order
        ready = []                      # copied, not launched: (frame, piece), in copy order
        inflight = collections.deque()  # (done event, [(frame, piece)])
        parts = [self.pieces(a) for a in arrivals]  # (after measure_copy_rate, if the caller ran it)
        offset = [0] * len(arrivals)    # slab offset of each admitted frame
        launched = [0] * len(arrivals)  # pieces launched
        finished = [0] * len(arrivals)  # pieces whose launch completed
        order = [collections.deque() for _ in self.specs]  # admitted frames of each stream, oldest first
        copy_ev, launch_ev = {}, []  # trace_gpu: (start, end) timing events per piece copy and per launch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if trace_gpu:
            ref = torch.cuda.Event(enable_timing=True)
            ref.record(self.copy_stream)
        done = 0
        launches = 0
        while done < len(arrivals):
            now = time.perf_counter() - t0
            while pending and arrivals[pending[0]].t <= now:
                waiting.append(pending.popleft())
            # admission by the device-memory budget, in arrival order; each piece is copied on the copy stream
            while waiting:
                k = waiting[0]
                a = arrivals[k]
                s = self.specs[a.stream]
                off = self.ring.alloc(a.T * s.F * s.N)
                if off is None:
                    break
                waiting.popleft()
                offset[k] = off
                order[a.stream].append(k)
                recs[k].admitted = time.perf_counter() - t0
                src = self._frame_view(a).view(-1)
                row = s.F * s.N
                with torch.cuda.stream(self.copy_stream):
                    for p, (u0, u1) in enumerate(parts[k]):
                        if trace_gpu:
                            ev0 = torch.cuda.Event(enable_timing=True)
                            ev0.record(self.copy_stream)
                        self.ring.buf[off + u0 * row:off + u1 * row].copy_(src[u0 * row:u1 * row], non_blocking=True)
                        ev = torch.cuda.Event(enable_timing=trace_gpu)
                        ev.record(self.copy_stream)
                        copying.append((k, p, ev))
                        if trace_gpu:
                            copy_ev[(k, p)] = (ev0, ev)
            while copying and copying[0][2].query():
                k, p, _ = copying.popleft()
                if p == 0:
                    recs[k].copied = time.perf_counter() - t0
                ready.append((k, p))
            # one launch over copied pieces in copy order, at most one per stream, each stream's frames in
            # arrival order. All pieces of a launch finish together, so the launch stays close to FIFO:
            # a piece whose work is more than the launch's so far (and more than small_ms) starts the next
            # launch instead (older work never waits for a larger, younger piece), and younger pieces join
            # the oldest one only up to join_frac of its work, or small_ms (a younger frame never holds up
            # an older one by much)
            if ready and len(inflight) < max_inflight:
                chosen, seen, rest, work, cut = [], set(), [], 0.0, False
                head = 0.0  # the first (oldest) piece's work
                for k, p in ready:
                    a = arrivals[k]
                    u0, u1 = parts[k][p]
                    w = self.frame_ms(a) * (u1 - u0) / a.T
                    eligible = a.stream not in seen and order[a.stream][0] == k and launched[k] == p
                    if cut or not eligible or (chosen and (w > max(work, small_ms)
                                                           or work - head + w > max(small_ms, join_frac * head))):
                        cut = cut or eligible
                        rest.append((k, p))
                    else:
                        seen.add(a.stream)
                        chosen.append((k, p))
                        if not head:
                            head = w
                        work += w
                ready = rest
                if chosen:
                    cors, xs = [], []
                    for k, p in chosen:
                        a = arrivals[k]
                        s = self.specs[a.stream]
                        u0, u1 = parts[k][p]
                        row = s.F * s.N
                        cors.append(self.cors[a.stream])
                        xs.append(self.ring.buf[offset[k] + u0 * row:offset[k] + u1 * row].view(u1 - u0, s.F, s.N))
                    if trace_gpu:
                        ev0 = torch.cuda.Event(enable_timing=True)
                        ev0.record(self.compute_stream)
                    accumulate_batch(cors, xs, stream=self.compute_stream)
                    launches += 1
                    t_launch = time.perf_counter() - t0
                    for k, p in chosen:
                        a = arrivals[k]
                        if p == 0:
                            recs[k].launched = t_launch
                        launched[k] += 1
                        if launched[k] == len(parts[k]):  # the frame's last piece: its stream moves on
                            order[a.stream].popleft()
                            self._after_frame(a.stream)
                    ev = torch.cuda.Event(enable_timing=trace_gpu)
                    ev.record(self.compute_stream)
                    inflight.append((ev, chosen))
                    if trace_gpu:
                        launch_ev.append((ev0, ev, list(chosen), t_launch))
            while inflight and inflight[0][0].query():
                _, chosen = inflight.popleft()
                t = time.perf_counter() - t0
                for k, p in chosen:
                    finished[k] += 1
                    if finished[k] == len(parts[k]):
                        recs[k].done = t
                        self.ring.free(offset[k])
                        done += 1
            if not (inflight and inflight[0][0].query()) and not copying and not ready:
                time.sleep(20e-6)
        seconds = time.perf_counter() - t0 - arrivals[0].t
        trace = {}
        if trace_gpu:  # milliseconds on the GPU clock after the run's start
            torch.cuda.synchronize()
            trace["copies"] = {f"{k}.{p}": (ref.elapsed_time(a), ref.elapsed_time(b)) for (k, p), (a, b) in copy_ev.items()}
            trace["launches"] = [(ref.elapsed_time(a), ref.elapsed_time(b), [f"{k}.{p}" for k, p in ch], 1e3 * th)
                                 for a, b, ch, th in launch_ev]
        return RunStats("served", len(arrivals), seconds, [1e3 * (r.done - a.t) for r, a in zip(recs, arrivals)],
                        self.ops(arrivals), recs, launches, trace)

    # ---------------------------------------------------------------- plain
    def run_plain(self, arrivals: list[Arrival]) -> RunStats:
        """One frame per launch, in arrival order, each waited for before the next."""
        lat = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a in arrivals:
            while time.perf_counter() - t0 < a.t:
                pass
            s = self.specs[a.stream]
            src = self._frame_view(a)
            dst = self.ring.buf[:src.numel()]
            with torch.cuda.stream(self.compute_stream):
                dst.copy_(src.view(-1), non_blocking=True)
            accumulate_batch([self.cors[a.stream]], [dst.view(a.T, s.F, s.N)], stream=self.compute_stream)
            self._after_frame(a.stream)
            self.compute_stream.synchronize()
            lat.append(1e3 * (time.perf_counter() - t0 - a.t))
        seconds = time.perf_counter() - t0 - arrivals[0].t
        return RunStats("plain", len(arrivals), seconds, lat, self.ops(arrivals), launches=len(arrivals))
