"""Served streams at the served workload's own shapes, bit-exact against the oracle.

Four streams from the served workload's recipe, one per (N, F) corner of it:
N in {256, 1024, 2048}, F in {16, 64, 256}, frames of T = 1024..8192 samples
(multiples of 256) arriving by a Poisson process, integrations read out every
16 frames. Every readout is checked against the CPU oracle (Eq. 1 summed over
the integration's frames): sampled entries (tile edges and corners among
them), every autocorrelation, and the Freivalds row identity V w for random
small complex w, which checks every row of the matrix. Each stream's readouts
in the continuous-batching mix must also equal, bit for bit, the same stream
served alone, one frame per launch.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import freivalds_rows

pytestmark = pytest.mark.gpu

SPECS = [(256, 16), (2048, 16), (1024, 64), (256, 256)]  # (N, F)
FRAMES_PER_STREAM = 16
T_MIN, T_MAX = 1024, 8192


def make_arrivals(serve, rate_hz, pool_bytes, seed):
    rng = np.random.default_rng(seed)
    streams = rng.permutation(np.repeat(np.arange(len(SPECS)), FRAMES_PER_STREAM))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, streams.size))
    out = []
    for k, s in enumerate(streams):
        N, F = SPECS[s]
        T = 256 * int(rng.integers(T_MIN // 256, T_MAX // 256 + 1))
        off = 256 * int(rng.integers(0, (pool_bytes - T * F * N) // 256 + 1))
        out.append(serve.Arrival(float(t[k]), int(s), T, off))
    return out


def check_integration(V, x, rng):
    """V int32 [F][B][2] of the frames x (uint8 [sum T][F][N]) against the oracle."""
    import paper_1503_06203_gb300 as xe
    T, F, N = x.shape
    # tile edges and corners, and random entries
    e = np.unique(np.concatenate([np.arange(0, N, 64), np.arange(63, N, 64)]))
    ei, ej = np.meshgrid(e, e, indexing="ij")
    keep = ei.ravel() <= ej.ravel()
    ri, rj = rng.integers(0, N, 1500), rng.integers(0, N, 1500)
    ii = np.concatenate([ei.ravel()[keep], np.minimum(ri, rj)])
    jj = np.concatenate([ej.ravel()[keep], np.maximum(ri, rj)])
    ff = rng.integers(0, F, ii.size)
    ref = oracle.entries(x, np.stack([ff, ii, jj], 1))
    assert np.array_equal(V[ff, xe.packed_index(N, ii, jj)].astype(np.int64), ref)
    # every autocorrelation
    fa, ia = np.meshgrid(np.arange(F), np.arange(N), indexing="ij")
    ref = oracle.entries(x, np.stack([fa.ravel(), ia.ravel(), ia.ravel()], 1))
    assert np.array_equal(V[fa.ravel(), xe.packed_index(N, ia.ravel(), ia.ravel())].astype(np.int64), ref)
    # every row: Freivalds
    w = rng.integers(-3, 4, size=(F, N, 2)).astype(np.int64)
    assert np.array_equal(freivalds_rows(V, w), oracle.freivalds_rhs(x, w))


def test_served_config4_shapes_bit_exact():
    import torch

    import paper_1503_06203_gb300 as xe
    from paper_1503_06203_gb300 import serve
    xe.build()
    specs = [serve.StreamSpec(N, F) for N, F in SPECS]
    pool_bytes = 1 << 30
    pool_np = synth.gauss_flat(pool_bytes, 2.5, 1004)
    pool = torch.from_numpy(pool_np).pin_memory()
    arrivals = make_arrivals(serve, 500.0, pool_bytes, 44)  # bursty: frames queue and share launches
    srv = serve.Server(specs, T_MAX, pool, budget_bytes=6 << 30, readout_every=FRAMES_PER_STREAM)
    srv.keep_readouts = True
    srv.piece_bytes = 64 << 20  # most frames of these shapes then run in time pieces
    assert max(len(srv.pieces(a)) for a in arrivals) == srv.max_pieces
    st = srv.run_served(arrivals)
    pieces = sum(len(srv.pieces(a)) for a in arrivals)
    assert st.frames == len(arrivals) and st.launches < pieces  # several pieces shared launches
    served = [list(r) for r in srv.readouts]
    srv.close()
    rng = np.random.default_rng(45)
    for sid, (N, F) in enumerate(SPECS):
        mine = [a for a in arrivals if a.stream == sid]
        assert len(served[sid]) == len(mine) // FRAMES_PER_STREAM == 1
        # alone: the stream's own frames, one per launch
        alone = serve.Server([specs[sid]], T_MAX, pool, budget_bytes=1 << 30, readout_every=FRAMES_PER_STREAM)
        alone.keep_readouts = True
        alone.run_plain([serve.Arrival(a.t, 0, a.T, a.offset) for a in mine])
        assert len(alone.readouts[0]) == 1 and torch.equal(alone.readouts[0][0], served[sid][0])
        alone.close()
        # the oracle over the integration's frames, in arrival order
        x = np.concatenate([pool_np[a.offset:a.offset + a.T * F * N].reshape(a.T, F, N) for a in mine], axis=0)
        check_integration(served[sid][0].numpy(), x, rng)
