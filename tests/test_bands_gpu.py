"""Band-range handles (corr_create_bands): one frame's bands split across handles, as across GPUs.

Frequency bands are independent (Sec. I, Sec. IV), so a frame's bands can be
partitioned with no exchange. The ranges of a partition, concatenated in band
order, must give exactly the visibilities of one handle over every band, and
each range must equal the oracle over its bands.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xe():
    import paper_1503_06203_gb300 as xe
    xe.build()
    return xe


def whole_and_parts(xe, x_np, parts, feed):
    """feed(correlator, frame) adds the frame; returns (whole, [part visibilities])."""
    import torch
    T, F, N = x_np.shape
    x = torch.from_numpy(x_np).cuda()
    whole = xe.Correlator(N, F, T)
    feed(whole, x if feed is not host_feed else x_np)
    outs = []
    for f0, f1 in parts:
        c = xe.Correlator(N, F, T, bands=(f0, f1))
        assert (c.F, c.F_in, c.f0) == (f1 - f0, F, f0)
        feed(c, x if feed is not host_feed else x_np)
        outs.append(c.readout().cpu().numpy())
        assert c.status() == 0
    V = whole.readout().cpu().numpy()
    torch.cuda.synchronize()
    return V, outs


def dev_feed(c, x):
    c.accumulate(x)


def host_feed(c, x_np):
    c.accumulate_host(x_np)


@pytest.mark.parametrize("N,F,T", [(256, 8, 1000), (96, 5, 333), (100, 6, 257)])
@pytest.mark.parametrize("feed", [dev_feed, host_feed], ids=["device", "host"])
def test_band_halves_equal_whole_and_oracle(xe, N, F, T, feed):
    """Two halves and an uneven three-way split give the whole frame's visibilities, bit for bit."""
    x_np = synth.gauss(N, F, T, 2.5, 300 + N + F)
    for world in (2, 3):
        parts = [xe.band_range(r, world, F) for r in range(world)]
        V, outs = whole_and_parts(xe, x_np, parts, feed)
        assert np.array_equal(np.concatenate(outs, axis=0), V)
        assert np.array_equal(V.astype(np.int64), oracle.visibilities(x_np))
        for (f0, f1), P in zip(parts, outs):
            sub = np.ascontiguousarray(x_np[:, f0:f1, :])
            assert np.array_equal(P.astype(np.int64), oracle.visibilities(sub))


def test_band_handles_accumulate_and_offset_route(xe):
    """Two frames added into band handles, on the offset-encoded route (Eq. 3) too."""
    import torch
    N, F, T = 128, 6, 640
    xs = [synth.gauss(N, F, T, 2.5, 310 + k) for k in range(2)]
    for product in (0, 1, 2):
        outs = []
        for f0, f1 in [(0, 2), (2, 5), (5, 6)]:
            c = xe.Correlator(N, F, T, bands=(f0, f1))
            c.set_option(xe.CORR_OPT_PRODUCT, product)
            for x in xs:
                c.accumulate(torch.from_numpy(x).cuda())
            outs.append(c.readout().cpu().numpy())
        ref = oracle.visibilities(xs[0]) + oracle.visibilities(xs[1])
        assert np.array_equal(np.concatenate(outs, axis=0).astype(np.int64), ref), product


def test_band_handles_batched_and_gated(xe):
    """Band handles in one batched launch (with whole-band handles beside them) and in a gated launch."""
    import torch
    N, F, T = 64, 4, 512
    x_np = synth.gauss(N, F, T, 2.5, 320)
    x = torch.from_numpy(x_np).cuda()
    parts = [xe.Correlator(N, F, T, bands=(0, 1)), xe.Correlator(N, F, T, bands=(1, 4))]
    other_np = synth.gauss(96, 2, 384, 2.0, 321)
    other = xe.Correlator(96, 2, 384)
    xe.accumulate_batch(parts + [other], [x, x, torch.from_numpy(other_np).cuda()])
    V = np.concatenate([c.readout().cpu().numpy() for c in parts], axis=0)
    assert np.array_equal(V.astype(np.int64), oracle.visibilities(x_np))
    assert np.array_equal(other.readout().cpu().numpy().astype(np.int64), oracle.visibilities(other_np))
    # gated: gate handles over bands [1, 3), a period below one chunk (gate segments) and one above
    # (gate arithmetic)
    for G, period, phase in [(3, 96, 10), (4, 256, 200)]:
        gates = [xe.Correlator(N, F, T, bands=(1, 3)) for _ in range(G)]
        xe.accumulate_gated(gates, x, period, phase)
        ref = oracle.gated(np.ascontiguousarray(x_np[:, 1:3, :]), G, period, phase)
        for g in range(G):
            assert np.array_equal(gates[g].readout().cpu().numpy().astype(np.int64), ref[g]), (period, g)
    torch.cuda.synchronize()


def test_band_range_rejects_bad_ranges(xe):
    for f0, f1 in [(-1, 2), (2, 2), (3, 2), (0, 5)]:
        with pytest.raises(xe.XEngineError):
            xe.Correlator(64, 4, 128, bands=(f0, f1))
