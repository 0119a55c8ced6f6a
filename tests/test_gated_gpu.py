"""Gated correlation (Sec. IV) on the GPU against the oracle."""
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


@pytest.mark.parametrize("N,F,T,G,period,phase", [
    (64, 2, 1024, 4, 256, 0),      # gate edges on chunk boundaries
    (96, 3, 1000, 3, 100, 37),     # edges inside chunks, ragged end
    (17, 1, 777, 5, 777, 5),       # one period, unaligned rows (staging)
    (256, 2, 4096, 8, 512, 300),
    # periods of a chunk or more run the gate-arithmetic kernel: every chunk meets its gate in two runs,
    # gates of many chunks, a frame shorter than a period (gates without samples), many gates
    (64, 2, 1024, 2, 128, 50),
    (128, 1, 5000, 8, 16384, 1000),
    (64, 3, 300, 4, 1024, 900),
    (96, 1, 3000, 7, 1000, 999),
    (64, 1, 4096, 64, 4096, 17),
])
def test_gated_matches_oracle(xe, N, F, T, G, period, phase):
    import torch
    x = synth.gauss(N, F, T, 2.5, 80 + G)
    gates = [xe.Correlator(N, F, T) for _ in range(G)]
    xe.accumulate_gated(gates, torch.from_numpy(x).cuda(), period, phase)
    ref = oracle.gated(x, G, period, phase)
    for g, c in enumerate(gates):
        assert np.array_equal(c.readout().cpu().numpy().astype(np.int64), ref[g]), g
    # a second frame adds on
    x2 = synth.gauss(N, F, T, 2.0, 90 + G)
    xe.accumulate_gated(gates, torch.from_numpy(x2).cuda(), period, phase)
    ref2 = ref + oracle.gated(x2, G, period, phase)
    for g, c in enumerate(gates):
        assert np.array_equal(c.readout().cpu().numpy().astype(np.int64), ref2[g]), g
    torch.cuda.synchronize()


def test_gated_pulse(xe):
    """A pulse in gate 0's window shows up only in gate 0, with its closed form."""
    import torch
    N, F, T, G, period = 64, 2, 2048, 4, 256
    q = synth.gauss(1, 1, T, 3.0, 99)[:, 0, 0]
    x = np.full((T, F, N), 0x88, dtype=np.uint8)
    on = np.array([((t % period) * G // period) == 0 for t in range(T)])
    x[on] = q[on, None, None]
    gates = [xe.Correlator(N, F, T) for _ in range(G)]
    xe.accumulate_gated(gates, torch.from_numpy(x).cuda(), period, 0)
    qr, qi = (q[on] >> 4).astype(np.int64) - 8, (q[on] & 15).astype(np.int64) - 8
    V0 = gates[0].readout().cpu().numpy()
    assert (V0[:, :, 0] == int((qr * qr + qi * qi).sum())).all() and not V0[:, :, 1].any()
    for c in gates[1:]:
        assert not c.readout().cpu().numpy().any()
