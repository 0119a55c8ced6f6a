"""The lag-shift kernel (Sec. IV) against the oracle, and shift-then-correlate against the oracle."""
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


@pytest.mark.parametrize("N,F,T", [(64, 3, 500), (17, 2, 300), (256, 4, 2048), (1, 1, 5)])
def test_shift_matches_oracle(xe, N, F, T):
    import torch
    x = synth.gauss(N, F, T, 2.5, 50 + N)
    rng = np.random.default_rng(N)
    lags = rng.integers(-T // 3, T // 3, N).astype(np.int32)
    lags[0] = 0
    if N > 2:
        lags[1], lags[2] = T + 7, -T  # elements shifted entirely out of the frame
    y = xe.shift_lags(torch.from_numpy(x).cuda(), torch.from_numpy(lags).cuda())
    assert np.array_equal(y.cpu().numpy(), oracle.shift_lags(x, lags))


def test_shift_then_correlate(xe):
    import torch
    N, F, T = 128, 4, 4096
    x = synth.gauss(N, F, T, 2.5, 61)
    lags = np.random.default_rng(0).integers(-40, 40, N).astype(np.int32)
    xd = torch.from_numpy(x).cuda()
    y = xe.shift_lags(xd, torch.from_numpy(lags).cuda())
    with xe.Correlator(N, F, T) as c:
        c.accumulate(y)
        V = c.readout().cpu().numpy()
    assert np.array_equal(V.astype(np.int64), oracle.visibilities(oracle.shift_lags(x, lags)))
