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


def _lag_case(kind, N, T, rng):
    if kind == "uniform100":
        return rng.integers(-100, 100, N)
    if kind == "span_limit":  # block 0 spans exactly the ring's 512 samples, block 1 one more
        lags = rng.integers(-200, 200, N)
        lags[0], lags[1] = -256, 256
        if N > 65:
            lags[64], lags[65] = -257, 256
        return lags
    if kind == "span_limit_wide":  # 128-element blocks: block 0 spans exactly the ring's 256 samples, block 1 one more
        lags = rng.integers(-100, 100, N)
        lags[0], lags[1] = -128, 128
        lags[128], lags[129] = -129, 128
        return lags
    if kind == "const_pos":
        return np.full(N, 300)
    if kind == "beyond_pos":
        return np.full(N, T + 100)
    if kind == "beyond_neg":
        return np.full(N, -(T + 100))
    if kind == "small":
        return rng.integers(-3, 4, N)
    if kind == "extreme":  # int32 ends: every such element is empty
        lags = rng.integers(-50, 50, N)
        lags[::7] = np.iinfo(np.int32).min
        lags[3::7] = np.iinfo(np.int32).max
        return lags
    raise ValueError(kind)


# Streaming (TMA ring) path: N % 16 == 0 and 16-byte aligned buffers; blocks of
# 64 elements below N = 128, of 128 from there. The cases cover ragged element
# blocks (N = 80, 176), ragged T, several time segments (T = 8192), each
# width's lag-range limit and one past it, constant lags, elements shifted out
# entirely and the int32 ends of the lag range.
@pytest.mark.parametrize("N,F,T,kind", [
    (80, 3, 1000, "uniform100"),
    (64, 2, 3000, "span_limit"),
    (256, 2, 3000, "span_limit_wide"),
    (176, 3, 1500, "uniform100"),
    (64, 1, 5000, "const_pos"),
    (64, 2, 700, "beyond_pos"),
    (64, 2, 700, "beyond_neg"),
    (256, 8, 8192, "uniform100"),
    (16, 1, 129, "small"),
    (96, 2, 2500, "extreme"),
])
def test_shift_streaming_matches_oracle(xe, N, F, T, kind):
    import torch
    x = synth.gauss(N, F, T, 2.5, 70 + N + T)
    lags = _lag_case(kind, N, T, np.random.default_rng(N * 31 + T)).astype(np.int32)
    y = xe.shift_lags(torch.from_numpy(x).cuda(), torch.from_numpy(lags).cuda())
    assert np.array_equal(y.cpu().numpy(), oracle.shift_lags(x, lags))


def test_shift_unaligned_input(xe):
    """An input starting one byte past an aligned address takes the staged kernel; same result."""
    import torch
    N, F, T = 64, 2, 1500
    x = synth.gauss(N, F, T, 2.5, 91)
    lags = np.random.default_rng(5).integers(-90, 90, N).astype(np.int32)
    buf = torch.empty(x.size + 1, dtype=torch.uint8, device="cuda")
    xin = buf[1:].view(T, F, N)
    xin.copy_(torch.from_numpy(x))
    y = xe.shift_lags(xin, torch.from_numpy(lags).cuda())
    assert np.array_equal(y.cpu().numpy(), oracle.shift_lags(x, lags))
