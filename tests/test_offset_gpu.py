"""The offset-encoded operand route (Eq. 3; CORR_OPT_PRODUCT = 2) against the oracle, bit-exact.

The library multiplies the encoded nibbles (unsigned), seeds the output with
offset terms built from per-element nibble sums, and adds the folded products
onto them. The first test checks that algebra on the CPU with numpy; the rest
run the CUDA route and compare with the oracle's plain definition.
"""
import numpy as np
import pytest

import oracle
import synth


def test_three_product_offset_algebra():
    """Re, Im from encoded products plus the offset terms equal the plain definition (CPU, numpy)."""
    for N, F, T, seed in [(7, 2, 50, 1), (16, 1, 300, 2), (3, 3, 1, 3)]:
        x = synth.uniform(N, F, T, 40 + seed)
        Xr = (x >> 4).astype(np.int64)
        Xi = (x & 15).astype(np.int64)
        E1 = np.einsum("tfi,tfj->fij", Xr, Xr)
        E2 = np.einsum("tfi,tfj->fij", Xi, Xi)
        E3 = np.einsum("tfi,tfj->fij", Xr + Xi, Xr - Xi + 15)
        R, I = Xr.sum(0), Xi.sum(0)  # [F][N]
        Ri, Ii, Rj, Ij = R[:, :, None], I[:, :, None], R[:, None, :], I[:, None, :]
        re = E1 + E2 - 8 * (Ri + Rj + Ii + Ij) + 128 * T
        im = (E3 - E1 + E2) - 7 * Ri - 23 * Ii - 8 * Rj + 8 * Ij
        full = oracle.visibilities_full(x)
        assert np.array_equal(re, full[..., 0]) and np.array_equal(im, full[..., 1])


@pytest.fixture(scope="module")
def xe():
    import paper_1503_06203_gb300 as xe
    xe.build()
    return xe


def enc_vis(xe, x, reps=1, split=0):
    import torch
    T, F, N = x.shape
    with xe.Correlator(N, F, T) as c:
        c.set_option(xe.CORR_OPT_PRODUCT, 2)
        c.set_option(xe.CORR_OPT_SPLIT, split)
        assert c.get_option(xe.CORR_OPT_PRODUCT) == 2
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        for _ in range(reps):
            c.accumulate(xd)
        V = c.readout().cpu().numpy()
        assert c.status() == 0
    return V.astype(np.int64)


@pytest.mark.gpu
@pytest.mark.parametrize("N,F,T", [(16, 4, 256), (1, 1, 16), (17, 3, 33), (63, 2, 64), (65, 1, 130),
                                   (100, 3, 300), (129, 2, 257), (256, 4, 1000), (300, 2, 640), (48, 5, 4096)])
def test_offset_route_matches_oracle(xe, N, F, T):
    x = synth.uniform(N, F, T, 500 + N + T) if (N + T) % 2 else synth.gauss(N, F, T, 2.5, 600 + N * F + T)
    assert np.array_equal(enc_vis(xe, x), oracle.visibilities(x))


@pytest.mark.gpu
def test_offset_route_adds_and_splits(xe):
    """Seeds are added onto resident sums (second frame) and time-split items add atomically onto seeds."""
    N, F, T = 64, 2, 8192
    x = synth.gauss(N, F, T, 2.5, 77)
    ref = oracle.visibilities(x)
    assert np.array_equal(enc_vis(xe, x, reps=2), 2 * ref)
    assert np.array_equal(enc_vis(xe, x, split=4), ref)
    assert np.array_equal(enc_vis(xe, x, reps=2, split=4), 2 * ref)


@pytest.mark.gpu
def test_offset_route_host_input(xe):
    N, F, T = 96, 3, 3000
    x = synth.gauss(N, F, T, 2.5, 78)
    with xe.Correlator(N, F, T) as c:
        c.set_option(xe.CORR_OPT_PRODUCT, 2)
        c.accumulate_host(x)
        V = c.readout().cpu().numpy().astype(np.int64)
    assert np.array_equal(V, oracle.visibilities(x))


@pytest.mark.gpu
@pytest.mark.parametrize("byte,re_per_sample", [(0x00, 128), (0xFF, 98)])
def test_offset_route_extremes_wrap_exactly(xe, byte, re_per_sample):
    """Constant -8-8i (all-zero codes) and 7+7i (0xFF): the encoded products wrap int32 for long
    integrations, the final sums are still exact."""
    import torch
    T = 1 << 22
    with xe.Correlator(16, 1, T) as c:
        c.set_option(xe.CORR_OPT_PRODUCT, 2)
        c.accumulate(torch.full((T, 1, 16), byte, dtype=torch.uint8, device="cuda"))
        V = c.readout().cpu().numpy().astype(np.int64)
    assert (V[0, :, 0] == re_per_sample * T).all() and not V[0, :, 1].any()
