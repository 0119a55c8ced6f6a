"""Parity at the full workload sizes, in the launch configuration the benchmark times.

N=256, F=256, T=16384 (Pathfinder shape) is compared in full against the
oracle; N=8192, F=4, T=2048 (large N with a common tone) on sampled entries,
every autocorrelation, the Freivalds identity for every row, and the
closed form of its tone-only variant.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def xe():
    import paper_1503_06203_gb300 as xe
    xe.build()
    return xe


def run(xe, x):
    import torch
    T, F, N = x.shape
    c = xe.Correlator(N, F, T)
    c.accumulate(torch.from_numpy(x).cuda())
    V = c.readout().cpu().numpy()
    assert c.status() == 0
    c.close()
    return V


def freivalds_check(x, V, seed=0):
    """sum_j V_ij w_j (V extended to the full Hermitian matrix) == oracle's O(NT) right-hand side."""
    T, F, N = x.shape
    rng = np.random.default_rng(seed)
    w = rng.integers(-3, 4, size=(F, N, 2)).astype(np.int64)
    rhs = oracle.freivalds_rhs(x, w)
    iu, ju = np.triu_indices(N)
    for f in range(F):
        wc = w[f, :, 0] + 1j * w[f, :, 1]
        Vc = V[f, :, 0].astype(np.float64) + 1j * V[f, :, 1].astype(np.float64)
        # upper part U (i <= j) applied to w, plus the strictly-lower part conj(U^T) applied to w
        t1 = Vc * wc[ju]
        off = iu != ju
        t2 = np.conj(Vc[off]) * wc[iu[off]]
        lhs_re = np.bincount(iu, weights=t1.real, minlength=N) + np.bincount(ju[off], weights=t2.real, minlength=N)
        lhs_im = np.bincount(iu, weights=t1.imag, minlength=N) + np.bincount(ju[off], weights=t2.imag, minlength=N)
        lhs = lhs_re + 1j * lhs_im
        # values stay below 2^53, so float64 sums are exact here
        assert np.array_equal(np.rint(lhs.real).astype(np.int64), rhs[f, :, 0])
        assert np.array_equal(np.rint(lhs.imag).astype(np.int64), rhs[f, :, 1])


def test_pathfinder_full(xe):
    x = synth.PATHFINDER.make()
    V = run(xe, x)
    ref = oracle.visibilities(x)
    assert np.array_equal(V.astype(np.int64), ref)


def test_large_n_sampled_and_freivalds(xe):
    fr = synth.LARGE_N
    x = fr.make()
    V = run(xe, x)
    N, F = fr.N, fr.F
    rng = np.random.default_rng(2)
    K = 20000
    f = rng.integers(0, F, K)
    i = rng.integers(0, N, K)
    j = rng.integers(0, N, K)
    i, j = np.minimum(i, j), np.maximum(i, j)
    # include the corners of the triangle and the tile edges
    edge = np.array([0, 63, 64, 127, 128, N - 65, N - 64, N - 1])
    ei, ej = np.meshgrid(edge, edge)
    keep = ei.ravel() <= ej.ravel()
    f = np.concatenate([f, np.zeros(keep.sum(), dtype=np.int64), np.full(keep.sum(), F - 1)])
    i = np.concatenate([i, ei.ravel()[keep], ei.ravel()[keep]])
    j = np.concatenate([j, ej.ravel()[keep], ej.ravel()[keep]])
    ref = oracle.entries(x, np.stack([f, i, j], 1))
    got = V[f, xe.packed_index(N, i, j)].astype(np.int64)
    assert np.array_equal(got, ref)
    # every autocorrelation
    re = (x >> 4).astype(np.int64) - 8
    im = (x & 15).astype(np.int64) - 8
    p = xe.packed_index(N, np.arange(N), np.arange(N))
    assert np.array_equal(V[:, p, 0], (re * re + im * im).sum(axis=0))
    assert not V[:, p, 1].any()
    freivalds_check(x, V)


def test_large_n_tone_only_closed_form(xe):
    fr = synth.LARGE_N_TONE_ONLY
    x = fr.make()
    V = run(xe, x)
    t = np.arange(fr.T)
    qr = np.clip(np.rint(3 * np.cos(2 * np.pi * fr.tone_k * t / fr.T)), -8, 7)
    qi = np.clip(np.rint(3 * np.sin(2 * np.pi * fr.tone_k * t / fr.T)), -8, 7)
    expect = int((qr * qr + qi * qi).sum())
    assert (V[:, :, 0] == expect).all()
    assert not V[:, :, 1].any()


def test_max_n_sampled_autos_freivalds_and_closed_form(xe):
    """N = CORR_MAX_N = 16384 (32,896 tiles per band, a 1.07 GB packed triangle): sampled entries at tile
    edges and at random, every autocorrelation, and the Freivalds identity for every row against the oracle;
    then one identical sequence on every element, whose visibilities are all (sum |q_t|^2, 0)."""
    from conftest import freivalds_rows
    N, F, T = xe.CORR_MAX_N, 1, 256
    x = synth.gauss(N, F, T, 2.5, 1601)
    V = run(xe, x)
    rng = np.random.default_rng(16)
    e = np.unique(np.concatenate([np.arange(0, N, 64), np.arange(63, N, 64)]))[::7]
    ei, ej = np.meshgrid(e, e, indexing="ij")
    keep = ei.ravel() <= ej.ravel()
    ri, rj = rng.integers(0, N, 3000), rng.integers(0, N, 3000)
    ii = np.concatenate([ei.ravel()[keep], np.minimum(ri, rj), np.arange(N)])
    jj = np.concatenate([ej.ravel()[keep], np.maximum(ri, rj), np.arange(N)])
    ff = np.zeros_like(ii)
    assert np.array_equal(V[ff, xe.packed_index(N, ii, jj)].astype(np.int64),
                          oracle.entries(x, np.stack([ff, ii, jj], 1)))
    w = rng.integers(-3, 4, size=(F, N, 2)).astype(np.int64)
    assert np.array_equal(freivalds_rows(V, w), oracle.freivalds_rhs(x, w))
    # closed form: one sequence q_t on every element
    q = synth.gauss(1, 1, T, 3.0, 1602)[:, 0, 0]
    xs = np.repeat(q[:, None, None], N, axis=2).astype(np.uint8)
    qr, qi = (q >> 4).astype(np.int64) - 8, (q & 15).astype(np.int64) - 8
    Vs = run(xe, np.ascontiguousarray(xs))
    assert (Vs[0, :, 0] == int((qr * qr + qi * qi).sum())).all() and not Vs[0, :, 1].any()
