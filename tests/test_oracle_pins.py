"""Pins of the CPU oracle to facts fixed outside it (no GPU).

Each test pins the oracle against something other than itself: hand-worked
cases from Eq. 1, brute force with Python complex numbers, a numpy matmul
special case, Hermitian symmetry, the autocorrelation identity, the closed
form for identical sequences, the Freivalds identity and the Eq. 3 offset
identity. A plausible slip (swapped nibbles, a flipped Im sign, i and j
exchanged, a dropped term, a wrong packed index or band stride) fails at
least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import read_decode_cases, read_hand_cases


def decode_np(x):
    # decoding restated for the brute-force pins; itself pinned by test_decode_golden
    return (x >> 4).astype(np.int64) - 8, (x & 15).astype(np.int64) - 8


def test_decode_golden():
    """Single-byte excess-8 decoding (Sec. III) against the hand-decoded table."""
    for b, re, im in read_decode_cases():
        x = np.array([[[b]]], dtype=np.uint8)
        V = oracle.visibilities(x)
        # an auto of one sample is |x|^2 = re^2 + im^2, Im = 0
        assert tuple(V[0, 0]) == (re * re + im * im, 0), hex(b)
        # the cross term against 1+0i (byte 0x98) reads x * conj(1) = (re, im)
        x2 = np.array([[[b, 0x98]]], dtype=np.uint8)
        V2 = oracle.visibilities(x2)
        assert tuple(V2[0, 1]) == (re, im), hex(b)
        # and against 0+1i (byte 0x89): x * conj(i) = x * (-i) = (im, -re)
        x3 = np.array([[[b, 0x89]]], dtype=np.uint8)
        assert tuple(oracle.visibilities(x3)[0, 1]) == (im, -re), hex(b)


@pytest.mark.parametrize("case", read_hand_cases(), ids=lambda c: c[0])
def test_hand_cases(case):
    """Hand-worked Eq. 1 visibilities (tests/golden/hand_cases.txt)."""
    name, N, F, T, x, Vexp = case
    V = oracle.visibilities(x)
    for (f, i, j), val in Vexp.items():
        assert tuple(V[f, oracle.packed_index(N, i, j)]) == val, (name, f, i, j)
    assert len(Vexp) == F * oracle.baselines(N)


def test_all_byte_pairs_brute_force():
    """Every byte value against every byte value (N=2, T=1): Python complex X*conj(Y)."""
    vals = np.arange(256, dtype=np.uint8)
    a, b = np.meshgrid(vals, vals, indexing="ij")
    x = np.stack([a.ravel(), b.ravel()], axis=1).reshape(1, -1, 2).astype(np.uint8)  # T=1, F=65536, N=2
    V = oracle.visibilities(np.ascontiguousarray(x))
    # each byte decoded once with Python integers: value = nibble - 8, high nibble real
    dec = [complex((v >> 4) - 8, (v & 15) - 8) for v in range(256)]
    A, Bv = a.ravel(), b.ravel()
    for k in range(65536):  # every one of the 256 x 256 byte pairs
        X, Y = dec[int(A[k])], dec[int(Bv[k])]
        z = X * Y.conjugate()
        assert (int(V[k, 1, 0]), int(V[k, 1, 1])) == (int(z.real), int(z.imag)), k
        assert (int(V[k, 0, 0]), int(V[k, 0, 1])) == (int((X * X.conjugate()).real), 0), k
        assert (int(V[k, 2, 0]), int(V[k, 2, 1])) == (int((Y * Y.conjugate()).real), 0), k


@pytest.mark.parametrize("N,F,T,seed", [(1, 1, 1, 1), (3, 2, 5, 2), (8, 3, 16, 3), (5, 1, 13, 4)])
def test_brute_force_complex(N, F, T, seed):
    """Tiny inputs: the definition enumerated with Python complex numbers."""
    x = synth.uniform(N, F, T, seed)
    V = oracle.visibilities(x)
    re, im = decode_np(x)
    for f in range(F):
        for i in range(N):
            for j in range(i, N):
                z = sum(complex(re[t, f, i], im[t, f, i]) * complex(re[t, f, j], -im[t, f, j]) for t in range(T))
                assert tuple(V[f, oracle.packed_index(N, i, j)]) == (int(z.real), int(z.imag))


@pytest.mark.parametrize("N,F,T,seed", [(16, 4, 256, 1000), (37, 3, 200, 5), (64, 2, 1000, 6)])
def test_numpy_matmul_special_case(N, F, T, seed):
    """Re = Xr Xr^T + Xi Xi^T, Im = Xi Xr^T - Xr Xi^T per band (numpy int64 matmul)."""
    x = synth.uniform(N, F, T, seed) if seed != 6 else synth.gauss(N, F, T, 2.5, seed)
    V = oracle.visibilities(x)
    re, im = decode_np(x)
    iu, ju = np.triu_indices(N)
    for f in range(F):
        Xr, Xi = re[:, f, :].T, im[:, f, :].T  # [N][T]
        R = Xr @ Xr.T + Xi @ Xi.T
        I = Xi @ Xr.T - Xr @ Xi.T
        assert np.array_equal(V[f, :, 0], R[iu, ju])
        assert np.array_equal(V[f, :, 1], I[iu, ju])


def test_packed_index_row_major():
    """p(i,j) walks the upper triangle row by row, autos first in each row."""
    N = 7
    order = [(i, j) for i in range(N) for j in range(i, N)]
    assert [oracle.packed_index(N, i, j) for i, j in order] == list(range(len(order)))


@pytest.mark.parametrize("N,F,T", [(12, 3, 40), (33, 2, 64)])
def test_hermitian_and_packing(N, F, T):
    """The full square is Hermitian (Sec. II.A) and the packed triangle is its upper part."""
    x = synth.gauss(N, F, T, 2.5, 11)
    full = oracle.visibilities_full(x)
    assert np.array_equal(full[:, :, :, 0], full[:, :, :, 0].transpose(0, 2, 1))
    assert np.array_equal(full[:, :, :, 1], -full[:, :, :, 1].transpose(0, 2, 1))
    V = oracle.visibilities(x)
    iu, ju = np.triu_indices(N)
    assert np.array_equal(V, full[:, iu, ju, :])


def test_autos_are_power():
    """V[f,i,i] = (sum_t xr^2 + xi^2, 0)."""
    x = synth.gauss(50, 3, 333, 3.0, 12)
    V = oracle.visibilities(x)
    re, im = decode_np(x)
    p = np.array([oracle.packed_index(50, i, i) for i in range(50)])
    assert np.array_equal(V[:, p, 0], (re * re + im * im).sum(axis=0))
    assert not V[:, p, 1].any()


def test_identical_sequences_closed_form():
    """Every element carries one sequence q_t: every visibility is (sum |q_t|^2, 0).

    The tone-only generator (sigma = 0) gives q_t = (rint(3 cos th), rint(3 sin th)),
    th = 2 pi k t / T, identical for all elements and bands.
    """
    N, F, T, k = 64, 2, 2048, synth.TONE_K
    x = synth.gauss(N, F, T, 0.0, 1, tone_amp=3.0, tone_k=k)
    t = np.arange(T)
    qr = np.clip(np.rint(3 * np.cos(2 * np.pi * k * t / T)), -8, 7)
    qi = np.clip(np.rint(3 * np.sin(2 * np.pi * k * t / T)), -8, 7)
    expect = int((qr * qr + qi * qi).sum())
    V = oracle.visibilities(x)
    assert (V[:, :, 0] == expect).all() and not V[:, :, 1].any()
    # and one repeated byte: 0x97 = 1-1i everywhere -> (2T, 0)
    x = np.full((256, 4, 16), 0x97, dtype=np.uint8)
    V = oracle.visibilities(x)
    assert (V[:, :, 0] == 512).all() and not V[:, :, 1].any()


def test_freivalds_identity():
    """sum_j V_ij w_j over the full Hermitian V equals sum_t x_i sum_j conj(x_j) w_j."""
    N, F, T = 40, 3, 300
    x = synth.gauss(N, F, T, 2.5, 13)
    rng = np.random.default_rng(0)
    w = rng.integers(-3, 4, size=(F, N, 2)).astype(np.int64)
    r = oracle.freivalds_rhs(x, w)
    full = oracle.visibilities_full(x)
    Vc = full[..., 0] + 1j * full[..., 1]
    lhs = np.einsum("fij,fj->fi", Vc, w[..., 0] + 1j * w[..., 1])
    assert np.array_equal(lhs.real.astype(np.int64), r[..., 0])
    assert np.array_equal(lhs.imag.astype(np.int64), r[..., 1])
    # brute force for one band, one row, with Python complex numbers
    re, im = decode_np(x)
    i = 7
    z = 0
    for t in range(T):
        s = sum(complex(re[t, 0, j], -im[t, 0, j]) * complex(w[0, j, 0], w[0, j, 1]) for j in range(N))
        z += complex(re[t, 0, i], im[t, 0, i]) * s
    assert (int(z.real), int(z.imag)) == tuple(r[0, i])


def test_eq3_offset_identity():
    """Eq. 3: encoded-value products plus the offsets give the signed correlation."""
    N, F, T = 20, 2, 77
    x = synth.uniform(N, F, T, 14)
    ur, ui = (x >> 4).astype(np.int64), (x & 15).astype(np.int64)
    Boff = oracle.offset_terms(x)
    V = oracle.visibilities(x)
    iu, ju = np.triu_indices(N)
    for f in range(F):
        Ur, Ui = ur[:, f, :].T, ui[:, f, :].T
        Renc = (Ur @ Ur.T + Ui @ Ui.T)[iu, ju]
        Ienc = (Ui @ Ur.T - Ur @ Ui.T)[iu, ju]
        assert np.array_equal(Renc + Boff[f, :, 0], V[f, :, 0])
        assert np.array_equal(Ienc + Boff[f, :, 1], V[f, :, 1])


def test_entries_match_packed():
    N, F, T = 70, 3, 129
    x = synth.gauss(N, F, T, 2.0, 15)
    V = oracle.visibilities(x)
    rng = np.random.default_rng(1)
    f = rng.integers(0, F, 200)
    i = rng.integers(0, N, 200)
    j = rng.integers(0, N, 200)
    i, j = np.minimum(i, j), np.maximum(i, j)
    e = oracle.entries(x, np.stack([f, i, j], 1))
    assert np.array_equal(e, V[f, oracle.packed_index(N, i, j)])
    # lower-triangle requests give the conjugate
    e2 = oracle.entries(x, np.stack([f, j, i], 1))
    assert np.array_equal(e2[:, 0], e[:, 0]) and np.array_equal(e2[:, 1], -e[:, 1])


def test_extreme_magnitudes():
    """All samples -8-8i: |Re| reaches the 128-per-sample bound the overflow guard uses."""
    x = np.zeros((1000, 1, 3), dtype=np.uint8)
    V = oracle.visibilities(x)
    assert (V[0, :, 0] == 128 * 1000).all() and not V[0, :, 1].any()
    # Im bound: X = -8+7i, Y = 7-8i... |Im| = |XiYr - XrYi| = |49 - 64| ; max over values is 120
    best = max(abs(xi * yr - xr * yi) for xr, xi, yr, yi in itertools.product(range(-8, 8), repeat=4))
    assert best == 120


def test_thread_count_invariance():
    x = synth.gauss(45, 5, 100, 2.5, 16)
    assert np.array_equal(oracle.visibilities(x, 1), oracle.visibilities(x, 7))


def test_shift_lags_pins():
    """Sec. IV lag shift: zero lag is the identity; a lag moves samples in time, zero-filled."""
    N, F, T = 6, 2, 40
    x = synth.uniform(N, F, T, 21)
    assert np.array_equal(oracle.shift_lags(x, np.zeros(N)), x)
    lags = np.array([0, 3, -2, T + 5, -T, 1], dtype=np.int32)
    y = oracle.shift_lags(x, lags)
    for i, L in enumerate(lags):
        for t in range(T):
            src = t - L
            want = x[src, :, i] if 0 <= src < T else np.full(F, 0x88, np.uint8)
            assert np.array_equal(y[t, :, i], want), (i, t)
    # shifting by L then by -L restores the samples that stayed inside the frame
    z = oracle.shift_lags(oracle.shift_lags(x, lags), -lags)
    for i, L in enumerate(lags):
        keep = [t for t in range(T) if 0 <= t + L < T]
        assert np.array_equal(z[keep, :, i], x[keep, :, i])


def test_shift_lags_compensates_a_delay():
    """Element 1 is element 0 delayed by d samples; shifting element 1 by -d aligns them, so
    V01 becomes element 0's autocorrelation over the samples both still hold."""
    N, F, T, d = 2, 1, 200, 17
    base = synth.gauss(1, F, T, 2.5, 22)[:, :, 0]
    x = np.full((T, F, N), 0x88, dtype=np.uint8)
    x[:, :, 0] = base
    x[d:, :, 1] = base[:T - d]          # delayed copy
    y = oracle.shift_lags(x, np.array([0, -d], dtype=np.int32))
    V = oracle.visibilities(y)
    part = np.ascontiguousarray(x[:T - d, :, :1])  # samples 0 .. T-d-1 of element 0
    auto = oracle.visibilities(part)[0, 0]
    assert tuple(V[0, 1]) == (auto[0], 0)


def test_gated_pins():
    """Sec. IV gating: one gate is the plain correlation; gates partition the samples."""
    x = synth.gauss(12, 2, 300, 2.5, 23)
    plain = oracle.visibilities(x)
    assert np.array_equal(oracle.gated(x, 1, 37, 5)[0], plain)
    for G, period, phase in [(4, 64, 0), (3, 50, 17), (8, 300, 299)]:
        V = oracle.gated(x, G, period, phase)
        assert np.array_equal(V.sum(axis=0), plain)
    # hand-derived gates for period 4, G 2, phase 1: t = 0..7 -> 0,1,1,0,0,1,1,0
    T = 8
    xs = np.full((T, 1, 2), 0x88, dtype=np.uint8)
    for t in range(T):
        xs[t, 0, 0] = 0x98 + t  # element 0 = 1 + (t)i... distinct samples
    V = oracle.gated(xs, 2, 4, 1)
    gates = [0, 1, 1, 0, 0, 1, 1, 0]
    for g in range(2):
        want = sum(int((xs[t, 0, 0] >> 4) - 8) ** 2 + int((xs[t, 0, 0] & 15) - 8) ** 2 for t in range(T) if gates[t] == g)
        assert V[g, 0, 0, 0] == want


def test_gated_pulse_closed_form():
    """A common pulse in gate 0's window only: gate 0 holds (sum |q|^2, 0) on every baseline, others zero."""
    N, F, T, G, period = 16, 2, 512, 4, 64
    q = synth.gauss(1, 1, T, 3.0, 24)[:, 0, 0]
    x = np.full((T, F, N), 0x88, dtype=np.uint8)
    on = np.array([((t % period) * G // period) == 0 for t in range(T)])
    x[on] = q[on, None, None]
    V = oracle.gated(x, G, period, 0)
    qr, qi = (q[on] >> 4).astype(np.int64) - 8, (q[on] & 15).astype(np.int64) - 8
    assert (V[0, :, :, 0] == int((qr * qr + qi * qi).sum())).all() and not V[0, :, :, 1].any()
    assert not V[1:].any()


def test_freivalds_rows_helper():
    """The test helper that forms V w from a packed triangle (Hermitian extension) against the oracle's rhs."""
    from conftest import freivalds_rows
    x = synth.gauss(70, 3, 150, 2.5, 25)
    w = np.random.default_rng(2).integers(-3, 4, size=(3, 70, 2)).astype(np.int64)
    assert np.array_equal(freivalds_rows(oracle.visibilities(x), w), oracle.freivalds_rhs(x, w))
