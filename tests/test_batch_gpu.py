"""Batched uneven frames in one persistent launch (replayed as a CUDA graph) against the oracle."""
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


def small_batch(count, seed, tmax=1024):
    """The uneven-frame recipe with T capped so the oracle stays fast."""
    out = []
    for fr in synth.batched_frames(count, seed):
        T = min(fr.T, tmax)
        N = min(fr.N, 512)
        F = min(fr.F, 8)
        out.append(synth.Frame(N, F, T, "gauss", fr.sigma, fr.seed))
    return out


def run_batch(xe, frames, cors=None, reps=1):
    import torch
    cors = cors or [xe.Correlator(f.N, f.F, f.T) for f in frames]
    xs = [f.make() for f in frames]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    for _ in range(reps):
        xe.accumulate_batch(cors, xd)
    outs = [c.readout().cpu().numpy() for c in cors]
    torch.cuda.synchronize()
    return cors, xs, outs


def test_batch_matches_oracle(xe):
    frames = small_batch(12, 1003)
    _, xs, outs = run_batch(xe, frames)
    for x, V in zip(xs, outs):
        assert np.array_equal(V.astype(np.int64), oracle.visibilities(x))


def test_batch_graph_replay_and_rebuild(xe):
    """Same sizes twice (graph replay with new frames), then new sizes (rebuild); results add up."""
    import torch
    frames = small_batch(5, 77)
    cors = [xe.Correlator(f.N, f.F, f.T) for f in frames]
    xs1 = [f.make() for f in frames]
    xs2 = [synth.gauss(f.N, f.F, f.T, 2.0, f.seed + 99) for f in frames]
    xe.accumulate_batch(cors, [torch.from_numpy(x).cuda() for x in xs1])
    xe.accumulate_batch(cors, [torch.from_numpy(x).cuda() for x in xs2])
    for c, a, b in zip(cors, xs1, xs2):
        assert np.array_equal(c.readout(reset=True).cpu().numpy().astype(np.int64),
                              oracle.visibilities(a) + oracle.visibilities(b))
    # a different batch (fewer frames, other sizes) rebuilds the graph
    sub = cors[1:4]
    xs3 = [synth.gauss(c.N, c.F, c.T, 3.0, 5 + k) for k, c in enumerate(sub)]
    xe.accumulate_batch(sub, [torch.from_numpy(x).cuda() for x in xs3])
    for c, x in zip(sub, xs3):
        assert np.array_equal(c.readout().cpu().numpy().astype(np.int64), oracle.visibilities(x))
    torch.cuda.synchronize()


def test_batch_rejects_duplicates_and_overflow(xe):
    import torch
    c = xe.Correlator(64, 1, 256)
    x = torch.zeros((256, 1, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(xe.XEngineError):
        xe.accumulate_batch([c, c], [x, x])
    T = 8 * 1024 * 1024
    big = xe.Correlator(16, 1, T)
    xb = torch.zeros((T, 1, 16), dtype=torch.uint8, device="cuda")
    xe.accumulate_batch([big], [xb])
    with pytest.raises(xe.XEngineError) as ei:  # 2 * 2^23 = 16777216 > 16777215
        xe.accumulate_batch([big], [xb])
    assert ei.value.code == -4
    assert big.samples == T
    V = big.readout().cpu().numpy()
    assert (V[0, :, 0] == 128 * T).all() and not V[0, :, 1].any()


@pytest.mark.slow
def test_full_uneven_batch_sampled_and_freivalds(xe):
    """All 64 frames of the uneven-frame workload in one launch: sampled entries, autos, Freivalds per frame."""
    import torch
    frames = synth.batched_frames()
    cors = [xe.Correlator(f.N, f.F, f.T) for f in frames]
    xs = [f.make() for f in frames]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    xe.accumulate_batch(cors, xd)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    for k, (fr, c, x) in enumerate(zip(frames, cors, xs)):
        V = c.readout().cpu().numpy()
        K = 300
        f = rng.integers(0, fr.F, K)
        i = rng.integers(0, fr.N, K)
        j = rng.integers(0, fr.N, K)
        i, j = np.minimum(i, j), np.maximum(i, j)
        assert np.array_equal(V[f, xe.packed_index(fr.N, i, j)].astype(np.int64),
                              oracle.entries(x, np.stack([f, i, j], 1))), k
        w = rng.integers(-3, 4, size=(fr.F, fr.N, 2)).astype(np.int64)
        rhs = oracle.freivalds_rhs(x, w)
        iu, ju = np.triu_indices(fr.N)
        for b in range(fr.F):
            wc = w[b, :, 0] + 1j * w[b, :, 1]
            Vc = V[b, :, 0].astype(np.float64) + 1j * V[b, :, 1].astype(np.float64)
            t1 = Vc * wc[ju]
            off = iu != ju
            t2 = np.conj(Vc[off]) * wc[iu[off]]
            lr = np.bincount(iu, weights=t1.real, minlength=fr.N) + np.bincount(ju[off], weights=t2.real, minlength=fr.N)
            li = np.bincount(iu, weights=t1.imag, minlength=fr.N) + np.bincount(ju[off], weights=t2.imag, minlength=fr.N)
            assert np.array_equal(np.rint(lr).astype(np.int64), rhs[b, :, 0]), (k, b)
            assert np.array_equal(np.rint(li).astype(np.int64), rhs[b, :, 1]), (k, b)


def test_batch_time_split_and_ring_reuse(xe):
    """A lone frame with few tiles and a long time axis is cut into time ranges (atomic adds onto
    zeroed, then onto resident sums); ten launches of changing sizes cycle through every launch set."""
    import torch
    N, F, T = 64, 1, 8192  # one tile, 64 chunks: split across many CTAs
    c = xe.Correlator(N, F, T)
    xs = [synth.gauss(N, F, T, 2.5, 600 + k) for k in range(2)]
    for x in xs:
        xe.accumulate_batch([c], [torch.from_numpy(x).cuda()])
    assert np.array_equal(c.readout(reset=True).cpu().numpy().astype(np.int64),
                          oracle.visibilities(xs[0]) + oracle.visibilities(xs[1]))
    frames = small_batch(10, 31)
    cors = [xe.Correlator(f.N, f.F, f.T) for f in frames]
    for k in range(10):
        sub = list(range(k % 5, len(frames), 1 + k % 3))
        xk = [synth.gauss(frames[i].N, frames[i].F, frames[i].T, 2.5, 700 + 10 * k + i) for i in sub]
        xe.accumulate_batch([cors[i] for i in sub], [torch.from_numpy(x).cuda() for x in xk])
        for i, x in zip(sub, xk):
            assert np.array_equal(cors[i].readout(reset=True).cpu().numpy().astype(np.int64),
                                  oracle.visibilities(x)), (k, i)
    torch.cuda.synchronize()


def test_batch_frames_that_fill_the_gpu_run_alone(xe):
    """Frames whose tiles fill every SM CORR_BATCH_ALONE_WAVES times run alone (single-frame kernel),
    the rest share the batched launch: every result equals the oracle, twice in a row (adds onto
    resident sums), with the routes mixed in one call. Time pieces (fewer samples than the handle's
    T) of such frames run alone where the handle's schedule keeps tiles whole, and share the
    batched launch where it splits the time axis."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    big_f = -(-xe.CORR_BATCH_ALONE_WAVES * sms // 36)  # N = 512: 36 tiles per band
    even_f = big_f  # the fewest bands from there whose tiles fill whole waves of SMs: no time split
    while (36 * even_f) % sms:
        even_f += 1
    shapes = [(512, big_f, 256), (64, 2, 300), (1024, -(-xe.CORR_BATCH_ALONE_WAVES * sms // 136), 128),
              (200, 3, 1000), (512, big_f, 384), (512, even_f, 256)]
    alone = [xe.batch_runs_alone(N, F, sms) for N, F, _ in shapes]
    assert alone == [True, False, True, False, True, True]
    split = [(np.asarray(xe.plan_schedule(N, F, T, sms)[0])[:, 2] != 0).any() for N, F, T in shapes]
    assert not split[5] and split[4]  # piece 5 runs alone over whole tiles; piece 4 stays shared
    cors = [xe.Correlator(N, F, T) for N, F, T in shapes]
    xs = [synth.gauss(N, F, T, 2.5, 900 + k) for k, (N, F, T) in enumerate(shapes)]
    xs[4] = np.ascontiguousarray(xs[4][:200])  # 200 of the handle's 384 samples
    xs[5] = np.ascontiguousarray(xs[5][:200])  # 200 of 256: a ragged last chunk
    xd = [torch.from_numpy(x).cuda() for x in xs]
    for _ in range(2):
        xe.accumulate_batch(cors, xd)
    for k, (c, x) in enumerate(zip(cors, xs)):
        assert np.array_equal(c.readout().cpu().numpy().astype(np.int64), 2 * oracle.visibilities(x)), k
    torch.cuda.synchronize()
