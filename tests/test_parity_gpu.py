"""GPU parity: the CUDA library against the CPU oracle, element by element (bit-exact).

Integer arithmetic has one correct answer, so the tolerance is zero.
"""
import ctypes

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


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_vis(xe, x, reps=1):
    import torch
    T, F, N = x.shape
    c = xe.Correlator(N, F, T)
    xd = to_dev(x)
    for _ in range(reps):
        c.accumulate(xd)
    V = c.readout()
    torch.cuda.synchronize()
    assert c.status() == 0
    out = V.cpu().numpy()
    c.close()
    return out


def assert_exact(V_gpu, V_ref):
    assert V_gpu.shape == V_ref.shape
    assert np.abs(V_ref).max(initial=0) < 2 ** 31
    bad = np.argwhere(V_gpu.astype(np.int64) != V_ref)
    assert bad.size == 0, f"{len(bad)} mismatches, first at {bad[:5].tolist()}"


SHAPES = [
    # (N, F, T): tiny config, ragged N around the 64-element tile, ragged T around the 128-sample stage
    (16, 4, 256), (1, 1, 16), (2, 3, 17), (15, 2, 100), (17, 3, 33), (32, 1, 1), (63, 2, 64), (64, 2, 64),
    (65, 1, 130), (100, 3, 300), (127, 1, 129), (128, 2, 63), (129, 2, 257), (200, 2, 1000), (256, 4, 1000),
    (300, 2, 640), (512, 1, 128), (48, 5, 4096),
]


@pytest.mark.parametrize("N,F,T", SHAPES)
def test_parity_small(xe, N, F, T):
    x = synth.uniform(N, F, T, 1000 + N + 7 * F + T) if (N + T) % 2 else synth.gauss(N, F, T, 2.5, N * F + T)
    assert_exact(gpu_vis(xe, x), oracle.visibilities(x))


def test_parity_tiny_config(xe):
    x = synth.TINY.make()
    assert_exact(gpu_vis(xe, x), oracle.visibilities(x))


def test_two_frames_add(xe):
    """Results are added to the previous results (Sec. III): V(a then b) = V(a) + V(b)."""
    import torch
    N, F, T = 200, 3, 512
    a, b = synth.gauss(N, F, T, 2.5, 1), synth.gauss(N, F, T, 3.0, 2)
    c = xe.Correlator(N, F, T)
    c.accumulate(to_dev(a))
    c.accumulate(to_dev(b))
    V = c.readout().cpu().numpy()
    assert c.samples == 2 * T
    assert_exact(V, oracle.visibilities(a) + oracle.visibilities(b))
    # reset starts a new integration
    c.readout(reset=True)
    assert c.samples == 0
    Z = c.readout().cpu().numpy()
    assert not Z.any()
    c.accumulate(to_dev(b))
    assert_exact(c.readout().cpu().numpy(), oracle.visibilities(b))
    torch.cuda.synchronize()


def test_split_time_path(xe):
    """Few tiles and a long integration: the time axis is split across CTAs (atomic adds)."""
    N, F, T = 64, 2, 8192
    x = synth.gauss(N, F, T, 2.5, 3)
    assert_exact(gpu_vis(xe, x), oracle.visibilities(x))
    assert_exact(gpu_vis(xe, x, reps=2), 2 * oracle.visibilities(x))


def test_extreme_values_to_the_sample_cap(xe):
    """All samples -8-8i up to the int32 cap: Re = 128 * 16777215 = 2147483520 exactly."""
    import torch
    T = xe.CORR_MAX_SAMPLES
    x = torch.zeros((T, 1, 16), dtype=torch.uint8, device="cuda")
    c = xe.Correlator(16, 1, T)
    c.accumulate(x)
    V = c.readout().cpu().numpy()
    assert (V[0, :, 0] == 128 * T).all() and not V[0, :, 1].any()
    with pytest.raises(xe.XEngineError) as ei:
        c.accumulate(x)
    assert ei.value.code == -4  # CORR_EOVERFLOW, nothing launched
    assert (c.readout().cpu().numpy()[0, :, 0] == 128 * T).all()
    c.close()


def test_overflow_guard_counts_samples(xe):
    T = 4 * 1024 * 1024
    c = xe.Correlator(16, 1, T)
    import torch
    x = torch.full((T, 1, 16), 0x88, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        c.accumulate(x)
    with pytest.raises(xe.XEngineError):
        c.accumulate(x)  # 4 * 2^22 = 16777216 > cap
    c.reset()
    c.accumulate(x)
    assert c.samples == T
    c.close()


def test_unaligned_input_pointer(xe):
    """A frame starting at an odd address goes through the aligned staging copy."""
    import torch
    N, F, T = 96, 2, 300
    x = synth.gauss(N, F, T, 2.5, 4)
    buf = torch.zeros(x.size + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = torch.from_numpy(x.ravel()).cuda()
    view = buf[1:].view(T, F, N)
    assert view.data_ptr() % 16 == 1
    c = xe.Correlator(N, F, T)
    c.accumulate(view)
    assert_exact(c.readout().cpu().numpy(), oracle.visibilities(x))


@pytest.mark.parametrize("N,F,T", [(256, 4, 1000), (17, 3, 777), (64, 8, 4096)])
def test_host_input_path(xe, N, F, T):
    """Host frames are copied in time chunks that overlap compute; same result."""
    import torch
    x = synth.gauss(N, F, T, 2.5, 5)
    c = xe.Correlator(N, F, T)
    pinned = torch.from_numpy(x).pin_memory()
    c.accumulate_host(pinned)
    c.accumulate_host(x)  # pageable works too
    out = np.empty((F, xe.baselines(N), 2), dtype=np.int32)
    c.readout_host(out, reset=True)
    c.synchronize()
    assert_exact(out, 2 * oracle.visibilities(x))


# (192, 8, 4096): input larger than output, two time chunks per frame; the others: output
# larger, one chunk per frame, so consecutive calls alternate the two chunk buffers
# ((512, 2, 300) with a ragged chunk, (100, 3, 200) with N % 16 != 0, rows padded in the copy)
@pytest.mark.parametrize("N,F,T", [(192, 8, 4096), (512, 2, 300), (100, 3, 200)])
def test_host_frames_back_to_back(xe, N, F, T):
    """Frame k+1's copies may overlap frame k's correlation and readout: each readout still
    holds exactly its own frame."""
    import torch
    frames = [synth.gauss(N, F, T, 2.0 + 0.5 * k, 80 + k) for k in range(4)]
    pinned = [torch.from_numpy(x).pin_memory() for x in frames]
    outs = [torch.empty((F, xe.baselines(N), 2), dtype=torch.int32).pin_memory() for _ in frames]
    c = xe.Correlator(N, F, T)
    for _ in range(2):  # twice: the second pass reuses the chunk buffers across calls
        for xh, o in zip(pinned, outs):
            c.accumulate_host(xh)
            c.readout_host(o, reset=True)
        c.synchronize()
        for x, o in zip(frames, outs):
            assert_exact(o.numpy(), oracle.visibilities(x))
    c.close()


def test_caller_owned_accumulators(xe):
    import torch
    N, F, T = 130, 2, 256
    x = synth.gauss(N, F, T, 2.5, 6)
    acc = torch.full((F * xe.baselines(N) * 2,), 12345, dtype=torch.int32, device="cuda")
    c = xe.Correlator(N, F, T, acc=acc)
    c.accumulate(to_dev(x))
    torch.cuda.synchronize()
    assert_exact(acc.view(F, -1, 2).cpu().numpy(), oracle.visibilities(x))


def test_streams_are_ordered(xe):
    import torch
    N, F, T = 128, 4, 2048
    a, b = synth.gauss(N, F, T, 2.5, 7), synth.gauss(N, F, T, 2.5, 8)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    da, db = to_dev(a), to_dev(b)
    torch.cuda.synchronize()
    c = xe.Correlator(N, F, T)
    c.accumulate(da, stream=s1)
    c.accumulate(db, stream=s2)
    out = torch.empty((F, xe.baselines(N), 2), dtype=torch.int32, device="cuda")
    c.readout(out, stream=s1)
    s1.synchronize()
    assert_exact(out.cpu().numpy(), oracle.visibilities(a) + oracle.visibilities(b))


def test_batch_call(xe):
    import torch
    frames = [(64, 3, 512), (200, 1, 256), (17, 2, 130)]
    cs, xs, refs = [], [], []
    for k, (N, F, T) in enumerate(frames):
        x = synth.gauss(N, F, T, 2.5, 40 + k)
        cs.append(xe.Correlator(N, F, T))
        xs.append(to_dev(x))
        refs.append(oracle.visibilities(x))
    xe.accumulate_batch(cs, xs)
    for c, r in zip(cs, refs):
        assert_exact(c.readout().cpu().numpy(), r)
    torch.cuda.synchronize()


@pytest.mark.parametrize("host", [False, True], ids=["device", "host"])
def test_overlapped_readouts(xe, host):
    """Readouts overlapped with the next integration (two accumulator sets): five integrations of two
    frames each, read out on a copy stream, each equal to the oracle; mixed with a plain readout; the
    host-input path; destroy with a copy out still in flight."""
    import torch
    N, F, T = 96, 3, 333
    frames = [synth.gauss(N, F, T, 2.5, 800 + k) for k in range(10)]
    c = xe.Correlator(N, F, T)
    cs = torch.cuda.Stream()
    outs = []
    for k in range(5):
        for x in frames[2 * k:2 * k + 2]:
            if k == 3:
                c.accumulate_host(x)
            else:
                c.accumulate(to_dev(x))
        if k == 2:  # a plain readout in between (with reset)
            outs.append(c.readout(reset=True).cpu())
            continue
        o = torch.empty((F, xe.baselines(N), 2), dtype=torch.int32, device="cpu" if host else "cuda")
        outs.append(c.readout_async(o.pin_memory() if host else o, cs))
    cs.synchronize()
    torch.cuda.synchronize()
    for k, o in enumerate(outs):
        ref = oracle.visibilities(frames[2 * k]) + oracle.visibilities(frames[2 * k + 1])
        assert_exact(o.cpu().numpy(), ref)
    # an empty integration reads as zeros; destroy waits for the copy out
    z = torch.full((F, xe.baselines(N), 2), 5, dtype=torch.int32, device="cuda")
    c.readout_async(z, cs)
    c.close()
    cs.synchronize()
    assert not z.cpu().numpy().any()
