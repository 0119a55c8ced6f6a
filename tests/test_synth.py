"""The seeded input generator: C library against its numpy restatement (no GPU)."""
import numpy as np
import pytest

import synth


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: the first outputs are published widely
    # (e.g. in the reference implementation accompanying xoshiro).
    assert synth.draw(0, 0) == 0xE220A8397B1DCDAF
    assert synth.draw(0, 1) == 0x6E789E6AA1B965F4
    assert int(synth.draw_np(0, np.array([0, 1], dtype=np.uint64))[1]) == 0x6E789E6AA1B965F4


@pytest.mark.parametrize("N,F,T,seed", [(16, 4, 256, 1000), (7, 3, 11, 2), (1, 1, 1, 3)])
def test_uniform_matches_numpy(N, F, T, seed):
    assert np.array_equal(synth.uniform(N, F, T, seed), synth.uniform_np(N, F, T, seed))


@pytest.mark.parametrize("N,F,T,sigma,tone", [(33, 5, 64, 2.5, 0.0), (20, 2, 128, 2.5, 3.0), (8, 1, 256, 0.0, 3.0)])
def test_gauss_matches_numpy(N, F, T, sigma, tone):
    a = synth.gauss(N, F, T, sigma, 77, tone, synth.TONE_K)
    b = synth.gauss_np(N, F, T, sigma, 77, tone, synth.TONE_K)
    assert np.array_equal(a, b)


def test_thread_invariance():
    a = synth.gauss(64, 8, 300, 2.5, 5, nthreads=1)
    b = synth.gauss(64, 8, 300, 2.5, 5, nthreads=13)
    assert np.array_equal(a, b)


def test_gauss_statistics():
    x = synth.gauss(256, 16, 512, 2.5, 1001)
    re = (x >> 4).astype(np.int64) - 8
    im = (x & 15).astype(np.int64) - 8
    assert abs(re.mean()) < 0.02 and abs(im.mean()) < 0.02
    assert 2.4 < re.std() < 2.6 and 2.4 < im.std() < 2.6
    assert re.min() == -8 and re.max() == 7


def test_batched_recipe():
    fr = synth.batched_frames()
    assert len(fr) == 64
    assert all(f.N in synth.BATCH_N_CHOICES and 1 <= f.F <= 64 and 512 <= f.T <= 8192 and f.T % 256 == 0
               and 1.5 <= f.sigma <= 3.5 for f in fr)
    assert fr == synth.batched_frames()


def test_gauss_flat_is_the_flat_generator():
    """The multithreaded flat form gives the same bytes as one long row (the counter is the flat index)."""
    for n in (1 << 16, 3 * 4096 + 256, 777):
        assert np.array_equal(synth.gauss_flat(n, 2.5, 4242), synth.gauss(n, 1, 1, 2.5, 4242).reshape(-1))


def test_small_frames_recipe():
    """Small uneven frames: seeded, within the recipe's ranges, and the same on every call."""
    fr = synth.small_frames()
    assert len(fr) == 64 and fr == synth.small_frames()
    assert all(f.N in (64, 128, 256) and 1 <= f.F <= 8 and f.T in (512, 768, 1024) and 1.5 <= f.sigma <= 3.5
               for f in fr)
