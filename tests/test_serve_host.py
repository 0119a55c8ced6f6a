"""Host logic of the serving loop (no GPU): the in-flight budget allocator and the arrival recipe."""
import random

import pytest

pytest.importorskip("torch")

from paper_1503_06203_gb300 import serve  # noqa: E402


def test_slab_never_overlaps_live_frames():
    r = serve.SlabAllocator(10000, device=None)
    rnd = random.Random(3)
    held = []
    for _ in range(30000):
        if rnd.random() < 0.55:
            n = rnd.randint(1, 3000)
            off = r.alloc(n)
            if off is not None:
                n2 = (n + 255) // 256 * 256
                assert 0 <= off and off + n2 <= r.size
                assert all(off + n2 <= a or off >= b for a, b in held)
                held.append((off, off + n2))
        elif held:
            a, _ = held.pop(rnd.randrange(len(held)))  # frames may finish out of admission order
            r.free(a)
    for a, _ in held:
        r.free(a)
    assert r.used == 0 and r.free_blocks == [[0, r.size]]


def test_slab_respects_budget():
    r = serve.SlabAllocator(4096, device=None)
    assert r.alloc(4096) == 0
    assert r.alloc(1) is None
    r.free(0)
    assert r.alloc(2048) == 0 and r.alloc(2048) == 2048 and r.alloc(256) is None
    with pytest.raises(ValueError):
        r.alloc(5000)


def test_slab_reuses_space_freed_out_of_order():
    """A block freed while an older one is still live is reusable at once (no head-of-line blocking)."""
    r = serve.SlabAllocator(3 * 256, device=None)
    a, b, c = r.alloc(256), r.alloc(256), r.alloc(256)
    assert (a, b, c) == (0, 256, 512) and r.alloc(1) is None
    r.free(b)                  # the middle frame finishes first
    assert r.alloc(256) == b   # its space is taken at once
    r.free(a)
    r.free(c)
    r.free(b)
    assert r.free_blocks == [[0, 768]] and r.used == 0


def test_poisson_arrivals_recipe():
    specs = [serve.StreamSpec(256, 16), serve.StreamSpec(1024, 64)]
    arr = serve.poisson_arrivals(100.0, 500, 2, 1024, 8192, 1 << 30, specs, 5)
    assert len(arr) == 500
    assert all(b.t > a.t for a, b in zip(arr, arr[1:]))
    assert all(a.T % 256 == 0 and 1024 <= a.T <= 8192 for a in arr)
    assert all(a.offset + a.T * specs[a.stream].F * specs[a.stream].N <= 1 << 30 for a in arr)
    mean_gap = (arr[-1].t - arr[0].t) / 499
    assert 0.008 < mean_gap < 0.012
