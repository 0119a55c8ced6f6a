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


def test_pieces_cover_each_frame_once():
    """Time pieces of served frames: whole 256-sample blocks, in order, covering [0, T), at most max_pieces."""
    from paper_1503_06203_gb300 import serve
    srv = serve.Server.__new__(serve.Server)  # the piece rule needs only the specs and its knobs
    srv.specs = [serve.StreamSpec(2048, 256), serve.StreamSpec(64, 1)]
    srv.piece_bytes, srv.max_pieces = 512 << 20, 4
    for sid, T in [(0, 8192), (0, 1024), (0, 256), (1, 100), (1, 8192), (0, 7936)]:
        p = srv.pieces(serve.Arrival(0.0, sid, T, 0))
        assert p[0][0] == 0 and p[-1][1] == T and 1 <= len(p) <= 4
        assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
        assert all(u0 % 256 == 0 and u1 > u0 for u0, u1 in p)
    assert len(srv.pieces(serve.Arrival(0.0, 0, 8192, 0))) == 4   # 4 GiB frame: capped at 4
    assert len(srv.pieces(serve.Arrival(0.0, 1, 8192, 0))) == 1   # 0.5 MB frame: whole


def test_piece_count_cost_model():
    """Without a fixed piece size the count follows the copy rate: a slow link cuts a large frame into
    pieces (its copy hides behind the correlation), a fast one keeps it nearly whole, small frames stay whole."""
    from paper_1503_06203_gb300 import serve
    srv = serve.Server.__new__(serve.Server)
    srv.specs = [serve.StreamSpec(2048, 256), serve.StreamSpec(256, 16)]
    srv.piece_bytes, srv.max_pieces, srv.piece_cost_ms, srv.hbm_gbs = 0, 4, 2.0, 6000.0
    big, small = serve.Arrival(0.0, 0, 8192, 0), serve.Arrival(0.0, 1, 8192, 0)
    srv.h2d_gbs = 20.0
    assert srv.piece_count(big) == 4 and srv.piece_count(small) == 1
    srv.h2d_gbs = 210.0
    assert 1 <= srv.piece_count(big) <= 2 and srv.piece_count(small) == 1
