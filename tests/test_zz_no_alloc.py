"""The allocation-free entry point corr_correlate_noalloc, called through the C ABI.

Some callers cannot allocate device memory at the moment they correlate: an
application whose device memory belongs to its own pool allocator may not
have memory taken behind that allocator's back, and a real-time host that
reserves every byte before it starts forbids allocation on its processing
path. corr_correlate_noalloc serves them: the caller passes the frame and
the output, and the kernel's work list and fault word live in a fixed array
inside the library.

Every call rewrites that one array, so each case makes two calls in a row and
checks both. Each output is checked against the CPU oracle (the plain Eq. 1
definition) and against the regular entry points (corr_create /
corr_accumulate / corr_readout); the visibilities are integers, so the
tolerance is zero. This file is collected last, so that a run stopping at
the first failure has run every other test first.
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


def regular_path(xe, x):
    import torch
    T, F, N = x.shape
    c = xe.Correlator(N, F, T)
    c.accumulate(x)
    V = c.readout()
    torch.cuda.synchronize()
    assert c.status() == 0
    c.close()
    return V.cpu().numpy()


def noalloc_call(x, out, status):
    """Raw C-ABI call (no Python wrapper logic in between)."""
    import torch
    from paper_1503_06203_gb300._lib import lib
    T, F, N = x.shape
    return lib().corr_correlate_noalloc(ctypes.c_void_p(x.data_ptr()), N, F, T, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(status.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def sampled_oracle_check(xe, x_np, V, rng, K=2000):
    """Entries at tile edges and corners plus random ones, and every autocorrelation, against the oracle."""
    T, F, N = x_np.shape
    edges = np.unique(np.clip(np.concatenate([np.arange(0, N, 64), np.arange(63, N, 64), [N - 1]]), 0, N - 1))
    ei, ej = np.meshgrid(edges, edges, indexing="ij")
    ei, ej = ei.ravel(), ej.ravel()
    keep = ei <= ej
    ri = rng.integers(0, N, K)
    rj = rng.integers(0, N, K)
    ii = np.concatenate([ei[keep], np.minimum(ri, rj), np.arange(N)])
    jj = np.concatenate([ej[keep], np.maximum(ri, rj), np.arange(N)])
    ff = rng.integers(0, F, ii.size)
    ff[-N:] = np.arange(N) % F
    ref = oracle.entries(x_np, np.stack([ff, ii, jj], 1))
    assert np.array_equal(V[ff, xe.packed_index(N, ii, jj)].astype(np.int64), ref)


# (N, F, T): several tiles and a ragged tail. The first four split the time axis
# (atomic adds onto a zeroed output); the last two leave it whole (stores of
# whole tiles, which must cover every baseline): (80, 2, 100) has one 128-sample
# chunk and an N % 64 tail, (2048, 8, 256) has more tiles than four per CTA.
CASES = [(256, 4, 1000), (64, 2, 8192), (16, 4, 256), (512, 3, 333), (80, 2, 100), (2048, 8, 256)]


@pytest.mark.parametrize("N,F,T", CASES)
def test_noalloc_matches_oracle_and_regular_path_twice(xe, N, F, T):
    import torch
    rng = np.random.default_rng(N + F + T)
    for k in range(2):  # two calls in a row: the shared array is rewritten each time
        x_np = synth.gauss(N, F, T, 2.5, 70 + k)
        x = torch.from_numpy(x_np).cuda()
        # prefilled with a value no visibility takes here, so a baseline left unwritten shows
        out = torch.full((F, xe.baselines(N), 2), -7, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert noalloc_call(x, out, status) == 0, xe.last_error()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        V = out.cpu().numpy()
        assert np.array_equal(V, regular_path(xe, x))
        if N * N * F * T <= 2 ** 30:
            assert np.array_equal(V.astype(np.int64), oracle.visibilities(x_np))
        else:
            sampled_oracle_check(xe, x_np, V, rng)


def test_noalloc_rejects_oversized_and_unaligned(xe):
    import torch
    from paper_1503_06203_gb300._lib import CORR_EINVAL
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # 8192 elements x 8 bands = 66,048 tiles > 65,536 work items: rejected before any launch
    big = torch.zeros((1, 8, 8192), dtype=torch.uint8, device="cuda")
    assert noalloc_call(big, out, status) == CORR_EINVAL
    assert "work-list" in xe.last_error()
    # N not a multiple of 16 (no staging copy on this path)
    odd = torch.zeros((4, 1, 17), dtype=torch.uint8, device="cuda")
    assert noalloc_call(odd, out, status) == CORR_EINVAL
