"""The allocation-free entry point corr_correlate_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory at call time (stream
capture into a CUDA graph, a foreign pool allocator, real-time hosts); its
work list lives in a fixed array inside the library. Its output must equal
the regular entry points' (corr_create / corr_accumulate / corr_readout)
exactly, call after call, since every call reuses the shared array. This
file is collected last so that a run stopping at the first failure has run
everything else first.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("N,F,T", [(256, 4, 1000), (64, 2, 8192), (16, 4, 256), (512, 3, 333)])
def test_noalloc_matches_regular_path_twice(xe, N, F, T):
    import torch
    frames = [synth.gauss(N, F, T, 2.5, 70 + k) for k in range(2)]
    for x_np in frames:  # two calls in a row: the shared array is rewritten each time
        x = torch.from_numpy(x_np).cuda()
        out = torch.full((F, xe.baselines(N), 2), -7, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert noalloc_call(x, out, status) == 0, xe.last_error()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        # integer visibilities: the tolerance is zero
        assert np.array_equal(out.cpu().numpy(), regular_path(xe, x))


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
