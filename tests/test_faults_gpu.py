"""Failure handling on the GPU without faulting it: host deadlines, failed allocations, bad calls,
and a bounded device wait that runs out."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xe():
    import paper_1503_06203_gb300 as xe
    xe.build()
    return xe


def test_synchronize_deadline_runs_out_while_busy(xe):
    """A short host deadline on a long frame returns CORR_ETIMEOUT; waiting longer then succeeds."""
    import torch
    N, F, T = 2048, 16, 16384  # about 0.3 s of work
    x = torch.randint(0, 256, (T, F, N), dtype=torch.uint8, device="cuda")
    with xe.Correlator(N, F, T) as c:
        torch.cuda.synchronize()
        c.accumulate(x)
        with pytest.raises(xe.XEngineError) as ei:
            c.synchronize(timeout_ms=0)
        assert ei.value.code == xe.CORR_ETIMEOUT
        c.synchronize(timeout_ms=60000)
        assert c.status() == 0  # a host deadline is not a device fault: nothing sticky


def test_allocation_failure_is_reported(xe):
    """Accumulators larger than the device's memory: CORR_ENOMEM from corr_create, nothing leaked."""
    import torch
    from paper_1503_06203_gb300._lib import CORR_ENOMEM, lib
    free0, total = torch.cuda.mem_get_info()
    N = 16384
    F = int(total // (N * (N + 1) // 2 * 8)) + 2  # accumulators larger than the whole device
    assert not lib().corr_create(N, F, 1024)
    assert "cudaMalloc" in xe.last_error() or "accumulators" in xe.last_error()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)
    with xe.Correlator(64, 1, 128) as c:  # the device still works
        c.accumulate(torch.zeros((128, 1, 64), dtype=torch.uint8, device="cuda"))
        assert int(c.readout()[0, 0, 0]) == 128 * 128


def test_bad_frames_rejected_before_launch(xe):
    import torch
    with xe.Correlator(64, 2, 256) as c:
        n0 = c.kernel_launches
        with pytest.raises(ValueError):
            c.accumulate(torch.zeros((256, 2, 63), dtype=torch.uint8, device="cuda"))
        from paper_1503_06203_gb300._lib import CORR_EINVAL, lib
        assert lib().corr_accumulate(c.handle, None, None) == CORR_EINVAL
        assert c.kernel_launches == n0 and c.status() == 0


def test_device_wait_runs_out_and_the_context_survives(xe):
    """A bounded device wait on a barrier nothing arrives on ends with an error status (no trap,
    no hang); correlation afterwards is still bit-exact."""
    import torch
    import oracle
    import synth
    for polls in (1, 64, 4096):
        assert xe.selftest_wait_timeout(polls) == xe.CORR_ETIMEOUT
    assert "ran out" in xe.last_error()
    with pytest.raises(xe.XEngineError):
        from paper_1503_06203_gb300 import check
        check(xe.selftest_wait_timeout(0))  # polls outside [1, 2^20]: rejected before launch
    x = synth.gauss(96, 2, 300, 2.5, 91)
    with xe.Correlator(96, 2, 300) as c:
        c.accumulate(torch.from_numpy(x).cuda())
        V = c.readout().cpu().numpy().astype(np.int64)
        assert c.status() == 0
    assert np.array_equal(V, oracle.visibilities(x))


def test_split_change_on_a_busy_handle_is_refused(xe):
    """Changing the time split rebuilds the schedule, so the handle must be idle: while a long correlation
    is still running the call returns CORR_EBUSY and changes nothing; once it is done the change is taken,
    and the results stay exact."""
    import torch

    import oracle
    import synth
    from paper_1503_06203_gb300._lib import CORR_EBUSY
    N, F, T = 2048, 16, 16384  # about 0.3 s of work
    x = torch.zeros((T, F, N), dtype=torch.uint8, device="cuda")
    c = xe.Correlator(N, F, T)
    torch.cuda.synchronize()
    c.accumulate(x)
    with pytest.raises(xe.XEngineError) as ei:
        c.set_option(xe.CORR_OPT_SPLIT, 2)
    assert ei.value.code == CORR_EBUSY and c.get_option(xe.CORR_OPT_SPLIT) == 0
    c.synchronize()
    c.set_option(xe.CORR_OPT_SPLIT, 2)
    assert c.get_option(xe.CORR_OPT_SPLIT) == 2
    small = synth.gauss(200, 2, 300, 2.5, 9)
    with xe.Correlator(200, 2, 300) as d:
        d.accumulate(torch.from_numpy(small).cuda())
        d.synchronize()
        d.set_option(xe.CORR_OPT_SPLIT, 2)
        d.reset()
        d.accumulate(torch.from_numpy(small).cuda())
        assert np.array_equal(d.readout().cpu().numpy().astype(np.int64), oracle.visibilities(small))
    c.close()
