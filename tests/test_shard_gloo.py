"""The multi-GPU path on CPU: two gloo ranks, no data-path collective, max-over-ranks timing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr = bench.rank_frame(synth.PATHFINDER, rank)
    seeds = [None] * world
    dist.all_gather_object(seeds, (fr.seed, fr.N, fr.F, fr.T))
    t = bench._max_over_ranks(world, 10.0 + rank)  # rank r "took" 10 + r ms
    if rank == 0:
        out.put((seeds, t, bench.aggregate_tops(world, 1e12, 4, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_logic():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    seeds, t, tops = q.get()
    assert len({s[0] for s in seeds}) == 2            # each rank its own frame: disjoint work
    assert all(s[1:] == seeds[0][1:] for s in seeds)  # same shape on every rank (weak scaling)
    assert t == 11.0                                  # the slowest rank's time
    assert abs(tops - 2 * 1e12 * 4 / 11e-3 / 1e12) < 1e-9


def test_band_range_partitions_every_band_once():
    """The band split of one frame across GPUs: contiguous, in rank order, every band exactly once."""
    from paper_1503_06203_gb300 import band_range
    for F in (1, 2, 3, 7, 16, 64, 256):
        for world in (1, 2, 3, 4, 8):
            ranges = [band_range(r, world, F) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == F
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [f1 - f0 for f0, f1 in ranges]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def _band_rank_main(rank, world, port, out):
    """Rank r correlates only its bands of one shared frame (CPU oracle); the test gathers the parts."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1503_06203_gb300 import band_range
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = synth.gauss(48, 5, 200, 2.5, 77)  # the same seeded frame on every rank
    f0, f1 = band_range(rank, world, x.shape[1])
    part = oracle.visibilities(np.ascontiguousarray(x[:, f0:f1, :]), 1)
    parts = [None] * world
    dist.all_gather_object(parts, (f0, f1, part))  # in the test only: the data path has no exchange
    if rank == 0:
        out.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_band_split_equals_whole():
    import numpy as np
    import torch.multiprocessing as mp

    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_band_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = q.get()  # read before joining: rank 0 blocks on a full pipe until the parent reads
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert [(p[0], p[1]) for p in parts] == [(0, 3), (3, 5)]
    whole = oracle.visibilities(synth.gauss(48, 5, 200, 2.5, 77))
    assert np.array_equal(np.concatenate([p[2] for p in parts], axis=0), whole)
