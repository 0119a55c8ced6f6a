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
