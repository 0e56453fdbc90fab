"""The N > 1 path of bench.py on CPU: gloo ranks, world size 2.

Each rank runs its own replica; the timed region is the maximum over ranks
and the whole-job throughput counts every rank's points. No GPU is used."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    elapsed = [0.5, 0.8][rank]  # rank 1 is the slow one
    t = bench.max_over_ranks(elapsed, dist, "cpu")
    out[rank] = (t, bench.replica_throughput(1000, 3, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == pytest.approx(0.8) and out[1][0] == pytest.approx(0.8)
    assert out[0][1] == pytest.approx(2 * 1000 * 3 / 0.8)


def test_single_process_is_its_own_maximum():
    import bench

    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.replica_throughput(10, 2, 1, 4.0) == 5.0
