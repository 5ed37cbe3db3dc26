"""The replica (weak-scaling) bookkeeping of the benchmark on two gloo ranks:
the slowest rank sets the time, all ranks' units count, shards are disjoint."""

import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2411_06224_gb300 import replicas

    rate, tmax = replicas.throughput(units_per_rank=3, seconds=1.0 + rank)  # rank 1 is slower
    mine = replicas.shard(list(range(10)), rank, world)
    out[rank] = (rate, tmax, mine)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_throughput_and_shards():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0[1] == pytest.approx(2.0) and r1[1] == pytest.approx(2.0)  # max over ranks
    assert r0[0] == pytest.approx(3 * 2 / 2.0)  # all ranks' units / slowest time
    assert sorted(r0[2] + r1[2]) == list(range(10)) and not set(r0[2]) & set(r1[2])


def test_single_process_is_identity():
    from paper_2411_06224_gb300 import replicas

    assert replicas.max_over_ranks(1.5) == 1.5
    assert replicas.throughput(4, 2.0) == (2.0, 2.0)
