"""The multi-GPU form of the benchmark is replicas only: each rank localises
its own array and the job's throughput is all ranks' blocks over the slowest
rank's time.  Checked here with two CPU processes over gloo."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    mx = bench.max_over_ranks(local_ms)
    out[rank] = (ws, r, bench.replica_seed(r), mx,
                 bench.job_throughput(100, 4, ws, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_distinct_arrays():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (ws, r, seed, mx, thr) in res.items():
        assert ws == 2 and r == rank
        assert mx == 150.0
        assert thr == pytest.approx(100 * 4 * 2 / 0.150)
    assert res[0][2] != res[1][2]  # each replica has its own workload


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(100, 10, 1, 1000.0) == pytest.approx(1000.0)
