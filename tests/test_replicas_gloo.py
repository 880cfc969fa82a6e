"""The multi-GPU form of the benchmark runs independent replicas (one per rank, no collective on
the data path): its host logic is exercised here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1904_02603_gb300 import datagen


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = datagen.WORKLOADS["uniform_100x3_1e4"]
        ds, iseed = bench.replica_seeds(w, rank)
        t, _, _ = datagen.make(w, data_seed=ds, init_seed=iseed)
        mine = 10.0 + 5.0 * rank  # each rank's own elapsed time
        slowest = bench.max_over_ranks(mine, world, device="cpu")
        out[rank] = (slowest, int(t.idx[:, :50].sum()), float(t.val[:50].sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_run_distinct_replicas():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1:] != res[1][1:]  # different seeds: different replicas


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(4, 1000, 10, 2000.0) == pytest.approx(4 * 1000 * 10 / 2.0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
