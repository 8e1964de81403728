"""The N > 1 path of bench.py on CPU with two gloo ranks: every rank works on its own
independent problem (replicas, weak scaling), the reported time is the slowest rank's and
the rate counts the units of all ranks.  No GPU and no data-path collective involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2310_20285_gb300 import datagen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + 0.5 * rank                 # rank 1 is the slower one
        t_max = bench.max_over_ranks(t_local, dist, torch.device("cpu"))
        X, _, _, _, S = datagen.workload_kernel_bench(n=64, seed=bench.replica_seed(rank))
        out.put((rank, t_max, bench.aggregate_rate(64 * 64, world, t_max), float(X.sum()), float(S.sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]                      # max over ranks on every rank
    assert res[0][2] == pytest.approx(2 * 64 * 64 / 1.5)          # units of both ranks / slowest time
    assert res[0][3] != res[1][3] and res[0][4] != res[1][4]      # independent problems per rank


def test_single_process_path_needs_no_process_group():
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.aggregate_rate(100.0, 1, 2.0) == 50.0
    assert bench.replica_seed(0) != bench.replica_seed(1)
