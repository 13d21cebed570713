"""The multi-rank (one process per GPU) host logic of the benchmark, on CPU
with the gloo backend and world size 2: every rank draws a disjoint workload
of the same size (weak scaling, no data-path collective), and the job's step
time is the slowest rank's."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2011_12984_b300 import gen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        p = gen.mass_action(64, seed=bench.shard_seed(gen.DEFAULT_SEED, rank))
        t_local = 0.25 + 0.5 * rank                   # the ranks' own step times
        t = bench.slowest_rank_time(torch, dist, t_local, "cpu")
        dist.barrier()
        out[rank] = (t, float(p.y0[:8].sum()), int(p.y_off[-1]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_take_the_slowest_time():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 0.75            # max over ranks, on every rank
    assert res[0][1] != res[1][1]                    # disjoint workloads
    for r in range(ws):                              # each as the single-rank run of its seed
        p = gen.mass_action(64, seed=bench.shard_seed(gen.DEFAULT_SEED, r))
        assert res[r][1] == float(p.y0[:8].sum()) and res[r][2] == int(p.y_off[-1])


def test_single_rank_time_is_its_own():
    assert bench.slowest_rank_time(torch, None, 0.3, "cpu") == 0.3
    assert bench.shard_seed(5, 0) == 5
