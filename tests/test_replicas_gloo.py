"""Multi-GPU runs are independent replicas (the path is not sharded): two gloo ranks on the
CPU check the benchmark's whole-job aggregation (max time over ranks, summed work) and that
replicas draw disjoint random streams (distinct run ids give distinct end states)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import OracleRun
    ms, work = bench.aggregate_replicas(100.0 + 50.0 * rank, 1000.0 * (rank + 1), world)
    # each rank's replica: same workload shape, run ids offset by rank
    args = type("A", (), {"rows": 4, "cols": 4, "gens": 3})()
    shs = bench.shapes(args, rank)
    o = OracleRun(4, 4, island_size=32, p_ben=shs[0].p_ben, run_id=shs[0].run_id, seed=shs[0].seed)
    o.step(3)
    digest = int(o.snapshot().view("uint32").sum())
    import torch
    d = torch.tensor([digest], dtype=torch.int64)
    all_d = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_d, d)
    out[rank] = (ms, work, shs[0].run_id, [int(x.item()) for x in all_d])
    dist.destroy_process_group()


def test_two_rank_aggregation_and_distinct_replicas():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 150.0          # slowest rank's time
    assert r0[1] == r1[1] == 3000.0         # summed work
    assert r0[2] != r1[2]                   # distinct run ids
    assert r0[3][0] != r0[3][1]             # distinct end states
