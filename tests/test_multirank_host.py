"""The multi-rank path of bench.py on the CPU: two gloo ranks on 127.0.0.1.
Each rank detects its own batch (replicas: systems are independent, no
collective on the data path); the job's time is the slowest rank's, its
throughput the units of all ranks over that time."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2504_09820_gb300 import workload as wl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the slowest rank's time, on every rank
        t = bench.max_over_ranks(1.5 + rank, dist)
        # each rank's own batch: a checksum of its first chunk, gathered
        spec = bench.workload_spec(rank)
        d = wl.generate(spec, chunks=[0])
        mine = torch.tensor([float(np.abs(d["H"]).sum()), float(spec.seed)], dtype=torch.float64)
        allv = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allv, mine)
        out[rank] = (t, [tuple(v.tolist()) for v in allv])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5                   # max over ranks, on both ranks
    g0, g1 = res[0][1], res[1][1]
    assert g0 == g1                                        # the same gathered view on both ranks
    assert g0[0][1] != g0[1][1] and g0[0][0] != g0[1][0]   # distinct seeds and channels per rank


def test_job_rate_and_single_rank():
    assert bench.job_rate(2, 16384, 10, 0.5) == pytest.approx(655360.0)
    assert bench.job_rate(1, 100, 4, 2.0) == pytest.approx(200.0)
    assert bench.max_over_ranks(3.25) == 3.25              # no process group: the value itself


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    """Under torchrun only rank 0 runs (and prints) the CPU oracle's line."""
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
