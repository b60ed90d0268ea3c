"""The bench's multi-rank host logic on two CPU ranks (gloo): every rank
solves its own instance (replicas, no collective on the data path), the job's
time is the slowest rank's and its units are every rank's; the reference arm
runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import inputs


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank instance: distinct seeds give distinct sample draws
        base = dict(inputs.CONFIGS["n31_N8"])
        seed = bench.rank_seed(base["seed"], rank)
        xi = inputs.draw_xi(seed, base["N"], base["K"])
        total_s = 1.0 + rank               # rank 1 is the slower one
        units = 10.0 * (rank + 1)
        value, t, u = bench.job_throughput(total_s, units, dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, (seed, float(xi[0, 0])))
        out[rank] = (value, t, u, gathered)
    finally:
        dist.destroy_process_group()


def test_job_throughput_and_rank_seeds_over_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        value, t, u, gathered = out[r]
        assert t == 2.0                    # max over ranks
        assert u == 30.0                   # sum over ranks
        assert value == pytest.approx(15.0)
        (s0, x0), (s1, x1) = gathered
        assert s0 != s1 and x0 != x1       # independent instances


def test_single_rank_is_the_local_number():
    value, t, u = bench.job_throughput(2.5, 5.0)
    assert (value, t, u) == (2.0, 2.5, 5.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        config = "n31_N8"
        gpus = 2
        steps = 1
        warmup = 0

    assert bench.run_reference(Args(), 2, 1) is None
    assert capsys.readouterr().out == ""
