"""Host logic of bench.py: replica aggregation across ranks (gloo, 2 processes on CPU).

Under torchrun every rank runs its own copy of the workload; the timed region is the
slowest rank's, and the whole-job value is all ranks' steps over that time.  The
reference arm runs on rank 0 only.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 0.25 if rank == 1 else 0.1  # rank 1 is the slow one
        t = bench.max_over_ranks(mine, world, "cpu")
        value, _ = bench.aggregate([t] * world, [10] * world)
        out[rank] = (t, value, bench.dist_env())
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, free_port(), out), nprocs=world,
                           start_method="spawn", join=True)
        got = dict(out)
    for r in range(world):
        t, value, env = got[r]
        assert t == 0.25
        assert value == pytest.approx(world * 10 / 0.25)
        assert env == (world, r, r)


def test_aggregate_and_single_process():
    assert bench.max_over_ranks(0.5, 1, "cpu") == 0.5
    v, t = bench.aggregate([0.1, 0.2, 0.4], [5, 5, 5])
    assert t == 0.4 and v == pytest.approx(15 / 0.4)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.parse_args(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert bench.reference_arm(args) is None
