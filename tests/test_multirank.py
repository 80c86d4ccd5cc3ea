"""Multi-GPU is replicas only: every rank advances its own grid and the only
collectives are the barrier and the reductions of the timings.  That host
logic runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 1000 (r + 1) cells, (r + 1) * 10 ms for 5 steps
        rate, slowest = bench.weak_scaling_rate(1000 * (rank + 1), 5, 0.010 * (rank + 1))
        env = bench.dist_env()
        dist.barrier()
        out[rank] = (rate, slowest, env)
    finally:
        dist.destroy_process_group()


def test_weak_scaling_rate_over_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        rate, slowest, env = out[r]
        # all ranks agree: (1000 + 2000) cells x 5 steps / the slowest 20 ms
        assert slowest == pytest.approx(0.020)
        assert rate == pytest.approx(3000 * 5 / 0.020)
        assert env == (r, world, r)


def test_single_process_rate_is_local():
    rate, slowest = bench.weak_scaling_rate(4096, 10, 0.5)
    assert (rate, slowest) == (4096 * 10 / 0.5, 0.5)


def _reference_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))

    class Args:
        steps, warmup, gpus = 1, 0, world

    if rank != 0:
        out[rank] = bench.run_reference(Args())   # the other ranks exit 0 without work


def test_reference_arm_runs_on_rank_zero_only():
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_reference_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[1] == 0
