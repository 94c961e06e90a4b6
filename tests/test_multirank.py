"""bench.py's multi-rank host logic on CPU ranks (gloo, world size 2).

On several GPUs the fit shards by replica set with no data-path collective
("replicas only"): each rank runs its own copy and the only exchanges are
the barrier and the max over ranks of the step time.  These tests run that
logic as two CPU processes: rendezvous, barrier, max-over-ranks, the
whole-job throughput, and the reference arm leaving the work to rank 0.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, dist = bench.dist_init(world)
    assert (r, w) == (rank, world) and dist is not None
    dist.barrier()
    step_ms = 1.0 + rank  # rank 1 is the slower one
    ms = bench.max_over_ranks(dist, step_ms)
    value = bench.job_throughput(450600, w, ms)

    class Args:
        gpus, steps, warmup = world, 1, 0
    ref = bench.run_reference(Args, r, w, dist) if r != 0 else "skipped"
    out[rank] = (ms, value, ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_barrier_max_and_throughput(monkeypatch):
    world = 2
    # the ranks are CPU processes (gloo) even where a GPU is visible
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "")
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ms, value, ref = out[rank]
        assert ms == 2.0                      # the slowest rank's step time
        assert value == pytest.approx(450600 * 2 / 2e-3)
    assert out[1][2] is None                  # the reference arm runs on rank 0 only


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1) == (0, 1, None)
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.job_throughput(100, 1, 1.0) == pytest.approx(1e5)
