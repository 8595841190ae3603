"""Host logic of bench.py's multi-rank path (replicas only) on CPU: world-size-2 gloo
process group, max-over-ranks timing, whole-job throughput, and the reference arm's
rank-0-only rule."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench._dist() == (world, rank, rank)
    ms = bench.reduce_max(dist, 10.0 + 5.0 * rank, "cpu")      # rank 1 is the slowest
    value = bench.job_value(1000, world, 50, ms)
    # the reference arm: ranks other than 0 exit without work or output
    class A:
        steps, warmup, gpus = 3, 3, world
    rc = bench.run_reference(A) if rank != 0 else 0
    out[rank] = (ms, value, rc)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_over_ranks_and_job_value():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000 * 50 / 15e-3)
    assert res[1][2] == 0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(None, 3.5, "cpu") == 3.5
    assert bench.job_value(500000, 1, 1000, 800.0) == pytest.approx(6.25e8)
