"""The multi-GPU path is replicas only: every rank renders its own views and only timings are
combined (barrier, maximum over ranks).  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    ms = 2.0 + rank  # rank 1 is the slower replica
    m = bench.max_over_ranks(ms, world)
    out[rank] = (m, bench.whole_job_mpix_s(world, 1920 * 1080, m))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_replicas_combine_timings():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 3.0
    expect = 2 * 1920 * 1080 / 3.0e-3 / 1e6
    assert abs(out[0][1] - expect) < 1e-9 * expect


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, 1) == 1.5
    bench.barrier(1)
