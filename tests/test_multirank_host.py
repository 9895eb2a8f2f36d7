"""The host side of the multi-GPU launch (one replica per rank, no collective on
the data path): two ranks on CPU with the gloo backend take the slowest rank's
step time and report the whole-job rate."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(dist, torch, 10.0 + 3.0 * rank, "cpu")
        q.put((rank, ms, bench.job_rate(world, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = []
    try:
        for _ in range(2):
            out.append(q.get(timeout=120))
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert sorted(r for r, _, _ in out) == [0, 1]
    for _, ms, rate in out:
        assert ms == 13.0
        assert rate == pytest.approx(2 * 1000.0 / 13.0)


def test_single_process_needs_no_group():
    import torch
    import bench
    assert bench.max_over_ranks(None, torch, 7.5, "cpu") == 7.5
    assert bench.job_rate(1, 500.0) == 2.0
