"""The N > 1 path of bench.py on CPU: ranks are independent replicas of the
fit, joined only by a barrier and the maximum of their timed totals.  Two
gloo ranks on 127.0.0.1 stand in for two GPUs."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed steps of (r + 1) ms and e2e steps of 10 - r ms
        steps = 4
        lm_ms = [float(rank + 1)] * steps
        e2e_ms = [float(10 - rank)] * steps
        dist.barrier()
        lm_total, e2e_total = bench.rank_max_totals([lm_ms, e2e_ms], torch.device("cpu"), dist)
        q.put((rank, lm_total, e2e_total, bench.job_rate(world, steps, lm_total)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_gather_takes_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, lm_total, e2e_total, rate in got:
        # every rank sees the slowest rank's totals: 4 x 2 ms and 4 x 10 ms
        assert lm_total == pytest.approx(8.0)
        assert e2e_total == pytest.approx(40.0)
        # 2 ranks x 4 steps in 8 ms
        assert rate == pytest.approx(1000.0)


def test_single_rank_totals_and_rate():
    lm_total, e2e_total = bench.rank_max_totals([[1.0, 2.0], [3.0]], torch.device("cpu"))
    assert (lm_total, e2e_total) == (3.0, 3.0)
    assert bench.job_rate(1, 2, lm_total) == pytest.approx(2 / 3e-3)
