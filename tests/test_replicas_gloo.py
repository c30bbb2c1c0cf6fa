"""Host logic of the multi-replica bench (one independent problem per rank,
no collective on the data path): two `gloo` ranks on the CPU agree on the
slowest replica's time and on the whole-job rate, and draw distinct problems."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp



def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import workloads as W
    r, w, lr = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        seconds = 1.0 + r  # rank 1 is the slow replica
        slowest = bench.max_over_ranks(seconds, dist, device="cpu")
        wl = W.config("c2", seed=r)
        units = wl.P * wl.T * wl.G
        out.put((r, w, lr, slowest, bench.whole_job_rate(units, w, slowest),
                 float(wl.plant.masses[0])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_report_slowest_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import workloads as W
    wl = W.config("c2")
    for r, (rank, world, local_rank, slowest, rate, _) in enumerate(res):
        assert (rank, world, local_rank) == (r, 2, r)
        assert slowest == 2.0
        assert rate == wl.P * wl.T * wl.G * 2 / 2.0
    assert res[0][5] != res[1][5]  # each replica solves its own seeded problem
