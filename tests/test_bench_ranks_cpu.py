"""Multi-process (gloo, world size 2, CPU) check of bench.py's rank logic:
each rank times its own replica; the job's time is the maximum over ranks and
its work the sum, so value = total particle-steps / slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = [1.5, 4.0][rank]
    work = [100.0, 300.0][rank]
    tmax = bench.max_over_ranks(t, torch, dist)
    wsum = bench.sum_over_ranks(work, torch, dist)
    out.put((rank, tmax, wsum, bench._dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_max_time_and_summed_work_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, wsum, env in res:
        assert tmax == 4.0 and wsum == 400.0
        assert env[0] == rank and env[1] == 2


def test_single_process_reductions_are_identity():
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.sum_over_ranks(7.0) == 7.0
