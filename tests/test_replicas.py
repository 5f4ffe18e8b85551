"""Multi-rank path of bench.py (replicas: each rank solves its own
frequencies, the job's time is the slowest rank's) on two gloo ranks over
CPU, the way torchrun launches it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    plan = [bench.frequency_index(i, w, r, 10) for i in range(13)]
    ms = bench.reduce_max_ms(100.0 + 50.0 * rank, w, "cpu")
    dist.barrier()
    q.put((r, plan, ms))
    dist.destroy_process_group()


def test_two_rank_replica_schedule_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    plans = [o[1] for o in out]
    # at every step the two ranks solve different frequencies, together the sweep
    for step in range(13):
        assert plans[0][step] != plans[1][step]
    assert sorted(plans[0][:5] + plans[1][:5]) == list(range(10))
    # both ranks report the slowest rank's time
    assert all(o[2] == 150.0 for o in out)
