"""The multi-GPU path of the bench on CPU ranks (gloo, world size 2).

Views are independent, so ranks share no data: each rank synthesises its own
camera pair (weak scaling) and the only cross-rank steps are the barrier and the
reduction of the timing (slowest rank) and of the view count.  These tests run that
logic with two gloo processes; the oracle stands in for the GPU work so that each
rank's views really depend only on its own pair."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from synth import scene, weights
        seed = bench.rank_pair_seed(rank)
        left, right = scene.stereo_pair(seed, 32, 48, 4.0)
        view = oracle.vinet_forward(weights.he_init(0), left, right, 0.5)
        dist.barrier()
        ms_local = 100.0 + 50.0 * rank          # rank 1 is the slower one
        t_max, value = bench.reduce_ranks(ms_local, 7, dist)
        dist.barrier()
        q.put((rank, seed, float(view.mean()), t_max, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    [p.start() for p in procs]
    res = sorted(q.get(timeout=300) for _ in procs)
    [p.join(timeout=60) for p in procs]
    assert all(p.exitcode == 0 for p in procs)
    (r0, s0, m0, t0, v0), (r1, s1, m1, t1, v1) = res
    assert s0 != s1 and m0 != m1                 # each rank worked on its own pair
    assert t0 == t1 == 150.0                     # slowest rank's time on every rank
    assert abs(v0 - 14 / 0.150) < 1e-9 and v0 == v1   # all views over the slowest time


def test_single_rank_reduction():
    t, v = bench.reduce_ranks(200.0, 7, None)
    assert t == 200.0 and abs(v - 35.0) < 1e-12
