"""The N > 1 path of bench.py on CPU: two gloo ranks (world size 2).

Each rank must draw its own independent system (seed index offset by rank),
the timing collective must return the maximum over ranks on every rank, and
the whole-job rate must count every rank's units over that maximum.  No GPU:
the process group is gloo on 127.0.0.1.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

from paper_2509_21471_gb300 import dist as pdist, workloads as wl


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(r, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(r))
    pdist.init("gloo")
    try:
        assert pdist.world_size() == world and pdist.rank() == r
        # independent systems: different seeds, deterministic per rank
        x, _ = wl.clustered_3d(n=1000, seed_index=pdist.seed_index(1))
        x2, _ = wl.clustered_3d(n=1000, seed_index=pdist.seed_index(1, r))
        assert np.array_equal(x, x2)
        digest = torch.tensor([float(np.sum(x * np.arange(1, 4)))], dtype=torch.float64)
        got = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        tdist.all_gather(got, digest)
        # the slowest rank's time on every rank
        pdist.barrier()
        t = pdist.max_over_ranks(1.5 * (r + 1))
        rate = pdist.job_rate(1000, 3, t)
        out[r] = (float(got[0]), float(got[1]), t, rate)
    finally:
        pdist.finish()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert set(out.keys()) == {0, 1}
    d0, d1, t0, r0 = out[0]
    assert out[1][:2] == (d0, d1)
    assert d0 != d1                                   # the ranks hold different systems
    assert t0 == out[1][2] == 3.0                     # max over ranks, seen by both
    assert r0 == out[1][3] == 2 * 1000 * 3 / 3.0      # all ranks' units over the max time
