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


# ----------------------------------------------------------------- one system
def _csr_near(tree):
    off = np.zeros(len(tree.leaves) + 1, np.int64)
    lst = []
    for i, nl in enumerate(tree.near):
        lst.extend(X for X, _ in nl)
        off[i + 1] = len(lst)
    return off, np.asarray(lst, np.int64)


def _shard_worker(r, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(r))
    pdist.init("gloo")
    try:
        from oracle import near as onear
        from oracle.tree import Tree
        from oracle.window import ProlateWindow
        from oracle.params import bandlimit_c
        from paper_2509_21471_gb300 import dmk
        rng = wl.rng_for(7)
        x = wl.gaussian_mixture_points(rng, 3000, 3, 6, 0.05)     # every rank: all coordinates
        f = wl.forces(rng, 3000, 3)
        tree = Tree(x, 40, periodic=True)
        off, nl = _csr_near(tree)
        begin, cost = dmk.partition_leaves(tree.leaf_count, off, nl, world)
        b, e = int(begin[r]), int(begin[r + 1])
        # owner of every point from the partition (points of a leaf range are contiguous in sorted order)
        owner = np.empty(3000, np.int64)
        for q in range(world):
            s0 = tree.leaf_start[begin[q]] if begin[q] < len(tree.leaves) else 3000
            s1 = tree.leaf_start[begin[q + 1]] if begin[q + 1] < len(tree.leaves) else 3000
            owner[tree.perm[s0:s1]] = q
        mine = np.nonzero(owner == r)[0]
        halo = dmk.halo_leaves(off, nl, b, e)
        halo_pts = np.concatenate([tree.leaf_points(int(X)) for X in halo]) if len(halo) else np.zeros(0, np.int64)
        # coverage: every near leaf of an owned leaf is owned or in the halo
        need = {int(X) for i in range(b, e) for X, _ in tree.near[i]}
        assert need <= set(range(b, e)) | set(int(X) for X in halo)
        # densities: only this rank's rows are known before the exchange
        vals = torch.full((3000, 3), float("nan"), dtype=torch.float64)
        vals[torch.as_tensor(mine)] = torch.as_tensor(f[mine])
        pdist.halo_exchange(vals, owner, halo_pts)
        f_here = vals.numpy()
        assert np.array_equal(f_here[halo_pts], f[halo_pts])
        kern = dict(win=ProlateWindow(bandlimit_c(1e-6)), stokeslet=True)
        u_mine = onear.near_lists(tree, kern, f=f_here, targets=mine)   # NaN if a needed row were missing
        out[r] = (mine, u_mine, int(cost[r]), len(halo_pts))
    finally:
        pdist.finish()


def test_one_system_sharded_over_two_gloo_ranks():
    """One periodic system split over two ranks by issued pairs: each rank
    receives its halo's densities (point-to-point, gloo) and its near field
    over its own targets equals the single-rank result exactly."""
    from oracle import near as onear
    from oracle.tree import Tree
    from oracle.window import ProlateWindow
    from oracle.params import bandlimit_c
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_shard_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    rng = wl.rng_for(7)
    x = wl.gaussian_mixture_points(rng, 3000, 3, 6, 0.05)
    f = wl.forces(rng, 3000, 3)
    u_all = onear.near_lists(Tree(x, 40, periodic=True), dict(win=ProlateWindow(bandlimit_c(1e-6)), stokeslet=True),
                             f=f)
    seen = np.zeros(3000, bool)
    for r in range(world):
        mine, u_mine, cost, nhalo = out[r]
        assert np.all(np.isfinite(u_mine))
        assert np.array_equal(u_mine, u_all[mine])
        assert not np.any(seen[mine])
        seen[mine] = True
        assert 0 < nhalo < 3000
    assert seen.all()                                   # the ranks' targets cover the system once
    c0, c1 = out[0][2], out[1][2]
    assert abs(c0 - c1) < 0.25 * (c0 + c1)               # issued pairs balanced


def test_partition_edge_cases():
    from paper_2509_21471_gb300 import dmk
    counts = np.array([5, 0, 7, 3], np.int32)
    off = np.array([0, 2, 4, 6, 8], np.int32)
    nl = np.array([0, 1, 0, 1, 2, 3, 2, 3], np.int32)
    b, cost = dmk.partition_leaves(counts, off, nl, 1)
    assert list(b) == [0, 4] and cost[0] == 5 * 5 + 0 + 7 * 10 + 3 * 10
    b, cost = dmk.partition_leaves(counts, off, nl, 7)          # more ranks than leaves
    assert b[0] == 0 and b[-1] == 4 and np.all(np.diff(b) >= 0) and cost.sum() == 125
    assert len(dmk.halo_leaves(off, nl, 0, 4)) == 0              # the whole tree has no halo
    assert list(dmk.halo_leaves(off, nl, 2, 4)) == []
    assert list(dmk.halo_leaves(off, nl, 0, 1)) == [1]
    b0, _ = dmk.partition_leaves(np.zeros(0, np.int32), np.zeros(1, np.int32), np.zeros(0, np.int32), 3)
    assert list(b0) == [0, 0, 0, 0]
