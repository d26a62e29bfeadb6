"""Pins for oracle/tree.py against brute-force geometry (Sec. 6.1 Step 1)."""
import itertools

import numpy as np
import pytest

from oracle.tree import Tree
from paper_2509_21471_gb300 import workloads as wl


def _cases():
    rng = np.random.default_rng(7)
    return [
        ("uniform3d", wl.uniform_points(rng, 600, 3), 16, False),
        ("clustered3d", wl.gaussian_mixture_points(rng, 600, 3, 3, 0.02), 8, False),
        ("clustered3d-per", wl.gaussian_mixture_points(rng, 500, 3, 2, 0.01, 0.0, 1.0), 8, True),
        ("uniform2d-per", wl.uniform_points(rng, 400, 2), 6, True),
        ("clustered2d", wl.gaussian_mixture_points(rng, 500, 2, 3, 0.003), 5, False),
        ("root-leaf", wl.uniform_points(rng, 5, 3), 10, False),
        ("root-leaf-per", wl.uniform_points(rng, 5, 3), 10, True),
    ]


@pytest.mark.parametrize("name,x,ns,per", _cases(), ids=[c[0] for c in _cases()])
def test_tree_invariants_and_near_lists(name, x, ns, per):
    tr = Tree(x, ns, periodic=per)
    d = tr.dim
    nl = len(tr.leaves)
    # leaves partition the unit box
    vol = np.sum(np.ldexp(1.0, -d * tr.leaf_level))
    assert abs(vol - 1.0) < 1e-15
    # capacity (no leaf at the finest level here)
    assert np.all(tr.leaf_count <= ns)
    # every point lies in its leaf's box
    for i in range(nl):
        lo, hi = tr.leaf_box(i)
        P = tr.leaf_points(i)
        assert np.all(tr.cell[P] >= lo) and np.all(tr.cell[P] < hi)
    images = list(itertools.product((-1, 0, 1), repeat=d)) if per else [(0,) * d]
    size = np.left_shift(np.int64(1), (tr.M - tr.leaf_level).astype(np.int64))
    blo = tr.leaf_coords * size[:, None]
    bhi = blo + size[:, None]
    for i in range(nl):
        brute = set()
        for q in images:
            sh = -np.array(q, dtype=np.int64) * (2 ** tr.M)
            touch = np.all((blo[i] <= bhi + sh) & (blo + sh <= bhi[i]), axis=1)
            for j in np.nonzero(touch)[0]:
                brute.add((int(j), q))
            # level restriction (Step 1(b))
            assert np.all(np.abs(tr.leaf_level[touch] - tr.leaf_level[i]) <= 1)
        assert set(tr.near[i]) == brute
        assert len(tr.near[i]) == len(brute)          # no duplicates


def test_level_restriction_refines_beyond_capacity_rule():
    rng = np.random.default_rng(8)
    x = np.concatenate([wl.gaussian_mixture_points(rng, 400, 3, 1, 0.002), wl.uniform_points(rng, 20, 3)])
    tr = Tree(x, 4)
    # some leaves were split only for the level restriction: they hold few points
    # while their parent held <= n_s points
    parents = {}
    for (lev, c) in tr.leaves:
        if lev > 0:
            parents.setdefault((lev - 1, tuple(v >> 1 for v in c)), 0)
    small = 0
    for (lev, c) in parents:
        cnt = np.sum(np.all((tr.cell >> (tr.M - lev)) == np.array(c), axis=1))
        small += cnt <= 4
    assert small > 0
    assert max(tr.leaf_level) >= 6


def test_morton_order_and_point_ranges():
    rng = np.random.default_rng(9)
    x = wl.uniform_points(rng, 300, 3)
    tr = Tree(x, 10)
    assert np.all(np.diff(tr.leaf_anchor_key.astype(np.float64)) > 0)
    assert np.all(np.diff(tr.key[tr.perm].astype(np.float64)) >= 0)
    assert tr.leaf_count.sum() == 300
