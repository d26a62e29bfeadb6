"""Pins for oracle/near.py: neighbour-list traversal vs brute force, the
r -> 0 limit, the periodic tie-in with the Gaussian Ewald total, FD gradients."""
import numpy as np
import pytest

from oracle import near, ewald, kernels3d as k3
from oracle.tree import Tree
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl

WIN6 = ProlateWindow(bandlimit_c(1e-6))
WIN40 = ProlateWindow(40.0)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("per", [False, True])
@pytest.mark.parametrize("clustered", [False, True])
def test_lists_equal_brute_force_3d(per, clustered):
    rng = np.random.default_rng(21 + 2 * per + clustered)
    N = 400
    x = (wl.gaussian_mixture_points(rng, N, 3, 3, 0.03) if clustered else wl.uniform_points(rng, N, 3))
    f = wl.forces(rng, N, 3)
    g = wl.stresslet_strengths(rng, N, 3)
    n = wl.unit_normals(rng, N, 3)
    tr = Tree(x, 12, periodic=per)
    kern = dict(win=WIN6, stokeslet=True, stresslet=True)
    a = near.near_lists(tr, kern, f=f, g=g, n=n)
    b = near.near_brute(tr, kern, f=f, g=g, n=n)
    assert rel(a, b) < 1e-14
    assert len(set(tr.leaf_level.tolist())) > 1 or not clustered


def test_two_point_limit_is_textbook_stokeslet():
    # Two close points in a single root leaf: nu = 1/2 and S_R -> S - phi(0)/(2 pi nu) delta.
    r = 1e-6
    x = np.array([[0.1, 0.2, -0.05], [0.1 + 0.6 * r, 0.2 - 0.8 * r, -0.05]])
    f = np.array([[1.0, -2.0, 0.5], [0.3, 0.7, -1.1]])
    tr = Tree(x, 4)
    u = near.near_lists(tr, dict(win=WIN6, stokeslet=True), f=f)
    a = float(WIN6.phi(0.0)) / np.pi                     # phi(0)/(2 pi nu), nu = 1/2
    d = x[0] - x[1]
    ref0 = k3.stokeslet(d) @ f[1] - a * f[1] - a * f[0]
    assert np.max(np.abs(u[0] - ref0)) < (WIN6.c * r) ** 2 * 10 * np.abs(ref0).max()


def test_uniform_periodic_near_plus_fourier_is_gaussian_ewald():
    # All leaves at level 1 -> nu = r_2 = 1/4 for every pair (Eq. (three_part_sum)
    # with a single level): near component + PSWF Fourier part + zero mode must
    # equal the split-independent periodic total.
    rng = np.random.default_rng(31)
    N = 24
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3, zero_mean=True)
    g = wl.stresslet_strengths(rng, N, 3)
    n = wl.unit_normals(rng, N, 3)
    tr = Tree(x, N - 1, periodic=True)
    assert np.all(tr.leaf_level == 1)
    kern = dict(win=WIN40, stokeslet=True, stresslet=True)
    u_near = near.near_lists(tr, kern, f=f, g=g, n=n)
    split = ewald.prolate_split_3d(WIN40, 0.25, kmax=2.2 * 40.0 / 0.25)
    u_far = ewald.ewald_sum(x, f=f, g=g, n=n, split=split, parts=("fourier", "zero"))
    u_ref = ewald.ewald_sum(x, f=f, g=g, n=n, split=ewald.gaussian_split_3d(0.1))
    assert rel(u_near + u_far, u_ref) < 5e-12


def test_gradient_matches_fd_with_tree_fixed():
    rng = np.random.default_rng(41)
    N = 300
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3)
    tr = Tree(x, 20)
    kern = dict(win=WIN6, stokeslet=True)
    tset = np.array([3, 77, 150, 299])
    _, G = near.near_lists(tr, kern, f=f, targets=tset, want_grad=True)
    h = 1e-6
    w0 = tr.w.copy()
    for row, t in enumerate(tset):
        for m in range(3):
            tr.w = w0.copy(); tr.w[t, m] += h
            up = near.near_lists(tr, kern, f=f, targets=[t])[0]
            tr.w = w0.copy(); tr.w[t, m] -= h
            um = near.near_lists(tr, kern, f=f, targets=[t])[0]
            fd = (up - um) / (2 * h)
            # FD rounding ~ 1e-16 |u| / h with |u| = O(1) from the self term
            assert np.max(np.abs(fd - G[row, :, m])) < 1e-6 * np.abs(G[row]).max() + 1e-8
    tr.w = w0


def test_pair_counts_consistent():
    rng = np.random.default_rng(51)
    x = wl.uniform_points(rng, 500, 3)
    tr = Tree(x, 32)
    issued, useful = near.pair_counts(tr)
    assert 0 < useful < issued
    # brute-force useful pairs with the pair rule
    nu = near.nu_of_levels(tr.point_level[:, None], tr.point_level[None, :])
    d = tr.w[:, None, :] - tr.w[None, :, :]
    r2 = near._r2(d)
    assert useful == int(np.count_nonzero((r2 < nu * nu) & (r2 > 0)))


@pytest.mark.parametrize("per", [False, True])
def test_separate_targets_lists_equal_brute_force(per):
    """Targets that are not sources (Sec. 1): the leaf-list traversal from
    each target's containing leaf equals brute force over all sources and
    images; targets in empty leaves and on other leaf levels included."""
    rng = np.random.default_rng(31 + per)
    xs = wl.gaussian_mixture_points(rng, 350, 3, 3, 0.04)
    xt = np.concatenate([wl.uniform_points(rng, 120, 3), wl.gaussian_mixture_points(rng, 80, 3, 3, 0.04)])
    f = wl.forces(rng, 350, 3)
    g = wl.stresslet_strengths(rng, 350, 3)
    n = wl.unit_normals(rng, 350, 3)
    tr = Tree(xs, 10, periodic=per)
    kern = dict(win=WIN6, stokeslet=True, stresslet=True)
    a = near.near_targets(tr, kern, xt, f=f, g=g, n=n)
    b = near.near_targets_brute(tr, kern, xt, f=f, g=g, n=n)
    assert rel(a, b) < 1e-14
    _, leaf = tr.locate(xt)
    assert np.any(tr.leaf_count[leaf] == 0)          # some targets sit in empty leaves


def test_separate_targets_at_the_sources_drop_only_the_self_term():
    """Targets placed exactly at the sources see every pair but the r = 0 one,
    so the result is the near component minus the self term -phi(0)/(2 pi nu_t) f_t."""
    rng = np.random.default_rng(33)
    xs = wl.uniform_points(rng, 300, 3)
    f = wl.forces(rng, 300, 3)
    tr = Tree(xs, 16)
    kern = dict(win=WIN6, stokeslet=True)
    u = near.near_lists(tr, kern, f=f)
    ut = near.near_targets(tr, kern, xs, f=f)
    nu_t = np.ldexp(1.0, -(tr.point_level + 1))
    self_term = (-float(WIN6.phi(0.0)) / (2 * np.pi * nu_t))[:, None] * f
    assert rel(ut, u - self_term) < 1e-14
    assert rel(ut, u) > 1e-3
