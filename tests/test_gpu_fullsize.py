"""Parity at the full workload sizes, in the launch configuration the bench
times (the paper's leaf capacity for eps, one plan per evaluation).

Every tree is compared with the oracle tree exactly (integers); velocities are
compared on seeded samples of targets, which the oracle evaluates one leaf at a
time (relative l2 over the sample): FP64 <= 1e-12, MIXED <= 10 eps.

Workloads (seeded, synthetic; recipes in paper_2509_21471_gb300/workloads.py):
  * 3D free space, 1e6 points from 8 Gaussians (sigma 0.02), Stokeslet,
    eps = 1e-6 and 1e-10;
  * 2D periodic unit square, 1e6 uniform points, Stokeslet + stresslet with the
    k = 0 stresslet term, eps = 1e-8;
  * 256 independent 3D systems (1e3..1e5 points, log-uniform; half uniform,
    half clustered), 16 force columns, one plan, eps = 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import near as onear, direct as odirect, kernels2d as k2
from oracle.tree import Tree
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl
from tests.helpers import rel_l2, assert_tree_equal

pytestmark = pytest.mark.gpu

N_SAMPLE = 256


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False))


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_clustered_1e6_stokeslet(dmk, eps):
    x, f = wl.clustered_3d(1_000_000)
    xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
    res = {}
    for prec in (dmk.FP64, dmk.MIXED):
        p = dmk.Plan(xd, eps=eps, precision=prec)
        res[prec] = p.eval(fd).cpu().numpy()
        p.sync_status()
        if prec == dmk.FP64:
            ns = p.stats()["leaf_capacity"]
            gtree = p.tree()
        p.close()
    tr = Tree(x, ns)
    assert_tree_equal(gtree, tr)
    tset = _sample(len(x), N_SAMPLE, 101)
    u_ref = onear.near_lists(tr, dict(win=ProlateWindow(bandlimit_c(eps)), stokeslet=True), f=f, targets=tset)
    assert rel_l2(res[dmk.FP64][tset], u_ref) < 1e-12
    assert rel_l2(res[dmk.MIXED][tset], u_ref) < 10 * eps


def test_periodic_2d_1e6_stokeslet_stresslet(dmk):
    eps = 1e-8
    x, f, g, n = wl.periodic_2d(1_000_000)
    dev = [torch.as_tensor(a, device="cuda") for a in (x, f, g, n)]
    res = {}
    for prec in (dmk.FP64, dmk.MIXED):
        p = dmk.Plan(dev[0], eps=eps, periodic=True, kernels=dmk.STOKESLET | dmk.STRESSLET, precision=prec)
        res[prec] = p.eval(dev[1], dev[2], dev[3]).cpu().numpy()
        p.sync_status()
        if prec == dmk.FP64:
            ns = p.stats()["leaf_capacity"]
            gtree = p.tree()
        p.close()
    tr = Tree(x, ns, periodic=True)
    assert_tree_equal(gtree, tr)
    tset = _sample(len(x), N_SAMPLE, 102)
    kern = dict(k2d=k2.Kernel2D(ProlateWindow(bandlimit_c(eps, stokeslet=True, stresslet=True))),
                stokeslet=True, stresslet=True)
    u_ref = onear.near_lists(tr, kern, f=f, g=g, n=n, targets=tset)
    u_ref = u_ref + odirect.stresslet_zero_mode(tr.w, g, n, targets=tset)
    assert rel_l2(res[dmk.FP64][tset], u_ref) < 1e-12
    assert rel_l2(res[dmk.MIXED][tset], u_ref) < 10 * eps


def _system_leaf_ranges(gt, n_sys, dim):
    """Leaf ranges of the systems of a batched plan: each system's leaves tile
    its unit box, so their volumes 2^(-dim*level) add up to exactly one."""
    lv = gt["leaf_level"].astype(np.int64)
    top = int(lv.max()) if len(lv) else 0
    vol = np.left_shift(np.int64(1), dim * (top - lv))
    cum = np.cumsum(vol)
    full = np.int64(1) << (dim * top)
    ends = np.searchsorted(cum, full * np.arange(1, n_sys + 1)) + 1
    assert np.array_equal(cum[ends - 1], full * np.arange(1, n_sys + 1))
    starts = np.concatenate([[0], ends[:-1]])
    return list(zip(starts, ends))


def test_batched_256_systems_16_columns(dmk):
    eps = 1e-6
    x, F, offs = wl.batched_3d()
    n_sys = len(offs) - 1
    xd, Fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(F, device="cuda")
    res = {}
    for prec in (dmk.FP64, dmk.MIXED):
        p = dmk.Plan(xd, eps=eps, precision=prec, n_rhs=16, offsets=offs)
        res[prec] = p.eval(Fd).cpu().numpy()
        p.sync_status()
        if prec == dmk.FP64:
            ns = p.stats()["leaf_capacity"]
            gt = p.tree()
        p.close()
    del Fd
    ranges = _system_leaf_ranges(gt, n_sys, 3)
    sizes = np.diff(offs)
    half = n_sys // 2
    pick = sorted({int(np.argmin(sizes[:half])), int(np.argmax(sizes[:half])),
                   half + int(np.argmin(sizes[half:])), half + int(np.argmax(sizes[half:])), 77, 201})
    win = ProlateWindow(bandlimit_c(eps))
    for k in pick:
        sl = slice(offs[k], offs[k + 1])
        tr = Tree(x[sl], ns)
        a, b = ranges[k]
        assert b - a == len(tr.leaves), k
        assert np.array_equal(gt["leaf_level"][a:b], tr.leaf_level)
        assert np.array_equal(gt["leaf_coords"][a:b], tr.leaf_coords)
        assert np.array_equal(gt["leaf_count"][a:b], tr.leaf_count)
        assert np.array_equal(gt["perm"][sl] - offs[k], tr.perm)       # FP64 plan: Morton order
        for i in range(len(tr.leaves)):
            e0, e1 = gt["near_off"][a + i], gt["near_off"][a + i + 1]
            got = {(int(gt["near_leaf"][e]) - a, tuple(int(v) for v in gt["near_q"][e])) for e in range(e0, e1)}
            assert got == set(tr.near[i]), (k, i)
        tset = _sample(sizes[k], 64, 200 + k)
        for col in (0, 7, 15):
            u_ref = onear.near_lists(tr, dict(win=win, stokeslet=True), f=F[sl][:, :, col], targets=tset)
            assert rel_l2(res[dmk.FP64][sl][tset, :, col], u_ref) < 1e-12, (k, col)
            assert rel_l2(res[dmk.MIXED][sl][tset, :, col], u_ref) < 10 * eps, (k, col)
