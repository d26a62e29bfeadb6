"""Separate targets (the sums of Sec. 1 at points that need not be sources):
GPU parity against the oracle's near component at targets (tree of the
sources; each target takes the leaf containing it, its level in nu_ts and that
leaf's near list, no self term), through the C ABI.

Cases: targets in empty leaves (uniform targets, clustered sources), targets on
other levels than their neighbours, 2D and 3D, free space and periodic (the
stresslet k = 0 term at the targets), several force columns, MIXED with FP32
pair terms and below eps 2e-7 (FP64 pair terms), gradients at the targets,
empty target and source sets.  FP64 <= 1e-12, MIXED <= 10 eps, and element-wise
checks on every target.
"""
import zlib

import numpy as np
import pytest
import torch

from oracle import near as onear, direct as odirect, kernels2d as k2
from oracle.tree import Tree
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


def _kern(dim, kernels, eps):
    st, sl = bool(kernels & 1), bool(kernels & 2)
    win = ProlateWindow(bandlimit_c(eps, stokeslet=st, stresslet=sl))
    if dim == 3:
        return dict(win=win, stokeslet=st, stresslet=sl)
    return dict(k2d=k2.Kernel2D(win), stokeslet=st, stresslet=sl)


CASES = [
    # name, dim, periodic, kernels, eps, n_src, n_trg, ns, n_rhs
    ("3d-free-stokeslet", 3, False, 1, 1e-6, 3000, 2000, 40, 1),
    ("3d-free-both-eps1e-10", 3, False, 3, 1e-10, 2000, 1500, 40, 1),
    ("3d-periodic-both", 3, True, 3, 1e-6, 2500, 1800, 48, 1),
    ("3d-free-4-columns", 3, False, 1, 1e-6, 2000, 2500, 32, 4),
    ("2d-periodic-both-eps1e-8", 2, True, 3, 1e-8, 3000, 2000, 40, 1),
    ("2d-free-stokeslet", 2, False, 1, 1e-6, 2000, 3000, 30, 1),
]


@pytest.mark.parametrize("name,dim,periodic,kernels,eps,n_src,n_trg,ns,n_rhs", CASES, ids=[c[0] for c in CASES])
def test_separate_targets_parity(dmk, name, dim, periodic, kernels, eps, n_src, n_trg, ns, n_rhs):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    xs = wl.gaussian_mixture_points(rng, n_src, dim, 4, 0.04)            # clustered sources
    xt = np.concatenate([wl.uniform_points(rng, n_trg // 2, dim),       # targets in empty leaves too
                         wl.gaussian_mixture_points(rng, n_trg - n_trg // 2, dim, 4, 0.04)])
    f = wl.forces(rng, n_src, dim, n_rhs=n_rhs, zero_mean=periodic)
    g = wl.stresslet_strengths(rng, n_src, dim)
    nrm = wl.unit_normals(rng, n_src, dim)
    tr = Tree(xs, ns, periodic=periodic)
    _, tleaf = tr.locate(xt)
    assert np.any(tr.leaf_count[tleaf] == 0)
    kern = _kern(dim, kernels, eps)
    cols = [f] if n_rhs == 1 else [f[:, :, k] for k in range(n_rhs)]
    refs = []
    for k, fk in enumerate(cols):
        use_t = kernels & 2 and k == 0
        u = onear.near_targets(tr, kern, xt, f=fk if kernels & 1 else None, g=g if use_t else None,
                               n=nrm if use_t else None)
        if periodic and use_t:
            wt, _ = tr.locate(xt)
            u = u + odirect.stresslet_zero_mode(tr.w, g, nrm, wt=wt)
        refs.append(u)
    for prec in (dmk.FP64, dmk.MIXED):
        p = dmk.Plan(torch.as_tensor(xs, device="cuda"), targets=torch.as_tensor(xt, device="cuda"), eps=eps,
                     periodic=periodic, kernels=kernels, precision=prec, leaf_capacity=ns, n_rhs=n_rhs)
        args = [torch.as_tensor(f, device="cuda") if kernels & 1 else None]
        args += ([torch.as_tensor(g, device="cuda"), torch.as_tensor(nrm, device="cuda")] if kernels & 2
                 else [None, None])
        u = p.eval(*args).cpu().numpy()
        p.sync_status()
        st = p.stats()
        p.close()
        assert u.shape[0] == n_trg
        got = [u] if n_rhs == 1 else [u[:, :, k] for k in range(n_rhs)]
        tol = 1e-12 if prec == dmk.FP64 else 10 * eps
        for uk, rk in zip(got, refs):
            assert rel_l2(uk, rk) < tol, (prec, rel_l2(uk, rk))
            scale = np.linalg.norm(rk) / np.sqrt(rk.size)
            assert np.max(np.abs(uk - rk)) < 1e3 * tol * scale
        assert st["useful_pairs"] > 0


@pytest.mark.parametrize("precision", [0, 1])
def test_separate_targets_gradient(dmk, precision):
    """Velocity gradient at separate targets (one-sided FP64 pass in both
    precisions) against the oracle's derivative of the residual Stokeslet."""
    rng = np.random.default_rng(640 + precision)
    eps = 1e-8
    xs = wl.gaussian_mixture_points(rng, 2500, 3, 4, 0.05)
    xt = wl.uniform_points(rng, 1500, 3)
    f = wl.forces(rng, 2500, 3)
    tr = Tree(xs, 40)
    u_ref, G_ref = onear.near_targets(tr, _kern(3, 1, eps), xt, f=f, want_grad=True)
    p = dmk.Plan(torch.as_tensor(xs, device="cuda"), targets=torch.as_tensor(xt, device="cuda"), eps=eps,
                 precision=precision, leaf_capacity=40)
    u, G = p.eval_grad(torch.as_tensor(f, device="cuda"), want_u=True)
    p.sync_status()
    p.close()
    assert rel_l2(u.cpu().numpy(), u_ref) < 1e-12
    assert rel_l2(G.cpu().numpy(), G_ref) < 1e-12


def test_targets_at_the_sources_equal_eval_without_self_term(dmk):
    """Targets placed exactly at the sources: every pair but the r = 0 one, so
    u_targets = u - u_self with u from the plan without separate targets."""
    rng = np.random.default_rng(650)
    x = wl.uniform_points(rng, 3000, 3)
    f = wl.forces(rng, 3000, 3)
    tr = Tree(x, 48)
    u_ref = onear.near_targets(tr, _kern(3, 1, 1e-8), x, f=f)
    xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
    p = dmk.Plan(xd, targets=xd.clone(), eps=1e-8, precision=dmk.FP64, leaf_capacity=48)
    q = dmk.Plan(xd, eps=1e-8, precision=dmk.FP64, leaf_capacity=48)
    ut, u = p.eval(fd).cpu().numpy(), q.eval(fd).cpu().numpy()
    p.close()
    q.close()
    assert rel_l2(ut, u_ref) < 1e-12
    assert rel_l2(u - ut, u - u_ref) < 1e-10            # the difference is the self term alone
    assert rel_l2(ut, u) > 1e-3


@pytest.mark.parametrize("n_src,n_trg", [(0, 500), (800, 0), (0, 0)])
def test_separate_targets_empty_sets(dmk, n_src, n_trg):
    rng = np.random.default_rng(660)
    xs = torch.as_tensor(wl.uniform_points(rng, n_src, 3), device="cuda")
    xt = torch.as_tensor(wl.uniform_points(rng, n_trg, 3), device="cuda")
    f = torch.as_tensor(wl.forces(rng, n_src, 3), device="cuda")
    for prec in (0, 1):
        p = dmk.Plan(xs, targets=xt, eps=1e-6, precision=prec, leaf_capacity=40)
        u = p.eval(f)
        p.sync_status()
        assert u.shape == (n_trg, 3)
        assert torch.all(u == 0).item()
        p.close()


@pytest.mark.parametrize("dim,kernels,eps", [(3, 1, 1e-6), (3, 2, 1e-6), (2, 3, 1e-6), (3, 1, 1e-9)])
def test_linear_scaling_workload_parity(dmk, dim, kernels, eps):
    """The perturbed sphere / circle workload (N_S = N_T, Sec. 8) at a size the
    oracle finishes in seconds, with the paper's leaf capacity for eps."""
    xs, xt, f, g, nrm = wl.linear_scaling(4000, dim=dim)
    ns = 1200 if dim == 3 else 240
    tr = Tree(xs, ns if dim == 3 else 60)
    kern = _kern(dim, kernels, eps)
    u_ref = onear.near_targets(tr, kern, xt, f=f if kernels & 1 else None, g=g if kernels & 2 else None,
                               n=nrm if kernels & 2 else None)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    for prec in (dmk.FP64, dmk.MIXED):
        p = dmk.Plan(dev(xs), targets=dev(xt), eps=eps, kernels=kernels, precision=prec,
                     leaf_capacity=ns if dim == 3 else 60)
        u = p.eval(dev(f) if kernels & 1 else None, dev(g) if kernels & 2 else None,
                   dev(nrm) if kernels & 2 else None).cpu().numpy()
        p.sync_status()
        p.close()
        assert rel_l2(u, u_ref) < (1e-12 if prec == dmk.FP64 else 10 * eps)
