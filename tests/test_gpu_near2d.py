"""GPU parity of the 2D near-field pass (App. B kernels) against the FP64 oracle.

The FP64 path evaluates m_d, m_o, m_td, m_to from polynomial tables fitted to
the same App. B quadratures the oracle sums directly (table error ~1e-14
relative), so the bound is relative l2 <= 1e-12 as in 3D.  The mixed path
meets 10 * eps: FP32 pair terms (FP32 log, two-sum accumulation) for
eps >= 2e-7, FP64 pair terms after an FP32 candidate test below that.
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
from tests.helpers import rel_l2, assert_tree_equal, hilbert_order

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def mixed_tol(eps):
    return 10 * eps


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


_KERN = {}


def _kernel2d(eps, kernels):
    key = (eps, kernels)
    if key not in _KERN:
        _KERN[key] = k2.Kernel2D(ProlateWindow(bandlimit_c(eps, stokeslet=bool(kernels & 1),
                                                           stresslet=bool(kernels & 2))))
    return _KERN[key]


def _oracle(x, f, g, n, eps, ns, periodic, kernels, targets=None):
    tr = Tree(x, ns, periodic=periodic)
    kern = dict(k2d=_kernel2d(eps, kernels), stokeslet=bool(kernels & 1), stresslet=bool(kernels & 2))
    u = onear.near_lists(tr, kern, f=f if kernels & 1 else None, g=g if kernels & 2 else None,
                         n=n if kernels & 2 else None, targets=targets)
    if periodic and kernels & 2:
        u = u + odirect.stresslet_zero_mode(tr.w, g, n, targets=targets)
    return tr, u


def _run(dmk, x, f=None, g=None, n=None, eps=1e-6, ns=40, periodic=False, precision=0, kernels=1):
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, periodic=periodic, kernels=kernels,
                 precision=precision, leaf_capacity=ns)
    u = p.eval(f, g, n)
    p.sync_status()
    return p, u.cpu().numpy()


CASES = [
    # name, N, clustered, periodic, kernels, ns, eps
    ("2d-uniform-3000-stokeslet", 3000, False, False, 1, 40, 1e-6),
    ("2d-clustered-3000-both", 3000, True, False, 3, 30, 1e-6),
    ("2d-periodic-2500-both-eps1e-8", 2500, False, True, 3, 40, 1e-8),
    ("2d-periodic-clustered-stresslet", 1500, True, True, 2, 20, 1e-10),
    ("2d-uniform-800-eps1e-3", 800, False, False, 3, 25, 1e-3),
    ("2d-periodic-1200-stokeslet-eps1e-12", 1200, False, True, 1, 30, 1e-12),
]


@pytest.mark.parametrize("name,N,clustered,periodic,kernels,ns,eps", CASES, ids=[c[0] for c in CASES])
def test_tree_and_near_parity_2d(dmk, name, N, clustered, periodic, kernels, ns, eps):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    x = wl.gaussian_mixture_points(rng, N, 2, 6, 0.02) if clustered else wl.uniform_points(rng, N, 2)
    f = wl.forces(rng, N, 2, zero_mean=periodic)
    g = wl.stresslet_strengths(rng, N, 2)
    n = wl.unit_normals(rng, N, 2)
    tr, u_ref = _oracle(x, f, g, n, eps, ns, periodic, kernels)
    args = dict(f=f if kernels & 1 else None, g=g if kernels & 2 else None, n=n if kernels & 2 else None)
    p64, u64 = _run(dmk, x, eps=eps, ns=ns, periodic=periodic, precision=0, kernels=kernels, **args)
    assert_tree_equal(p64.tree(), tr)
    e64 = rel_l2(u64, u_ref)
    assert e64 < FP64_TOL, e64
    scale = np.linalg.norm(u_ref) / np.sqrt(u_ref.size)
    assert np.max(np.abs(u64 - u_ref)) < 1e3 * FP64_TOL * scale
    p32, u32 = _run(dmk, x, eps=eps, ns=ns, periodic=periodic, precision=1, kernels=kernels, **args)
    e32 = rel_l2(u32, u_ref)
    assert e32 < mixed_tol(eps), e32
    p64.close()
    p32.close()


@pytest.mark.parametrize("N", [0, 1, 2, 33])
def test_tiny_inputs_2d(dmk, N):
    rng = np.random.default_rng(50 + N)
    x = wl.uniform_points(rng, N, 2)
    f = wl.forces(rng, N, 2)
    for prec in (0, 1):
        p, u = _run(dmk, x, f=f, eps=1e-6, ns=8, precision=prec)
        if N == 0:
            assert u.shape == (0, 2)
            continue
        _, u_ref = _oracle(x, f, None, None, 1e-6, 8, False, 1)
        assert rel_l2(u, u_ref) < (FP64_TOL if prec == 0 else 1e-5)
        p.close()


def test_faces_and_coincident_2d(dmk):
    rng = np.random.default_rng(91)
    x = wl.uniform_points(rng, 500, 2)
    x[:20] = np.round(x[:20] * 4) / 4             # on cell faces and corners, incl. +-1/2
    x[30:35] = x[40]                               # coincident points (pair terms skipped)
    f = wl.forces(rng, 500, 2)
    for periodic in (False, True):
        for ns in (10, 600):                       # deep tree / everything in the root leaf
            tr, u_ref = _oracle(x, f, None, None, 1e-6, ns, periodic, 1)
            for prec in (0, 1):
                p, u = _run(dmk, x, f=f, eps=1e-6, ns=ns, periodic=periodic, precision=prec)
                assert_tree_equal(p.tree(), tr, hilbert_order(prec, 1e-6))
                assert rel_l2(u, u_ref) < (FP64_TOL if prec == 0 else 1e-5)
                p.close()


def test_several_columns_2d(dmk):
    """n_rhs = 3 force columns: each column equals a one-column evaluation."""
    rng = np.random.default_rng(17)
    N, ns, eps = 1500, 30, 1e-6
    x = wl.uniform_points(rng, N, 2)
    F = wl.forces(rng, N, 2, n_rhs=3)
    for prec, tol in ((0, FP64_TOL), (1, 10 * eps)):
        p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, precision=prec, leaf_capacity=ns, n_rhs=3)
        U = p.eval(torch.as_tensor(F, device="cuda")).cpu().numpy()
        p.sync_status()
        for k in range(3):
            _, u_ref = _oracle(x, F[:, :, k], None, None, eps, ns, False, 1)
            assert rel_l2(U[:, :, k], u_ref) < tol
        p.close()


def test_gradient_rejected_2d(dmk):
    x = wl.uniform_points(np.random.default_rng(3), 100, 2)
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=1e-6)
    with pytest.raises(dmk.DMKError) as ei:
        p.eval_grad(torch.zeros(100, 2, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 3
    p.close()
