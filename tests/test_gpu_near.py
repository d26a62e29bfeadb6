"""GPU parity of the near-field pass against the FP64 oracle (through the C ABI).

Tolerances: the FP64 path evaluates the same formulas as the oracle, with
polynomial kernel tables fitted to ~1e-15 relative and a different summation
order, so relative l2 <= 1e-12.  The mixed path must meet 10 * eps: FP32
pair terms with two-sum accumulation for eps >= 2e-7 (their error, ~1e-7 to
2e-6 in l2, is set by FP32 rounding of the pair terms), float-float pair terms
below that (one force column; the MIXED gradient takes float-float pair terms at
every eps).
"""
import zlib

import numpy as np
import pytest
import torch

from oracle import near as onear, direct as odirect
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


def _run(dmk, x, f=None, g=None, n=None, eps=1e-6, ns=64, periodic=False, precision=0, kernels=None):
    kernels = kernels or ((1 if f is not None else 0) | (2 if g is not None else 0))
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, periodic=periodic, kernels=kernels,
                 precision=precision, leaf_capacity=ns)
    u = p.eval(f, g, n)
    p.sync_status()
    return p, u.cpu().numpy()


def _oracle(x, f, g, n, eps, ns, periodic, kernels):
    tr = Tree(x, ns, periodic=periodic)
    win = ProlateWindow(bandlimit_c(eps, stokeslet=bool(kernels & 1), stresslet=bool(kernels & 2)))
    kern = dict(win=win, stokeslet=bool(kernels & 1), stresslet=bool(kernels & 2))
    u = onear.near_lists(tr, kern, f=f if kernels & 1 else None, g=g if kernels & 2 else None,
                         n=n if kernels & 2 else None)
    if periodic and kernels & 2:
        u = u + odirect.stresslet_zero_mode(tr.w, g, n)
    return tr, u


CASES = [
    # name, N, clustered, periodic, kernels, ns, eps
    ("uniform-2000-stokeslet", 2000, False, False, 1, 64, 1e-6),
    ("clustered-3000-both", 3000, True, False, 3, 32, 1e-6),
    ("periodic-2000-both", 2000, False, True, 3, 50, 1e-6),
    ("clustered-periodic-stresslet", 1500, True, True, 2, 24, 1e-8),
    ("uniform-1000-eps1e-10", 1000, False, False, 1, 40, 1e-10),
    ("uniform-700-eps1e-3", 700, False, False, 3, 30, 1e-3),
    ("clustered-2000-both-eps1e-9", 2000, True, False, 3, 32, 1e-9),
    ("periodic-1500-both-eps1e-8", 1500, False, True, 3, 40, 1e-8),
    ("uniform-800-eps1e-12", 800, False, False, 1, 30, 1e-12),
    ("clustered-1200-both-eps1e-12", 1200, True, False, 3, 30, 1e-12),
    ("periodic-1000-stresslet-eps1e-11", 1000, False, True, 2, 30, 1e-11),
]


@pytest.mark.parametrize("name,N,clustered,periodic,kernels,ns,eps", CASES, ids=[c[0] for c in CASES])
def test_tree_and_near_parity(dmk, name, N, clustered, periodic, kernels, ns, eps):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    x = wl.gaussian_mixture_points(rng, N, 3, 8, 0.02) if clustered else wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3)
    g = wl.stresslet_strengths(rng, N, 3)
    n = wl.unit_normals(rng, N, 3)
    tr, u_ref = _oracle(x, f, g, n, eps, ns, periodic, kernels)
    args = dict(f=f if kernels & 1 else None, g=g if kernels & 2 else None, n=n if kernels & 2 else None)
    p64, u64 = _run(dmk, x, eps=eps, ns=ns, periodic=periodic, precision=0, kernels=kernels, **args)
    assert_tree_equal(p64.tree(), tr)
    e64 = rel_l2(u64, u_ref)
    assert e64 < FP64_TOL, e64
    p32, u32 = _run(dmk, x, eps=eps, ns=ns, periodic=periodic, precision=1, kernels=kernels, **args)
    e32 = rel_l2(u32, u_ref)
    assert e32 < mixed_tol(eps), e32
    # element-wise: every target within a few times the l2 bound
    scale = np.linalg.norm(u_ref) / np.sqrt(u_ref.size)
    assert np.max(np.abs(u64 - u_ref)) < 1e3 * FP64_TOL * scale
    p64.close()
    p32.close()


@pytest.mark.parametrize("eps", [1e-6, 1e-8, 1e-10])
def test_gradient_parity(dmk, eps):
    """FP64 and MIXED velocity gradients against the oracle's derivative of the
    residual Stokeslet (MIXED: float-float pair terms at every eps), 10 eps."""
    rng = np.random.default_rng(77)
    N, ns = 1200, 40
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3)
    tr = Tree(x, ns)
    win = ProlateWindow(bandlimit_c(eps))
    u_ref, G_ref = onear.near_lists(tr, dict(win=win, stokeslet=True), f=f, want_grad=True)
    for prec, tol in ((0, FP64_TOL), (1, 10 * eps)):
        p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, precision=prec, leaf_capacity=ns)
        u, G = p.eval_grad(torch.as_tensor(f, device="cuda"), want_u=True)
        p.sync_status()
        assert rel_l2(u.cpu().numpy(), u_ref) < (FP64_TOL if prec == 0 else 10 * eps)
        assert rel_l2(G.cpu().numpy(), G_ref) < tol, (prec, rel_l2(G.cpu().numpy(), G_ref))
        p.close()


@pytest.mark.parametrize("N", [0, 1, 2, 33])
def test_tiny_inputs(dmk, N):
    rng = np.random.default_rng(5 + N)
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3)
    for prec in (0, 1):
        p, u = _run(dmk, x, f=f, eps=1e-6, ns=8, precision=prec)
        if N == 0:
            assert u.shape == (0, 3)
            continue
        tr, u_ref = _oracle(x, f, None, None, 1e-6, 8, False, 1)
        assert rel_l2(u, u_ref) < (FP64_TOL if prec == 0 else 1e-5)


def test_faces_coincident_and_single_leaf(dmk):
    rng = np.random.default_rng(9)
    x = wl.uniform_points(rng, 400, 3)
    x[:20] = np.round(x[:20] * 4) / 4            # on box faces, edges, corners (incl. +-1/2)
    x[20] = 0.5
    x[21] = -0.5
    x[30:35] = x[40]                              # coincident points (their pair terms are skipped)
    f = wl.forces(rng, 400, 3)
    for ns in (10, 500):                          # deep-ish tree / everything in the root leaf
        tr, u_ref = _oracle(x, f, None, None, 1e-6, ns, False, 1)
        for prec in (0, 1):
            p, u = _run(dmk, x, f=f, eps=1e-6, ns=ns, precision=prec)
            assert_tree_equal(p.tree(), tr, hilbert_order(prec, 1e-6))
            assert rel_l2(u, u_ref) < (FP64_TOL if prec == 0 else 1e-5)


def test_out_of_range_point_is_reported(dmk):
    x = np.zeros((10, 3))
    x[3, 1] = 0.75
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=1e-6)
    with pytest.raises(dmk.DMKError) as ei:
        p.sync_status()
    assert ei.value.code == 2


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("periodic", [False, True])
def test_nonfinite_point_is_reported(dmk, bad, periodic):
    x = np.zeros((10, 3))
    x[4, 2] = bad
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=1e-6, periodic=periodic)
    with pytest.raises(dmk.DMKError) as ei:
        p.sync_status()
    assert ei.value.code == 1
    p.close()


def test_points_on_the_box_faces_are_in_range(dmk):
    """w = 0 and w = 1 exactly (x = -1/2, +1/2) are inside the free-space box;
    w = 1 + 2^-50 is not."""
    rng = np.random.default_rng(77)
    x = wl.uniform_points(rng, 300, 3)
    x[:8] = [[-0.5, -0.5, -0.5], [0.5, 0.5, 0.5], [-0.5, 0.5, 0.0], [0.5, -0.5, 0.25],
             [0.0, 0.5, -0.5], [-0.0, 0.0, 0.5], [0.5, 0.5, -0.5], [-0.5, -0.5, 0.5]]
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=1e-6, leaf_capacity=8)
    p.sync_status()
    tr = Tree(x, 8)
    assert_tree_equal(p.tree(), tr, hilbert_order(dmk.MIXED, 1e-6))
    p.close()
    y = x.copy()
    y[5, 0] = 0.5 + 2.0 ** -50
    q = dmk.Plan(torch.as_tensor(y, device="cuda"), eps=1e-6, leaf_capacity=8)
    with pytest.raises(dmk.DMKError) as ei:
        q.sync_status()
    assert ei.value.code == 2
    q.close()


@pytest.mark.parametrize("dim", [3, 2])
def test_refinement_to_the_maximum_level(dmk, dim):
    """40 coincident points and a tight pair with n_s = 8: the tree refines to
    the maximum level M (21 in 3D, 31 in 2D) at that spot, the leaf there keeps
    all its points, and level restriction cascades out from it.  Tree parity
    is exact; coincident pairs are skipped on both sides."""
    rng = np.random.default_rng(1234 + dim)
    x = wl.uniform_points(rng, 600, dim)
    x[:40] = x[40]                                   # 41 coincident points
    x[41] = x[40] + 1e-9                             # a near neighbour far below the finest cell
    f = wl.forces(rng, 600, dim)
    ns = 8
    tr = Tree(x, ns)
    assert int(tr.leaf_level.max()) == {3: 21, 2: 31}[dim]
    if dim == 3:
        win = ProlateWindow(bandlimit_c(1e-6))
        u_ref = onear.near_lists(tr, dict(win=win, stokeslet=True), f=f)
    else:
        from oracle import kernels2d as k2
        u_ref = onear.near_lists(tr, dict(k2d=k2.Kernel2D(ProlateWindow(bandlimit_c(1e-6))), stokeslet=True), f=f)
    for prec in (0, 1):
        p, u = _run(dmk, x, f=f, eps=1e-6, ns=ns, precision=prec)
        assert_tree_equal(p.tree(), tr, hilbert_order(prec, 1e-6))
        assert rel_l2(u, u_ref) < (FP64_TOL if prec == 0 else 1e-5)
        p.close()
