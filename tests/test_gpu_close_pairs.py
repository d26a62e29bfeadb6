"""Nearly coincident points in shallow leaves (MIXED precision, and FP64).

FP32 and float-float pair terms start from leaf-relative coordinates, whose
rounding error is a relative error of the displacement x of about
2^-23 h / r (FP32; h the leaf side) or 2^-48 h / r (float-float).  For the
closest pairs that term is also the largest (S_R -> S as r -> 0, App. A.1),
so the library takes pairs with r <= nu/16 (FP32) or r <= nu/1024
(float-float) in FP64 from the FP64 coordinates.  Here partners are planted at
r = 1e-5, 1e-7 and 1e-9 of the leaf side next to points of leaves on levels 1
and 2 (n_s large), where FP32 leaf-relative coordinates cannot resolve them
(at 1e-9 h the two points round to the same FP32 coordinates), and the
per-target error is checked, not only the aggregate l2:
  * planted points (their velocity is dominated by the close pair):
    |u_t - u_ref,t| / |u_ref,t| <= 10 eps (MIXED), 1e-11 (FP64);
  * every target: |u_t - u_ref,t| / max(|u_ref,t|, rms(u_ref)) <= 10 eps
    (MIXED), 1e-11 (FP64).
"""
import zlib

import numpy as np
import pytest
import torch

from oracle import near as onear, kernels2d as k2
from oracle.tree import Tree
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

R_FRACS = (1e-5, 1e-7, 1e-9)


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


def _planted(rng, dim, n0, ns, per_frac=10):
    """n0 uniform points plus, for each r_frac, per_frac partners at r_frac x
    (leaf side of the base point's leaf) in a random direction."""
    x0 = wl.uniform_points(rng, n0, dim)
    tr0 = Tree(x0, ns)
    base = rng.choice(n0, per_frac * len(R_FRACS), replace=False)
    partners = []
    for k, b in enumerate(base):
        h = 2.0 ** -int(tr0.point_level[b])
        d = rng.standard_normal(dim)
        d /= np.linalg.norm(d)
        partners.append(x0[b] + R_FRACS[k // per_frac] * h * d)
    x = np.concatenate([x0, np.array(partners)])
    planted = np.concatenate([base, n0 + np.arange(len(base))])
    return x, planted, tr0


def _per_target(u, u_ref, planted):
    du = np.linalg.norm(u - u_ref, axis=1)
    nr = np.linalg.norm(u_ref, axis=1)
    rms = np.sqrt(np.mean(nr ** 2))
    return float(np.max(du[planted] / nr[planted])), float(np.max(du / np.maximum(nr, rms)))


CASES = [
    # dim, kernels, eps, n_rhs
    (3, 1, 1e-6, 1),
    (3, 3, 1e-6, 1),
    (3, 1, 1e-6, 4),
    (3, 1, 1e-10, 1),
    (3, 3, 1e-10, 1),
    (2, 3, 1e-6, 1),
    (2, 3, 1e-8, 1),
]


@pytest.mark.parametrize("dim,kernels,eps,n_rhs", CASES)
def test_close_pairs_per_target(dmk, dim, kernels, eps, n_rhs):
    rng = np.random.default_rng(zlib.crc32(f"close{dim}{kernels}{eps}{n_rhs}".encode()))
    n0, ns = (3000, 800) if dim == 3 else (2000, 300)
    x, planted, tr0 = _planted(rng, dim, n0, ns)
    N = len(x)
    tr = Tree(x, ns)
    assert int(np.max(tr.leaf_level)) <= 2                  # shallow leaves
    f = wl.forces(rng, N, dim, n_rhs=n_rhs)
    g = wl.stresslet_strengths(rng, N, dim)
    nrm = wl.unit_normals(rng, N, dim)
    st, sl = bool(kernels & 1), bool(kernels & 2)
    c = bandlimit_c(eps, stokeslet=st, stresslet=sl)
    kern = dict(win=ProlateWindow(c), stokeslet=st, stresslet=sl)
    if dim == 2:
        kern = dict(k2d=k2.Kernel2D(ProlateWindow(c)), stokeslet=st, stresslet=sl)
    fcols = [f] if n_rhs == 1 else [f[:, :, k] for k in range(n_rhs)]
    refs = []
    for k, fk in enumerate(fcols):
        refs.append(onear.near_lists(tr, kern, f=fk if st else None, g=g if (sl and k == 0) else None,
                                     n=nrm if (sl and k == 0) else None))
    for prec in (dmk.FP64, dmk.MIXED):
        p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, kernels=kernels, precision=prec,
                     leaf_capacity=ns, n_rhs=n_rhs)
        args = [torch.as_tensor(f, device="cuda") if st else None]
        args += [torch.as_tensor(g, device="cuda"), torch.as_tensor(nrm, device="cuda")] if sl else [None, None]
        u = p.eval(*args).cpu().numpy()
        p.sync_status()
        p.close()
        ucols = [u] if n_rhs == 1 else [u[:, :, k] for k in range(n_rhs)]
        tol = 1e-11 if prec == dmk.FP64 else 10 * eps
        for uk, rk in zip(ucols, refs):
            e_planted, e_all = _per_target(uk, rk, planted)
            assert e_planted < tol, (prec, e_planted)
            assert e_all < tol, (prec, e_all)


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_close_pair_queue_overflow(dmk, eps):
    """Clusters of three nearly coincident points everywhere: the symmetric
    passes queue far more skipped pairs than the queue holds (max(1024, N/4)),
    so the marked-tile walk takes over; the result must not change."""
    rng = np.random.default_rng(99 + int(-np.log10(eps)))
    n0, ns = 1500, 800
    x0 = wl.uniform_points(rng, n0, 3)
    d1, d2 = rng.standard_normal((n0, 3)), rng.standard_normal((n0, 3))
    x = np.concatenate([x0, x0 + 1e-7 * d1, x0 + 3e-9 * d2])
    N = len(x)
    f = wl.forces(rng, N, 3)
    tr = Tree(x, ns)
    u_ref = onear.near_lists(tr, dict(win=ProlateWindow(bandlimit_c(eps)), stokeslet=True), f=f)
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, precision=dmk.MIXED, leaf_capacity=ns)
    u = p.eval(torch.as_tensor(f, device="cuda")).cpu().numpy()
    p.sync_status()
    p.close()
    e_planted, e_all = _per_target(u, u_ref, np.arange(N))
    assert e_all < 10 * eps, e_all
