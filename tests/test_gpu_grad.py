"""GPU gradient and autograd checks (row a7).

* eval_grad against central finite differences of eval (FP64, plan rebuilt at
  x +- h with the tree checked unchanged), and against the oracle gradient;
* the autograd function's dL/df and dL/dx for L = 1/2 |u - u_tgt|^2 (backward =
  one dmk_stokes_eval_adjoint call) against the oracle adjoint (dL/df = S[w],
  dL/dx = (grad u)^T w + (grad v)^T f, v = S[w]), and eval_adjoint directly;
* torch.autograd.gradcheck on a tiny system;
* the differentiation workload (3D periodic, N = 2e5 uniform, zero-mean forces,
  eps = 1e-8): directional finite differences of L on a 500-point subset.
"""
import numpy as np
import pytest
import torch

from oracle import near as onear
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


def _same_tree(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("leaf_level", "leaf_coords", "leaf_count", "near_leaf", "near_q"))


def test_eval_grad_matches_finite_differences(dmk):
    rng = np.random.default_rng(301)
    N, ns, eps, h = 3000, 48, 1e-6, 1e-6
    x = wl.uniform_points(rng, N, 3)
    f = torch.as_tensor(wl.forces(rng, N, 3), device="cuda")
    p0 = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, precision=dmk.FP64, leaf_capacity=ns)
    G = p0.eval_grad(f).cpu().numpy()
    tree0 = p0.tree()
    checked = 0
    num = den = 0.0
    for t in rng.choice(N, 40, replace=False):
        for m in range(3):
            us = []
            for sgn in (1, -1):
                xp = x.copy()
                xp[t, m] += sgn * h
                p = dmk.Plan(torch.as_tensor(xp, device="cuda"), eps=eps, precision=dmk.FP64, leaf_capacity=ns)
                ok = _same_tree(p.tree(), tree0)
                us.append(p.eval(f).cpu().numpy()[t])
                p.close()
                if not ok:
                    break
            if len(us) < 2 or not ok:
                continue
            checked += 1
            fd = (us[0] - us[1]) / (2 * h)
            num += np.sum((fd - G[t, :, m]) ** 2)
            den += np.sum(G[t, :, m] ** 2)
    assert checked >= 100 and den > 0
    assert np.sqrt(num / den) < 1e-5, np.sqrt(num / den)


def _oracle_adjoint(x, f, u_tgt, eps, ns, periodic):
    tr = Tree(x, ns, periodic=periodic)
    kern = dict(win=ProlateWindow(bandlimit_c(eps)), stokeslet=True)
    u, gu = onear.near_lists(tr, kern, f=f, want_grad=True)
    w = u - u_tgt
    v, gv = onear.near_lists(tr, kern, f=w, want_grad=True)
    gx = np.einsum("tjm,tj->tm", gu, w) + np.einsum("tjm,tj->tm", gv, f)
    return u, v, gx


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("precision,eps", [(0, 1e-8), (1, 1e-8), (1, 1e-6)])
def test_autograd_matches_oracle_adjoint(dmk, periodic, precision, eps):
    """Backward = one dmk_stokes_eval_adjoint call.  FP64: round-off bounds;
    MIXED (float-float pair terms at both eps): 10 eps."""
    rng = np.random.default_rng(302 + periodic)
    N, ns = 1500, 40
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3, zero_mean=True)
    u_tgt = 0.1 * rng.standard_normal((N, 3))
    u_o, gf_o, gx_o = _oracle_adjoint(x, f, u_tgt, eps, ns, periodic)
    xt = torch.as_tensor(x, device="cuda").requires_grad_(True)
    ft = torch.as_tensor(f, device="cuda").requires_grad_(True)
    u = dmk.near_stokeslet(xt, ft, eps=eps, leaf_capacity=ns, periodic=periodic, precision=precision)
    L = 0.5 * ((u - torch.as_tensor(u_tgt, device="cuda")) ** 2).sum()
    L.backward()
    tol = (1e-12, 1e-12, 1e-11) if precision == 0 else (10 * eps, 10 * eps, 10 * eps)
    assert rel_l2(u.detach().cpu().numpy(), u_o) < tol[0]
    assert rel_l2(ft.grad.cpu().numpy(), gf_o) < tol[1]
    assert rel_l2(xt.grad.cpu().numpy(), gx_o) < tol[2]


@pytest.mark.parametrize("precision", [0, 1])
def test_eval_adjoint_clustered_matches_oracle(dmk, precision):
    """dmk_stokes_eval_adjoint on clustered points (leaves on several levels,
    coarse-neighbour pairs) against the oracle adjoint, and twice in a row
    (the adjoint workspace is reused)."""
    rng = np.random.default_rng(311)
    N, ns, eps = 2500, 24, 1e-10
    x = wl.gaussian_mixture_points(rng, N, 3, 8, 0.03)
    f = wl.forces(rng, N, 3)
    w = wl.forces(rng, N, 3)
    tr = Tree(x, ns)
    kern = dict(win=ProlateWindow(bandlimit_c(eps)), stokeslet=True)
    _, gu = onear.near_lists(tr, kern, f=f, want_grad=True)
    v_o, gv = onear.near_lists(tr, kern, f=w, want_grad=True)
    gx_o = np.einsum("tjm,tj->tm", gu, w) + np.einsum("tjm,tj->tm", gv, f)
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, precision=precision, leaf_capacity=ns)
    fd, wd = torch.as_tensor(f, device="cuda"), torch.as_tensor(w, device="cuda")
    tol = 1e-11 if precision == 0 else 10 * eps
    for _ in range(2):
        v, gx = p.eval_adjoint(fd, wd)
        p.sync_status()
        assert rel_l2(v.cpu().numpy(), v_o) < tol
        assert rel_l2(gx.cpu().numpy(), gx_o) < tol
    p.close()


def test_gradcheck_tiny(dmk):
    rng = np.random.default_rng(303)
    N = 24
    x = torch.as_tensor(wl.uniform_points(rng, N, 3) * 0.4, device="cuda").requires_grad_(True)
    f = torch.as_tensor(wl.forces(rng, N, 3), device="cuda").requires_grad_(True)
    fn = lambda xx, ff: dmk.near_stokeslet(xx, ff, eps=1e-10, leaf_capacity=6)
    assert torch.autograd.gradcheck(fn, (x, f), eps=1e-7, atol=1e-6, rtol=1e-5)


def test_differentiation_workload_fd(dmk):
    """3D periodic unit cube, N = 2e5 uniform, zero-mean forces, eps = 1e-8;
    L = 1/2 |u - u_tgt|^2 with u_tgt from the forces plus a seeded 0.1 N(0,1)
    perturbation; directional FD of L w.r.t. the first 500 points.
    h = 1e-7: the central-difference truncation error scales as h^2 and points
    with close neighbours (gradients ~3e4) need it below 1e-5 (measured:
    3.6e-6 at h = 1e-6, 3.5e-8 at h = 1e-7)."""
    eps, h = 1e-8, 1e-7
    x, f = wl.periodic_3d(n=200_000)
    rng = wl.rng_for(4, extra=1)
    xi = rng.standard_normal(f.shape)
    xd = torch.as_tensor(x, device="cuda")
    fd_ = torch.as_tensor(f, device="cuda")
    p0 = dmk.Plan(xd, eps=eps, periodic=True, precision=dmk.FP64)
    u_tgt = p0.eval(torch.as_tensor(f + 0.1 * xi, device="cuda"))
    tree0 = p0.tree()
    p0.close()
    xt = xd.clone().requires_grad_(True)
    ft = fd_.clone().requires_grad_(True)
    u = dmk.near_stokeslet(xt, ft, eps=eps, periodic=True)
    L = 0.5 * ((u - u_tgt) ** 2).sum()
    L.backward()
    gx = xt.grad.cpu().numpy()

    def velocity(xx):
        p = dmk.Plan(torch.as_tensor(xx, device="cuda"), eps=eps, periodic=True, precision=dmk.FP64)
        same = _same_tree(p.tree(), tree0)
        u = p.eval(fd_)
        p.close()
        return u, same

    an, fdv = [], []
    for k in range(500):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        xp = x.copy(); xp[k] += h * d
        xm = x.copy(); xm[k] -= h * d
        up, sp = velocity(xp)
        um, sm = velocity(xm)
        if not (sp and sm):
            continue
        # L(x+) - L(x-) = 1/2 sum (u+ - u-) . (u+ + u- - 2 u_tgt), free of the
        # cancellation of subtracting two large totals
        dl = 0.5 * float(((up - um) * (up + um - 2 * u_tgt)).sum())
        an.append(gx[k] @ d)
        fdv.append(dl / (2 * h))
    assert len(an) >= 450
    an, fdv = np.array(an), np.array(fdv)
    assert np.linalg.norm(an - fdv) / np.linalg.norm(an) < 1e-5


@pytest.mark.parametrize("kernels,periodic", [(3, False), (2, True), (2, False)])
@pytest.mark.parametrize("precision", [0, 1])
def test_stresslet_gradient_matches_oracle(dmk, kernels, periodic, precision):
    """Gradient of the stresslet (and Stokeslet) near component against the
    oracle's derivative of Eq. (res_stresslet) (itself pinned by finite
    differences); periodic: plus the k = 0 term's -delta_jm sum g.n.  FP64
    pair terms in both precisions."""
    rng = np.random.default_rng(701 + kernels + 10 * periodic)
    N, ns, eps = 2000, 40, 1e-8
    x = wl.gaussian_mixture_points(rng, N, 3, 6, 0.05)
    f = wl.forces(rng, N, 3)
    g = wl.stresslet_strengths(rng, N, 3)
    n = wl.unit_normals(rng, N, 3)
    tr = Tree(x, ns, periodic=periodic)
    st, sl = bool(kernels & 1), bool(kernels & 2)
    kern = dict(win=ProlateWindow(bandlimit_c(eps, stokeslet=st, stresslet=sl)), stokeslet=st, stresslet=sl)
    u_ref, G_ref = onear.near_lists(tr, kern, f=f if st else None, g=g, n=n, want_grad=True)
    if periodic:
        from oracle import direct as odirect
        u_ref = u_ref + odirect.stresslet_zero_mode(tr.w, g, n)
        G_ref = G_ref - np.sum(g * n) * np.eye(3)[None, :, :]
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, periodic=periodic, kernels=kernels,
                 precision=precision, leaf_capacity=ns)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    u, G = p.eval_grad(dev(f) if st else None, dev(g), dev(n), want_u=True)
    p.sync_status()
    p.close()
    assert rel_l2(u.cpu().numpy(), u_ref) < 1e-12
    assert rel_l2(G.cpu().numpy(), G_ref) < 1e-12
