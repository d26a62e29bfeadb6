"""components = ALL: the DMK far field of Sec. 6 (3D) on the GPU.

* Far component alone: GPU (ALL minus NEAR on the same plan parameters) against
  the oracle's far field (oracle/dmk.py: proxy charges, plane waves, root,
  interpolation) on the same tree and the same (p, N1, N_per) - FP64 to
  round-off.
* Whole velocity: against the O(N^2) direct sum (free space) or the Gaussian
  Ewald sum at tolerance 1e-14 (periodic), relative l2 <= 10 eps (the stresslet
  at the Table 2 bandlimit reaches about 2 eps in the oracle as well).
* The 2000-point uniform free-space case with leaf capacity 64, eps 1e-6, FP64;
  clustered (adaptive, mixed leaf levels) cases; separate targets; eps 1e-10.
"""
import numpy as np
import pytest
import torch

from oracle import dmk as odmk
from oracle import direct, ewald, tree as otree, window
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


def _dev(a):
    return None if a is None else torch.as_tensor(a, device="cuda")


def _run(dmk, x, f, g, n, eps, prec, ns, periodic, comp, targets=None):
    kernels = (1 if f is not None else 0) | (2 if g is not None else 0)
    p = dmk.Plan(_dev(x), eps=eps, periodic=periodic, kernels=kernels, precision=prec, leaf_capacity=ns,
                 components=comp, targets=_dev(targets))
    u = p.eval(_dev(f), _dev(g), _dev(n)).cpu().numpy()
    info = p.far_info()
    p.close()
    return u, info


@pytest.mark.parametrize("periodic,kernels,ns", [(False, 1, 64), (True, 1, 40), (False, 2, 64), (True, 3, 40)])
def test_far_component_matches_oracle(dmk, periodic, kernels, ns):
    eps = 1e-6 if kernels == 1 else 1e-3
    rng = np.random.default_rng(11 + kernels + 10 * periodic)
    N = 1200
    x = wl.gaussian_mixture_points(rng, N, 3, 4, 0.08)
    f = wl.forces(rng, N, 3, zero_mean=periodic) if kernels & 1 else None
    g = wl.stresslet_strengths(rng, N, 3) if kernels & 2 else None
    nrm = wl.unit_normals(rng, N, 3) if kernels & 2 else None
    u_all, info = _run(dmk, x, f, g, nrm, eps, 0, ns, periodic, dmk.ALL)
    u_near, _ = _run(dmk, x, f, g, nrm, eps, 0, ns, periodic, dmk.NEAR)
    tcp, p, n1, nper = odmk.dmk_params(eps, stokeslet=bool(kernels & 1), stresslet=bool(kernels & 2))
    assert (info["p"], info["n1"]) == (p, n1)
    assert info["root_modes"] == (nper if periodic else info["root_modes"])
    win = window.ProlateWindow(tcp * np.pi / 3)
    T = otree.Tree(x, ns, periodic=periodic)
    assert info["max_level"] == T.leaf_level.max()
    F = odmk.FarField(T, win, p, n1, nper)
    u_far = F.far(f, g, nrm)
    assert rel_l2(u_all - u_near, u_far) < 1e-11, rel_l2(u_all - u_near, u_far)


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-5)])
def test_uniform_2000_leaf64_matches_direct_sum(dmk, prec, tol):
    """3D free-space Stokeslet, N = 2000 uniform, forces N(0,1), eps 1e-6,
    leaf capacity 64, against the O(N^2) direct FP64 sum."""
    x, f = wl.small_uniform_3d()
    u, info = _run(dmk, x, f, None, None, 1e-6, prec, 64, False, dmk.ALL)
    assert info["fp32"] == prec
    ref = direct.direct_sum(x, f)
    assert rel_l2(u, ref) < tol, rel_l2(u, ref)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kernels", [1, 2, 3])
def test_clustered_free_space_matches_direct_sum(dmk, prec, kernels):
    eps = 1e-6
    rng = np.random.default_rng(40 + kernels)
    N = 4000
    x = wl.gaussian_mixture_points(rng, N, 3, 8, 0.03)
    f = wl.forces(rng, N, 3) if kernels & 1 else None
    g = wl.stresslet_strengths(rng, N, 3) if kernels & 2 else None
    nrm = wl.unit_normals(rng, N, 3) if kernels & 2 else None
    u, info = _run(dmk, x, f, g, nrm, eps, prec, 48, False, dmk.ALL)
    assert info["max_level"] >= 4
    ref = direct.direct_sum(x, f, g, nrm)
    assert rel_l2(u, ref) < 10 * eps, rel_l2(u, ref)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kernels", [1, 3])
def test_periodic_matches_ewald(dmk, prec, kernels):
    eps = 1e-6
    rng = np.random.default_rng(60 + kernels)
    N = 2000
    x = wl.gaussian_mixture_points(rng, N, 3, 4, 0.1)
    f = wl.forces(rng, N, 3, zero_mean=True) if kernels & 1 else None
    g = wl.stresslet_strengths(rng, N, 3) if kernels & 2 else None
    nrm = wl.unit_normals(rng, N, 3) if kernels & 2 else None
    u, _ = _run(dmk, x, f, g, nrm, eps, prec, 40, True, dmk.ALL)
    ref = ewald.ewald_sum(x, f, g, nrm, split=ewald.gaussian_split_3d(0.08))
    assert rel_l2(u, ref) < 10 * eps, rel_l2(u, ref)


def test_separate_targets_match_direct_sum(dmk):
    eps = 1e-6
    rng = np.random.default_rng(77)
    xs, xt, f, g, nrm = wl.linear_scaling(3000)
    for prec in (0, 1):
        u, info = _run(dmk, xs, f, g, nrm, eps, prec, 64, False, dmk.ALL, targets=xt)
        assert u.shape == (3000, 3)
        # direct sum at separate targets: every source counts (no self pair)
        ref = np.zeros_like(u)
        from oracle import kernels3d as k3
        for i in range(len(xt)):
            d = xt[i][None, :] - xs
            ref[i] = (np.einsum("pjl,pl->j", k3.stokeslet(d), f)
                      + np.einsum("pjlm,pl,pm->j", k3.stresslet(d), g, nrm))
        assert rel_l2(u, ref) < 10 * eps, (prec, rel_l2(u, ref))


def test_eps_1e10_fp64_matches_direct_sum(dmk):
    eps = 1e-10
    rng = np.random.default_rng(90)
    N = 2000
    x = wl.gaussian_mixture_points(rng, N, 3, 8, 0.05)
    f = wl.forces(rng, N, 3)
    u, info = _run(dmk, x, f, None, None, eps, 0, 150, False, dmk.ALL)
    assert info["fp32"] == 0
    ref = direct.direct_sum(x, f)
    assert rel_l2(u, ref) < 10 * eps, rel_l2(u, ref)


def test_root_leaf_and_empty_cases(dmk):
    rng = np.random.default_rng(5)
    x = wl.uniform_points(rng, 50, 3)                     # one leaf: the root
    f = wl.forces(rng, 50, 3)
    u, info = _run(dmk, x, f, None, None, 1e-6, 0, 64, False, dmk.ALL)
    assert info["boxes"] == 1
    assert rel_l2(u, direct.direct_sum(x, f)) < 1e-5
    # empty set of separate targets
    u, _ = _run(dmk, x, f, None, None, 1e-6, 0, 64, False, dmk.ALL, targets=np.zeros((0, 3)))
    assert u.shape == (0, 3)


def test_traced_evaluation_matches_eval_and_times_every_stage(dmk):
    rng = np.random.default_rng(21)
    x = torch.as_tensor(wl.gaussian_mixture_points(rng, 20000, 3, 8, 0.05), device="cuda")
    f = torch.as_tensor(wl.forces(rng, 20000, 3), device="cuda")
    for comp in (dmk.ALL, dmk.NEAR):
        p = dmk.Plan(x, eps=1e-6, precision=dmk.MIXED, leaf_capacity=256, components=comp)
        u = p.eval(f).cpu().numpy()
        u2, ms = p.eval_traced(f)
        assert np.array_equal(u, u2.cpu().numpy())
        assert list(ms) == list(dmk.Plan.STAGES)
        assert all(v >= 0.0 for v in ms.values()) and ms["near"] > 0.0
        if comp == dmk.ALL:
            assert ms["leaf_charges"] > 0.0 and ms["outgoing"] > 0.0 and ms["leaf_eval"] > 0.0
        else:
            assert sum(v for k, v in ms.items() if k != "near") == 0.0
        p.close()


@pytest.mark.parametrize("eps,kernels", [(1e-3, 1), (1e-5, 3), (1e-6, 1), (1e-6, 3), (2e-7, 1)])
def test_tensor_core_leaf_kernels_match_fp32_pipe(dmk, monkeypatch, eps, kernels):
    """MIXED: the tcgen05 leaf charges and leaf evaluation (split-TF32 products, row
    widths 16 / 24 / 32, 48 / 64 / 80 charge columns) against the FP32-pipe kernels on
    the same plan, and both against the direct sum."""
    rng = np.random.default_rng(500 + kernels)
    N = 5000
    x = wl.gaussian_mixture_points(rng, N, 3, 8, 0.05)
    f = wl.forces(rng, N, 3) if kernels & 1 else None
    g = wl.stresslet_strengths(rng, N, 3) if kernels & 2 else None
    nrm = wl.unit_normals(rng, N, 3) if kernels & 2 else None
    monkeypatch.setenv("DMK_STOKES_FAR_TC", "1")
    u_tc, info = _run(dmk, x, f, g, nrm, eps, 1, 150, False, dmk.ALL)
    monkeypatch.setenv("DMK_STOKES_FAR_TC", "0")
    u_pipe, _ = _run(dmk, x, f, g, nrm, eps, 1, 150, False, dmk.ALL)
    assert info["fp32"] == 1
    assert rel_l2(u_tc, u_pipe) < max(1e-5, eps), rel_l2(u_tc, u_pipe)
    ref = direct.direct_sum(x, f, g, nrm)
    assert rel_l2(u_tc, ref) < 10 * eps, rel_l2(u_tc, ref)


def test_tensor_core_wait_limit_is_reported_and_the_device_stays_usable(dmk):
    """The bounded wait of the tensor-core kernels run out on purpose (an mbarrier
    that nothing completes, ~1 ms limit): reported as the kernels report it, tensor
    memory freed, and the device still evaluates a plan correctly afterwards."""
    assert dmk.tc_wait_selftest() is True
    x, f = wl.small_uniform_3d()
    u, info = _run(dmk, x, f, None, None, 1e-6, 1, 64, False, dmk.ALL)
    assert info["fp32"] == 1
    assert rel_l2(u, direct.direct_sum(x, f)) < 1e-5
