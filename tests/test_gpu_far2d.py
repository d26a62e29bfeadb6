"""components = ALL in 2D: the DMK far field with the App. B kernels on the GPU.

* Far component alone: GPU (ALL minus NEAR on the same plan parameters) against
  the oracle's 2D far field (oracle/dmk.py FarField on the same tree and the
  same p, N1, N_per): proxy charges, merges, plane waves with 9 colleagues, the
  root (periodic series or the truncated kernel with R = 1 + sqrt 2 and
  K_corr = (1 - log R)/(4 pi)), interpolation - FP64 to round-off.
* Whole velocity: against the O(N^2) 2D direct sum (free space) or the 2D
  Gaussian Ewald sum at tolerance 1e-14 (periodic), relative l2 <= 10 eps, in
  FP64 and MIXED; separate targets; eps 1e-10; a root-only tree.
"""
import numpy as np
import pytest
import torch

from oracle import dmk as odmk
from oracle import direct, ewald, tree as otree, window
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


def _density(rng, N, kernels, periodic):
    f = wl.forces(rng, N, 2, zero_mean=periodic) if kernels & 1 else None
    g = wl.stresslet_strengths(rng, N, 2) if kernels & 2 else None
    nrm = wl.unit_normals(rng, N, 2) if kernels & 2 else None
    return f, g, nrm


@pytest.mark.parametrize("periodic,kernels,ns,eps", [(False, 1, 30, 1e-6), (True, 1, 25, 1e-6),
                                                     (False, 2, 30, 1e-3), (True, 3, 25, 1e-3),
                                                     (False, 3, 20, 1e-9)])
def test_far_component_matches_oracle_2d(dmk, periodic, kernels, ns, eps):
    rng = np.random.default_rng(211 + kernels + 10 * periodic)
    N = 1200
    x = wl.gaussian_mixture_points(rng, N, 2, 4, 0.08)
    f, g, nrm = _density(rng, N, kernels, periodic)
    u_all, info = _run(dmk, x, f, g, nrm, eps, 0, ns, periodic, dmk.ALL)
    u_near, _ = _run(dmk, x, f, g, nrm, eps, 0, ns, periodic, dmk.NEAR)
    tcp, p, n1, nper = odmk.dmk_params(eps, stokeslet=bool(kernels & 1), stresslet=bool(kernels & 2))
    assert (info["p"], info["n1"]) == (p, n1)
    if periodic:
        assert info["root_modes"] == nper
    win = window.ProlateWindow(tcp * np.pi / 3)
    T = otree.Tree(x, ns, periodic=periodic)
    assert info["max_level"] == T.leaf_level.max() and info["max_level"] >= 3
    u_far = odmk.FarField(T, win, p, n1, nper).far(f, g, nrm)
    assert rel_l2(u_all - u_near, u_far) < 1e-11, rel_l2(u_all - u_near, u_far)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kernels", [1, 2, 3])
def test_clustered_free_space_matches_direct_sum_2d(dmk, prec, kernels):
    eps = 1e-6
    rng = np.random.default_rng(240 + kernels)
    N = 3000
    x = wl.gaussian_mixture_points(rng, N, 2, 8, 0.03)
    f, g, nrm = _density(rng, N, kernels, False)
    u, info = _run(dmk, x, f, g, nrm, eps, prec, 40, False, dmk.ALL)
    assert info["max_level"] >= 4 and info["fp32"] == prec
    ref = direct.direct_sum(x, f, g, nrm)
    assert rel_l2(u, ref) < 10 * eps, rel_l2(u, ref)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kernels", [1, 3])
def test_periodic_matches_ewald_2d(dmk, prec, kernels):
    eps = 1e-6
    rng = np.random.default_rng(260 + kernels)
    N = 500
    x = wl.gaussian_mixture_points(rng, N, 2, 4, 0.1)
    f, g, nrm = _density(rng, N, kernels, True)
    u, _ = _run(dmk, x, f, g, nrm, eps, prec, 12, True, dmk.ALL)
    ref = ewald.ewald_sum(x, f, g, nrm, split=ewald.gaussian_split_2d(0.08))
    assert rel_l2(u, ref) < 10 * eps, rel_l2(u, ref)


def test_separate_targets_match_direct_sum_2d(dmk):
    from oracle.direct import stokeslet_2d, stresslet_2d
    eps = 1e-6
    rng = np.random.default_rng(277)
    xs = wl.gaussian_mixture_points(rng, 2500, 2, 6, 0.05)
    xt = wl.uniform_points(rng, 2000, 2)
    f, g, nrm = _density(rng, 2500, 3, False)
    ref = np.zeros((2000, 2))
    for i in range(2000):
        d = xt[i][None, :] - xs
        ref[i] = (np.einsum("pjl,pl->j", stokeslet_2d(d), f) + np.einsum("pjlm,pl,pm->j", stresslet_2d(d), g, nrm))
    for prec in (0, 1):
        u, _ = _run(dmk, xs, f, g, nrm, eps, prec, 40, False, dmk.ALL, targets=xt)
        assert u.shape == (2000, 2)
        assert rel_l2(u, ref) < 10 * eps, (prec, rel_l2(u, ref))


def test_eps_1e10_fp64_matches_direct_sum_2d(dmk):
    eps = 1e-10
    rng = np.random.default_rng(290)
    N = 2500
    x = wl.gaussian_mixture_points(rng, N, 2, 8, 0.05)
    f = wl.forces(rng, N, 2)
    u, info = _run(dmk, x, f, None, None, eps, 0, 60, False, dmk.ALL)
    assert info["fp32"] == 0
    ref = direct.direct_sum(x, f)
    assert rel_l2(u, ref) < 10 * eps, rel_l2(u, ref)


def test_root_leaf_and_empty_cases_2d(dmk):
    rng = np.random.default_rng(25)
    x = wl.uniform_points(rng, 40, 2)                     # one leaf: the root
    f = wl.forces(rng, 40, 2)
    u, info = _run(dmk, x, f, None, None, 1e-6, 0, 64, False, dmk.ALL)
    assert info["boxes"] == 1
    assert rel_l2(u, direct.direct_sum(x, f)) < 1e-5
    u, _ = _run(dmk, x, f, None, None, 1e-6, 0, 64, False, dmk.ALL, targets=np.zeros((0, 2)))
    assert u.shape == (0, 2)
