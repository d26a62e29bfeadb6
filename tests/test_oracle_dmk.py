"""Pins of the oracle's DMK far field (oracle/dmk.py) against things other than itself.

* Parameters: the rules for (3c/pi, p, N1, N_per) reproduce every row of Table 2
  (Stokeslet and stresslet).
* Proxy basis: the Lagrange basis at the Chebyshev points reproduces polynomials of
  degree < p exactly (numpy's polynomial evaluation) and is cardinal at the nodes.
* Truncated biharmonic kernel: the closed form of Eq. (Btrunc_hat), both branches,
  equals the radial Fourier transform of B^R of Eq. (Btrunc) computed by quadrature.
* Every level of the downward pass: the plane-wave colleague interaction equals the
  same sum done in real space with the residual kernels of Sec. 5.2
  (K_D,l = K_R(r_l) - K_R(r_l+1), pinned in test_oracle_kernels3d.py), on an
  adaptive tree with coarse and fine neighbours, free space and periodic,
  Stokeslet and stresslet; a wrong phase sign, level scale, Hermitian weight or
  kernel term fails here.
* Root: the free-space truncated kernel equals K - K_R(1) summed directly (plus
  the K_M(0) self value); the periodic Fourier series equals the Fourier part of a
  prolate Ewald split at nu = 1 (oracle/ewald.py, pinned by Gaussian Ewald).
* Totals (Sec. 7): near + far against the direct sum on 5000 uniform points with
  Table 2 parameters, relative l2 <= eps (Stokeslet); the periodic total against
  Gaussian Ewald.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import dmk, direct, ewald, near, tree as otree, window
from paper_2509_21471_gb300 import workloads as wl
from tests.helpers import rel_l2

TABLE2 = {   # eps: (3c/pi, p, N1, N_per) for the Stokeslet and the stresslet
    "stokeslet": {1e-3: (10, 12, 19, 3), 1e-6: (17, 23, 33, 5), 1e-9: (25, 33, 49, 9), 1e-12: (31, 44, 61, 11)},
    "stresslet": {1e-3: (9, 11, 17, 3), 1e-6: (17, 22, 33, 5), 1e-9: (25, 33, 49, 9), 1e-12: (32, 44, 63, 11)},
}


@pytest.mark.parametrize("kernel", ["stokeslet", "stresslet"])
def test_parameters_reproduce_table2(kernel):
    for eps, row in TABLE2[kernel].items():
        got = dmk.dmk_params(eps, stokeslet=kernel == "stokeslet", stresslet=kernel == "stresslet")
        assert tuple(got) == row, (eps, got, row)


def test_lagrange_basis_is_exact_on_polynomials():
    p = 13
    xi = dmk.cheb_nodes(p)
    assert np.allclose(np.sort(xi), np.sort(np.cos((2 * np.arange(p) + 1) * np.pi / (2 * p))))
    assert np.allclose(dmk.lagrange(xi, xi), np.eye(p), atol=1e-13)
    rng = np.random.default_rng(0)
    coef = rng.standard_normal(p)                     # degree p - 1
    t = rng.uniform(-1, 1, 50)
    L = dmk.lagrange(xi, t)
    assert np.allclose(np.polyval(coef, xi) @ L, np.polyval(coef, t), atol=1e-11)
    # anterpolation is the transpose: charges keep the total
    assert np.allclose(L.sum(axis=0), 1.0, atol=1e-12)


def test_truncated_biharmonic_closed_form_matches_quadrature():
    R = dmk.R_TRUNC

    def BR(r):                                         # Eq. (Btrunc), d = 3
        return -(r - R / 2 - r * r / (2 * R)) / (8 * np.pi)

    for k in [1e-4, 1e-3, 0.2, 1.0, 3.7, 11.0]:
        # 3D radial transform of a radial function: (4 pi / k) int_0^R B(r) r sin(k r) dr
        val = 4 * np.pi / k * quad(lambda r: BR(r) * r * np.sin(k * r), 0.0, R, limit=200, epsabs=1e-15,
                                   epsrel=1e-12)[0]
        got = float(dmk.B_trunc_hat(np.array([k]))[0])
        assert abs(got - val) <= 1e-9 * max(1.0, abs(val)), (k, got, val)


def _setup(N, ns, periodic, eps, kernels, seed):
    rng = np.random.default_rng(seed)
    x = wl.gaussian_mixture_points(rng, N, 3, 3, 0.08)
    f = wl.forces(rng, N, 3, zero_mean=periodic) if kernels & 1 else None
    g = wl.stresslet_strengths(rng, N, 3) if kernels & 2 else None
    n = wl.unit_normals(rng, N, 3) if kernels & 2 else None
    tcp, p, n1, nper = dmk.dmk_params(eps, stokeslet=bool(kernels & 1), stresslet=bool(kernels & 2))
    win = window.ProlateWindow(tcp * np.pi / 3)
    T = otree.Tree(x, ns, periodic=periodic)
    return x, f, g, n, win, T, dmk.FarField(T, win, p, n1, nper)


@pytest.mark.parametrize("periodic,kernels", [(False, 1), (False, 3), (True, 3)])
def test_each_level_matches_real_space_difference_kernels(periodic, kernels):
    N, ns = (150, 9) if periodic else (400, 16)         # the periodic exact sum loops over 27 images
    x, f, g, n, win, T, F = _setup(N, ns, periodic, 1e-3, kernels, 10 + kernels + 5 * periodic)
    levels = np.unique(T.leaf_level)
    assert len(levels) >= 2 and F.maxlev >= 3          # adaptive: coarse and fine neighbours
    # relative to each level's own sum at eps = 1e-3 (the stresslet at the Table 2 bandlimit
    # reaches about ten times eps per level; a wrong term is off by order one)
    tol = 5e-3 if kernels == 1 else 3e-2
    for lev in range(F.maxlev + 1):
        a = F.far(f, g, n, levels=[lev], want_root=False)
        b = dmk.level_exact(T, win, lev, f, g, n)
        if np.linalg.norm(b) == 0.0:
            assert np.linalg.norm(a) < 1e-12
            continue
        assert rel_l2(a, b) < tol, (lev, rel_l2(a, b))


def test_free_space_root_matches_direct_sum():
    x, f, g, n, win, T, F = _setup(300, 16, False, 1e-6, 3, 3)
    a = F.far(f, g, n, levels=[], want_root=True)
    b = dmk.root_exact_free(T, win, f, g, n)
    assert rel_l2(a, b) < 1e-6


def test_periodic_root_matches_prolate_ewald_fourier_part():
    x, f, g, n, win, T, F = _setup(300, 16, True, 1e-6, 3, 4)
    a = F.far(f, g, n, levels=[], want_root=True)
    split = ewald.prolate_split_3d(win, 1.0, 2.0 * win.c)
    b = ewald.ewald_sum(x, f, g, n, split=split, parts=("fourier",))
    # N_per modes a side truncate the series at the eps level (about 2 eps with the stresslet)
    assert rel_l2(a, b) < 5e-6


@pytest.mark.parametrize("eps,ns", [(1e-3, 64), (1e-6, 200)])
def test_total_matches_direct_sum_on_5000_uniform_points(eps, ns):
    """Sec. 7: relative l2 error of the DMK sum against the direct sum, 5000 uniform
    points, Table 2 parameters, at most eps."""
    rng = np.random.default_rng(5)
    x = wl.uniform_points(rng, 5000, 3)
    f = wl.forces(rng, 5000, 3)
    tcp, p, n1, nper = dmk.dmk_params(eps)
    win = window.ProlateWindow(tcp * np.pi / 3)
    T = otree.Tree(x, ns)
    u = near.near_lists(T, dict(win=win, stokeslet=True, stresslet=False), f) + dmk.FarField(T, win, p, n1, nper).far(f)
    assert rel_l2(u, direct.direct_sum(x, f)) < eps


def test_periodic_total_matches_gaussian_ewald():
    eps = 1e-3
    rng = np.random.default_rng(6)
    x = wl.uniform_points(rng, 900, 3)
    f = wl.forces(rng, 900, 3, zero_mean=True)
    g = wl.stresslet_strengths(rng, 900, 3)
    n = wl.unit_normals(rng, 900, 3)
    tcp, p, n1, nper = dmk.dmk_params(eps, stokeslet=True, stresslet=True)
    win = window.ProlateWindow(tcp * np.pi / 3)
    T = otree.Tree(x, 16, periodic=True)
    u = (near.near_lists(T, dict(win=win, stokeslet=True, stresslet=True), f, g, n)
         + direct.stresslet_zero_mode(T.w, g, n)
         + dmk.FarField(T, win, p, n1, nper).far(f, g, n))
    ref = ewald.ewald_sum(x, f, g, n, split=ewald.gaussian_split_3d(0.1))
    # the stresslet at the Table 2 bandlimit reaches about 2 eps (a reading stated with the design)
    assert rel_l2(u, ref) < 3 * eps


def test_truncated_biharmonic_2d_closed_form_matches_hankel_quadrature():
    from scipy.special import j0
    R = 1.0 + np.sqrt(2.0)

    def BR(r):                                         # Eq. (Btrunc), d = 2
        return (r * r * np.log(r) - r * r / 2 - r * r * np.log(R) + R * R / 2) / (8 * np.pi)

    for k in [1e-4, 1e-3, 0.2, 1.0, 3.7, 11.0]:
        # 2D transform of a radial function: 2 pi int_0^R B(r) J0(k r) r dr
        val = 2 * np.pi * quad(lambda r: BR(r) * j0(k * r) * r, 0.0, R, limit=200, epsabs=1e-15, epsrel=1e-12)[0]
        got = float(dmk.B_trunc_hat(np.array([k]), d=2)[0])
        assert abs(got - val) <= 1e-9 * max(1.0, abs(val)), (k, got, val)


def test_2d_levels_root_and_total_match_exact_sums():
    """The same pins in 2D (App. B kernels): each level against the real-space
    difference-kernel sum, the root against K - K_R(1), and near + far against the
    2D direct sum, free space, Stokeslet + stresslet, eps 1e-3."""
    from oracle import kernels2d as k2
    eps = 1e-3
    rng = np.random.default_rng(12)
    N = 220
    x = wl.gaussian_mixture_points(rng, N, 2, 3, 0.08)
    f = wl.forces(rng, N, 2)
    g = wl.stresslet_strengths(rng, N, 2)
    n = wl.unit_normals(rng, N, 2)
    tcp, p, n1, nper = dmk.dmk_params(eps, stokeslet=True, stresslet=True)
    win = window.ProlateWindow(tcp * np.pi / 3)
    kern = k2.Kernel2D(win)
    T = otree.Tree(x, 12)
    F = dmk.FarField(T, win, p, n1, nper)
    assert F.maxlev >= 3 and len(np.unique(T.leaf_level)) >= 2
    for lev in range(F.maxlev + 1):
        a = F.far(f, g, n, levels=[lev], want_root=False)
        b = dmk.level_exact(T, kern, lev, f, g, n)
        if np.linalg.norm(b) > 0:
            assert rel_l2(a, b) < 3e-2, (lev, rel_l2(a, b))
    a = F.far(f, g, n, levels=[], want_root=True)
    assert rel_l2(a, dmk.root_exact_free(T, kern, f, g, n)) < 1e-3
    u = near.near_lists(T, dict(k2d=kern, stokeslet=True, stresslet=True), f, g, n) + F.far(f, g, n)
    assert rel_l2(u, direct.direct_sum(x, f, g, n)) < 3 * eps


def test_2d_periodic_total_matches_gaussian_ewald():
    from oracle import kernels2d as k2
    eps = 1e-3
    rng = np.random.default_rng(13)
    N = 300
    x = wl.uniform_points(rng, N, 2)
    f = wl.forces(rng, N, 2, zero_mean=True)
    g = wl.stresslet_strengths(rng, N, 2)
    n = wl.unit_normals(rng, N, 2)
    tcp, p, n1, nper = dmk.dmk_params(eps, stokeslet=True, stresslet=True)
    win = window.ProlateWindow(tcp * np.pi / 3)
    kern = k2.Kernel2D(win)
    T = otree.Tree(x, 12, periodic=True)
    u = (near.near_lists(T, dict(k2d=kern, stokeslet=True, stresslet=True), f, g, n)
         + direct.stresslet_zero_mode(T.w, g, n) + dmk.FarField(T, win, p, n1, nper).far(f, g, n))
    ref = ewald.ewald_sum(x, f, g, n, split=ewald.gaussian_split_2d(0.08))
    assert rel_l2(u, ref) < 3 * eps
