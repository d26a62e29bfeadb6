"""Pins for oracle/kernels2d.py (2D residual kernels by App. B).

Against scipy's Bessel functions (series branch), the exact cancellation of
the low-order terms, sigma-invariance of the 2D Gaussian Ewald sum, the
prolate split at two scales reproducing it (pins the 2D nu-scaling and the
log nu self term), compact support at the cutoff, a divergence-free residual
Stokeslet (ties m_d to m_o) and the tree-based 2D near component.
"""
from math import factorial

import numpy as np
import pytest
from scipy.special import j0, j1

from oracle import kernels2d as k2, ewald, near
from oracle.tree import Tree
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("kind", ["d", "o", "td", "to"])
def test_series_match_scipy_bessel(kind):
    z = np.linspace(0.6, 2.4, 13)
    J0, J1 = j0(z), j1(z)
    direct = {"d": J0 - J1 / z, "o": (2 * J1 - z * J0) / z ** 3,
              "td": (4 * J1 - 2 * z * J0 - z ** 2 * J1) / z ** 3,
              "to": ((8 / 3) * J1 - (4 / 3) * z * J0 - z ** 2 * J1 / 3) / z ** 5}[kind]
    assert np.max(np.abs(k2._series(kind, z) - direct) / np.abs(direct)) < 1e-12


def test_low_order_terms_cancel_exactly():
    a0 = lambda m: (-1) ** m / (4.0 ** m * factorial(m) ** 2)
    a1 = lambda m: (-1) ** m / (2.0 * 4.0 ** m * factorial(m) * factorial(m + 1))
    assert 2 * a1(0) - a0(0) == 0.0                                          # o: z^1
    assert 4 * a1(0) - 2 * a0(0) == 0.0                                      # td: z^1
    assert abs((8 / 3) * a1(0) - (4 / 3) * a0(0)) < 1e-16                    # to: z^1
    assert abs((8 / 3) * a1(1) - (4 / 3) * a0(1) - a1(0) / 3) < 1e-16        # to: z^3


def test_truncated_biharmonic_hat():
    k = np.array([0.5 / k2.R_TRUNC * (1 - 1e-9), 0.5 / k2.R_TRUNC * (1 + 1e-9)])
    v = k2.bhat_trunc_2d(k)
    assert abs(v[0] - v[1]) < 1e-8 * abs(v[0])
    assert abs(k2.bhat_trunc_2d(np.array([0.0]))[0] - k2.R_TRUNC ** 4 / 64) < 1e-15


def _inputs(N, seed):
    rng = np.random.default_rng(seed)
    x = wl.uniform_points(rng, N, 2)
    f = wl.forces(rng, N, 2, zero_mean=True)
    g = wl.stresslet_strengths(rng, N, 2)
    n = wl.unit_normals(rng, N, 2)
    return x, f, g, n


@pytest.mark.parametrize("which", ["stokeslet", "stresslet"])
def test_gaussian_ewald_2d_sigma_invariant(which):
    x, f, g, n = _inputs(8, 61)
    kw = dict(f=f) if which == "stokeslet" else dict(g=g, n=n)
    u1 = ewald.ewald_sum(x, split=ewald.gaussian_split_2d(0.08), **kw)
    u2 = ewald.ewald_sum(x, split=ewald.gaussian_split_2d(0.12), **kw)
    assert rel(u1, u2) < 1e-12


@pytest.mark.parametrize("which", ["stokeslet", "stresslet"])
@pytest.mark.parametrize("nu", [0.5, 0.25])
def test_prolate_split_2d_reproduces_gaussian_ewald(which, nu):
    x, f, g, n = _inputs(8, 62)
    kw = dict(f=f) if which == "stokeslet" else dict(g=g, n=n)
    u_g = ewald.ewald_sum(x, split=ewald.gaussian_split_2d(0.1), **kw)
    kern = k2.Kernel2D(ProlateWindow(40.0))
    u_p = ewald.ewald_sum(x, split=ewald.prolate_split_2d(kern, nu, kmax=2.2 * 40.0 / nu), **kw)
    assert rel(u_p, u_g) < 1e-12


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-8])
def test_residual_2d_vanishes_at_cutoff(eps):
    kern = k2.Kernel2D(ProlateWindow(bandlimit_c(eps, True, True)))
    one = np.array([1.0])
    assert abs(kern.m_d(one)[0]) < 10 * eps                 # A(1) = -log 1 - m_d(1)
    assert abs(2.0 - kern.m_o(one)[0]) < 10 * eps           # C(1) ~ 2 - m_o(1)
    assert abs(kern.m_td(one)[0]) < 200 * eps               # D(1) ~ -m_td(1)
    assert abs(4.0 / 3.0 - kern.m_to(one)[0]) < 200 * eps   # E(1) ~ 6 m_to(1) - 8


def test_residual_stokeslet_2d_divergence_free():
    kern = k2.Kernel2D(ProlateWindow(bandlimit_c(1e-6)))
    nu, h = 0.25, 1e-6
    rng = np.random.default_rng(63)
    for _ in range(5):
        x = rng.standard_normal(2)
        x *= rng.uniform(0.1, 0.9) * nu / np.linalg.norm(x)
        div = np.zeros(2)
        for j in range(2):
            e = np.zeros(2); e[j] = h
            dS = (k2.stokeslet_res(kern, (x + e)[None], nu)[0] - k2.stokeslet_res(kern, (x - e)[None], nu)[0]) / (2 * h)
            div += dS[j, :]
        assert np.max(np.abs(div)) < 1e-6 / np.linalg.norm(x)


@pytest.mark.parametrize("per", [False, True])
def test_lists_equal_brute_force_2d(per):
    rng = np.random.default_rng(64 + per)
    N = 250
    x = wl.gaussian_mixture_points(rng, N, 2, 3, 0.03)
    f = wl.forces(rng, N, 2)
    g = wl.stresslet_strengths(rng, N, 2)
    n = wl.unit_normals(rng, N, 2)
    tr = Tree(x, 10, periodic=per)
    kern = dict(k2d=k2.Kernel2D(ProlateWindow(bandlimit_c(1e-6))), stokeslet=True, stresslet=True)
    a = near.near_lists(tr, kern, f=f, g=g, n=n)
    b = near.near_brute(tr, kern, f=f, g=g, n=n)
    assert rel(a, b) < 1e-13


def test_uniform_periodic_2d_near_plus_fourier_is_gaussian_ewald():
    # all leaves at level 1 -> nu = 1/4; near component + Fourier part + zero
    # mode equals the split-independent 2D periodic total
    x, f, g, n = _inputs(16, 65)
    tr = Tree(x, 15, periodic=True)
    assert np.all(tr.leaf_level == 1)
    kern2 = k2.Kernel2D(ProlateWindow(40.0))
    u_near = near.near_lists(tr, dict(k2d=kern2, stokeslet=True, stresslet=True), f=f, g=g, n=n)
    split = ewald.prolate_split_2d(kern2, 0.25, kmax=2.2 * 40.0 / 0.25)
    u_far = ewald.ewald_sum(x, f=f, g=g, n=n, split=split, parts=("fourier", "zero"))
    u_ref = ewald.ewald_sum(x, f=f, g=g, n=n, split=ewald.gaussian_split_2d(0.1))
    assert rel(u_near + u_far, u_ref) < 1e-12
