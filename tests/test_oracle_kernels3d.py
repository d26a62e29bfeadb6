"""Pins for oracle/kernels3d.py: Thm 4.1, Cor. 4.1, Sec. 5.2, App. A, gradient.

Checks against Hasimoto's closed form, finite differences of B_R through the
differential operators D_S, D_T of App. A (Eqs. (dsf), (dtf)), textbook
Stokeslet values, divergence-free fields and the r -> 0 limits of App. A.1.
"""
import numpy as np
import pytest

from oracle import kernels3d as k3
from oracle.window import ProlateWindow, GaussianWindow
from oracle.params import bandlimit_c

WINS = [ProlateWindow(bandlimit_c(1e-6)), ProlateWindow(bandlimit_c(1e-10)), ProlateWindow(40.0)]


def test_textbook_stokeslet_and_stresslet():
    r = 0.3
    S = k3.stokeslet(np.array([r, 0.0, 0.0]))
    assert np.allclose(S, np.diag([2.0, 1.0, 1.0]) / (8 * np.pi * r), rtol=1e-15, atol=0)
    T = k3.stresslet(np.array([0.0, r, 0.0]))
    ref = np.zeros((3, 3, 3))
    ref[1, 1, 1] = -3.0 / (4 * np.pi * r * r)
    assert np.allclose(T, ref, rtol=1e-15, atol=0)


def test_gaussian_window_reproduces_hasimoto():
    # Thm 4.1 with phi_G must give the Hasimoto residual of Eq. (hasimoto-split)
    for sigma in (0.1, 0.3):
        g = GaussianWindow(sigma)
        r = np.linspace(0.01, 1.5, 40)
        assert np.max(np.abs(k3.B_res(g, r) - k3.B_res_hasimoto(sigma, r))) < 1e-16


@pytest.mark.parametrize("w", WINS)
def test_BR_compact_support_and_BM_equals_B(w):
    # Cor. 3.1 / Thm 3.1: B_R = 0 (B_M = B) for r > 1
    r = np.array([1.0, 1.01, 1.5, 3.0])
    assert np.max(np.abs(k3.B_res(w, r))) < 1e-16
    # and B_R is continuous at 1 from inside, of size ~ phi(1)
    assert abs(k3.B_res(w, 1.0 - 1e-9)) < 1e-8


def _d(fn, r, h, order):
    """Central finite differences (4th-order stencils)."""
    if order == 1:
        return (-fn(r + 2 * h) + 8 * fn(r + h) - 8 * fn(r - h) + fn(r - 2 * h)) / (12 * h)
    if order == 2:
        return (-fn(r + 2 * h) + 16 * fn(r + h) - 30 * fn(r) + 16 * fn(r - h) - fn(r - 2 * h)) / (12 * h * h)
    if order == 3:
        return (-fn(r + 3 * h) + 8 * fn(r + 2 * h) - 13 * fn(r + h) + 13 * fn(r - h)
                - 8 * fn(r - 2 * h) + fn(r - 3 * h)) / (8 * h ** 3)
    raise ValueError


@pytest.mark.parametrize("w", WINS[:2])
def test_residual_functions_are_DS_DT_of_BR(w):
    # App. A: Sdiag = -8pi (B_R' + r B_R''), Soffd = 8pi(-B_R' + r B_R''),
    #         Tdiag = -8pi r^2 B_R''', Toffd = 8pi(-B_R' + r B_R'' - r^2 B_R'''/3)  (d = 3)
    BR = lambda r: k3.B_res(w, r)
    r = np.linspace(0.1, 0.9, 17)
    b1, b2, b3 = _d(BR, r, 2e-3, 1), _d(BR, r, 2e-3, 2), _d(BR, r, 5e-3, 3)
    e = 8 * np.pi
    assert np.max(np.abs(-e * (b1 + r * b2) - k3.Sdiag(w, r))) < 1e-6
    assert np.max(np.abs(e * (-b1 + r * b2) - k3.Soffd(w, r))) < 1e-6
    assert np.max(np.abs(-e * r * r * b3 - k3.Tdiag(w, r))) < 5e-5
    assert np.max(np.abs(e * (-b1 + r * b2 - r * r * b3 / 3) - k3.Toffd(w, r))) < 5e-5


@pytest.mark.parametrize("w", WINS[:2])
def test_BR_derivatives_cor41(w):
    # Cor. 4.1: B_R' = -Phi/(8 pi), B_R'' = phi/(4 pi)
    r = np.linspace(0.05, 0.95, 19)
    BR = lambda r: k3.B_res(w, r)
    assert np.max(np.abs(_d(BR, r, 1e-3, 1) + w.Phi(r) / (8 * np.pi))) < 1e-10
    assert np.max(np.abs(_d(BR, r, 2e-3, 2) - w.phi(r) / (4 * np.pi))) < 1e-7


@pytest.mark.parametrize("w", WINS)
@pytest.mark.parametrize("nu", [0.5, 0.0625])
def test_residual_stokeslet_divergence_free(w, nu):
    rng = np.random.default_rng(3)
    h = 1e-5 * nu
    for _ in range(5):
        x = rng.standard_normal(3)
        x *= rng.uniform(0.1, 0.9) * nu / np.linalg.norm(x)
        div = np.zeros(3)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            dS = (k3.stokeslet_res(w, x + e, nu) - k3.stokeslet_res(w, x - e, nu)) / (2 * h)
            div += dS[j, :]
        scale = np.max(np.abs(k3.stokeslet(x))) / np.linalg.norm(x)
        assert np.max(np.abs(div)) < 1e-6 * scale


@pytest.mark.parametrize("w", WINS)
def test_self_limits(w):
    # App. A.1: S - S_R -> phi(0)/(2 pi nu) delta and T - T_R -> 0 as r -> 0
    nu = 0.25
    for r in (1e-4, 1e-5):
        x = r * np.array([0.6, -0.48, 0.64])
        SM = k3.stokeslet(x) - k3.stokeslet_res(w, x, nu)
        ref = -k3.stokeslet_self_coeff(w, nu) * np.eye(3)
        # S_M is smooth: the limit is approached as O((c r / nu)^2)
        assert np.max(np.abs(SM - ref)) < (w.c * r / nu) ** 2 * np.max(np.abs(ref))
        TM = k3.stresslet(x) - k3.stresslet_res(w, x, nu)
        # T_M(x) = O(phi''(0) r / nu^3) with |phi''(0)| ~ c phi(0): vanishes linearly
        assert np.max(np.abs(TM)) < w.c * float(w.phi(0.0)) * r / nu ** 3


@pytest.mark.parametrize("w", WINS)
def test_residual_kernels_vanish_beyond_nu_and_are_symmetric(w):
    nu = 0.125
    x = np.array([0.05, -0.09, 0.07])
    x = x / np.linalg.norm(x) * 1.01 * nu
    assert np.all(k3.stokeslet_res(w, x, nu) == 0.0)
    assert np.all(k3.stresslet_res(w, x, nu) == 0.0)
    y = x * 0.5
    S = k3.stokeslet_res(w, y, nu)
    T = k3.stresslet_res(w, y, nu)
    assert np.allclose(S, S.T, rtol=0, atol=1e-14 * np.abs(S).max())
    for perm in [(1, 0, 2), (0, 2, 1), (2, 1, 0)]:
        assert np.allclose(T, np.transpose(T, perm), rtol=0, atol=1e-14 * np.abs(T).max())
    # nu-scaling of Sec. 5.2 remark: S_R,nu(x) = S_R,1(x/nu)/nu, T_R,nu(x) = T_R,1(x/nu)/nu^2
    assert np.allclose(S, k3.stokeslet_res(w, y / nu, 1.0) / nu, rtol=1e-13, atol=0)
    assert np.allclose(T, k3.stresslet_res(w, y / nu, 1.0) / nu ** 2, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("w", WINS[:2])
def test_gradient_matches_finite_differences(w):
    nu = 0.25
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(6):
        x = rng.standard_normal(3)
        x *= rng.uniform(0.05, 0.95) * nu / np.linalg.norm(x)
        G = k3.stokeslet_res_grad(w, x, nu)
        fd = np.zeros((3, 3, 3))
        for m in range(3):
            e = np.zeros(3)
            e[m] = h
            fd[:, :, m] = (k3.stokeslet_res(w, x + e, nu) - k3.stokeslet_res(w, x - e, nu)) / (2 * h)
        assert np.max(np.abs(G - fd)) < 1e-6 * np.max(np.abs(G))


@pytest.mark.parametrize("w", WINS[:2] + [GaussianWindow(0.2)])
def test_stresslet_gradient_matches_finite_differences(w):
    """d_k T_R,jlm against central differences of T_R (pins the second
    derivative of the window, phi'', and every term of the product rule)."""
    nu = 0.25
    rng = np.random.default_rng(6)
    h = 1e-6
    for _ in range(6):
        x = rng.standard_normal(3)
        x *= rng.uniform(0.05, 0.95) * nu / np.linalg.norm(x)
        G = k3.stresslet_res_grad(w, x, nu)
        fd = np.zeros((3, 3, 3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            fd[..., k] = (k3.stresslet_res(w, x + e, nu, cut=False) - k3.stresslet_res(w, x - e, nu, cut=False)) / (2 * h)
        assert np.max(np.abs(G - fd)) < 1e-6 * np.max(np.abs(G))


@pytest.mark.parametrize("w", WINS[:2])
def test_window_second_derivative_matches_finite_differences(w):
    r = np.linspace(0.02, 0.98, 25)
    h = 1e-5
    fd = (w.dphi(r + h) - w.dphi(r - h)) / (2 * h)
    assert np.max(np.abs(w.d2phi(r) - fd)) < 1e-7 * np.max(np.abs(fd))
