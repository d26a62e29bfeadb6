"""Pins for oracle/window.py (PSWF, phi, Phi, phi-hat, gamma-hat).

Each check compares the oracle with something other than itself: scipy's
independent prolate routines, the defining integral equation, closed forms,
and finite differences.
"""
import numpy as np
import pytest
import scipy.special as sp

from oracle.window import ProlateWindow, GaussianWindow
from oracle.params import bandlimit_c, three_c_over_pi

C_TABLE = [bandlimit_c(e) for e in (1e-3, 1e-6, 1e-9, 1e-12)]


@pytest.mark.parametrize("c", [1.0, 5.0, 10.0] + C_TABLE)
def test_chi_matches_scipy_pro_cv(c):
    # Sec. 2.4: psi_0^c is the prolate of order 0; scipy computes its
    # characteristic value by an independent method.
    w = ProlateWindow(c)
    assert abs(w.chi - sp.pro_cv(0, 0, c)) <= 1e-12 * max(1.0, w.chi)


@pytest.mark.parametrize("c", [2.0, 5.0, 10.0])
def test_psi_proportional_to_scipy_pro_ang1(c):
    w = ProlateWindow(c)
    x = np.linspace(-0.95, 0.95, 41)
    s, _ = sp.pro_ang1(0, 0, c, x)
    ratio = w.psi(x) / s
    assert np.std(ratio) <= 1e-11 * abs(np.mean(ratio))


@pytest.mark.parametrize("c", C_TABLE + [40.0])
def test_integral_eigen_equation(c):
    # Sec. 2.4: lambda psi(x) = int_{-1}^1 psi(t) e^{ictx} dt (psi even -> cosine).
    w = ProlateWindow(c)
    t, wt = np.polynomial.legendre.leggauss(300)
    x = np.linspace(-1.0, 1.0, 50)
    rhs = (np.cos(c * np.outer(x, t)) * (wt * w.psi(t))).sum(axis=1)
    lhs = w.lam * w.psi(x)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(w.psi(x))) * max(1.0, abs(w.lam))
    # psi is even and normalised in L2[-1,1]
    assert np.allclose(w.psi(x), w.psi(-x), rtol=0, atol=1e-14)
    assert abs(np.dot(wt, w.psi(t) ** 2) - 1.0) < 1e-13


@pytest.mark.parametrize("c", C_TABLE)
def test_phihat_closed_form_equals_transform(c):
    # Eq. (wfunchat_prol_G): phi-hat(k) = psi(k/c)/psi(0) for |k| <= c
    w = ProlateWindow(c)
    k = np.linspace(0.0, c, 33)
    assert np.max(np.abs(w.phihat(k) - w.phihat_closed(k))) < 1e-13


@pytest.mark.parametrize("c", C_TABLE)
def test_Phi_properties(c):
    # Eq. (def_erfc_like_fcn): Phi(0) = int phi = 1, Phi(1) = 0, Phi' = -2 phi
    w = ProlateWindow(c)
    assert abs(w.Phi(0.0) - 1.0) < 1e-14
    assert abs(w.Phi(1.0)) < 1e-15 and abs(w.Phi(1.0 - 1e-13)) < 1e-12
    r = np.linspace(0.05, 0.95, 19)
    h = 1e-4
    fd = (-w.Phi(r + 2 * h) + 8 * w.Phi(r + h) - 8 * w.Phi(r - h) + w.Phi(r - 2 * h)) / (12 * h)
    assert np.max(np.abs(fd + 2.0 * w.phi(r))) < 1e-9 * c
    fd = (-w.phi(r + 2 * h) + 8 * w.phi(r + h) - 8 * w.phi(r - h) + w.phi(r - 2 * h)) / (12 * h)
    assert np.max(np.abs(fd - w.dphi(r))) < 1e-8 * c * c


@pytest.mark.parametrize("c", C_TABLE[:2])
def test_Legendre_antiderivatives_match_quadrature(c):
    w = ProlateWindow(c)
    r = np.array([0.0, 0.1, 0.37, 0.5, 0.81, 0.999])
    assert np.max(np.abs(w.Phi(r) - w.Phi_quad(r))) < 1e-14
    assert np.max(np.abs(w.I1(r) - w.I1_quad(r))) < 1e-14
    assert np.max(np.abs(w.I0(r) - w.I0_quad(r))) < 1e-14


def test_gaussian_generic_path_reproduces_erfc():
    # Special case: with the Gaussian window Phi is erfc(r/sigma).
    g = GaussianWindow(0.2)
    r = np.array([0.0, 0.05, 0.2, 0.4, 0.9])
    assert np.max(np.abs(g.Phi_quad(r, upper=g._tail) - sp.erfc(r / 0.2))) < 1e-14
    # and Eq. (gammaB_in_phi) gives the Hasimoto mollifier
    k = np.linspace(0.0, 60.0, 31)
    # k phi-hat'/2 amplifies rounding by k (up to 60 here)
    assert np.max(np.abs(g.gammahat(k) - g.gammahat_closed(k))) < 1e-12


@pytest.mark.parametrize("c", C_TABLE)
def test_gammahat_is_biharmonic_mollifier(c):
    # Def. 3.1: gamma-hat(0) = 1, gamma-hat''(0) = 0.
    w = ProlateWindow(c)
    assert abs(w.gammahat(0.0)[0] - 1.0) < 1e-13
    h = 2e-3
    d2 = (w.gammahat(h)[0] - 2 * w.gammahat(0.0)[0] + w.gammahat(-h)[0]) / h ** 2
    d2_phi = (w.phihat(h)[0] - 2 * w.phihat(0.0)[0] + w.phihat(-h)[0]) / h ** 2
    assert abs(d2) < 1e-6 and abs(d2_phi) > 1e-3   # phi-hat alone is not a mollifier


def test_gamma_1d_inverse_transform():
    # Eq. (biharmonic_screen_R): (1/pi) int_0^inf cos(kx) gamma-hat(k) dk = 3/2 phi + x phi'/2
    c = 40.0
    w = ProlateWindow(c)
    K = 2.2 * c
    t, wt = np.polynomial.legendre.leggauss(500)
    k = 0.5 * K * (t + 1.0)
    wk = 0.5 * K * wt
    gk = w.gammahat(k, n=500)
    x = np.linspace(0.0, 0.9, 10)
    inv = (np.cos(np.outer(x, k)) * (wk * gk)).sum(axis=1) / np.pi
    assert np.max(np.abs(inv - w.gamma1d(x))) < 1e-10


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9, 1e-12])
def test_stokeslet_residual_below_eps_at_cutoff(eps):
    # Table 2 choice of c: the residual Stokeslet functions are below eps at rho = 1.
    from oracle import kernels3d as k3
    w = ProlateWindow(bandlimit_c(eps))
    assert abs(k3.Sdiag(w, 1.0 - 1e-14, cut=False)) <= eps
    assert abs(k3.Soffd(w, 1.0 - 1e-14, cut=False)) <= eps


def test_table2_interpolation_reading():
    assert three_c_over_pi(1e-6) == 17 and three_c_over_pi(1e-12, "stresslet") == 32
    assert three_c_over_pi(1e-8) == 23 and three_c_over_pi(1e-10) == 27
    assert three_c_over_pi(1e-8, "stresslet") == 23 and three_c_over_pi(1e-10, "stresslet") == 28
