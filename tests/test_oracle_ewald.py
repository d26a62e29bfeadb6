"""Pins tying the prolate split to the classical Gaussian (Hasimoto) Ewald sum.

A periodic total is independent of how it is split.  The Gaussian Ewald sum is
checked for sigma-invariance; the prolate split (Sec. 5.2 real-space kernels,
the Fourier mollifier of Eq. (gammaB_in_phi) and the self term of Eq. (S_self))
must then reproduce it.  A wrong sign, factor or term in any of the three parts
would change the total.
"""
import numpy as np
import pytest

from oracle import ewald
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c


def _inputs(N, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((N, 3)) - 0.5
    f = rng.standard_normal((N, 3))
    f -= f.mean(axis=0)
    g = rng.standard_normal((N, 3))
    n = rng.standard_normal((N, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    return x, f, g, n


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("which", ["stokeslet", "stresslet"])
def test_gaussian_ewald_sigma_invariant(which):
    x, f, g, n = _inputs(7, 11)
    kw = dict(f=f) if which == "stokeslet" else dict(g=g, n=n)
    u1 = ewald.ewald_sum(x, split=ewald.gaussian_split_3d(0.09), **kw)
    u2 = ewald.ewald_sum(x, split=ewald.gaussian_split_3d(0.15), **kw)
    assert rel(u1, u2) < 1e-13


@pytest.mark.parametrize("which", ["stokeslet", "stresslet"])
@pytest.mark.parametrize("nu", [0.5, 0.25])
def test_prolate_split_reproduces_gaussian_ewald(which, nu):
    x, f, g, n = _inputs(6, 12)
    kw = dict(f=f) if which == "stokeslet" else dict(g=g, n=n)
    c = 40.0
    win = ProlateWindow(c)
    u_g = ewald.ewald_sum(x, split=ewald.gaussian_split_3d(0.12), **kw)
    u_p = ewald.ewald_sum(x, split=ewald.prolate_split_3d(win, nu, kmax=2.2 * c / nu), **kw)
    # rounding over ~4e4 Fourier modes; any wrong term would show at >= 1e-6
    assert rel(u_p, u_g) < 5e-12


def test_prolate_split_at_table2_c_is_eps_accurate():
    x, f, g, n = _inputs(6, 13)
    u_g = ewald.ewald_sum(x, f=f, split=ewald.gaussian_split_3d(0.12))
    for eps in (1e-3, 1e-6):
        win = ProlateWindow(bandlimit_c(eps))
        u_p = ewald.ewald_sum(x, f=f, split=ewald.prolate_split_3d(win, 0.5, kmax=3.0 * win.c / 0.5))
        assert rel(u_p, u_g) < eps
