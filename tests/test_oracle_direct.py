"""Pins for oracle/direct.py (Eq. (stokes_stress_sum) point sums, the 2D full
kernels) and for the periodic stresslet k = 0 term of Sec. 5.3.

None of these checks retypes a kernel: they compare layer potentials over a
sphere (3D) or a circle (2D), sampled by spectrally accurate quadrature, with
values fixed by calculus alone.

* Single layer of a uniform density f on a sphere of radius a: the velocity
  inside is the constant (2a/3) f (the translating-sphere result); on a circle
  of radius a its value at the centre is (a/2)(1/2 - log a) f.  This fixes the
  normalisation and both terms (delta and x x) of the Stokeslet.
* Single layer of the normal density n: zero everywhere (S is divergence free,
  so the flux identity closes), which needs the 1 : 1 ratio of the two terms.
* Double layer (stresslet) of a constant density c (rho = c (x) n, outward n):
  c inside the closed surface, 0 outside (Gauss's theorem: the stresslet is
  divergence free in the source point away from the target, and a small ball
  around the target contributes c in 2D and 3D).
* Periodic stresslet: every periodic image of a closed surface with constant
  density contributes 0 at a target outside it, so the periodic sum equals the
  free-space value (c inside, 0 outside).  The Fourier series with k != 0 has
  zero cell mean, so the k = 0 term must restore the mean c |Omega|; the
  formula u0 = -sum_s (x_t - x_s)(g_s . n_s) gives exactly that (a sign error
  gives -c |Omega|).  With a net source sum_s g_s . n_s != 0, translating every
  point leaves the Fourier and real-space parts unchanged, so the total must
  not change either: that fixes the target term of u0 against the source term.
"""
import numpy as np
import pytest

from oracle import direct, ewald


def _sphere(centre, a, n_th=24, n_ph=48):
    """Gauss-Legendre in cos(theta) x trapezoidal in phi: nodes, outward normals, weights."""
    z, wz = np.polynomial.legendre.leggauss(n_th)
    ph = 2.0 * np.pi * np.arange(n_ph) / n_ph
    Z, P = np.meshgrid(z, ph, indexing="ij")
    S = np.sqrt(1.0 - Z * Z)
    nrm = np.stack([S * np.cos(P), S * np.sin(P), Z], axis=-1).reshape(-1, 3)
    w = (wz[:, None] * np.full(n_ph, 2.0 * np.pi / n_ph)[None, :]).reshape(-1) * a * a
    return np.asarray(centre) + a * nrm, nrm, w


def _circle(centre, a, n=96):
    th = 2.0 * np.pi * np.arange(n) / n
    nrm = np.stack([np.cos(th), np.sin(th)], axis=1)
    return np.asarray(centre) + a * nrm, nrm, np.full(n, 2.0 * np.pi * a / n)


def _with_targets(xs, tg):
    """Sources followed by zero-density target points (a zero density adds nothing)."""
    return np.concatenate([xs, tg]), np.arange(len(xs), len(xs) + len(tg))


C3 = np.array([0.1, -0.05, 0.02])
C2 = np.array([0.1, -0.05])


def test_direct_3d_single_layer_uniform_density():
    a = 0.2
    xs, nrm, w = _sphere(C3, a)
    tg = C3 + np.array([[0.0, 0.0, 0.0], [0.06, -0.03, 0.05], [-0.1, 0.02, 0.0]])
    x, ti = _with_targets(xs, tg)
    f0 = np.array([0.3, -1.1, 0.7])
    f = np.zeros_like(x)
    f[: len(xs)] = f0[None, :] * w[:, None]
    u = direct.direct_sum(x, f=f, targets=ti)
    assert np.max(np.abs(u - (2.0 * a / 3.0) * f0[None, :])) < 1e-12


def test_direct_3d_single_layer_normal_density_vanishes():
    a = 0.2
    xs, nrm, w = _sphere(C3, a)
    tg = C3 + np.array([[0.05, 0.0, 0.0], [0.45, 0.1, 0.0], [0.0, -0.3, 0.2]])
    x, ti = _with_targets(xs, tg)
    f = np.zeros_like(x)
    f[: len(xs)] = nrm * w[:, None]
    u = direct.direct_sum(x, f=f, targets=ti)
    assert np.max(np.abs(u)) < 1e-12


def test_direct_3d_double_layer_jump():
    a = 0.2
    xs, nrm, w = _sphere(C3, a)
    tg = C3 + np.array([[0.0, 0.0, 0.0], [0.05, 0.04, -0.03], [0.45, 0.0, 0.0], [0.0, 0.3, -0.25]])
    x, ti = _with_targets(xs, tg)
    c = np.array([0.4, -0.9, 1.3])
    g = np.zeros_like(x)
    g[: len(xs)] = c[None, :] * w[:, None]
    n = np.zeros_like(x)
    n[: len(xs)] = nrm
    n[len(xs):] = [1.0, 0.0, 0.0]
    u = direct.direct_sum(x, g=g, n=n, targets=ti)
    assert np.max(np.abs(u[:2] - c[None, :])) < 1e-10
    assert np.max(np.abs(u[2:])) < 1e-10


@pytest.mark.parametrize("a", [0.2, 0.35])
def test_direct_2d_single_layer_centre(a):
    xs, nrm, w = _circle(C2, a)
    x, ti = _with_targets(xs, C2[None, :])
    f0 = np.array([0.8, -0.35])
    f = np.zeros_like(x)
    f[: len(xs)] = f0[None, :] * w[:, None]
    u = direct.direct_sum(x, f=f, targets=ti)
    assert np.max(np.abs(u[0] - 0.5 * a * (0.5 - np.log(a)) * f0)) < 1e-13


def test_direct_2d_single_layer_normal_density_vanishes():
    a = 0.2
    xs, nrm, w = _circle(C2, a)
    tg = C2 + np.array([[0.05, 0.02], [0.4, 0.1], [-0.1, -0.3]])
    x, ti = _with_targets(xs, tg)
    f = np.zeros_like(x)
    f[: len(xs)] = nrm * w[:, None]
    u = direct.direct_sum(x, f=f, targets=ti)
    assert np.max(np.abs(u)) < 1e-12


def test_direct_2d_double_layer_jump():
    a = 0.2
    xs, nrm, w = _circle(C2, a)
    tg = C2 + np.array([[0.0, 0.0], [0.06, -0.05], [0.4, 0.0], [-0.2, 0.25]])
    x, ti = _with_targets(xs, tg)
    c = np.array([-0.6, 1.2])
    g = np.zeros_like(x)
    g[: len(xs)] = c[None, :] * w[:, None]
    n = np.zeros_like(x)
    n[: len(xs)] = nrm
    n[len(xs):] = [1.0, 0.0]
    u = direct.direct_sum(x, g=g, n=n, targets=ti)
    assert np.max(np.abs(u[:2] - c[None, :])) < 1e-10
    assert np.max(np.abs(u[2:])) < 1e-10


def test_direct_sum_excludes_the_target_and_adds_pairs():
    # two points: each sees only the other, through the full kernels
    x = np.array([[0.1, 0.0, 0.0], [-0.2, 0.1, 0.05]])
    f = np.array([[1.0, 0.5, -0.2], [0.3, -0.7, 0.9]])
    u = direct.direct_sum(x, f=f)
    d = x[0] - x[1]
    r = np.linalg.norm(d)
    S = (np.eye(3) / r + np.outer(d, d) / r ** 3) / (8 * np.pi)
    assert np.allclose(u[0], S @ f[1], rtol=1e-14, atol=0)
    assert np.allclose(u[1], S @ f[0], rtol=1e-14, atol=0)


def test_periodic_stresslet_zero_mode_closed_surface_3d():
    """Ewald (Gaussian split) + u0 of a sphere with constant density = c inside, 0 outside."""
    a = 0.2
    xs, nrm, w = _sphere(C3, a, n_th=28, n_ph=56)
    tg = C3 + np.array([[0.0, 0.0, 0.0], [0.05, -0.04, 0.03], [0.0, 0.0, 0.34], [-0.33, 0.1, 0.0]])
    x, ti = _with_targets(xs, tg)
    c = np.array([0.7, -0.4, 1.1])
    g = np.zeros_like(x)
    g[: len(xs)] = c[None, :] * w[:, None]
    n = np.zeros_like(x)
    n[: len(xs)] = nrm
    n[len(xs):] = [0.0, 1.0, 0.0]
    split = ewald.gaussian_split_3d(0.2)
    u = ewald.ewald_sum(x, g=g, n=n, split=split, targets=ti)
    assert np.max(np.abs(u[:2] - c[None, :])) < 1e-9
    assert np.max(np.abs(u[2:])) < 1e-9
    # the k = 0 term supplies the cell mean c |Omega|: without it the sum is off by that
    u_nz = ewald.ewald_sum(x, g=g, n=n, split=split, targets=ti, parts=("real", "fourier"))
    vol = 4.0 / 3.0 * np.pi * a ** 3
    assert np.max(np.abs(u - u_nz - vol * c[None, :])) < 1e-9


def test_periodic_stresslet_zero_mode_closed_curve_2d():
    a = 0.2
    xs, nrm, w = _circle(C2, a, n=80)
    tg = C2 + np.array([[0.0, 0.0], [0.05, 0.08], [0.3, 0.0], [-0.1, -0.32]])
    x, ti = _with_targets(xs, tg)
    c = np.array([0.5, -1.3])
    g = np.zeros_like(x)
    g[: len(xs)] = c[None, :] * w[:, None]
    n = np.zeros_like(x)
    n[: len(xs)] = nrm
    n[len(xs):] = [1.0, 0.0]
    u = ewald.ewald_sum(x, g=g, n=n, split=ewald.gaussian_split_2d(0.15), targets=ti)
    assert np.max(np.abs(u[:2] - c[None, :])) < 1e-9
    assert np.max(np.abs(u[2:])) < 1e-9


@pytest.mark.parametrize("d", [2, 3])
def test_periodic_stresslet_translation_invariant_with_net_source(d):
    rng = np.random.default_rng(5)
    x = 0.6 * rng.random((6, d)) - 0.3
    g = rng.standard_normal((6, d))
    n = rng.standard_normal((6, d))
    n /= np.linalg.norm(n, axis=1)[:, None]
    G = np.sum(g * n)
    assert abs(G) > 0.1                                # a net source: the target term of u0 matters
    shift = np.array([0.12, -0.15, 0.07])[:d]
    split = ewald.gaussian_split_3d(0.15) if d == 3 else ewald.gaussian_split_2d(0.15)
    u1 = ewald.ewald_sum(x, g=g, n=n, split=split)
    u2 = ewald.ewald_sum(x + shift, g=g, n=n, split=split)
    assert np.max(np.abs(u1 - u2)) < 1e-11 * np.max(np.abs(u1))
    # the source term alone (target term dropped) would move by shift * G
    w1 = x + 0.5
    src_only = lambda w: np.sum(w * np.sum(g * n, axis=1)[:, None], axis=0)
    assert np.linalg.norm(src_only(w1 + shift) - src_only(w1)) > 0.01
