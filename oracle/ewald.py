"""Single-level periodic Ewald sums with a Gaussian or prolate split (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5.3, Eqs. (ewald_local), (ewald_far): on the unit cell,
    u(x_t) = sum_s sum*_p K_R(x_t - x_s + p) rho_s
           + sum_{k in 2 pi Z^d, k != 0} K-hat_M(k) sum_s e^{i k.(x_t - x_s)} rho_s
           + u_self + u0,
with the mollified kernels of Eqs. (moll_stokeslet), (moll_stresslet),
    S-hat_M = (k^2 delta - k k) B-hat_M,
    T-hat_M = i [ (k_m delta_jl + k_j delta_lm + k_l delta_mj) k^2 - 2 k_j k_l k_m ] B-hat_M,
    B-hat_M(k) = gamma-hat(k nu) / k^4          (Eq. (generalbiharkdefs), scale nu).
Gaussian split (Hasimoto, Eq. (hasimoto-split)): gamma-hat = exp(-k^2 s^2/4)(1 + k^2 s^2/4),
real-space functions from Sec. 5.2 with Phi = erfc(r/s); self -1/(2 pi^{3/2} s).
u0: Stokeslet 0, stresslet -sum_s (x_t - x_s)(g_s . n_s).

These totals are independent of the split (sigma, nu, window); that is what
the pins check.  3D and 2D; the 2D real-space part uses kernels2d.
"""
import itertools
import numpy as np

from . import kernels3d as k3
from .direct import stresslet_zero_mode


def _kvectors(d, kmax):
    m = int(np.ceil(kmax / (2.0 * np.pi)))
    rng = np.arange(-m, m + 1)
    grid = np.array(list(itertools.product(rng, repeat=d)), dtype=np.float64) * 2.0 * np.pi
    kk = np.sqrt(np.sum(grid * grid, axis=1))
    keep = (kk > 0) & (kk <= kmax)
    return grid[keep], kk[keep]


def ewald_sum(x, f=None, g=None, n=None, split=None, lo=None,
              parts=("real", "fourier", "self", "zero"), targets=None):
    """Periodic sum on the unit cell, at every point (or at the points whose
    indices are in ``targets``).

    split: dict with
      'real'  : callable(d[P, dim], which) -> kernel tensors for the residual
                part ('S' -> [P,d,d], 'T' -> [P,d,d,d]); zero beyond 'rcut'
      'rcut'  : real-space cutoff radius
      'ghat'  : callable(k) -> gamma-hat at the scale of the split
      'kmax'  : Fourier cutoff
      'self'  : Stokeslet self coefficient (u_self = self * f_t)
    parts: which of the four terms to include.
    """
    x = np.asarray(x, dtype=np.float64)
    N, d = x.shape
    lo = np.full(d, -0.5) if lo is None else np.asarray(lo)[:d]
    w = x - lo
    w = w - np.floor(w)
    tset = np.arange(N) if targets is None else np.asarray(targets)
    u = np.zeros((N, d))
    # ---- real space: all images within rcut ------------------------------
    R = int(np.ceil(split["rcut"])) + 1
    images = np.array(list(itertools.product(range(-R, R + 1), repeat=d)), dtype=np.float64)
    for t in (tset if "real" in parts else ()):
        dd = (w[t][None, None, :] - w[None, :, :]) + images[:, None, :]   # [img, s, d]
        dd = dd.reshape(-1, d)
        src = np.tile(np.arange(N), len(images))
        r = np.sqrt(np.sum(dd * dd, axis=1))
        m = (r > 0.0) & (r < split["rcut"])
        dd, src = dd[m], src[m]
        if f is not None:
            u[t] += np.einsum("pjl,pl->j", split["real"](dd, "S"), f[src])
        if g is not None:
            u[t] += np.einsum("pjlm,pl,pm->j", split["real"](dd, "T"), g[src], n[src])
    # ---- Fourier space ---------------------------------------------------
    kv, kk = _kvectors(d, split["kmax"]) if "fourier" in parts else (np.zeros((0, d)), np.zeros(0))
    Bh = split["ghat"](kk) / kk ** 4
    ph = np.exp(-1j * (w @ kv.T))                       # [s, k] e^{-i k.w_s}
    pt = np.exp(1j * (w[tset] @ kv.T))                  # [t, k] e^{+i k.w_t}
    if f is not None:
        rhat = ph.T @ f                                 # [k, d] sum_s f_s e^{-ik.w_s}
        kdot = np.sum(kv * rhat, axis=1)
        Shat_rho = (kk[:, None] ** 2 * rhat - kv * kdot[:, None]) * Bh[:, None]
        u[tset] += np.real(pt @ Shat_rho)
    if g is not None:
        Gh = np.einsum("sk,sl,sm->klm", ph, g, n)       # [k, l, m]
        Gk = np.einsum("klm,km->kl", Gh, kv)            # G_jm k_m   (j = l index)
        GTk = np.einsum("klm,kl->km", Gh, kv)           # G_lj k_l   (j = m index)
        tr = np.einsum("kll->k", Gh)
        kGk = np.einsum("kl,klm,km->k", kv, Gh, kv)
        That_rho = 1j * Bh[:, None] * (kk[:, None] ** 2 * (Gk + kv * tr[:, None] + GTk)
                                        - 2.0 * kv * kGk[:, None])
        u[tset] += np.real(pt @ That_rho)
        if "zero" in parts:
            u[tset] += stresslet_zero_mode(w, g, n, targets=tset)
    if f is not None and "self" in parts:
        u[tset] += split["self"] * f[tset]
    return u if targets is None else u[tset]


def gaussian_split_3d(sigma, tol=1e-16):
    """Hasimoto split with Gaussian width sigma."""
    from .window import GaussianWindow
    win = GaussianWindow(sigma)
    rcut = sigma * np.sqrt(-np.log(tol)) + 1e-12
    kmax = 2.0 / sigma * np.sqrt(-np.log(tol))
    return dict(
        real=lambda dd, which: (k3.stokeslet_res(win, dd, 1.0, cut=False) if which == "S"
                                else k3.stresslet_res(win, dd, 1.0, cut=False)),
        rcut=rcut, kmax=kmax, ghat=win.gammahat_closed,
        self=-1.0 / (2.0 * np.pi ** 1.5 * sigma))


def prolate_split_3d(win, nu, kmax):
    """Prolate split at scale nu (nu <= 1/2 keeps the real part to nearest images)."""
    return dict(
        real=lambda dd, which: (k3.stokeslet_res(win, dd, nu) if which == "S"
                                else k3.stresslet_res(win, dd, nu)),
        rcut=nu, kmax=kmax, ghat=lambda k: win.gammahat(k * nu, n=600),
        self=k3.stokeslet_self_coeff(win, nu))


def gaussian_split_2d(sigma, tol=1e-16):
    """2D Hasimoto split: real-space residual by the App. B route with the
    Gaussian mollifier (no compact support, cut at erfc-level tol)."""
    from .window import GaussianWindow
    from . import kernels2d as k2
    win = GaussianWindow(sigma)
    kern = k2.Kernel2D(win)
    rcut = sigma * np.sqrt(-np.log(tol)) + 1e-12
    kmax = 2.0 / sigma * np.sqrt(-np.log(tol))
    return dict(
        real=lambda dd, which: (k2.stokeslet_res(kern, dd, 1.0, cut=False) if which == "S"
                                else k2.stresslet_res(kern, dd, 1.0, cut=False)),
        rcut=rcut, kmax=kmax, ghat=win.gammahat_closed,
        self=k2.stokeslet_self_coeff(kern, 1.0))


def prolate_split_2d(kern, nu, kmax):
    """2D prolate split at scale nu, kern a kernels2d.Kernel2D."""
    from . import kernels2d as k2
    win = kern.win
    return dict(
        real=lambda dd, which: (k2.stokeslet_res(kern, dd, nu) if which == "S"
                                else k2.stresslet_res(kern, dd, nu)),
        rcut=nu, kmax=kmax, ghat=lambda k: win.gammahat(k * nu, n=600),
        self=k2.stokeslet_self_coeff(kern, nu))
