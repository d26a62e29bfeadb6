"""Direct O(N^2) sums and the periodic stresslet zero mode (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. (stokes_stress_sum): free-space point sums, source = target excluded:
    u_j(x_t) = sum_{s != t} S_jl(x_t - x_s) f_s,l
    u_j(x_t) = sum_{s != t} T_jlm(x_t - x_s) g_s,l n_s,m
with the kernels of Eqs. (stokeslet_def_deriv), (stresslet_def_deriv).

Sec. 5.3 after Eq. (ewald_far): for the periodic stresslet the k = 0 term is
    u0(x_t) = - sum_s (x_t - x_s) (g_s . n_s),
taken with in-cell coordinates (reading); the Stokeslet k = 0 term is zero.
"""
import numpy as np

from . import kernels3d as k3


def stokeslet_2d(x):
    """Full 2D Stokeslet (1/4pi)(-delta log r + x x / r^2)."""
    x = np.asarray(x, dtype=np.float64)
    r2 = np.sum(x * x, axis=-1)
    eye = np.eye(2)
    return (-0.5 * np.log(r2)[..., None, None] * eye
            + x[..., :, None] * x[..., None, :] / r2[..., None, None]) / (4.0 * np.pi)


def stresslet_2d(x):
    """Full 2D stresslet -(1/pi) x x x / r^4."""
    x = np.asarray(x, dtype=np.float64)
    r2 = np.sum(x * x, axis=-1)
    xxx = x[..., :, None, None] * x[..., None, :, None] * x[..., None, None, :]
    return -xxx / (np.pi * r2[..., None, None, None] ** 2)


def direct_sum(x, f=None, g=None, n=None, targets=None):
    """Free-space direct sum over all sources s != t (plain loop over targets)."""
    x = np.asarray(x, dtype=np.float64)
    N, d = x.shape
    tset = np.arange(N) if targets is None else np.asarray(targets)
    u = np.zeros((len(tset), d))
    S_fn = k3.stokeslet if d == 3 else stokeslet_2d
    T_fn = k3.stresslet if d == 3 else stresslet_2d
    for row, t in enumerate(tset):
        m = np.ones(N, dtype=bool)
        m[t] = False
        dd = x[t][None, :] - x[m]
        if f is not None:
            u[row] += np.einsum("pjl,pl->j", S_fn(dd), f[m])
        if g is not None:
            u[row] += np.einsum("pjlm,pl,pm->j", T_fn(dd), g[m], n[m])
    return u


def stresslet_zero_mode(w, g, n, targets=None, wt=None):
    """u0(x_t) = -sum_s (w_t - w_s)(g_s . n_s), as a plain double loop; the
    targets are the points (all, or the indices in targets) or, with wt, the
    separate in-cell target coordinates wt."""
    w = np.asarray(w, dtype=np.float64)
    N, d = w.shape
    if wt is None:
        tset = np.arange(N) if targets is None else np.asarray(targets)
        wt = w[tset]
    wt = np.asarray(wt, dtype=np.float64)
    gn = np.sum(g * n, axis=1)
    u = np.zeros((len(wt), d))
    for row in range(len(wt)):
        u[row] = -np.sum((wt[row][None, :] - w) * gn[:, None], axis=0)
    return u
