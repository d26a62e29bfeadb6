"""2D residual Stokeslet and stresslet kernels by App. B (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

App. B, Eqs. (win_stokeslet_detail), (win_stresslet_detail), (msdiag), (STterms),
(dFterms), (msdiag0): the mollified kernels are radial integrals of derivatives
of F_k(r) = J0(kr) against the truncated biharmonic B-hat^R (Eq. (Btrunc_hat),
R = 1 + sqrt(2), Sec. 2.3) and the mollifier gamma-hat (Eq. (gammaB_in_phi)):

    M(r) = (1/2pi) int_0^K F_term(k, r) B-hat^R(k) gamma-hat(k) k dk,

plus 2 r (1 - log R) for the Stokeslet diagonal term (Eq. (msdiag)).  The
residual is the full kernel minus the mollified one, written in the factored
forms of Sec. 5.2 with the 2D full functions Sdiag = -2 r log r, Soffd = 2 r,
Tdiag = 0, Toffd = (4/3) r (read off Eqs. (stokeslet_def_deriv),
(stresslet_def_deriv)).

With z = k r the four terms of Eq. (dFterms) for d = 2 are
    F_Sdiag = 8 pi k (z J0 - J1),            F_Soffd = 8 pi k (2 J1 - z J0),
    F_Tdiag = 8 pi k (4 J1 - 2 z J0 - z^2 J1),
    F_Toffd = 8 pi k ((8/3) J1 - (4/3) z J0 - z^2 J1 / 3),
which vanish like z, z^3, z^3 and z^5.  This module returns the smooth even
functions (unit scale nu = 1, argument s = r^2)
    m_d = Mdiag / r,  m_o = Moffd / r^3,  m_td = MTdiag / r^3,  m_to = MToffd / r^5
using power series of the Bessel combinations for z < 2 (they cancel there).

Readings (the paper leaves them open):
  * the k-integral is truncated at K = c (the prolate bandlimit; Sec. 7 uses
    K_max = c for the prolate window), by Gauss-Legendre on [0, K];
  * scaling by nu (Sec. 5.2 remark, carried to 2D by homogeneity of B-hat):
    S_R,nu(x) = S_R,1(x/nu), T_R,nu(x) = T_R,1(x/nu)/nu, and the self term is
    -S_M,nu(0) f = (-m_d(0) + 2 log nu) f / (8 pi).
Assembled per pair (r < nu, rho = r/nu):
    S_R f = [(-log rho^2 - m_d) f + (2/r^2 - m_o/nu^2)(x.f) x] / (8 pi)
    T_R:(g n) = [-m_td/nu^2 (g (x.n) + x (g.n) + n (x.g))
                 + (-8/r^4 + 6 m_to/nu^4) x (x.g)(x.n)] / (8 pi)
"""
import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.special import j0, j1

R_TRUNC = 1.0 + np.sqrt(2.0)


def _series(kind, z, terms=40):
    """Power series (in z) of the four Bessel combinations divided by their
    leading power, from J0 = sum (-1)^m (z/2)^{2m}/(m!)^2 and
    J1 = sum (-1)^m (z/2)^{2m+1}/(m!(m+1)!)."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    # coefficient of z^(2m+1) in J1 and of z^(2m) in J0
    from math import factorial
    for m in range(terms):
        a0 = (-1) ** m / (4.0 ** m * factorial(m) ** 2)               # J0: z^{2m}
        a1 = (-1) ** m / (2.0 * 4.0 ** m * factorial(m) * factorial(m + 1))   # J1: z^{2m+1}
        if kind == "d":      # J0 - J1/z  -> z^{2m}: a0 - a1
            c, p = a0 - a1, 2 * m
        elif kind == "o":    # (2 J1 - z J0)/z^3 -> z^{2m+1}(2 a1 - a0) / z^3
            c, p = 2 * a1 - a0, 2 * m - 2
        elif kind == "td":   # (4 J1 - 2 z J0 - z^2 J1)/z^3
            # z^{2m+1}: 4 a1_m - 2 a0_m - a1_{m-1}
            a1p = 0.0 if m == 0 else (-1) ** (m - 1) / (2.0 * 4.0 ** (m - 1) * factorial(m - 1) * factorial(m))
            c, p = 4 * a1 - 2 * a0 - a1p, 2 * m - 2
        elif kind == "to":   # ((8/3) J1 - (4/3) z J0 - z^2 J1 / 3)/z^5
            a1p = 0.0 if m == 0 else (-1) ** (m - 1) / (2.0 * 4.0 ** (m - 1) * factorial(m - 1) * factorial(m))
            c, p = (8.0 / 3.0) * a1 - (4.0 / 3.0) * a0 - a1p / 3.0, 2 * m - 4
        else:
            raise ValueError(kind)
        if p < 0:
            continue          # these low powers cancel exactly (checked in the tests)
        out = out + c * z ** p
    return out


def bessel_combo(kind, z):
    """G_kind(z) for z >= 0 (direct Bessel formulas for z >= 2, series below)."""
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    small = z < 2.0
    out[small] = _series(kind, z[small])
    zl = z[~small]
    J0, J1 = j0(zl), j1(zl)
    if kind == "d":
        out[~small] = J0 - J1 / zl
    elif kind == "o":
        out[~small] = (2 * J1 - zl * J0) / zl ** 3
    elif kind == "td":
        out[~small] = (4 * J1 - 2 * zl * J0 - zl ** 2 * J1) / zl ** 3
    elif kind == "to":
        out[~small] = ((8.0 / 3.0) * J1 - (4.0 / 3.0) * zl * J0 - zl ** 2 * J1 / 3.0) / zl ** 5
    else:
        raise ValueError(kind)
    return out


def bhat_trunc_2d(k):
    """B-hat^R(k) = (1 - J0(Rk) - (1/2) R k J1(Rk)) / k^4 (Eq. (Btrunc_hat), d = 2)."""
    k = np.asarray(k, dtype=np.float64)
    z = R_TRUNC * k
    small = z < 0.5
    zs = np.where(small, z, 0.5)
    # series: 1 - J0 - z J1/2 = sum_{m>=2} (-1)^m (z/2)^{2m} (1/(m!)^2 - 1/(m!(m-1)!)) ... computed termwise
    from math import factorial
    ser = np.zeros_like(zs)
    for m in range(2, 25):
        c = -((-1) ** m) / (4.0 ** m * factorial(m) ** 2) - ((-1) ** (m - 1)) / (4.0 ** (m - 1) * 4.0 * factorial(m - 1) * factorial(m))
        ser = ser + c * zs ** (2 * m)
    zl = np.where(small, 0.5, z)
    direct = 1.0 - j0(zl) - 0.5 * zl * j1(zl)
    num = np.where(small, ser, direct)
    kk = np.where(k > 0, k, 1.0)
    return np.where(k > 0, num / kk ** 4, R_TRUNC ** 4 / 64.0)


class Kernel2D:
    """2D residual functions m_d, m_o, m_td, m_to for a window (prolate or Gaussian)."""

    def __init__(self, win, K=None, nquad=160):
        self.win = win
        gaussian = hasattr(win, "gammahat_closed")
        if K is None:
            K = 12.0 / win.sigma if gaussian else win.c
        self.K = float(K)
        x, w = npleg.leggauss(nquad)
        self.k = 0.5 * self.K * (x + 1.0)
        self.wk = 0.5 * self.K * w
        gh = win.gammahat_closed(self.k) if gaussian else win.gammahat(self.k, n=600)
        self.weight = self.wk * bhat_trunc_2d(self.k) * gh

    def _integral(self, kind, power, rho):
        rho = np.atleast_1d(np.asarray(rho, dtype=np.float64))
        z = np.outer(rho, self.k)
        return 4.0 * (bessel_combo(kind, z) * (self.k ** power * self.weight)).sum(axis=1)

    def m_d(self, rho):
        return self._integral("d", 3, rho) + 2.0 * (1.0 - np.log(R_TRUNC))

    def m_o(self, rho):
        return self._integral("o", 5, rho)

    def m_td(self, rho):
        return self._integral("td", 5, rho)

    def m_to(self, rho):
        return self._integral("to", 7, rho)

    def self_md0(self):
        """lim_{r->0} Mdiag(r)/r = 2 int_0^K B-hat^R gamma-hat k^3 dk + 2(1 - log R) (Eqs. (msdiag0), (msdiag))."""
        return 2.0 * float((self.k ** 3 * self.weight).sum()) + 2.0 * (1.0 - np.log(R_TRUNC))


def stokeslet_res(k2, x, nu, cut=True):
    """S_R,jl(x) at scale nu (2D)."""
    x = np.asarray(x, dtype=np.float64)
    r2 = np.sum(x * x, axis=-1)
    nu = np.broadcast_to(np.asarray(nu, dtype=np.float64), r2.shape)
    rho = np.sqrt(r2) / nu
    inside = (rho < 1.0) | (not cut)
    A = (-np.log(rho * rho) - k2.m_d(rho.ravel()).reshape(rho.shape)) / (8 * np.pi)
    C = (2.0 / r2 - k2.m_o(rho.ravel()).reshape(rho.shape) / nu ** 2) / (8 * np.pi)
    A = np.where(inside, A, 0.0)
    C = np.where(inside, C, 0.0)
    return A[..., None, None] * np.eye(2) + C[..., None, None] * x[..., :, None] * x[..., None, :]


def stresslet_res(k2, x, nu, cut=True):
    """T_R,jlm(x) at scale nu (2D)."""
    x = np.asarray(x, dtype=np.float64)
    r2 = np.sum(x * x, axis=-1)
    nu = np.broadcast_to(np.asarray(nu, dtype=np.float64), r2.shape)
    rho = np.sqrt(r2) / nu
    inside = (rho < 1.0) | (not cut)
    D = -k2.m_td(rho.ravel()).reshape(rho.shape) / (8 * np.pi * nu ** 2)
    E = (-8.0 / r2 ** 2 + 6.0 * k2.m_to(rho.ravel()).reshape(rho.shape) / nu ** 4) / (8 * np.pi)
    D = np.where(inside, D, 0.0)
    E = np.where(inside, E, 0.0)
    eye = np.eye(2)
    sym = (eye[:, :, None] * x[..., None, None, :] + eye[None, :, :] * x[..., :, None, None]
           + eye[:, None, :] * x[..., None, :, None])
    xxx = x[..., :, None, None] * x[..., None, :, None] * x[..., None, None, :]
    return D[..., None, None, None] * sym + E[..., None, None, None] * xxx


def stokeslet_self_coeff(k2, nu):
    """u_self = coeff * f_t, coeff = (-m_d(0) + 2 log nu) / (8 pi) (App. B.1 with the 2D nu-scaling)."""
    return (-k2.self_md0() + 2.0 * np.log(nu)) / (8 * np.pi)


def stokeslet_res_grad(k2, x, nu):
    raise NotImplementedError("the 2D gradient is not part of the oracle")
