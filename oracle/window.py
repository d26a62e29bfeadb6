"""Window functions phi and the biharmonic mollifier gamma-hat (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2.4, Eqs. (PSWFhat), (wfunchat_prol_G), (wfunc_prol_G): psi_0^c is the order-zero prolate spheroidal wave
function on [-1, 1]; the prolate window is

    phi(r)     = psi_0^c(r) / int_{-1}^{1} psi_0^c(t) dt,   |r| <= 1, and 0 beyond,
    phi-hat(k) = psi_0^c(k/c) / psi_0^c(0)          (Fourier transform of phi).

Cor. 4.1, Eq. (def_erfc_like_fcn): Phi(r) = 2 int_r^inf phi(t) dt.
Sec. 4, Eq. (gammaB_in_phi): gamma-hat(k) = phi-hat(k) - k phi-hat'(k) / 2.

psi_0^c is computed the standard way for prolates (Bouwkamp; Xiao, Rokhlin and
Yarvin 2001): expand in orthonormal Legendre polynomials p_k = sqrt(k+1/2) P_k,
in which the prolate differential operator

    L psi = -((1 - x^2) psi')' + c^2 x^2 psi

is  diag(k(k+1)) + c^2 (X^2),  X the Jacobi matrix of multiplication by x
(x p_k = a_{k+1} p_{k+1} + a_k p_{k-1},  a_k = k / sqrt(4k^2 - 1), from the
Legendre three-term recurrence).  psi_0^c is the eigenvector of the smallest
eigenvalue chi_0 within the even subspace.  Sign: psi_0^c(0) > 0.

The Gaussian window of Eq. (wfunc_prol_G), phi_G(r) = exp(-r^2/sigma^2)/(sigma sqrt(pi)),
is provided for special-case pins (it must reproduce erfc and the Hasimoto split).
"""
import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.special import erfc


def _gauss_legendre(n):
    x, w = npleg.leggauss(n)
    return x, w


class _WindowBase:
    """Generic window: phi, phi' supplied by a subclass; integrals by quadrature.

    The quadrature versions (suffix _quad) use composite Gauss-Legendre rules and
    serve both the Gaussian window and as an independent check of the closed
    Legendre antiderivatives used by the prolate window.
    """

    support = np.inf  # phi == 0 for r > support

    def phi(self, r):
        raise NotImplementedError

    def dphi(self, r):
        raise NotImplementedError

    # ---- integrals of phi by composite Gauss-Legendre on [a, b] ----
    def _int_quad(self, f, a, b, panels=64, order=24):
        x, w = _gauss_legendre(order)
        edges = np.linspace(a, b, panels + 1)
        tot = 0.0
        for lo, hi in zip(edges[:-1], edges[1:]):
            h = 0.5 * (hi - lo)
            t = lo + h * (x + 1.0)
            tot += h * np.dot(w, f(t))
        return tot

    def I0_quad(self, r):
        """int_0^r phi(s) ds."""
        return np.array([self._int_quad(self.phi, 0.0, ri) for ri in np.atleast_1d(r)])

    def I1_quad(self, r):
        """int_0^r s phi(s) ds."""
        return np.array([self._int_quad(lambda s: s * self.phi(s), 0.0, ri)
                         for ri in np.atleast_1d(r)])

    def Phi_quad(self, r, upper=None):
        """Phi(r) = 2 int_r^inf phi (Eq. (def_erfc_like_fcn)); 'upper' truncates the infinite range."""
        upper = self.support if upper is None else upper
        out = []
        for ri in np.atleast_1d(r):
            out.append(0.0 if ri >= upper else 2.0 * self._int_quad(self.phi, ri, upper))
        return np.array(out)

    # ---- Fourier transforms (1D cosine transforms of the even function phi) ----
    def phihat(self, k, n=400):
        """phi-hat(k) = int phi(t) e^{-ikt} dt = 2 int_0^R phi(t) cos(kt) dt."""
        R = self.support if np.isfinite(self.support) else self._tail
        k = np.atleast_1d(np.asarray(k, dtype=np.float64))
        x, w = _gauss_legendre(n)
        t = 0.5 * R * (x + 1.0)
        wt = 0.5 * R * w
        return 2.0 * (np.cos(np.outer(k, t)) * (wt * self.phi(t))).sum(axis=1)

    def dphihat(self, k, n=400):
        """d/dk phi-hat(k) = -2 int_0^R t phi(t) sin(kt) dt."""
        R = self.support if np.isfinite(self.support) else self._tail
        k = np.atleast_1d(np.asarray(k, dtype=np.float64))
        x, w = _gauss_legendre(n)
        t = 0.5 * R * (x + 1.0)
        wt = 0.5 * R * w
        return -2.0 * (np.sin(np.outer(k, t)) * (wt * t * self.phi(t))).sum(axis=1)

    def gammahat(self, k, n=400):
        """Biharmonic mollifier gamma-hat(k) = phi-hat(k) - k phi-hat'(k)/2 (Eq. (gammaB_in_phi))."""
        k = np.atleast_1d(np.asarray(k, dtype=np.float64))
        return self.phihat(k, n) - 0.5 * k * self.dphihat(k, n)

    def gamma1d(self, x):
        """1D inverse transform of gamma-hat, 3/2 phi + x phi'/2 (Eq. (biharmonic_screen_R))."""
        return 1.5 * self.phi(x) + 0.5 * x * self.dphi(x)


class ProlateWindow(_WindowBase):
    """Prolate window phi = psi_0^c / int psi_0^c, truncated at r = 1 (Eq. (wfunc_prol_G))."""

    support = 1.0

    def __init__(self, c, nterms=None):
        self.c = float(c)
        nt = int(nterms) if nterms else int(self.c) + 48   # number of even terms
        n = 2 * nt + 2
        k = np.arange(1, n, dtype=np.float64)
        a = k / np.sqrt(4.0 * k * k - 1.0)                   # Jacobi off-diagonal
        X = np.diag(a, 1) + np.diag(a, -1)
        X2 = (X @ X)[: 2 * nt: 2, : 2 * nt: 2]               # even-even block of x^2
        ke = np.arange(0, 2 * nt, 2, dtype=np.float64)
        M = np.diag(ke * (ke + 1.0)) + self.c ** 2 * X2
        evals, evecs = np.linalg.eigh(M)
        self.chi = float(evals[0])
        beta = evecs[:, 0]                                   # orthonormal-basis coefs
        coef = np.zeros(2 * nt)
        coef[::2] = beta * np.sqrt(ke + 0.5)                 # standard P_k coefs
        if npleg.legval(0.0, coef) < 0.0:
            coef = -coef
        self.psi_coef = coef                                 # ||psi||_{L2[-1,1]} = 1
        self.psi_int = 2.0 * coef[0]                         # int_{-1}^1 psi = 2 c_0
        self.lam = self.psi_int / npleg.legval(0.0, coef)    # lambda_0^c (Sec. 2.4, the eigen-relation above Eq. (PSWFhat))
        self.phi_coef = coef / self.psi_int
        self.dphi_coef = npleg.legder(self.phi_coef)
        self.d2phi_coef = npleg.legder(self.dphi_coef)
        self.I0_coef = npleg.legint(self.phi_coef, lbnd=0.0)            # int_0^x phi
        self.I1_coef = npleg.legint(npleg.legmulx(self.phi_coef), lbnd=0.0)  # int_0^x s phi

    def psi(self, x):
        return npleg.legval(np.asarray(x, dtype=np.float64), self.psi_coef)

    def _masked(self, coef, r, outside):
        r = np.asarray(r, dtype=np.float64)
        val = npleg.legval(np.clip(r, -1.0, 1.0), coef)
        return np.where(np.abs(r) <= 1.0, val, outside)

    def phi(self, r):
        return self._masked(self.phi_coef, r, 0.0)

    def dphi(self, r):
        return self._masked(self.dphi_coef, r, 0.0)

    def d2phi(self, r):
        return self._masked(self.d2phi_coef, r, 0.0)

    def I0(self, r):
        """int_0^r phi(s) ds for r >= 0 (constant 1/2 beyond the support)."""
        r = np.asarray(r, dtype=np.float64)
        return np.where(r <= 1.0, npleg.legval(np.minimum(r, 1.0), self.I0_coef),
                        npleg.legval(1.0, self.I0_coef))

    def I1(self, r):
        """int_0^r s phi(s) ds for r >= 0."""
        r = np.asarray(r, dtype=np.float64)
        return np.where(r <= 1.0, npleg.legval(np.minimum(r, 1.0), self.I1_coef),
                        npleg.legval(1.0, self.I1_coef))

    def I1_inf(self):
        """int_0^inf s phi(s) ds."""
        return float(npleg.legval(1.0, self.I1_coef))

    def Phi(self, r):
        """Phi(r) = 2 int_r^1 phi(t) dt for 0 <= r <= 1, 0 beyond (Eq. (def_erfc_like_fcn))."""
        r = np.asarray(r, dtype=np.float64)
        top = npleg.legval(1.0, self.I0_coef)
        return np.where(r < 1.0, 2.0 * (top - npleg.legval(np.minimum(r, 1.0), self.I0_coef)), 0.0)

    def phihat_closed(self, k):
        """phi-hat(k) = psi_0^c(k/c)/psi_0^c(0), valid for |k| <= c (Eq. (wfunchat_prol_G))."""
        return self.psi(np.asarray(k) / self.c) / self.psi(0.0)


class GaussianWindow(_WindowBase):
    """Gaussian window phi_G(r) = exp(-r^2/sigma^2)/(sigma sqrt(pi)) (Eq. (wfunc_prol_G))."""

    def __init__(self, sigma):
        self.sigma = float(sigma)
        self._tail = 12.0 * self.sigma      # exp(-144) is far below FP64 resolution

    def phi(self, r):
        r = np.asarray(r, dtype=np.float64)
        return np.exp(-(r / self.sigma) ** 2) / (self.sigma * np.sqrt(np.pi))

    def dphi(self, r):
        r = np.asarray(r, dtype=np.float64)
        return -2.0 * r / self.sigma ** 2 * self.phi(r)

    def d2phi(self, r):
        r = np.asarray(r, dtype=np.float64)
        return (4.0 * r * r / self.sigma ** 4 - 2.0 / self.sigma ** 2) * self.phi(r)

    def Phi(self, r):
        """Closed form: Phi_G = erfc(r/sigma) (Gaussian case of Eq. (harmonic_split))."""
        return erfc(np.asarray(r, dtype=np.float64) / self.sigma)

    def I0(self, r):
        return 0.5 * (1.0 - self.Phi(r))

    def I1(self, r):
        r = np.asarray(r, dtype=np.float64)
        return self.sigma / (2.0 * np.sqrt(np.pi)) * (1.0 - np.exp(-(r / self.sigma) ** 2))

    def I1_inf(self):
        return self.sigma / (2.0 * np.sqrt(np.pi))

    def phihat_closed(self, k):
        """exp(-k^2 sigma^2 / 4) (Eq. (wfunchat_prol_G))."""
        return np.exp(-(np.asarray(k, dtype=np.float64) * self.sigma) ** 2 / 4.0)

    def gammahat_closed(self, k):
        """Hasimoto mollifier exp(-k^2 s^2/4)(1 + k^2 s^2/4) (Eq. (hasimoto-split); Sec. 3 after Eq. (3.13))."""
        q = (np.asarray(k, dtype=np.float64) * self.sigma) ** 2 / 4.0
        return np.exp(-q) * (1.0 + q)
