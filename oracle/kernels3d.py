"""3D residual biharmonic, Stokeslet and stresslet kernels (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Thm 4.1, Eq. (BR_gen):
    B_R(r) = -(1/8pi) ( r - 2r int_0^r phi + 2 int_0^r s phi - 2 int_0^inf s phi ).
Sec. 5.2, Eqs. (res_stokeslet), (Soffdiag), (res_stresslet), (T-offd), rho = r/nu:
    S_R,jl = Sdiag(rho) delta_jl / (8 pi r) + Soffd(rho) x_j x_l / (8 pi r^3)
    Sdiag = Phi - 2 rho phi,   Soffd = Phi + 2 rho phi
    T_R,jlm = (delta_jl x_m + delta_lm x_j + delta_mj x_l) / (8 pi r^3) Tdiag(rho)
              - (3 / 4pi) x_j x_l x_m / r^5 Toffd(rho)
    Tdiag = -2 rho^2 phi',     Toffd = Phi + 2 rho phi - (2/3) rho^2 phi'
The remark closing Sec. 5.2 scales by a length nu: the real-space functions are
evaluated at r/nu and nothing else changes.  Eq. (S_self): the Stokeslet self
term is -phi(0)/(2 pi) rho_t at nu = 1; S is homogeneous of degree -1, so at
scale nu it is -phi(0)/(2 pi nu) rho_t.  The stresslet self term is zero.

Reading (cutoff): the prolate window is truncated at r = 1, so the residual
kernels are taken to be exactly zero for rho >= 1 (strict r < nu inclusion).

Full kernels, Eqs. (stokeslet_def_deriv), (stresslet_def_deriv):
    S_jl = (delta_jl / r + x_j x_l / r^3) / (8 pi),   T_jlm = -(3/4pi) x_j x_l x_m / r^5.

Gradient of S_R (derived here by differentiating Eq. (res_stokeslet) with
Phi' = -2 phi from Eq. (def_erfc_like_fcn)): writing S_R = A(r) delta + C(r) x x,
    d_m S_R,jl = A'(r) x_m/r delta_jl + C'(r) x_m/r x_j x_l + C (delta_jm x_l + delta_lm x_j)
    A' = (rho Sdiag'(rho) - Sdiag(rho)) / (8 pi r^2),  C' = (rho Soffd'(rho) - 3 Soffd(rho)) / (8 pi r^4)
    Sdiag' = -4 phi - 2 rho phi',  Soffd' = 2 rho phi'.
"""
import numpy as np

EIGHT_PI = 8.0 * np.pi


# ---------------------------------------------------------------- biharmonic
def B_full(r):
    """B(r) = -r / (8 pi) in R^3, Eq. (biharmonic_green_def)."""
    return -np.asarray(r, dtype=np.float64) / EIGHT_PI


def B_res(win, r):
    """Residual biharmonic B_R(r), Thm 4.1 Eq. (BR_gen)."""
    r = np.asarray(r, dtype=np.float64)
    return -(r - 2.0 * r * win.I0(r) + 2.0 * win.I1(r) - 2.0 * win.I1_inf()) / EIGHT_PI


def B_res_hasimoto(sigma, r):
    """Hasimoto residual biharmonic, Eq. (hasimoto-split)."""
    from scipy.special import erfc
    r = np.asarray(r, dtype=np.float64)
    return (-r / EIGHT_PI * erfc(r / sigma)
            + sigma / (8.0 * np.pi ** 1.5) * np.exp(-(r / sigma) ** 2))


# ---------------------------------------------------------- radial functions
def Sdiag(win, rho, cut=True):
    rho = np.asarray(rho, dtype=np.float64)
    v = win.Phi(rho) - 2.0 * rho * win.phi(rho)
    return np.where(rho < 1.0, v, 0.0) if cut else v


def Soffd(win, rho, cut=True):
    rho = np.asarray(rho, dtype=np.float64)
    v = win.Phi(rho) + 2.0 * rho * win.phi(rho)
    return np.where(rho < 1.0, v, 0.0) if cut else v


def Tdiag(win, rho, cut=True):
    rho = np.asarray(rho, dtype=np.float64)
    v = -2.0 * rho ** 2 * win.dphi(rho)
    return np.where(rho < 1.0, v, 0.0) if cut else v


def Toffd(win, rho, cut=True):
    rho = np.asarray(rho, dtype=np.float64)
    v = win.Phi(rho) + 2.0 * rho * win.phi(rho) - (2.0 / 3.0) * rho ** 2 * win.dphi(rho)
    return np.where(rho < 1.0, v, 0.0) if cut else v


def dSdiag(win, rho):
    rho = np.asarray(rho, dtype=np.float64)
    return -4.0 * win.phi(rho) - 2.0 * rho * win.dphi(rho)


def dSoffd(win, rho):
    rho = np.asarray(rho, dtype=np.float64)
    return 2.0 * rho * win.dphi(rho)


def dTdiag(win, rho):
    """d/drho of Tdiag = -2 rho^2 phi'."""
    rho = np.asarray(rho, dtype=np.float64)
    return -4.0 * rho * win.dphi(rho) - 2.0 * rho ** 2 * win.d2phi(rho)


def dToffd(win, rho):
    """d/drho of Toffd = Phi + 2 rho phi - (2/3) rho^2 phi', with Phi' = -2 phi."""
    rho = np.asarray(rho, dtype=np.float64)
    return (2.0 / 3.0) * rho * win.dphi(rho) - (2.0 / 3.0) * rho ** 2 * win.d2phi(rho)


# ------------------------------------------------------------------ tensors
def stokeslet(x):
    """Full 3D Stokeslet S_jl(x) for displacement(s) x[..., 3]."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=-1))
    eye = np.eye(3)
    return (eye / r[..., None, None]
            + x[..., :, None] * x[..., None, :] / r[..., None, None] ** 3) / EIGHT_PI


def stresslet(x):
    """Full 3D stresslet T_jlm(x)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=-1))
    xxx = x[..., :, None, None] * x[..., None, :, None] * x[..., None, None, :]
    return -3.0 / (4.0 * np.pi) * xxx / r[..., None, None, None] ** 5


def stokeslet_res(win, x, nu, cut=True):
    """S_R,jl(x) at scale nu, Eq. (res_stokeslet) with the nu-scaling remark."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=-1))
    rho = r / nu
    A = Sdiag(win, rho, cut) / (EIGHT_PI * r)
    C = Soffd(win, rho, cut) / (EIGHT_PI * r ** 3)
    return (A[..., None, None] * np.eye(3)
            + C[..., None, None] * x[..., :, None] * x[..., None, :])


def stresslet_res(win, x, nu, cut=True):
    """T_R,jlm(x) at scale nu, Eq. (res_stresslet)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=-1))
    rho = r / nu
    D = Tdiag(win, rho, cut) / (EIGHT_PI * r ** 3)
    O = -3.0 / (4.0 * np.pi) * Toffd(win, rho, cut) / r ** 5
    eye = np.eye(3)
    sym = (eye[:, :, None] * x[..., None, None, :]       # delta_jl x_m
           + eye[None, :, :] * x[..., :, None, None]     # delta_lm x_j
           + np.transpose(eye)[:, None, :] * x[..., None, :, None])  # delta_mj x_l
    xxx = x[..., :, None, None] * x[..., None, :, None] * x[..., None, None, :]
    return D[..., None, None, None] * sym + O[..., None, None, None] * xxx


def stokeslet_self_coeff(win, nu):
    """u_self = coeff * f_t with coeff = -phi(0) / (2 pi nu), Eq. (S_self)."""
    return -float(win.phi(0.0)) / (2.0 * np.pi * nu)


def stokeslet_res_grad(win, x, nu):
    """d_m S_R,jl(x) as array [..., j, l, m] (derivative of Eq. (res_stokeslet))."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=-1))
    rho = r / nu
    inside = rho < 1.0
    sd, so = Sdiag(win, rho, False), Soffd(win, rho, False)
    dsd, dso = dSdiag(win, rho), dSoffd(win, rho)
    C = np.where(inside, so / (EIGHT_PI * r ** 3), 0.0)
    dA = np.where(inside, (rho * dsd - sd) / (EIGHT_PI * r ** 2), 0.0)
    dC = np.where(inside, (rho * dso - 3.0 * so) / (EIGHT_PI * r ** 4), 0.0)
    eye = np.eye(3)
    xh = x / r[..., None]
    xx = x[..., :, None] * x[..., None, :]
    g = (dA[..., None, None, None] * eye[:, :, None] * xh[..., None, None, :]
         + dC[..., None, None, None] * xx[..., :, :, None] * xh[..., None, None, :]
         + C[..., None, None, None] * (eye[:, None, :] * x[..., None, :, None]
                                       + eye[None, :, :] * x[..., :, None, None]))
    return g


def stresslet_res_grad(win, x, nu):
    """d_k T_R,jlm(x) as array [..., j, l, m, k] (derivative of Eq. (res_stresslet)):
    T_R = D(r) (delta_jl x_m + delta_lm x_j + delta_mj x_l) + O(r) x_j x_l x_m with
    D = Tdiag/(8 pi r^3), O = -(3/4pi) Toffd/r^5, so
    d_k T_R = D' x_k/r sym + D (delta_jl delta_mk + delta_lm delta_jk + delta_mj delta_lk)
              + O' x_k/r x_j x_l x_m + O (delta_jk x_l x_m + x_j delta_lk x_m + x_j x_l delta_mk),
    D' = (rho Tdiag' - 3 Tdiag)/(8 pi r^4),  O' = -(3/4pi)(rho Toffd' - 5 Toffd)/r^6."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=-1))
    rho = r / nu
    inside = rho < 1.0
    td, to = Tdiag(win, rho, False), Toffd(win, rho, False)
    D = np.where(inside, td / (EIGHT_PI * r ** 3), 0.0)
    O = np.where(inside, -3.0 / (4.0 * np.pi) * to / r ** 5, 0.0)
    dD = np.where(inside, (rho * dTdiag(win, rho) - 3.0 * td) / (EIGHT_PI * r ** 4), 0.0)
    dO = np.where(inside, -3.0 / (4.0 * np.pi) * (rho * dToffd(win, rho) - 5.0 * to) / r ** 6, 0.0)
    e = np.eye(3)
    xh = x / r[..., None]
    sym = (e[:, :, None] * x[..., None, None, :] + e[None, :, :] * x[..., :, None, None]
           + np.transpose(e)[:, None, :] * x[..., None, :, None])                       # [.., j, l, m]
    xxx = x[..., :, None, None] * x[..., None, :, None] * x[..., None, None, :]
    dsym = (e[:, :, None, None] * e[None, None, :, :] + e[None, :, :, None] * e[:, None, None, :]
            + np.transpose(e)[:, None, :, None] * e[None, :, None, :])                   # [j, l, m, k]
    dxxx = (e[:, None, None, :] * x[..., None, :, None, None] * x[..., None, None, :, None]
            + x[..., :, None, None, None] * e[None, :, None, :] * x[..., None, None, :, None]
            + x[..., :, None, None, None] * x[..., None, :, None, None] * e[None, None, :, :])
    return (dD[..., None, None, None, None] * sym[..., None] * xh[..., None, None, None, :]
            + D[..., None, None, None, None] * dsym
            + dO[..., None, None, None, None] * xxx[..., None] * xh[..., None, None, None, :]
            + O[..., None, None, None, None] * dxxx)
