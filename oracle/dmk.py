"""DMK far field in 3D: proxy charges, plane-wave colleague interactions, the
root kernel and interpolation down the tree (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The method (Sec. 6.1 Steps 1(c), 2, 3; Sec. 6.2; Sec. 7), as this file takes it:

  * Split.  Eq. (three_part_sum) with the multilevel kernels of Sec. 3:
        K = K_M,0 + sum_{l} K_D,l + K_R,
    K_M,l the mollified kernel at scale r_l = 2^-l (Remark after Eq. (ewalds3):
    the Fourier signature at level l is the level-0 one evaluated at k r_l),
    K_D,l = K_M,l+1 - K_M,l.  A leaf at level L takes part in its own level's
    difference step, so its residual is at scale r_{L+1}: the near component
    (oracle.near) and this far component add up to the whole sum.
    Fourier signatures (Eqs. (moll_stokeslet), (moll_stresslet)):
        S-hat = (k^2 delta - k k) B-hat,
        T-hat = i [(k_m delta_jl + k_j delta_lm + k_l delta_mj) k^2 - 2 k_j k_l k_m] B-hat,
        B-hat of K_D,l = (gamma-hat(k r_{l+1}) - gamma-hat(k r_l)) / k^4.
  * Proxy grids (Step 1(c)).  Every box B (centre c_B, side r) carries p^3
    tensor-product points z = c_B + (r/2) xi, xi Chebyshev points of the first
    kind on [-1, 1] (reading: the paper says "scaled Chebyshev nodes").
  * Upward pass (Step 2).  Leaf proxy charges q_j = sum_s L_j(xi_s) rho_s
    (the transpose of interpolation, L_j the tensor Lagrange basis); a parent
    takes sum over children of L_j(child proxy points) q_child.  rho is f
    (Stokeslet, 3 components) or g (x) n (stresslet, 3 x 3).
  * Plane waves (Sec. 7).  At level l, k = h m with h = 2 pi / (3 r_l) and
    m in [-(N1-1)/2, (N1-1)/2]^3; the integral of Eq. (ewalds3) becomes the
    trapezoidal sum (h / 2pi)^3 sum_m.  Outgoing expansion of box C:
        O_C(m) = K-hat_D,l(hm) . sum_j q_j e^{-i h m.(z_j - c_C)}
    (the kernel contraction is applied to the outgoing side, the remark after
    Step 4).  Colleague C of B sits at c_C = c_B + r delta, delta in {-1,0,1}^3
    (periodic images included, Sec. 6.2), so
        I_B(m) = sum_C e^{-2 pi i m.delta / 3} O_C(m),
        pot_B(z_i) += Re (h/2pi)^3 sum_m e^{i h m.(z_i - c_B)} I_B(m).
    With h (z - c) = pi xi / 3 every level uses the same matrices.
  * Root (Step 3(a), Sec. 5.3, Sec. 6.2).  Periodic: the Fourier series of
    K_M,0 on the unit cell over k = 2 pi kappa, kappa != 0,
    |kappa_i| <= (N_per - 1)/2, sampled on the root proxy grid.  Free space:
    the truncated kernel of Eq. (Bmollhat_trunc), B-hat^R gamma-hat with
    R = 1 + sqrt(3) (Eq. (Btrunc_hat)), by the trapezoidal rule with spacing
    h0 = 2 pi / (2 + 2 sqrt 3) over |k_i| <= c + h0 (reading: the kernel
    B^R * gamma is supported in r <= R + 1 and the separations in the unit
    box are at most sqrt 3, so that period has no aliasing), plus the
    constant K_corr = 1/(4 pi R) times sum_s f_s for the Stokeslet.
  * Downward pass (Step 3(b)).  Coarse to fine: a box's potential grid is
    interpolated to its children, and each box adds its colleagues' level-l
    plane waves.  A leaf evaluates its grid at its points by the same
    Lagrange basis.
  * Parameters (Table 2).  3c/pi and p are interpolated linearly in log10 eps
    between the table rows and rounded up; N1 = 2 (3c/pi) - 1 and
    N_per = 2 floor(c / 2pi) + 1, which reproduce every row of the table.

In 2D (App. B) the same steps run on p x p grids with N1 x N1 modes, 9
colleagues, (h/2pi)^2, R = 1 + sqrt(2) and K_corr = (1 - log R)/(4 pi) (Sec. 5.3).
The difference kernels K_D,l = K_R(r_l) - K_R(r_l+1) are compactly supported,
so their Fourier transforms carry no constant and take the same
(gamma-hat(k r_{l+1}) - gamma-hat(k r_l)) / k^4 form as in 3D.
"""
import itertools
import math
import numpy as np

from . import kernels3d as k3
from .params import three_c_over_pi

TABLE2_P = {
    "stokeslet": {-3: 12, -6: 23, -9: 33, -12: 44},
    "stresslet": {-3: 11, -6: 22, -9: 33, -12: 44},
}
R_TRUNC = 1.0 + math.sqrt(3.0)


def _interp_row(rows, eps):
    e = math.log10(eps)
    keys = sorted(rows)
    for lo, hi in zip(keys[:-1], keys[1:]):
        if lo - 1e-9 <= e <= hi + 1e-9:
            t = (e - lo) / (hi - lo)
            return int(math.ceil(rows[lo] + t * (rows[hi] - rows[lo]) - 1e-9))
    raise ValueError("eps outside Table 2 range [1e-12, 1e-3]")


def dmk_params(eps, stokeslet=True, stresslet=False):
    """(3c/pi, p, N1, N_per) for the requested kernels (Table 2 and the rules above)."""
    names = [k for k, on in (("stokeslet", stokeslet), ("stresslet", stresslet)) if on]
    tcp = max(three_c_over_pi(eps, k) for k in names)
    p = max(_interp_row(TABLE2_P[k], eps) for k in names)
    c = tcp * math.pi / 3.0
    return tcp, p, 2 * tcp - 1, 2 * int(math.floor(c / (2.0 * math.pi))) + 1


def cheb_nodes(p):
    """Chebyshev points of the first kind, cos((2j+1) pi / (2p))."""
    j = np.arange(p, dtype=np.float64)
    return np.cos((2.0 * j + 1.0) * np.pi / (2.0 * p))


def lagrange(nodes, t):
    """L[j, i] = prod_{k != j} (t_i - x_k) / (x_j - x_k)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    p = len(nodes)
    L = np.ones((p, len(t)))
    for j in range(p):
        for k in range(p):
            if k != j:
                L[j] *= (t - nodes[k]) / (nodes[j] - nodes[k])
    return L


def _apply3(A, X):
    """Y[a, b, c, ...] = sum_{ijk} A[a, i] A[b, j] A[c, k] X[i, j, k, ...]."""
    Y = np.tensordot(A, X, axes=([1], [0]))                          # a j k ...
    Y = np.moveaxis(np.tensordot(A, Y, axes=([1], [1])), 0, 1)       # a b k ...
    Y = np.moveaxis(np.tensordot(A, Y, axes=([1], [2])), 0, 2)       # a b c ...
    return Y


def _apply3_each(A0, A1, A2, X):
    Y = np.tensordot(A0, X, axes=([1], [0]))
    Y = np.moveaxis(np.tensordot(A1, Y, axes=([1], [1])), 0, 1)
    Y = np.moveaxis(np.tensordot(A2, Y, axes=([1], [2])), 0, 2)
    return Y


def stokeslet_hat(kv, Bh, rh):
    """(k^2 delta - k k) B-hat . rho-hat for k vectors kv[..., 3], rho-hat[..., 3]."""
    k2 = np.sum(kv * kv, axis=-1)
    kdot = np.sum(kv * rh, axis=-1)
    return Bh[..., None] * (k2[..., None] * rh - kv * kdot[..., None])


def stresslet_hat(kv, Bh, G):
    """i [(k_m d_jl + k_j d_lm + k_l d_mj) k^2 - 2 k_j k_l k_m] B-hat G_lm, G[..., l, m]."""
    k2 = np.sum(kv * kv, axis=-1)
    Gk = np.einsum("...lm,...m->...l", G, kv)          # sum_m G_jm k_m   (j = l)
    GTk = np.einsum("...lm,...l->...m", G, kv)         # sum_l G_lj k_l   (j = m)
    tr = np.einsum("...ll->...", G)
    kGk = np.einsum("...l,...lm,...m->...", kv, G, kv)
    return 1j * Bh[..., None] * (k2[..., None] * (Gk + kv * tr[..., None] + GTk)
                                 - 2.0 * kv * kGk[..., None])


def B_trunc_hat(k, d=3):
    """B-hat^R(k), Eq. (Btrunc_hat), R = 1 + sqrt(d); the k -> 0 limits are R^4/120 (3D)
    and R^4/64 (2D), reached through the Taylor series of the same brackets."""
    from scipy.special import j0, j1
    k = np.asarray(k, dtype=np.float64)
    R = 1.0 + math.sqrt(d)
    kr = k * R
    out = np.empty(k.shape)
    m = kr > 1e-2
    x = kr[m]
    if d == 3:
        out[m] = (1.0 + 0.5 * np.cos(x) - 1.5 * np.sin(x) / x) / k[m] ** 4
    else:
        out[m] = (1.0 - j0(x) - 0.5 * x * j1(x)) / k[m] ** 4
    s = ~m
    x = kr[s]
    if d == 3:
        # x^4/120 - x^6/2520 + x^8/120960 (divided by k^4)
        out[s] = R ** 4 * (1.0 / 120.0 - x ** 2 / 2520.0 + x ** 4 / 120960.0)
    else:
        # 1 - J0(x) - x J1(x)/2 = x^4/64 - x^6/1152 + x^8/49152 (divided by k^4)
        out[s] = R ** 4 * (1.0 / 64.0 - x ** 2 / 1152.0 + x ** 4 / 49152.0)
    return out


def K_corr(d):
    """The constant of the truncated free-space Stokeslet (Sec. 5.3 after Eq. (Bmollhat_trunc))."""
    R = 1.0 + math.sqrt(d)
    return 1.0 / (4.0 * np.pi * R) if d == 3 else (1.0 - math.log(R)) / (4.0 * np.pi)


def _applyd(As, X, d):
    """Y[a1..ad, ...] = sum_i prod_k As[k][a_k, i_k] X[i1..id, ...] (one matrix per axis)."""
    Y = X
    for ax in range(d):
        Y = np.moveaxis(np.tensordot(As[ax], Y, axes=([1], [ax])), 0, ax)
    return Y


class FarField:
    """The far component of the DMK sum on an oracle.tree.Tree (2D or 3D)."""

    def __init__(self, tree, win, p, n1, nper):
        self.tree, self.win = tree, win
        self.d = d = tree.dim
        self.p, self.n1, self.nper = int(p), int(n1), int(nper)
        self.xi = cheb_nodes(self.p)
        # child proxy points in the parent's coordinates: ((2o - 1) + xi) / 2
        self.T = [lagrange(self.xi, ((2 * o - 1) + self.xi) / 2.0) for o in (0, 1)]   # [a, i]
        M = (self.n1 - 1) // 2
        self.m1 = np.arange(-M, M + 1, dtype=np.float64)
        self.E = np.exp(-1j * np.pi * np.outer(self.m1, self.xi) / 3.0)   # [m, j] outgoing
        # boxes: every ancestor of a leaf
        boxes = set()
        for (lev, c) in tree.leaves:
            for l in range(lev, -1, -1):
                boxes.add((l, tuple(v >> (lev - l) for v in c)))
        self.boxes = boxes
        self.maxlev = max(l for (l, _) in boxes)
        self.by_level = [sorted(b for b in boxes if b[0] == l) for l in range(self.maxlev + 1)]
        self._modes = {}

    # ------------------------------------------------------------- helpers
    def _is_leaf(self, B):
        return B in self.tree.leafset

    def _children(self, B):
        lev, c = B
        d = self.d
        return [((lev + 1, tuple(2 * c[a] + o[a] for a in range(d))), o)
                for o in self.tree.child_offsets]

    def _colleagues(self, B):
        """(box, delta) for every existing box at B's level touching B (images in
        the periodic case; delta is the offset of the colleague's image in units
        of the box side)."""
        lev, c = B
        d = self.d
        n = 2 ** lev
        out = []
        for dl in itertools.product((-1, 0, 1), repeat=d):
            raw = tuple(c[a] + dl[a] for a in range(d))
            if self.tree.periodic:
                pos = tuple(v % n for v in raw)
            else:
                if any(v < 0 or v >= n for v in raw):
                    continue
                pos = raw
            if (lev, pos) in self.boxes:
                out.append(((lev, pos), np.array(dl, dtype=np.float64)))
        return out

    def _centre(self, B):
        lev, c = B
        r = 2.0 ** -lev
        return (np.array(c, dtype=np.float64) + 0.5) * r, r

    def _local(self, B, w):
        cB, r = self._centre(B)
        return (w - cB[None, :]) / (0.5 * r)

    def _level_Bhat(self, lev, k):
        """B-hat of K_D,lev times (h/2pi)^d."""
        r = 2.0 ** -lev
        h = 2.0 * np.pi / (3.0 * r)
        g = self.win.gammahat(k.ravel() * (0.5 * r), n=600) - self.win.gammahat(k.ravel() * r, n=600)
        g = g.reshape(k.shape)
        out = np.zeros(k.shape)
        nz = k > 0.0
        out[nz] = g[nz] / k[nz] ** 4 * (h / (2.0 * np.pi)) ** self.d
        return out

    def _grid(self, axis_values):
        return np.stack(np.meshgrid(*([axis_values] * self.d), indexing="ij"), axis=-1)

    # ------------------------------------------------------------- passes
    def charges(self, f=None, g=None, n=None):
        """Upward pass: proxy charges of every box, {box: (qS[p]*d + [d], qT[p]*d + [d, d])}."""
        tree, p, d = self.tree, self.p, self.d
        shp = (p,) * d
        q = {}
        for i, L in enumerate(tree.leaves):
            S = tree.leaf_points(i)
            qS = np.zeros(shp + (d,))
            qT = np.zeros(shp + (d, d))
            if len(S):
                xi = self._local(L, tree.w[S])
                A = [lagrange(self.xi, xi[:, a]) for a in range(d)]          # [j, s]
                idx = "abc"[:d]
                spec = ",".join(f"{x}s" for x in idx)
                if f is not None:
                    qS = np.einsum(f"{spec},sk->{idx}k", *A, f[S])
                if g is not None:
                    rho = g[S][:, :, None] * n[S][:, None, :]
                    qT = np.einsum(f"{spec},slm->{idx}lm", *A, rho)
            q[L] = (qS, qT)
        for lev in range(self.maxlev - 1, -1, -1):
            for B in self.by_level[lev]:
                if self._is_leaf(B):
                    continue
                qS = np.zeros(shp + (d,))
                qT = np.zeros(shp + (d, d))
                for (C, o) in self._children(B):
                    cS, cT = q[C]
                    As = [self.T[o[a]] for a in range(d)]
                    qS += _applyd(As, cS, d)
                    qT += _applyd(As, cT, d)
                q[B] = (qS, qT)
        return q

    def _level_modes(self, lev):
        """k vectors [N1]*d + [d] and (h/2pi)^d B-hat of K_D,lev (computed once per level)."""
        if lev not in self._modes:
            r = 2.0 ** -lev
            h = 2.0 * np.pi / (3.0 * r)
            kv = h * self._grid(self.m1)
            kk = np.sqrt(np.sum(kv * kv, axis=-1))
            self._modes[lev] = (kv, self._level_Bhat(lev, kk))
        return self._modes[lev]

    def outgoing(self, lev, qS, qT, want_S, want_T):
        """Kernel-contracted outgoing plane waves O(m)[N1]*d + [d] at level lev."""
        kv, Bh = self._level_modes(lev)
        d = self.d
        O = np.zeros(Bh.shape + (d,), dtype=np.complex128)
        if want_S:
            O += stokeslet_hat(kv, Bh, _applyd([self.E] * d, qS, d))
        if want_T:
            O += stresslet_hat(kv, Bh, _applyd([self.E] * d, qT, d))
        return O

    def root(self, qS, qT, want_S, want_T):
        """Root potential on the root proxy grid [p]*d + [d]."""
        d = self.d
        if self.tree.periodic:
            K = (self.nper - 1) // 2
            kap = np.arange(-K, K + 1, dtype=np.float64)
            # z - c_0 = xi / 2 on the unit cell
            E0 = np.exp(-1j * np.pi * np.outer(kap, self.xi))
            kv = 2.0 * np.pi * self._grid(kap)
            kk = np.sqrt(np.sum(kv * kv, axis=-1))
            Bh = np.zeros(kk.shape)
            nz = kk > 0.0
            Bh[nz] = self.win.gammahat(kk[nz], n=600) / kk[nz] ** 4
        else:
            h0 = 2.0 * np.pi / (2.0 + 2.0 * math.sqrt(d))
            M0 = int(math.ceil(self.win.c / h0)) + 1
            mv = np.arange(-M0, M0 + 1, dtype=np.float64)
            E0 = np.exp(-1j * 0.5 * h0 * np.outer(mv, self.xi))
            kv = h0 * self._grid(mv)
            kk = np.sqrt(np.sum(kv * kv, axis=-1))
            Bh = (B_trunc_hat(kk.ravel(), d) * self.win.gammahat(kk.ravel(), n=600)).reshape(kk.shape)
            Bh *= (h0 / (2.0 * np.pi)) ** d
        O = np.zeros(kk.shape + (d,), dtype=np.complex128)
        if want_S:
            O += stokeslet_hat(kv, Bh, _applyd([E0] * d, qS, d))
        if want_T:
            O += stresslet_hat(kv, Bh, _applyd([E0] * d, qT, d))
        return np.real(_applyd([np.conj(E0).T] * d, O, d))

    def far(self, f=None, g=None, n=None, levels=None, want_root=True):
        """u_far at every point (caller order).  levels: which difference levels
        to include (default all); want_root: include K_M,0 (and K_corr)."""
        tree, p, d = self.tree, self.p, self.d
        want_S, want_T = f is not None, g is not None
        q = self.charges(f, g, n)
        pot = {B: np.zeros((p,) * d + (d,)) for B in self.boxes}
        root = (0, (0,) * d)
        if want_root:
            pot[root] += self.root(q[root][0], q[root][1], want_S, want_T)
        EtH = np.conj(self.E).T                                            # [j, m] incoming
        w3 = np.exp(-2j * np.pi * self.m1 / 3.0)                           # e^{-2 pi i m / 3}
        for lev in range(self.maxlev + 1):
            if levels is None or lev in levels:
                outs = {B: self.outgoing(lev, q[B][0], q[B][1], want_S, want_T)
                        for B in self.by_level[lev]}
                for B in self.by_level[lev]:
                    I = np.zeros_like(outs[B])
                    for (C, dl) in self._colleagues(B):
                        ph = np.ones((1,) * d)
                        for a in range(d):
                            shape = [1] * d
                            shape[a] = len(self.m1)
                            ph = ph * (w3 ** dl[a]).reshape(shape)
                        I += ph[..., None] * outs[C]
                    pot[B] += np.real(_applyd([EtH] * d, I, d))
            if lev < self.maxlev:
                for B in self.by_level[lev]:
                    if self._is_leaf(B):
                        continue
                    for (C, o) in self._children(B):
                        pot[C] += _applyd([self.T[o[a]].T for a in range(d)], pot[B], d)
        u = np.zeros((tree.N, d))
        idx = "abc"[:d]
        spec = ",".join(f"{x}s" for x in idx)
        for i, L in enumerate(tree.leaves):
            S = tree.leaf_points(i)
            if len(S) == 0:
                continue
            xi = self._local(L, tree.w[S])
            A = [lagrange(self.xi, xi[:, a]) for a in range(d)]
            u[S] = np.einsum(f"{spec},{idx}k->sk", *A, pot[L])
        if want_root and want_S and not tree.periodic:
            u += np.sum(f, axis=0)[None, :] * K_corr(d)
        return u


# ------------------------------------------------------------------ exact parts
def _kernels(d, kern):
    """(residual Stokeslet, residual stresslet, self coefficient, full Stokeslet,
    full stresslet) for the dimension; kern is the window (3D) or a
    kernels2d.Kernel2D (2D)."""
    if d == 3:
        return (lambda x, nu: k3.stokeslet_res(kern, x, nu), lambda x, nu: k3.stresslet_res(kern, x, nu),
                lambda nu: k3.stokeslet_self_coeff(kern, nu), k3.stokeslet, k3.stresslet)
    from . import kernels2d as k2
    from .direct import stokeslet_2d, stresslet_2d
    return (lambda x, nu: k2.stokeslet_res(kern, x, nu), lambda x, nu: k2.stresslet_res(kern, x, nu),
            lambda nu: k2.stokeslet_self_coeff(kern, nu), stokeslet_2d, stresslet_2d)


def level_exact(tree, kern, lev, f=None, g=None, n=None):
    """The level-lev difference component summed in real space:
    sum over (s, image) whose level-lev box is a colleague of t's level-lev
    box of K_D,lev(x_t - x_s - image) rho_s, with
    K_D,lev = K_R(r_lev) - K_R(r_lev+1) (the residual kernels of Sec. 5.2 / App. B)
    and K_D,lev(0) from the self terms.  Points whose leaves are coarser than lev
    have no level-lev box and take no part.  kern: the window (3D) or a
    kernels2d.Kernel2D (2D)."""
    d = tree.dim
    N = tree.N
    r0, r1 = 2.0 ** -lev, 2.0 ** -(lev + 1)
    u = np.zeros((N, d))
    box = tree.cell >> (tree.M - lev)                                     # [N, d]
    n_side = 2 ** lev
    idx = np.nonzero(tree.point_level >= lev)[0]
    images = list(itertools.product((-1, 0, 1), repeat=d)) if tree.periodic else [(0,) * d]
    KS = _kernels(d, kern)
    for t in idx:
        # every (source, image) pair of t, evaluated in one call
        dds, Ss, sames = [], [], []
        for img in images:
            im = np.array(img, dtype=np.int64)
            bs = box[idx] + im[None, :] * n_side
            S = idx[np.all(np.abs(bs - box[t][None, :]) <= 1, axis=1)]
            if len(S) == 0:
                continue
            dds.append((tree.w[t][None, :] - tree.w[S]) - im[None, :].astype(np.float64))
            Ss.append(S)
            sames.append((S == t) & (not any(img)))
        if Ss:
            u[t] += _diff_pairs(KS, d, np.concatenate(dds), r0, r1, np.concatenate(sames), f, g, n,
                                np.concatenate(Ss))
    return u


def _diff_pairs(KS, d, dd, r0, r1, same, f, g, n, S):
    Sres, Tres, self_c = KS[0], KS[1], KS[2]
    out = np.zeros(d)
    m = ~same
    if np.any(m):
        x = dd[m]
        if f is not None:
            K = Sres(x, r0) - Sres(x, r1)
            out += np.einsum("pjl,pl->j", K, f[S[m]])
        if g is not None:
            K = Tres(x, r0) - Tres(x, r1)
            out += np.einsum("pjlm,pl,pm->j", K, g[S[m]], n[S[m]])
    if np.any(same) and f is not None:
        # K_D(0) = K_M(r1)(0) - K_M(r0)(0), K_M,nu(0) = -self coefficient
        coeff = -self_c(r1) + self_c(r0)
        out += coeff * f[S[same]].sum(axis=0)
    return out


def root_exact_free(tree, kern, f=None, g=None, n=None):
    """K_M,0 summed exactly in free space: sum_{s != t} (K - K_R(1)) rho_s
    + K_M,1(0) f_t.  kern: the window (3D) or a kernels2d.Kernel2D (2D)."""
    d = tree.dim
    N = tree.N
    w = tree.w
    Sres, Tres, self_c, Sfull, Tfull = _kernels(d, kern)
    u = np.zeros((N, d))
    for t in range(N):
        m = np.ones(N, dtype=bool)
        m[t] = False
        dd = w[t][None, :] - w[m]
        if f is not None:
            K = Sfull(dd) - Sres(dd, 1.0)
            u[t] += np.einsum("pjl,pl->j", K, f[m]) - self_c(1.0) * f[t]
        if g is not None:
            K = Tfull(dd) - Tres(dd, 1.0)
            u[t] += np.einsum("pjlm,pl,pm->j", K, g[m], n[m])
    return u
