"""Near (residual + self) component of the DMK sum (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5.3, Eq. (three_part_sum): u = u_far^0 + sum_l u_diff^l + u_local^L + u_self,
where L varies with the target's leaf.  Step 4 (Sec. 6.1) sums the residual
kernel directly over the near-neighbour leaves.

Reading of the residual scale for a pair (the paper does not spell it out for
adaptive trees): Step 2(a) gives every leaf at level l proxy charges for the
difference kernel K_D,l and Step 3(b) applies K_D,l to every box at level l,
leaves included; so the mollified part a pair (t, s) receives is K_M at level
min(L_t, L_s) + 1 and the residual left for the near field is

    K_R at scale nu_ts = r_{min(L_t, L_s) + 1} = 2^-(min(L_t, L_s) + 1),

with the self correction at nu_t = r_{L_t + 1} (Eq. (S_self)).  The residual
is supported in r < nu (Cor. 3.1), which the near lists always cover.

Pair displacement (both sides use exactly this FP64 order):
    d = (w_t - w_s) + q,     r2 = (d_0 d_0 + d_1 d_1) + d_2 d_2,
included iff 0 < r2 < nu^2.  Coincident distinct points (r2 == 0) are skipped
(the sum is singular there; reading).

Output: u[N, d] in the caller's point order:
    Stokeslet  u_j += S_R,jl(d) f_s,l          (Eq. (res_stokeslet))
    stresslet  u_j += T_R,jlm(d) g_s,l n_s,m   (Eq. (res_stresslet), strength g (x) n)
    self       u_t += -phi(0)/(2 pi nu_t) f_t   (Eq. (S_self); stresslet: 0)
Periodic stresslet zero mode (Sec. 5.3, after Eq. (ewald_far)) is separate:
see direct.stresslet_zero_mode.
"""
import numpy as np

from . import kernels3d as k3


def _r2(d):
    if d.shape[-1] == 3:
        return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    return d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]


def nu_of_levels(lt, ls):
    return np.ldexp(1.0, -(np.minimum(lt, ls) + 1))


def _pair_values(kern, d, nu, fs, gs, ns, want_grad):
    """Per-pair contributions K_R(d_p) rho_p, shape [p, dim] (and [p, dim, dim])."""
    dim = d.shape[-1]
    P = len(d)
    out = np.zeros((P, dim))
    grad = np.zeros((P, dim, dim)) if want_grad else None
    if P == 0:
        return out, grad
    if dim == 3:
        km = k3
        tab = kern["win"]
    else:
        from . import kernels2d as km
        tab = kern["k2d"]
    if kern.get("stokeslet") and fs is not None:
        out += np.einsum("pjl,pl->pj", km.stokeslet_res(tab, d, nu), fs)
        if want_grad:
            grad += np.einsum("pjlm,pl->pjm", km.stokeslet_res_grad(tab, d, nu), fs)
    if kern.get("stresslet") and gs is not None:
        out += np.einsum("pjlm,pl,pm->pj", km.stresslet_res(tab, d, nu), gs, ns)
        if want_grad:
            if dim != 3:
                raise NotImplementedError("the stresslet gradient is 3D")
            grad += np.einsum("pjlmk,pl,pm->pjk", km.stresslet_res_grad(tab, d, nu), gs, ns)
    return out, grad


def _pair_terms(kern, d, nu, fs, gs, ns, want_grad):
    """Sum over the given pairs of one target."""
    v, g = _pair_values(kern, d, nu, fs, gs, ns, want_grad)
    return v.sum(axis=0), (g.sum(axis=0) if want_grad else None)


def _self_coeff(kern, dim, nu):
    if not kern.get("stokeslet"):
        return 0.0
    if dim == 3:
        return k3.stokeslet_self_coeff(kern["win"], nu)
    from . import kernels2d as k2
    return k2.stokeslet_self_coeff(kern["k2d"], nu)


def near_lists(tree, kern, f=None, g=None, n=None, targets=None, want_grad=False):
    """Near component via the tree's near lists (Step 4).

    kern: dict(win=<window> (3D) or k2d=<2D kernel tables>, stokeslet=bool, stresslet=bool)
    targets: optional original indices to evaluate (default all).
    Returns u[len(targets), d] (and grad[len(targets), d, d] if want_grad).
    Loops over target leaves; all (target, source) pairs of a leaf pair are
    formed at once and the included ones summed per target.
    """
    d = tree.dim
    tset = np.arange(tree.N) if targets is None else np.asarray(targets)
    row_of = np.full(tree.N, -1, dtype=np.int64)
    row_of[tset] = np.arange(len(tset))
    u = np.zeros((len(tset), d))
    G = np.zeros((len(tset), d, d)) if want_grad else None
    by_leaf = {}
    for t in tset:
        by_leaf.setdefault(int(tree.point_leaf[t]), []).append(int(t))
    for B, T in by_leaf.items():
        T = np.array(T, dtype=np.int64)
        Lt = tree.leaf_level[B]
        tt, ds, nus, srcs = [], [], [], []
        for (X, q) in tree.near[B]:
            S = tree.leaf_points(X)
            if len(S) == 0:
                continue
            dd = ((tree.w[T][:, None, :] - tree.w[S][None, :, :])
                  + np.array(q, dtype=np.float64)[None, None, :])
            nu = float(nu_of_levels(Lt, tree.leaf_level[X]))
            r2 = _r2(dd)
            m = (r2 < nu * nu) & (r2 > 0.0)
            it, js = np.nonzero(m)
            tt.append(T[it])
            srcs.append(S[js])
            ds.append(dd[it, js])
            nus.append(np.full(len(it), nu))
        tl = np.concatenate(tt)
        dd = np.concatenate(ds)
        nu = np.concatenate(nus)
        ss = np.concatenate(srcs)
        vals, grads = _pair_values(kern, dd, nu,
                                   None if f is None else f[ss],
                                   None if g is None else g[ss],
                                   None if n is None else n[ss], want_grad)
        rows = row_of[tl]
        for j in range(d):
            u[:, j] += np.bincount(rows, weights=vals[:, j], minlength=len(tset))
            if want_grad:
                for m in range(d):
                    G[:, j, m] += np.bincount(rows, weights=grads[:, j, m], minlength=len(tset))
        if f is not None:
            u[row_of[T]] += _self_coeff(kern, d, float(np.ldexp(1.0, -(Lt + 1)))) * f[T]
    return (u, G) if want_grad else u


def near_targets(tree, kern, xt, f=None, g=None, n=None, want_grad=False):
    """Near component at separate target points xt (Sec. 1 states the sums
    for target points x_t that need not be sources).  The tree is the
    sources'; a target takes the level L_t of the leaf containing it, the pair
    rule nu_ts = r_{min(L_t, L_s)+1} and the near list of that leaf, and has
    no self term (it is not a source).  Pairs at r = 0 are skipped.
    want_grad: also the velocity gradient at the targets (Stokeslet)."""
    d = tree.dim
    wt, tleaf = tree.locate(xt)
    u = np.zeros((len(wt), d))
    G = np.zeros((len(wt), d, d)) if want_grad else None
    for B in np.unique(tleaf):
        T = np.nonzero(tleaf == B)[0]
        Lt = tree.leaf_level[B]
        tt, ds, nus, srcs = [], [], [], []
        for (X, q) in tree.near[B]:
            S = tree.leaf_points(X)
            if len(S) == 0:
                continue
            dd = (wt[T][:, None, :] - tree.w[S][None, :, :]) + np.array(q, dtype=np.float64)[None, None, :]
            nu = float(nu_of_levels(Lt, tree.leaf_level[X]))
            r2 = _r2(dd)
            it, js = np.nonzero((r2 < nu * nu) & (r2 > 0.0))
            tt.append(T[it])
            srcs.append(S[js])
            ds.append(dd[it, js])
            nus.append(np.full(len(it), nu))
        if not tt:
            continue
        tl, dd, nu, ss = (np.concatenate(a) for a in (tt, ds, nus, srcs))
        vals, grads = _pair_values(kern, dd, nu, None if f is None else f[ss], None if g is None else g[ss],
                                   None if n is None else n[ss], want_grad)
        for j in range(d):
            u[:, j] += np.bincount(tl, weights=vals[:, j], minlength=len(wt))
            if want_grad:
                for m in range(d):
                    G[:, j, m] += np.bincount(tl, weights=grads[:, j, m], minlength=len(wt))
    return (u, G) if want_grad else u


def near_targets_brute(tree, kern, xt, f=None, g=None, n=None):
    """The same by brute force over every source and periodic image, from the
    target's leaf level and each source's leaf level only."""
    import itertools
    d = tree.dim
    wt, tleaf = tree.locate(xt)
    images = list(itertools.product((-1, 0, 1), repeat=d)) if tree.periodic else [(0,) * d]
    u = np.zeros((len(wt), d))
    for row in range(len(wt)):
        nu_all = nu_of_levels(tree.leaf_level[tleaf[row]], tree.point_level)
        ds, nus, srcs = [], [], []
        for q in images:
            dd = (wt[row][None, :] - tree.w) + np.array(q, dtype=np.float64)[None, :]
            r2 = _r2(dd)
            m = (r2 < nu_all * nu_all) & (r2 > 0.0)
            ds.append(dd[m])
            nus.append(nu_all[m])
            srcs.append(np.nonzero(m)[0])
        dd, nu, ss = np.concatenate(ds), np.concatenate(nus), np.concatenate(srcs)
        u[row], _ = _pair_terms(kern, dd, nu, None if f is None else f[ss], None if g is None else g[ss],
                                None if n is None else n[ss], False)
    return u


def near_brute(tree, kern, f=None, g=None, n=None, targets=None, want_grad=False):
    """Same component by brute force over all sources and all periodic images,
    using only each point's leaf level (pins the near-list logic)."""
    d = tree.dim
    tset = np.arange(tree.N) if targets is None else np.asarray(targets)
    u = np.zeros((len(tset), d))
    G = np.zeros((len(tset), d, d)) if want_grad else None
    import itertools
    images = list(itertools.product((-1, 0, 1), repeat=d)) if tree.periodic else [(0,) * d]
    for row, t in enumerate(tset):
        Lt = tree.point_level[t]
        nu_all = nu_of_levels(Lt, tree.point_level)
        ds, nus, srcs = [], [], []
        for q in images:
            dd = (tree.w[t][None, :] - tree.w) + np.array(q, dtype=np.float64)[None, :]
            r2 = _r2(dd)
            m = (r2 < nu_all * nu_all) & (r2 > 0.0)
            ds.append(dd[m])
            nus.append(nu_all[m])
            srcs.append(np.nonzero(m)[0])
        dd, nu, ss = np.concatenate(ds), np.concatenate(nus), np.concatenate(srcs)
        val, gr = _pair_terms(kern, dd, nu,
                              None if f is None else f[ss],
                              None if g is None else g[ss],
                              None if n is None else n[ss], want_grad)
        if f is not None:
            val = val + _self_coeff(kern, d, float(np.ldexp(1.0, -(Lt + 1)))) * f[t]
        u[row] = val
        if want_grad:
            G[row] = gr
    return (u, G) if want_grad else u


def pair_counts(tree):
    """(issued, useful): issued = sum over targets of the points in their near
    leaves minus the target itself; useful = pairs with 0 < r2 < nu_ts^2."""
    issued = 0
    useful = 0
    for B in range(len(tree.leaves)):
        T = tree.leaf_points(B)
        if len(T) == 0:
            continue
        for (X, q) in tree.near[B]:
            S = tree.leaf_points(X)
            if len(S) == 0:
                continue
            issued += len(T) * len(S)
            dd = (tree.w[T][:, None, :] - tree.w[S][None, :, :]) + np.array(q, dtype=np.float64)
            nu = float(nu_of_levels(tree.leaf_level[B], tree.leaf_level[X]))
            r2 = _r2(dd)
            useful += int(np.count_nonzero((r2 < nu * nu) & (r2 > 0.0)))
        issued -= len(T)
    return issued, useful
