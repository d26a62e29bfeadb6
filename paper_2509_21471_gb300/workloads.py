"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method: it only draws points, forces,
normals and stresslet strengths with numpy's PCG64 generator.  The shapes follow
the paper's synthetic tests (uniform random points in the unit cube, Sec. 7;
clustered sets are what adaptive trees are for, Sec. 1 and Sec. 8).

All point sets live in [-1/2, 1/2]^d (the unit box of Sec. 1); "unit cube"
recipes are drawn in [0, 1]^d and shifted by -1/2.
"""
import numpy as np

SEED_BASE = 20250921


def rng_for(config_index, extra=0):
    return np.random.default_rng(SEED_BASE + int(config_index) + 1000 * int(extra))


def uniform_points(rng, n, dim):
    return rng.random((n, dim)) - 0.5


def gaussian_mixture_points(rng, n, dim, n_centres=8, sigma=0.02, lo=0.2, hi=0.8):
    """n points from n_centres equally weighted isotropic Gaussians (width sigma)
    with centres uniform in [lo, hi]^dim, clipped to [0, 1]^dim, shifted by -1/2."""
    centres = rng.uniform(lo, hi, size=(n_centres, dim))
    which = rng.integers(0, n_centres, size=n)
    x = centres[which] + sigma * rng.standard_normal((n, dim))
    return np.clip(x, 0.0, 1.0) - 0.5


def forces(rng, n, dim, n_rhs=1, zero_mean=False):
    """N(0,1) per component; layout [n][dim][n_rhs] (n_rhs == 1 -> [n][dim])."""
    f = rng.standard_normal((n, dim, n_rhs))
    if zero_mean:
        f -= f.mean(axis=0, keepdims=True)
    return f[:, :, 0] if n_rhs == 1 else f


def unit_normals(rng, n, dim):
    if dim == 2:
        th = rng.uniform(0.0, 2.0 * np.pi, size=n)
        return np.stack([np.cos(th), np.sin(th)], axis=1)
    v = rng.standard_normal((n, dim))
    return v / np.linalg.norm(v, axis=1)[:, None]


def stresslet_strengths(rng, n, dim):
    return rng.standard_normal((n, dim))


# ---------------------------------------------------------------- recipes
def small_uniform_3d(n=2000, seed_index=0):
    """3D free-space Stokeslet: N uniform points, forces N(0,1)."""
    rng = rng_for(seed_index)
    x = uniform_points(rng, n, 3)
    f = forces(rng, n, 3)
    return x, f


def clustered_3d(n=1_000_000, sigma=0.02, seed_index=1):
    """3D free-space nonuniform: mixture of 8 Gaussians, forces N(0,1)."""
    rng = rng_for(seed_index)
    x = gaussian_mixture_points(rng, n, 3, 8, sigma)
    f = forces(rng, n, 3)
    return x, f


def periodic_2d(n=1_000_000, seed_index=2):
    """2D periodic: uniform points, zero-mean forces, unit normals, strengths."""
    rng = rng_for(seed_index)
    x = uniform_points(rng, n, 2)
    f = forces(rng, n, 2, zero_mean=True)
    nrm = unit_normals(rng, n, 2)
    g = stresslet_strengths(rng, n, 2)
    return x, f, g, nrm


def batched_3d(n_sys=256, n_rhs=16, seed_index=3, nmin=1e3, nmax=1e5):
    """Many independent 3D systems, log-uniform sizes, half uniform / half clustered."""
    rng = rng_for(seed_index)
    sizes = np.round(10.0 ** rng.uniform(np.log10(nmin), np.log10(nmax), size=n_sys)).astype(np.int64)
    xs, fs = [], []
    for i, m in enumerate(sizes):
        if i < n_sys // 2:
            xs.append(uniform_points(rng, int(m), 3))
        else:
            xs.append(gaussian_mixture_points(rng, int(m), 3, 8, 0.05))
        fs.append(rng.standard_normal((int(m), 3, n_rhs)))
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(xs), np.concatenate(fs), offsets


def periodic_3d(n=200_000, seed_index=4):
    """3D periodic: uniform points, zero-mean forces."""
    rng = rng_for(seed_index)
    x = uniform_points(rng, n, 3)
    f = forces(rng, n, 3, zero_mean=True)
    return x, f


def perturbed_sphere_points(rng, n, radius=0.35, amp=0.15):
    """n points on the surface rho(theta, phi) = radius (1 + amp sin(3 theta) cos(4 phi))
    centred in the box, (cos theta, phi) uniform: the "perturbed sphere" point
    sets of the linear-scaling experiments (Sec. 8; the perturbation is not
    specified there, this one stays inside [-0.4025, 0.4025]^3)."""
    ct = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    th = np.arccos(ct)
    rr = radius * (1.0 + amp * np.sin(3.0 * th) * np.cos(4.0 * ph))
    st = np.sqrt(1.0 - ct * ct)
    return np.stack([rr * st * np.cos(ph), rr * st * np.sin(ph), rr * ct], axis=1)


def perturbed_circle_points(rng, n, radius=0.35, amp=0.15):
    """n points on the curve rho(theta) = radius (1 + amp cos(5 theta)), theta
    uniform: the "perturbed circle" of the 2D linear-scaling experiments (Sec. 8)."""
    th = rng.uniform(0.0, 2.0 * np.pi, n)
    rr = radius * (1.0 + amp * np.cos(5.0 * th))
    return np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1)


def linear_scaling(n, dim=3, seed_index=5):
    """Sources and as many separate targets on the perturbed sphere (3D) or
    circle (2D), forces N(0,1), stresslet strengths N(0,1) and unit normals
    (N_S = N_T = n, Sec. 8)."""
    rng = rng_for(seed_index, extra=int(n % 997))
    pts = perturbed_sphere_points if dim == 3 else perturbed_circle_points
    xs = pts(rng, n)
    xt = pts(rng, n)
    f = forces(rng, n, dim)
    g = stresslet_strengths(rng, n, dim)
    nrm = unit_normals(rng, n, dim)
    return xs, xt, f, g, nrm
