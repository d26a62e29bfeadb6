"""components = EWALD of a periodic 3D Stokeslet plan: the single-level PSWF
Ewald sum (Sec. 5.3, Eqs. (ewald_local), (ewald_far); the fast Ewald version
of Sec. 8): near pass on a uniform tree at scale nu plus the Fourier part by a
non-uniform FFT, against the oracle.

* the oracle's near component on the same uniform tree plus its Fourier sum
  over k != 0 (direct, not FFT) with the same split: 10 eps for MIXED, for FP64
  the NUFFT's own accuracy (about 10^-(w-1), w = ceil(log10(1/eps)) + 1 grid
  points per direction) also at 10 eps;
* the classical Gaussian (Hasimoto) Ewald total, independent of any split
  (pinned by sigma-invariance): 10 eps.
"""
import numpy as np
import pytest
import torch

from oracle import near as onear, ewald
from oracle.tree import Tree
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


def _gpu_total(dmk, x, f, eps, prec, ns):
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, periodic=True, precision=prec, leaf_capacity=ns,
                 components=dmk.EWALD)
    u = p.eval(torch.as_tensor(f, device="cuda")).cpu().numpy()
    p.sync_status()
    st = p.stats()
    p.close()
    return u, st


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_ewald_total_matches_oracle_split(dmk, eps):
    rng = np.random.default_rng(900 + int(-np.log10(eps)))
    N, ns = 2000, 500                                      # uniform tree at level 1: nu = 1/4
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3, zero_mean=True)
    win = ProlateWindow(bandlimit_c(eps))
    tr = Tree(x, ns, periodic=True)
    assert set(tr.leaf_level.tolist()) == {1}
    nu = 0.25
    u_ref = (onear.near_lists(tr, dict(win=win, stokeslet=True), f=f)
             + ewald.ewald_sum(x, f=f, split=ewald.prolate_split_3d(win, nu, kmax=1.3 * win.c / nu),
                               parts=("fourier",)))
    for prec in (0, 1):
        u, st = _gpu_total(dmk, x, f, eps, prec, ns)
        assert st["max_level"] == 1 and st["leaves"] == 8
        assert rel_l2(u, u_ref) < 10 * eps, (prec, rel_l2(u, u_ref))


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_ewald_total_matches_gaussian_ewald(dmk, eps):
    rng = np.random.default_rng(910 + int(-np.log10(eps)))
    N = 150
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3, zero_mean=True)
    u_ref = ewald.ewald_sum(x, f=f, split=ewald.gaussian_split_3d(0.12))
    for prec, ns in ((0, 20), (0, 4), (1, 20)):            # levels 1 and 2
        u, _ = _gpu_total(dmk, x, f, eps, prec, ns)
        assert rel_l2(u, u_ref) < 10 * eps, (prec, ns, rel_l2(u, u_ref))


def test_components_all_limits(dmk):
    x = torch.as_tensor(wl.uniform_points(np.random.default_rng(3), 500, 3), device="cuda")
    with pytest.raises(dmk.DMKError) as ei:                # the Ewald split is periodic only
        dmk.Plan(x, eps=1e-6, periodic=False, components=dmk.EWALD)
    assert ei.value.code == 3
    p = dmk.Plan(x, eps=1e-6, periodic=True, components=dmk.EWALD)
    f = torch.zeros((500, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dmk.DMKError) as ei:
        p.eval_grad(f)
    assert ei.value.code == 3
    with pytest.raises(dmk.DMKError) as ei:
        p.eval_noalloc(f)
    assert ei.value.code == 3
    p.close()


def test_bandlimit_override_table2_rows(dmk):
    """With the bandlimit given explicitly (3c/pi), the full sum's error against
    the Gaussian Ewald total falls with c, and Table 2's values of 3c/pi for
    eps = 1e-3, 1e-6, 1e-9 meet their eps (grid width of eps = 1e-12)."""
    rng = np.random.default_rng(930)
    N = 150
    x = wl.uniform_points(rng, N, 3)
    f = wl.forces(rng, N, 3, zero_mean=True)
    u_ref = ewald.ewald_sum(x, f=f, split=ewald.gaussian_split_3d(0.12))
    errs = {}
    for c3 in (6, 10, 17, 25):
        p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=1e-12, periodic=True, precision=0, leaf_capacity=20,
                     components=dmk.EWALD, bandlimit=c3)
        errs[c3] = rel_l2(p.eval(torch.as_tensor(f, device="cuda")).cpu().numpy(), u_ref)
        p.close()
    assert errs[6] > errs[10] > errs[17] > errs[25]
    assert errs[10] < 1e-3 and errs[17] < 1e-6 and errs[25] < 1e-9


def test_autotune_picks_the_fastest_candidate(dmk):
    """The autotuner times plan + eval per candidate leaf capacity (for the full
    periodic sum: the uniform level of the Ewald split) and returns the fastest;
    its result equals a plan built with that capacity."""
    rng = np.random.default_rng(940)
    N = 60000
    x = torch.as_tensor(wl.uniform_points(rng, N, 3), device="cuda")
    f = torch.as_tensor(wl.forces(rng, N, 3, zero_mean=True), device="cuda")
    best, times = dmk.autotune(x, f, candidates=(300, 3000, 30000), repeats=2, eps=1e-6, periodic=True,
                               precision=dmk.MIXED, components=dmk.EWALD)
    assert set(times) == {300, 3000, 30000} and all(t > 0 for t in times.values())
    assert times[best] == min(times.values())
    levels = set()
    for ns in times:
        p = dmk.Plan(x, eps=1e-6, periodic=True, precision=dmk.MIXED, components=dmk.EWALD, leaf_capacity=ns)
        levels.add(p.stats()["max_level"])
        p.close()
    assert levels == {1, 2, 3}                                   # three different splits
