"""Row a8: several force columns, many independent systems in one plan and one
near-field launch, and capture of the evaluation in a CUDA graph.

Every system is checked against the oracle run on that system alone (tree:
exact integer parity; near field: FP64 1e-12, mixed 10 eps); force columns
against the oracle column by column."""
import numpy as np
import pytest
import torch

from oracle import near as onear
from oracle.tree import Tree
from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from paper_2509_21471_gb300 import workloads as wl
from tests.helpers import rel_l2, leaf_hilbert_perm, hilbert_order

pytestmark = pytest.mark.gpu
EPS = 1e-6


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


def _oracle_u(x, f, ns, periodic=False):
    tr = Tree(x, ns, periodic=periodic)
    return tr, onear.near_lists(tr, dict(win=ProlateWindow(bandlimit_c(EPS)), stokeslet=True), f=f)


@pytest.mark.parametrize("n_rhs", [2, 4, 16])
@pytest.mark.parametrize("precision", [0, 1])
def test_force_columns_match_oracle(dmk, n_rhs, precision):
    rng = np.random.default_rng(400 + n_rhs + 50 * precision)
    N, ns = 1500, 40
    x = wl.uniform_points(rng, N, 3)
    F = rng.standard_normal((N, 3, n_rhs))
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=EPS, precision=precision, leaf_capacity=ns, n_rhs=n_rhs)
    U = p.eval(torch.as_tensor(F, device="cuda")).cpu().numpy()
    p.sync_status()
    assert U.shape == (N, 3, n_rhs)
    tol = 1e-12 if precision == 0 else 10 * EPS
    for k in sorted({0, n_rhs // 2, n_rhs - 1}):
        _, u_ref = _oracle_u(x, F[:, :, k], ns)
        assert rel_l2(U[:, :, k], u_ref) < tol, (k, rel_l2(U[:, :, k], u_ref))
    p.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_systems_match_per_system_oracle(dmk, precision):
    rng = np.random.default_rng(410 + precision)
    sizes = [1, 37, 800, 1500, 2100]
    xs, fs = [], []
    for i, m in enumerate(sizes):
        xs.append(wl.uniform_points(rng, m, 3) if i % 2 == 0 else wl.gaussian_mixture_points(rng, m, 3, 3, 0.05))
        fs.append(wl.forces(rng, m, 3))
    x, f = np.concatenate(xs), np.concatenate(fs)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    ns = 50
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=EPS, precision=precision, leaf_capacity=ns, offsets=offs)
    u = p.eval(torch.as_tensor(f, device="cuda")).cpu().numpy()
    p.sync_status()
    gt = p.tree()
    leaf_base = 0
    for k, m in enumerate(sizes):
        sl = slice(offs[k], offs[k + 1])
        tr, u_ref = _oracle_u(x[sl], f[sl], ns)
        assert rel_l2(u[sl], u_ref) < (1e-12 if precision == 0 else 10 * EPS), k
        if gt is not None:
            L = len(tr.leaves)
            lv = gt["leaf_level"][leaf_base: leaf_base + L]
            assert np.array_equal(lv, tr.leaf_level)
            assert np.array_equal(gt["leaf_coords"][leaf_base: leaf_base + L], tr.leaf_coords)
            assert np.array_equal(gt["leaf_count"][leaf_base: leaf_base + L], tr.leaf_count)
            expect = leaf_hilbert_perm(tr) if hilbert_order(precision, EPS) else tr.perm
            assert np.array_equal(gt["perm"][offs[k]: offs[k + 1]] - offs[k], expect)
            off = gt["near_off"]
            for i in range(L):
                e0, e1 = off[leaf_base + i], off[leaf_base + i + 1]
                got = {(int(gt["near_leaf"][e]) - leaf_base, tuple(int(v) for v in gt["near_q"][e]))
                       for e in range(e0, e1)}
                assert got == set(tr.near[i])
            leaf_base += L
    if gt is not None:
        assert leaf_base == len(gt["leaf_level"])
    p.close()


def test_batched_force_columns_match_single_systems(dmk):
    """Many systems x 16 force columns in one launch equal one plan per system."""
    x, F, offs = wl.batched_3d(n_sys=12, n_rhs=16, nmin=200, nmax=4000)
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=EPS, precision=dmk.MIXED, n_rhs=16, offsets=offs)
    U = p.eval(torch.as_tensor(F, device="cuda")).cpu().numpy()
    p.sync_status()
    for k in range(len(offs) - 1):
        sl = slice(offs[k], offs[k + 1])
        q = dmk.Plan(torch.as_tensor(x[sl], device="cuda"), eps=EPS, precision=dmk.MIXED, n_rhs=16)
        Uk = q.eval(torch.as_tensor(F[sl], device="cuda")).cpu().numpy()
        assert np.array_equal(U[sl], Uk), k
        q.close()
    p.close()


def test_eval_captured_in_cuda_graph(dmk):
    rng = np.random.default_rng(420)
    N = 20000
    x = torch.as_tensor(wl.gaussian_mixture_points(rng, N, 3, 8, 0.02), device="cuda")
    f_static = torch.zeros((N, 3, 16), dtype=torch.float64, device="cuda")
    u_static = torch.zeros((N, 3, 16), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = dmk.Plan(x, eps=EPS, precision=dmk.MIXED, n_rhs=16, stream=s)
        p.eval(f_static, out=u_static, stream=s)        # first use outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.eval(f_static, out=u_static, stream=s)
    for trial in range(2):
        F = torch.as_tensor(rng.standard_normal((N, 3, 16)), device="cuda")
        f_static.copy_(F)
        g.replay()
        torch.cuda.synchronize()
        ref = p.eval(F)
        assert torch.equal(u_static, ref), trial
    p.close()


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_one_column_eval_captured_in_cuda_graph(dmk, eps):
    """One force column, periodic Stokeslet + stresslet: FP32 pair terms at
    1e-6, float-float pair terms at 1e-9; the replay equals an eager call
    (up to the order of the zero-mode reductions)."""
    rng = np.random.default_rng(421)
    N = 8000
    x = torch.as_tensor(wl.uniform_points(rng, N, 3), device="cuda")
    ins = [torch.zeros((N, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    u_static = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = dmk.Plan(x, eps=eps, periodic=True, kernels=dmk.STOKESLET | dmk.STRESSLET, precision=dmk.MIXED,
                     stream=s)
        p.eval(*ins, out=u_static, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.eval(*ins, out=u_static, stream=s)
    for trial in range(2):
        new = [torch.as_tensor(wl.forces(rng, N, 3, zero_mean=True), device="cuda"),
               torch.as_tensor(wl.stresslet_strengths(rng, N, 3), device="cuda"),
               torch.as_tensor(wl.unit_normals(rng, N, 3), device="cuda")]
        for a, b in zip(ins, new):
            a.copy_(b)
        g.replay()
        torch.cuda.synchronize()
        ref = p.eval(*new)
        # the zero-mode sums are reduced with atomics: equal up to their order
        scale = float(ref.abs().max())
        assert torch.allclose(u_static, ref, rtol=0.0, atol=1e-13 * scale), trial
    p.close()
