"""dmk_stokes_eval_noalloc: the evaluation for callers that must not allocate
device memory when they evaluate (a CUDA stream capture that forbids
allocation calls, or an application whose device memory belongs to another
allocator with a fixed budget).  Its scratch is the library's static 64 MiB
device array instead of the plan's workspace.

Checked through the C ABI against dmk_stokes_eval, with the tolerances of the
other GPU tests, on two calls in a row (the array keeps the previous call's
contents, so the second call shows that what must start at zero is cleared).
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2509_21471_gb300 import workloads as wl
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmk(dmk_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmk_lib


def _pool_bytes():
    """Reserved and high-water bytes of the device's default memory pool, the
    pool the library's stream-ordered allocations come from (driver API:
    CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT = 5, CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8)."""
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    assert cu.cuInit(0) == 0
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    out = []
    for attr in (5, 8):
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        out.append(int(v.value))
    return out


@pytest.mark.parametrize("dim,precision,periodic,kernels,eps,n_rhs,tol", [
    (3, 1, False, 1, 1e-6, 1, 1e-5),      # mixed precision (FP32 pair terms), tolerance 10 eps
    (3, 0, True, 3, 1e-6, 1, 1e-12),      # FP64, periodic Stokeslet + stresslet (zero-mode sums)
    (3, 1, True, 2, 1e-6, 1, 1e-5),
    (3, 1, True, 3, 1e-9, 1, 1e-8),       # mixed below eps 2e-7: float-float pair terms
    (3, 1, False, 1, 1e-6, 16, 1e-5),     # 16 force columns (FP32 columns max(3, 16) per point)
    (2, 1, True, 3, 1e-8, 1, 1e-7),       # 2D periodic, float-float (192 B per point)
])
def test_noalloc_matches_eval_on_two_calls(dmk, dim, precision, periodic, kernels, eps, n_rhs, tol):
    rng = np.random.default_rng(2024 + 10 * precision + kernels + 100 * dim + n_rhs)
    N = 3000
    x = wl.gaussian_mixture_points(rng, N, dim, 8, 0.03)
    f = torch.as_tensor(wl.forces(rng, N, dim, n_rhs=n_rhs), device="cuda") if kernels & 1 else None
    g = torch.as_tensor(wl.stresslet_strengths(rng, N, dim), device="cuda") if kernels & 2 else None
    n = torch.as_tensor(wl.unit_normals(rng, N, dim), device="cuda") if kernels & 2 else None
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, periodic=periodic, kernels=kernels,
                 precision=precision, leaf_capacity=48, n_rhs=n_rhs)
    u_ref = p.eval(f, g, n).cpu().numpy()
    out = torch.empty_like(torch.as_tensor(u_ref, device="cuda"))
    p.eval_noalloc(f, g, n, out=out)                 # the first call looks the array up
    torch.cuda.synchronize()
    before = _pool_bytes()
    for _ in range(2):
        p.eval_noalloc(f, g, n, out=out)
        p.sync_status()
        assert rel_l2(out.cpu().numpy(), u_ref) < tol
    # the calls took nothing from the stream-ordered pool
    assert _pool_bytes() == before
    p.close()


def test_noalloc_replays_in_a_cuda_graph(dmk):
    """Captured once after a warm call, replayed with new forces: equal to eval."""
    rng = np.random.default_rng(2031)
    N = 4000
    x = torch.as_tensor(wl.gaussian_mixture_points(rng, N, 3, 8, 0.03), device="cuda")
    f_static = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    u_static = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = dmk.Plan(x, eps=1e-6, precision=dmk.FP64, stream=s)
        p.eval_noalloc(f_static, out=u_static, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.eval_noalloc(f_static, out=u_static, stream=s)
    for _ in range(2):
        F = torch.as_tensor(wl.forces(rng, N, 3), device="cuda")
        f_static.copy_(F)
        g.replay()
        torch.cuda.synchronize()
        ref = p.eval(F)
        assert rel_l2(u_static.cpu().numpy(), ref.cpu().numpy()) < 1e-14
    p.close()


def test_noalloc_rejects_float_float_plans_beyond_the_static_scratch(dmk):
    rng = np.random.default_rng(8)
    N = 240_000                       # mixed below eps 2e-7 in 3D: 296 B per point, 71 MB > 64 MiB
    x = torch.as_tensor(wl.uniform_points(rng, N, 3), device="cuda")
    f = torch.as_tensor(wl.forces(rng, N, 3), device="cuda")
    p = dmk.Plan(x, eps=1e-9, precision=1, leaf_capacity=512)
    with pytest.raises(dmk.DMKError) as ei:
        p.eval_noalloc(f)
    assert ei.value.code == 1 and "static scratch" in str(ei.value)
    p.close()


def test_noalloc_rejects_plans_beyond_the_static_scratch(dmk):
    rng = np.random.default_rng(7)
    N = 600_000                       # mixed precision needs 136 B per point: 81.6 MB > 64 MiB
    x = torch.as_tensor(wl.uniform_points(rng, N, 3), device="cuda")
    f = torch.as_tensor(wl.forces(rng, N, 3), device="cuda")
    p = dmk.Plan(x, eps=1e-6, precision=1, leaf_capacity=256)
    with pytest.raises(dmk.DMKError) as ei:
        p.eval_noalloc(f)
    assert ei.value.code == 1 and "static scratch" in str(ei.value)
    p.close()
