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


@pytest.mark.parametrize("precision,periodic,kernels,eps,tol", [
    (1, False, 1, 1e-6, 1e-5),      # mixed precision (FP32 pair terms), tolerance 10 eps
    (0, True, 3, 1e-6, 1e-12),      # FP64, periodic Stokeslet + stresslet (zero-mode sums)
    (1, True, 2, 1e-6, 1e-5),
    (1, True, 3, 1e-9, 1e-8),       # mixed below eps 2e-7: float-float pair terms
])
def test_noalloc_matches_eval_on_two_calls(dmk, precision, periodic, kernels, eps, tol):
    rng = np.random.default_rng(2024 + 10 * precision + kernels)
    N = 3000
    x = wl.gaussian_mixture_points(rng, N, 3, 8, 0.03)
    f = torch.as_tensor(wl.forces(rng, N, 3), device="cuda") if kernels & 1 else None
    g = torch.as_tensor(wl.stresslet_strengths(rng, N, 3), device="cuda") if kernels & 2 else None
    n = torch.as_tensor(wl.unit_normals(rng, N, 3), device="cuda") if kernels & 2 else None
    p = dmk.Plan(torch.as_tensor(x, device="cuda"), eps=eps, periodic=periodic, kernels=kernels,
                 precision=precision, leaf_capacity=48)
    u_ref = p.eval(f, g, n).cpu().numpy()
    for _ in range(2):
        u = p.eval_noalloc(f, g, n).cpu().numpy()
        p.sync_status()
        assert rel_l2(u, u_ref) < tol
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
