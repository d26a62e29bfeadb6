"""CPU-side checks of the C-ABI library: it loads, exports what the header
declares, validates arguments before touching the GPU, and its host-built
kernel tables agree with the oracle's residual functions."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.window import ProlateWindow
from oracle.params import bandlimit_c
from oracle import kernels3d as k3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dmk_stokes.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmk_stokes_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol(dmk_lib):
    lib = ctypes.CDLL(dmk_lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(dmk_lib.EXPORTED)


def test_invalid_arguments_rejected_without_gpu(dmk_lib):
    lib = dmk_lib._lib
    h = ctypes.c_void_p()
    o = dmk_lib.make_opts(dim=4)
    assert lib.dmk_stokes_plan(ctypes.byref(o), 0, None, 0, None, None, ctypes.byref(h)) == 1
    assert b"dim" in lib.dmk_stokes_last_error(None)
    o = dmk_lib.make_opts(eps=1e-14)
    assert lib.dmk_stokes_plan(ctypes.byref(o), 0, None, 0, None, None, ctypes.byref(h)) == 1
    # the Ewald split is periodic-3D-Stokeslet only; the DMK far field takes one column
    for kw in (dict(components=dmk_lib.EWALD), dict(components=dmk_lib.EWALD, periodic=True, kernels=3),
               dict(components=dmk_lib.EWALD, periodic=True, dim=2), dict(components=dmk_lib.ALL, n_rhs=4),
               dict(components=dmk_lib.ALL, dim=2, n_rhs=2)):
        o = dmk_lib.make_opts(**kw)
        assert lib.dmk_stokes_plan(ctypes.byref(o), 0, None, 0, None, None, ctypes.byref(h)) == 3, kw
    o = dmk_lib.make_opts(components=3)
    assert lib.dmk_stokes_plan(ctypes.byref(o), 0, None, 0, None, None, ctypes.byref(h)) == 1
    assert lib.dmk_stokes_far_info(None, None) == 7
    assert lib.dmk_stokes_tc_wait_selftest(None, None) == 1        # no output pointer: rejected before the GPU
    o = dmk_lib.make_opts()
    assert lib.dmk_stokes_plan(ctypes.byref(o), 10, None, 10, None, None, ctypes.byref(h)) == 1
    # targets are the sources (d_trg NULL) but n_trg != n_src
    assert lib.dmk_stokes_plan(ctypes.byref(o), 10, None, 5, None, None, ctypes.byref(h)) == 1
    # separate targets need a single system; a negative target count is rejected
    assert lib.dmk_stokes_plan(ctypes.byref(o), 0, None, -1, ctypes.c_void_p(8), None, ctypes.byref(h)) == 1
    assert lib.dmk_stokes_eval(None, None, None, None, None, None) == 7
    assert lib.dmk_stokes_sync_status(None) == 7
    lib.dmk_stokes_destroy(None)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-8, 1e-10, 1e-12])
def test_host_tables_match_oracle_residual_functions(dmk_lib, eps):
    c, phi0, gS = dmk_lib.kernel_table(3, eps, 0, kernels=3)
    w = ProlateWindow(bandlimit_c(eps, stokeslet=True, stresslet=True))
    assert abs(c - w.c) < 1e-14 * c
    assert abs(phi0 - float(w.phi(0.0))) < 1e-13
    rho = np.linspace(0.01, 0.999, 200)
    t = 2 * rho ** 2 - 1
    ref = {0: (k3.Sdiag(w, rho) - 1) / rho, 1: (k3.Soffd(w, rho) - 1) / rho,
           2: k3.Tdiag(w, rho) / rho, 3: (k3.Toffd(w, rho) - 1) / rho}
    for which, r in ref.items():
        _, _, p64 = dmk_lib.kernel_table(3, eps, which, kernels=3)
        _, _, p32 = dmk_lib.kernel_table(3, eps, which, fp32=True, kernels=3)
        v64 = np.polynomial.polynomial.polyval(t, p64)
        v32 = np.polynomial.polynomial.polyval(t, p32)
        scale = np.abs(r).max()
        assert np.max(np.abs(v64 - r)) < 2e-13 * scale, which
        assert len(p64) <= 32 and len(p32) <= 24          # compiled kernel sizes
        # FP32 tables drop the Chebyshev tail below eps/10 of max |f|
        assert np.max(np.abs(v32 - r)) < max(eps / 5, 3e-7) * scale, which
    # derivative tables (d/ds, s = rho^2) against finite differences of the oracle
    for which, base in ((4, 0), (5, 1)):
        _, _, pd = dmk_lib.kernel_table(3, eps, which, kernels=3)
        s = rho ** 2
        h = 1e-6
        f = lambda ss: ((k3.Sdiag if base == 0 else k3.Soffd)(w, np.sqrt(ss)) - 1) / np.sqrt(ss)
        fd = (f(s + h) - f(s - h)) / (2 * h)
        assert np.max(np.abs(np.polynomial.polynomial.polyval(t, pd) - fd)) < 1e-6 * np.abs(fd).max() + 1e-8


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-8, 1e-12])
def test_host_tables_2d_match_oracle(dmk_lib, eps):
    from oracle import kernels2d as k2
    kern = k2.Kernel2D(ProlateWindow(bandlimit_c(eps, stokeslet=True, stresslet=True)))
    rho = np.linspace(0.01, 0.999, 150)
    t = 2 * rho ** 2 - 1
    for which, fn in enumerate((kern.m_d, kern.m_o, kern.m_td, kern.m_to)):
        ref = fn(rho)
        _, _, p64 = dmk_lib.kernel_table(2, eps, which, kernels=3)
        _, _, p32 = dmk_lib.kernel_table(2, eps, which, fp32=True, kernels=3)
        scale = np.abs(ref).max()
        # m_to weighs k^7: near k = c the two sides' gamma-hat quadratures differ
        # by rounding, ~1e-12 of max|m_to| at small rho
        assert np.max(np.abs(np.polynomial.polynomial.polyval(t, p64) - ref)) < 5e-12 * scale, which
        assert np.max(np.abs(np.polynomial.polynomial.polyval(t, p32) - ref)) < max(eps / 5, 3e-7) * scale, which
        assert len(p64) <= 32 and len(p32) <= 24
    _, _, m0 = dmk_lib.kernel_table(2, eps, 6, kernels=3)
    assert abs(m0[0] - kern.self_md0()) < 1e-12 * abs(kern.self_md0())
