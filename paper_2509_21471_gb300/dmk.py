"""Thin Python binding of the C ABI in include/dmk_stokes.h (ctypes).

Argument marshalling only: every step of the near-field pass runs in the CUDA
library libdmk_stokes.so.  Importing this module fails loudly if the library
has not been built (``python -c "import __graft_entry__ as g; g.build()"``).
Torch is used for device memory and streams only.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmk_stokes.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (paper_2509_21471_gb300/build.py)")
_lib = ctypes.CDLL(LIB_PATH)

DMK_OK = 0
STATUS_NAMES = {0: "DMK_OK", 1: "DMK_ERR_INVALID_ARG", 2: "DMK_ERR_OUT_OF_RANGE", 3: "DMK_ERR_UNSUPPORTED",
                4: "DMK_ERR_NOMEM", 5: "DMK_ERR_CUDA", 6: "DMK_ERR_TIMEOUT", 7: "DMK_ERR_BAD_PLAN"}
STOKESLET, STRESSLET = 1, 2
FP64, MIXED = 0, 1
ALL, NEAR, EWALD = 0, 1, 2


class DMKError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("periodic", ctypes.c_int32), ("kernels", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("components", ctypes.c_int32),
                ("leaf_capacity", ctypes.c_int32), ("n_rhs", ctypes.c_int32), ("bandlimit", ctypes.c_int32),
                ("eps", ctypes.c_double), ("box_lo", ctypes.c_double * 3)]


_P = ctypes.c_void_p
_lib.dmk_stokes_plan.argtypes = [ctypes.POINTER(Opts), ctypes.c_int64, _P, ctypes.c_int64, _P, _P,
                                 ctypes.POINTER(_P)]
_lib.dmk_stokes_plan_batched.argtypes = [ctypes.POINTER(Opts), ctypes.c_int32, _P, _P, _P, ctypes.POINTER(_P)]
_lib.dmk_stokes_eval.argtypes = [_P, _P, _P, _P, _P, _P]
_lib.dmk_stokes_eval_grad.argtypes = [_P, _P, _P, _P, _P, _P, _P]
_lib.dmk_stokes_eval_adjoint.argtypes = [_P, _P, _P, _P, _P, _P]
_lib.dmk_stokes_eval_noalloc.argtypes = [_P, _P, _P, _P, _P, _P]
_lib.dmk_stokes_sync_status.argtypes = [_P]
_lib.dmk_stokes_plan_stats.argtypes = [_P, _P]
_lib.dmk_stokes_plan_tree.argtypes = [_P] + [_P] * 8
_lib.dmk_stokes_kernel_table.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P]
_lib.dmk_stokes_partition_leaves.argtypes = [ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, _P, _P]
_lib.dmk_stokes_halo_leaves.argtypes = [ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                        _P]
_lib.dmk_stokes_autotune.argtypes = [ctypes.POINTER(Opts), ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_int32, _P,
                                     ctypes.c_int32, _P, _P, _P]
_lib.dmk_stokes_far_info.argtypes = [_P, _P]
_lib.dmk_stokes_tc_wait_selftest.argtypes = [_P, _P]
_lib.dmk_stokes_eval_traced.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int32]
_lib.dmk_stokes_destroy.argtypes = [_P]
_lib.dmk_stokes_destroy.restype = None
_lib.dmk_stokes_last_error.argtypes = [_P]
_lib.dmk_stokes_last_error.restype = ctypes.c_char_p
for _name in ("dmk_stokes_plan", "dmk_stokes_plan_batched", "dmk_stokes_eval", "dmk_stokes_eval_noalloc",
              "dmk_stokes_eval_grad", "dmk_stokes_eval_adjoint",
              "dmk_stokes_sync_status", "dmk_stokes_plan_stats", "dmk_stokes_plan_tree",
              "dmk_stokes_kernel_table", "dmk_stokes_partition_leaves", "dmk_stokes_halo_leaves",
              "dmk_stokes_autotune"):
    getattr(_lib, _name).restype = ctypes.c_int

EXPORTED = ["dmk_stokes_plan", "dmk_stokes_plan_batched", "dmk_stokes_eval", "dmk_stokes_eval_noalloc",
            "dmk_stokes_eval_grad", "dmk_stokes_eval_adjoint",
            "dmk_stokes_sync_status", "dmk_stokes_plan_stats", "dmk_stokes_plan_tree", "dmk_stokes_kernel_table",
            "dmk_stokes_partition_leaves", "dmk_stokes_halo_leaves", "dmk_stokes_autotune", "dmk_stokes_far_info", "dmk_stokes_eval_traced", "dmk_stokes_tc_wait_selftest",
            "dmk_stokes_destroy", "dmk_stokes_last_error"]


def _check(code, handle=None):
    if code != DMK_OK:
        msg = _lib.dmk_stokes_last_error(handle)
        raise DMKError(code, msg.decode() if msg else "")


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _as_dev(t, dim, name, device, n_rhs=1):
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t, dtype=np.float64))
    t = t.to(device=device, dtype=torch.float64).contiguous()
    if n_rhs == 1 and t.dim() == 3 and t.shape[2] == 1:
        t = t[:, :, 0].contiguous()
    ok = (t.dim() == 2 and t.shape[1] == dim) if n_rhs == 1 else (t.dim() == 3 and t.shape[1:] == (dim, n_rhs))
    if not ok:
        raise ValueError(f"{name} must have shape [n, {dim}]" + ("" if n_rhs == 1 else f"[{n_rhs}]"))
    return t


def make_opts(dim=3, periodic=False, kernels=STOKESLET, precision=MIXED, components=NEAR,
              leaf_capacity=0, n_rhs=1, eps=1e-6, box_lo=None, bandlimit=0):
    o = Opts()
    o.dim, o.periodic, o.kernels, o.precision = dim, int(bool(periodic)), kernels, precision
    o.components, o.leaf_capacity, o.n_rhs, o.bandlimit = components, leaf_capacity, n_rhs, bandlimit
    o.eps = eps
    lo = [-0.5] * 3 if box_lo is None else list(box_lo) + [-0.5] * (3 - len(box_lo))
    for a in range(3):
        o.box_lo[a] = lo[a]
    return o


class Plan:
    """dmk_stokes_plan / dmk_stokes_plan_batched on CUDA tensors."""

    def __init__(self, x, eps=1e-6, dim=None, periodic=False, kernels=STOKESLET, precision=MIXED,
                 leaf_capacity=0, n_rhs=1, box_lo=None, offsets=None, stream=None, device=None, targets=None,
                 components=NEAR, bandlimit=0):
        device = device or (x.device if isinstance(x, torch.Tensor) and x.is_cuda else torch.device("cuda"))
        dim = dim or (x.shape[1])
        self.dim = dim
        self.kernels = kernels
        self.n_rhs = n_rhs
        self.device = device
        self._x = _as_dev(x, dim, "x", device)
        self.n = self._x.shape[0]
        self._t = None if targets is None else _as_dev(targets, dim, "targets", device)
        self.nt = self.n if targets is None else self._t.shape[0]     # rows of every output
        self.opts = make_opts(dim, periodic, kernels, precision, components, leaf_capacity, n_rhs, eps, box_lo,
                              bandlimit)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(device):
            sp = _stream_ptr(stream)
            if offsets is None:
                code = _lib.dmk_stokes_plan(ctypes.byref(self.opts), self.n, _ptr(self._x), self.nt, _ptr(self._t),
                                            sp, ctypes.byref(self._h))
            else:
                offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
                self._offs = offs
                code = _lib.dmk_stokes_plan_batched(ctypes.byref(self.opts), len(offs) - 1,
                                                    offs.ctypes.data_as(ctypes.c_void_p), _ptr(self._x), sp,
                                                    ctypes.byref(self._h))
        _check(code, None)

    # ------------------------------------------------------------------
    def _out_shape(self):
        return (self.nt, self.dim) if self.n_rhs == 1 else (self.nt, self.dim, self.n_rhs)

    def eval(self, f=None, g=None, n=None, out=None, stream=None):
        """dmk_stokes_eval: near component u [n, dim] or [n, dim, n_rhs] (float64, caller order)."""
        f = None if f is None else _as_dev(f, self.dim, "f", self.device, self.n_rhs)
        g = None if g is None else _as_dev(g, self.dim, "g", self.device)
        n = None if n is None else _as_dev(n, self.dim, "n", self.device)
        if out is None:
            out = torch.empty(self._out_shape(), dtype=torch.float64, device=self.device)
        code = _lib.dmk_stokes_eval(self._h, _ptr(f), _ptr(g), _ptr(n), _ptr(out), _stream_ptr(stream))
        _check(code, self._h)
        return out

    STAGES = ("near", "leaf_charges", "merge", "outgoing", "colleague", "incoming", "root", "interp", "leaf_eval")

    def eval_traced(self, f=None, g=None, n=None, out=None, stream=None):
        """dmk_stokes_eval_traced: (u, {stage: ms}) for one evaluation (host-synchronises)."""
        f = None if f is None else _as_dev(f, self.dim, "f", self.device, self.n_rhs)
        g = None if g is None else _as_dev(g, self.dim, "g", self.device)
        n = None if n is None else _as_dev(n, self.dim, "n", self.device)
        if out is None:
            out = torch.empty(self._out_shape(), dtype=torch.float64, device=self.device)
        ms = (ctypes.c_double * 9)()
        code = _lib.dmk_stokes_eval_traced(self._h, _ptr(f), _ptr(g), _ptr(n), _ptr(out), _stream_ptr(stream),
                                           ctypes.cast(ms, ctypes.c_void_p), 9)
        _check(code, self._h)
        return out, dict(zip(self.STAGES, [float(v) for v in ms]))

    def eval_noalloc(self, f=None, g=None, n=None, out=None, stream=None):
        """dmk_stokes_eval_noalloc: as eval, with the library's static scratch
        array instead of the plan's workspace (no device allocation)."""
        f = None if f is None else _as_dev(f, self.dim, "f", self.device, self.n_rhs)
        g = None if g is None else _as_dev(g, self.dim, "g", self.device)
        n = None if n is None else _as_dev(n, self.dim, "n", self.device)
        if out is None:
            out = torch.empty(self._out_shape(), dtype=torch.float64, device=self.device)
        code = _lib.dmk_stokes_eval_noalloc(self._h, _ptr(f), _ptr(g), _ptr(n), _ptr(out), _stream_ptr(stream))
        _check(code, self._h)
        return out

    def eval_grad(self, f=None, g=None, n=None, want_u=False, stream=None):
        """dmk_stokes_eval_grad: gradu [n, dim, dim] (and u if want_u); forces f
        (Stokeslet) and / or stresslet strengths g with orientations n."""
        f = None if f is None else _as_dev(f, self.dim, "f", self.device)
        g = None if g is None else _as_dev(g, self.dim, "g", self.device)
        n = None if n is None else _as_dev(n, self.dim, "n", self.device)
        gu = torch.empty((self.nt, self.dim, self.dim), dtype=torch.float64, device=self.device)
        u = torch.empty((self.nt, self.dim), dtype=torch.float64, device=self.device) if want_u else None
        code = _lib.dmk_stokes_eval_grad(self._h, _ptr(f), _ptr(g), _ptr(n), _ptr(u), _ptr(gu), _stream_ptr(stream))
        _check(code, self._h)
        return (u, gu) if want_u else gu

    def eval_adjoint(self, f, w, stream=None):
        """dmk_stokes_eval_adjoint: (dL/df, dL/dx), both [n, 3], for cotangent w = dL/du."""
        f = _as_dev(f, self.dim, "f", self.device)
        w = _as_dev(w, self.dim, "w", self.device)
        v = torch.empty((self.n, self.dim), dtype=torch.float64, device=self.device)
        gx = torch.empty((self.n, self.dim), dtype=torch.float64, device=self.device)
        code = _lib.dmk_stokes_eval_adjoint(self._h, _ptr(f), _ptr(w), _ptr(v), _ptr(gx), _stream_ptr(stream))
        _check(code, self._h)
        return v, gx

    def sync_status(self):
        _check(_lib.dmk_stokes_sync_status(self._h), self._h)

    def stats(self):
        s = (ctypes.c_int64 * 10)()
        _check(_lib.dmk_stokes_plan_stats(self._h, ctypes.cast(s, ctypes.c_void_p)), self._h)
        keys = ["leaves", "max_level", "near_entries", "tiles", "issued_pairs", "three_c_over_pi",
                "leaf_capacity", "points", "useful_pairs", "launches"]
        return dict(zip(keys, [int(v) for v in s]))

    def far_info(self):
        """Far-field sizes of a components=ALL plan (zeros otherwise)."""
        s = (ctypes.c_int32 * 8)()
        _check(_lib.dmk_stokes_far_info(self._h, ctypes.cast(s, ctypes.c_void_p)), self._h)
        keys = ["p", "n1", "root_modes", "boxes", "source_boxes", "target_boxes", "max_level", "fp32"]
        return dict(zip(keys, [int(v) for v in s]))

    def tree(self):
        """Host copy of the tree: dict of numpy arrays."""
        st = self.stats()
        L, E, N, d = st["leaves"], st["near_entries"], st["points"], self.dim
        arr = dict(perm=np.zeros(N, np.int32), leaf_level=np.zeros(L, np.int32), leaf_start=np.zeros(L, np.int32),
                   leaf_count=np.zeros(L, np.int32), leaf_coords=np.zeros((L, d), np.int64),
                   near_off=np.zeros(L + 1, np.int32), near_leaf=np.zeros(E, np.int32),
                   near_q=np.zeros((E, d), np.int32))
        ptrs = [arr[k].ctypes.data_as(ctypes.c_void_p) for k in
                ("perm", "leaf_level", "leaf_start", "leaf_count", "leaf_coords", "near_off", "near_leaf", "near_q")]
        _check(_lib.dmk_stokes_plan_tree(self._h, *ptrs), self._h)
        return arr

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.dmk_stokes_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_table(dim, eps, which, fp32=False, kernels=STOKESLET):
    """dmk_stokes_kernel_table (host only): (c, phi0, coefficients)."""
    c = ctypes.c_double()
    phi0 = ctypes.c_double()
    buf = np.zeros(64, np.float64)
    nt = ctypes.c_int32()
    _check(_lib.dmk_stokes_kernel_table(dim, eps, kernels, which, int(fp32), ctypes.byref(c), ctypes.byref(phi0),
                                        buf.ctypes.data_as(ctypes.c_void_p), 64, ctypes.byref(nt)))
    return c.value, phi0.value, buf[: nt.value].copy()


def autotune(x, f=None, g=None, n=None, candidates=(600, 1200, 2400), repeats=3, stream=None, **plan_kwargs):
    """dmk_stokes_autotune: (best leaf capacity, {candidate: median ms of plan + eval})."""
    x = _as_dev(x, x.shape[1], "x", x.device)
    dim = x.shape[1]
    o = make_opts(dim=dim, **{k: v for k, v in plan_kwargs.items() if k != "leaf_capacity"})
    nr = o.n_rhs
    f = None if f is None else _as_dev(f, dim, "f", x.device, nr)
    g = None if g is None else _as_dev(g, dim, "g", x.device)
    n = None if n is None else _as_dev(n, dim, "n", x.device)
    u = torch.empty((x.shape[0], dim) if nr == 1 else (x.shape[0], dim, nr), dtype=torch.float64, device=x.device)
    cand = _i32(candidates)
    ms = np.zeros(len(cand), np.float64)
    best = ctypes.c_int32()
    with torch.cuda.device(x.device):
        _check(_lib.dmk_stokes_autotune(ctypes.byref(o), x.shape[0], _ptr(x), _ptr(f), _ptr(g), _ptr(n), _ptr(u),
                                        len(cand), cand.ctypes.data_as(ctypes.c_void_p), repeats,
                                        _stream_ptr(stream), ms.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(best)))
    return int(cand[best.value]), {int(c): float(t) for c, t in zip(cand, ms)}


def tc_wait_selftest(stream=None):
    """dmk_stokes_tc_wait_selftest: True when a tensor-core wait that nothing
    completes ran out and was reported (the far field's failure path)."""
    out = ctypes.c_int32(0)
    _check(_lib.dmk_stokes_tc_wait_selftest(_stream_ptr(stream), ctypes.byref(out)), None)
    return bool(out.value)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def partition_leaves(leaf_count, near_off, near_leaf, n_ranks, leaf_tcount=None):
    """dmk_stokes_partition_leaves (host only): (leaf_begin [n_ranks + 1], cost per rank)."""
    lc, no, nl = _i32(leaf_count), _i32(near_off), _i32(near_leaf)
    tc = None if leaf_tcount is None else _i32(leaf_tcount)
    begin = np.zeros(n_ranks + 1, np.int32)
    cost = np.zeros(n_ranks, np.int64)
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    _check(_lib.dmk_stokes_partition_leaves(len(lc), p(lc), p(tc), p(no), p(nl), n_ranks, p(begin), p(cost)))
    return begin, cost


def halo_leaves(near_off, near_leaf, begin, end):
    """dmk_stokes_halo_leaves (host only): the near-list leaves outside [begin, end)."""
    no, nl = _i32(near_off), _i32(near_leaf)
    n = ctypes.c_int32()
    args = (len(no) - 1, no.ctypes.data_as(ctypes.c_void_p), nl.ctypes.data_as(ctypes.c_void_p), int(begin), int(end))
    _check(_lib.dmk_stokes_halo_leaves(*args, None, 0, ctypes.byref(n)))
    halo = np.zeros(max(n.value, 1), np.int32)
    _check(_lib.dmk_stokes_halo_leaves(*args, halo.ctypes.data_as(ctypes.c_void_p), len(halo), ctypes.byref(n)))
    return halo[: n.value]


def eval(x, f=None, g=None, n=None, **plan_kwargs):
    """One-shot plan + eval (allocates a plan per call)."""
    p = Plan(x, **plan_kwargs)
    try:
        return p.eval(f, g, n)
    finally:
        p.close()


class DMKStokesFn(torch.autograd.Function):
    """u = near-field Stokeslet(x, f) with gradients for f and x.

    The forward pass builds a plan from x (or uses the one given).  Backward
    holds the tree, hence every residual scale nu_ts, fixed:
      dL/df   = S[w]                  (S_R is even and symmetric: the operator is its own transpose)
      dL/dx_k = (grad u_k)^T w_k + (grad v_k)^T f_k,   v = S[w]
    both from one dmk_stokes_eval_adjoint call (a symmetric pass that
    recomputes the pair terms; nothing is stored per pair).
    """

    @staticmethod
    def forward(ctx, x, f, plan, plan_kwargs):
        if plan is None:
            plan = Plan(x.detach(), **plan_kwargs)   # released with the autograd graph
        ctx.plan = plan
        ctx.save_for_backward(f)
        return plan.eval(f.detach())

    @staticmethod
    def backward(ctx, w):
        (f,) = ctx.saved_tensors
        v, gx = ctx.plan.eval_adjoint(f.detach(), w)
        return (gx if ctx.needs_input_grad[0] else None), (v if ctx.needs_input_grad[1] else None), None, None


def near_stokeslet(x, f, plan=None, **plan_kwargs):
    """Differentiable near-field Stokeslet velocity u(x, f) (float64 tensors on CUDA).

    Without ``plan`` a plan (FP64 unless ``precision`` is given) is built from x
    in the forward pass; gradients hold its tree fixed."""
    plan_kwargs.setdefault("precision", FP64)
    return DMKStokesFn.apply(x, f, plan, plan_kwargs)
