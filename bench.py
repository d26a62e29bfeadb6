#!/usr/bin/env python
"""Benchmark: 3D free-space Stokeslet DMK sum on GB300.

Workload (one rank = one independent system, weak scaling): N = 1e6 points from
a mixture of 8 isotropic Gaussians (sigma = 0.02, centres uniform in
[0.2, 0.8]^3, clipped to the unit cube, shifted to [-1/2, 1/2]^3), forces
N(0, 1), eps = 1e-6 (3c/pi = 17, p = 23, N1 = 33, Table 2); the leaf capacity
is picked by the library's autotuner among 1024, 2048, 3072, 4096 and 6144.

One step = dmk_stokes_plan (kernel tables, Morton sort, adaptive tree, level
restriction, near lists, tiles, box hierarchy and far-field job lists) +
dmk_stokes_eval (near field + self term + far field: proxy charges, merges,
plane waves, root, interpolation, leaf evaluation) + dmk_stokes_destroy,
components = ALL, mixed precision.  value = targets / s over the timed steps;
the L2 is flushed (256 MB write) before every timed step.  The FP64 path is
measured on the same workload and reported beside it, with the stage times of
one evaluation (dmk_stokes_eval_traced), the near-field pair rates and the
near-field pass alone.

--impl reference times the FP64 CPU oracle's whole DMK sum (plain numpy, one
thread) on a bounded sample of the same recipe.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3D Stokeslet DMK targets/s at eps=1e-6, mixed vs FP64 on GPU; near-field Gpairs/s"
N_SM = 152
FP32_LANES_PER_SM = 128
# DRAM bytes per launch of the candidate dominant kernels at N = 5e5 (8-Gaussian recipe,
# eps 1e-6, MIXED), keyed by (stage, leaf capacity); filled from ncu captures
TRAFFIC_5E5 = {("near", 2048): 29.1e6, ("near", 3072): 29.1e6, ("near", 4096): 29.0e6,
               ("leaf_charges", 2048): 428.8e6, ("leaf_charges", 3072): 408.7e6, ("leaf_charges", 4096): 384.7e6,
               ("outgoing", 2048): 1299.4e6, ("outgoing", 3072): 1162.2e6, ("outgoing", 4096): 957.5e6,
               ("incoming", 2048): 1001.5e6, ("incoming", 3072): 892.7e6, ("incoming", 4096): 744.4e6,
               ("leaf_eval", 2048): 242.7e6, ("leaf_eval", 3072): 217.5e6, ("leaf_eval", 4096): 185.7e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--leaf-capacity", type=int, default=0, help="0 = paper's n_s for eps")
    ap.add_argument("--cpu-sample", type=int, default=1500, help="points in the oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (eps = 1e-10, 2D periodic, batched, gradient)")
    ap.add_argument("--ewald-only", type=int, default=0, metavar="N",
                    help="profiling aid: time only the full periodic sum (components = EWALD) of N uniform "
                         "points at --eps, plan reused, and print its own line")
    ap.add_argument("--sweep", action="store_true",
                    help="parameter sweep (Sec. 7): error of the periodic full sum (FP64) on 5000 uniform points "
                         "against the bandlimit c (3c/pi = 2..34) and the grid width w (eps = 1e-3..1e-12), "
                         "relative to 3c/pi = 36 at eps = 1e-12; prints its own line")
    ap.add_argument("--batched-only", type=int, default=0, metavar="N_SYS",
                    help="profiling aid: time only the mixed near field of the batched workload "
                         "(N_SYS systems x 16 columns, plan reused) and print its own line")
    return ap.parse_args()


def run_batched_only(args):
    """The batched workload at N_SYS systems, mixed precision, near field only:
    a small case of the several-column kernel for profiling."""
    import torch
    from paper_2509_21471_gb300 import dmk, workloads as wl
    x, F, offs = wl.batched_3d(n_sys=args.batched_only, seed_index=3)
    xd, Fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(F, device="cuda")
    Ud = torch.empty_like(Fd)
    p = dmk.Plan(xd, eps=1e-6, precision=dmk.MIXED, n_rhs=16, offsets=offs)
    for _ in range(max(1, args.warmup)):
        p.eval(Fd, out=Ud)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p.eval(Fd, out=Ud)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = p.stats()
    p.sync_status()
    p.close()
    t = sorted(ms)[len(ms) // 2] / 1e3
    print(json.dumps({"workload": "batched-systems-16-rhs", "n_systems": args.batched_only, "n_points": len(x),
                      "eps": 1e-6, "near_ms_median": 1e3 * t, "useful_pairs": st["useful_pairs"],
                      "gpairs_useful": st["useful_pairs"] / t / 1e9}), flush=True)


def run_ewald_only(args):
    """The periodic full sum at N uniform points, mixed precision: a small case
    of the Ewald far-field kernels (spreading, per-mode product, interpolation)."""
    import torch
    from paper_2509_21471_gb300 import dmk, workloads as wl
    x, f = wl.periodic_3d(n=args.ewald_only, seed_index=4)
    xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
    ud = torch.empty_like(fd)
    p = dmk.Plan(xd, eps=args.eps, periodic=True, precision=dmk.MIXED, components=dmk.EWALD)
    for _ in range(max(1, args.warmup)):
        p.eval(fd, out=ud)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p.eval(fd, out=ud)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = p.stats()
    p.sync_status()
    p.close()
    print(json.dumps({"workload": "3d-periodic-uniform-full-sum", "n_points": args.ewald_only, "eps": args.eps,
                      "uniform_level": st["max_level"], "eval_ms_median": sorted(ms)[len(ms) // 2]}), flush=True)


def run_sweep(args):
    """E(c, w): relative l2 error of the periodic Stokeslet full sum (single-level
    prolate Ewald split, FP64) on 5000 uniform points against the converged sum
    (3c/pi = 36, eps = 1e-12), for 3c/pi = 2..34 and the grid widths of eps =
    1e-3..1e-12; per row the fitted slope of log10 E in 3c/pi and the smallest
    3c/pi reaching E <= eps, beside Table 2's value."""
    import numpy as np
    import torch
    from paper_2509_21471_gb300 import dmk, workloads as wl
    x, f = wl.periodic_3d(n=5000, seed_index=6)
    xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")

    def total(c3, eps):
        p = dmk.Plan(xd, eps=eps, periodic=True, precision=dmk.FP64, components=dmk.EWALD, bandlimit=c3)
        u = p.eval(fd).cpu().numpy()
        p.sync_status()
        p.close()
        return u

    ref = total(36, 1e-12)
    table2 = {1e-3: 10, 1e-6: 17, 1e-9: 25, 1e-12: 31}
    rows = []
    for eps in (1e-3, 1e-6, 1e-9, 1e-12):
        c3s = list(range(2, 35, 2))
        errs = [float(np.linalg.norm(total(c3, eps) - ref) / np.linalg.norm(ref)) for c3 in c3s]
        ok = [c3 for c3, e in zip(c3s, errs) if e <= eps]
        # fitted where c limits the error: above 20x the row's floor (the grid width's accuracy)
        floor = min(errs)
        fit = [(c3, np.log10(e)) for c3, e in zip(c3s, errs) if e > 20 * floor and c3 >= 4]
        slope = float(np.polyfit([a for a, _ in fit], [b for _, b in fit], 1)[0]) if len(fit) > 2 else None
        rows.append({"eps": eps, "w": int(np.ceil(-np.log10(eps))) + 1, "three_c_over_pi": c3s, "rel_l2": errs,
                     "first_c3_meeting_eps": ok[0] if ok else None, "table2_c3": table2[eps],
                     "fit_slope_log10E_per_c3": slope})
    print(json.dumps({"sweep": "E(c, w) of the periodic Stokeslet full sum, 5000 uniform points, FP64",
                      "reference": "3c/pi = 36, eps = 1e-12", "rows": rows}), flush=True)


def workload_config(args, ns):
    return {"workload": "3d-free-stokeslet-clustered-8gauss, whole DMK sum (near + far field)",
            "n_points": args.n, "sigma": 0.02, "eps": args.eps, "leaf_capacity": ns,
            "kernels": "stokeslet", "rhs": 1, "l2": "flushed (256 MB write) before every timed step"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        import statistics
        reasons = set()
        for r in rows:
            if r["hw"].lower().startswith("active"):
                reasons.add("hw_slowdown")
            if r["hwt"].lower().startswith("active"):
                reasons.add("hw_thermal_slowdown")
            if r["swt"].lower().startswith("active"):
                reasons.add("sw_thermal_slowdown")
            if r["pcap"].lower().startswith("active"):
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# ------------------------------------------------------------ reference arm
def oracle_dmk_seconds(n_sample, eps, ns, seed_extra=0):
    """Seconds the FP64 oracle takes for the whole DMK sum (tree, near pass and the
    far field of Sec. 6) on the same recipe at n_sample points."""
    import numpy as np
    from paper_2509_21471_gb300 import workloads as wl
    from oracle import near as onear, dmk as odmk
    from oracle.tree import Tree
    from oracle.window import ProlateWindow
    rng = wl.rng_for(1, extra=10 + seed_extra)
    x = wl.gaussian_mixture_points(rng, n_sample, 3, 8, 0.02)
    f = wl.forces(rng, n_sample, 3)
    tcp, p, n1, nper = odmk.dmk_params(eps)
    win = ProlateWindow(tcp * np.pi / 3)
    t0 = time.perf_counter()
    tr = Tree(x, ns)
    u = onear.near_lists(tr, dict(win=win, stokeslet=True), f=f)
    u += odmk.FarField(tr, win, p, n1, nper).far(f)
    return time.perf_counter() - t0


def oracle_seconds_in_process(n_sample, eps, ns, threads, seed_extra=0):
    """oracle_dmk_seconds in a fresh Python process whose BLAS / OpenMP thread pools
    are limited to `threads` (None: the libraries' default, every core)."""
    env = dict(os.environ)
    if threads is not None:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    code = (f"import bench; print(bench.oracle_dmk_seconds({n_sample}, {eps!r}, {ns}, {seed_extra}))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, check=True)
    return float(r.stdout.strip().splitlines()[-1])


def oracle_timings(n_sample, eps, ns):
    """The oracle on the host cores: one thread, and every core through numpy's
    threaded BLAS (the oracle as it stands); one run each."""
    procs = os.cpu_count() or 1
    one = oracle_seconds_in_process(n_sample, eps, ns, 1)
    alln = oracle_seconds_in_process(n_sample, eps, ns, None)
    return one, alln, procs


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_s, ns = 600, 128          # per step: the oracle's whole DMK sum on a 600-point sample
    for _ in range(min(args.warmup, 1)):
        oracle_seconds_in_process(200, args.eps, ns, 1)
    times = [oracle_seconds_in_process(n_s, args.eps, ns, 1, k) for k in range(args.steps)]
    t = sum(times)
    v = n_s * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "targets/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, ns),
            "cpu_baseline": {"value": v, "unit": "targets/s", "cores": 1, "kind": "oracle",
                             "sample": f"same 8-Gaussian recipe at N={n_s} points per step, leaf capacity {ns}: "
                                       f"the oracle's whole DMK sum (tree, near pass, far field), numpy, 1 thread"},
            "e2e": {"value": v, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_extras(args, dmk, wl, timed, max_over_ranks, rank, k_mixed=3, k_fp64=2):
    from paper_2509_21471_gb300 import dist as pdist
    """The remaining workloads of the hot path, each timed per step (plan +
    eval, or forward + backward) and per near-field evaluation (plan reused),
    in both precisions.  Reported beside the headline; not part of it."""
    import numpy as np
    import torch

    def measure(make_plan, evaluate, n_targets, k):
        out = {}
        for name, prec in (("mixed", dmk.MIXED), ("fp64", dmk.FP64)):
            kk = k if prec == dmk.MIXED else k_fp64
            def step():
                p = make_plan(prec)
                evaluate(p)
                p.close()
            step()
            torch.cuda.synchronize()
            t_step = max_over_ranks(sum(timed(step, kk)) / kk / 1e3)
            p = make_plan(prec)
            evaluate(p)
            torch.cuda.synchronize()
            st = p.stats()
            t_near = max_over_ranks(sum(timed(lambda: evaluate(p), kk)) / kk / 1e3)
            p.close()
            out[name] = {"ms_per_step": 1e3 * t_step, "targets_per_s": n_targets / t_step,
                         "near_ms": 1e3 * t_near, "useful_pairs": st["useful_pairs"],
                         "gpairs_useful": st["useful_pairs"] / t_near / 1e9, "leaves": st["leaves"],
                         "leaf_capacity": st["leaf_capacity"]}
        out["speedup_mixed_over_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
        return out

    res = {}
    # 3D clustered, eps = 1e-10 (MIXED takes float-float pair terms below eps = 2e-7)
    x, f = wl.clustered_3d(n=args.n, sigma=0.02, seed_index=pdist.seed_index(1, rank))
    xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
    ud = torch.empty_like(fd)
    r = measure(lambda prec: dmk.Plan(xd, eps=1e-10, precision=prec), lambda p: p.eval(fd, out=ud), len(x), k_mixed)
    r.update(workload="3d-free-stokeslet-clustered-8gauss", n_points=len(x), eps=1e-10,
             mixed_pair_arith="float-float (eps < 2e-7)")
    res["clustered_3d_eps1e-10"] = r
    del xd, fd, ud

    # the whole DMK sum (near + far field) at eps = 1e-10: the far field in float64
    # in both precisions (MIXED: float-float near pair terms), N = 2e5 clustered
    x, f = wl.clustered_3d(n=200_000, sigma=0.02, seed_index=pdist.seed_index(1, rank))
    xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
    ud = torch.empty_like(fd)
    r = measure(lambda prec: dmk.Plan(xd, eps=1e-10, precision=prec, leaf_capacity=2048, components=dmk.ALL),
                lambda p: p.eval(fd, out=ud), len(x), 2)
    r.update(workload="3d-free-stokeslet-clustered-8gauss, whole DMK sum", n_points=len(x), eps=1e-10,
             note="near_ms here is the whole evaluation (near + far) with the plan reused")
    res["dmk_full_sum_clustered_3d_eps1e-10"] = r
    del xd, fd, ud

    # 2D periodic unit square, Stokeslet + stresslet (k = 0 term included), eps = 1e-8
    x, f, g, nrm = wl.periodic_2d(n=args.n, seed_index=pdist.seed_index(2, rank))
    xd, fd, gd, nd = (torch.as_tensor(a, device="cuda") for a in (x, f, g, nrm))
    ud = torch.empty_like(fd)
    r = measure(lambda prec: dmk.Plan(xd, eps=1e-8, periodic=True, kernels=dmk.STOKESLET | dmk.STRESSLET,
                                      precision=prec),
                lambda p: p.eval(fd, gd, nd, out=ud), len(x), k_mixed)
    r.update(workload="2d-periodic-stokeslet+stresslet-uniform", n_points=len(x), eps=1e-8,
             mixed_pair_arith="float-float (eps < 2e-7)")
    res["periodic_2d_eps1e-8"] = r
    # the same workload as the whole DMK sum (near + the 2D far field; far field in
    # float64 at eps 1e-8 in both precisions)
    r = measure(lambda prec: dmk.Plan(xd, eps=1e-8, periodic=True, kernels=dmk.STOKESLET | dmk.STRESSLET,
                                      precision=prec, components=dmk.ALL),
                lambda p: p.eval(fd, gd, nd, out=ud), len(x), 2)
    r.update(workload="2d-periodic-stokeslet+stresslet-uniform, whole DMK sum", n_points=len(x), eps=1e-8,
             note="near_ms here is the whole evaluation (near + far) with the plan reused")
    res["dmk_full_sum_periodic_2d_eps1e-8"] = r
    del xd, fd, gd, nd, ud

    # 256 independent 3D systems, 16 force columns, one plan and one launch
    x, F, offs = wl.batched_3d(seed_index=pdist.seed_index(3, rank))
    xd, Fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(F, device="cuda")
    Ud = torch.empty_like(Fd)
    r = measure(lambda prec: dmk.Plan(xd, eps=1e-6, precision=prec, n_rhs=16, offsets=offs),
                lambda p: p.eval(Fd, out=Ud), len(x), 2)
    r.update(workload="batched-256-systems-16-rhs", n_points=len(x), n_systems=len(offs) - 1, rhs=16, eps=1e-6,
             mixed_pair_arith="fp32")
    res["batched_256x16_eps1e-6"] = r
    del xd, Fd, Ud

    # differentiation: 3D periodic, N = 2e5, L = 1/2 |u - u_tgt|^2, gradients w.r.t. x and f
    x, f = wl.periodic_3d(n=200_000, seed_index=pdist.seed_index(4, rank))
    rng = wl.rng_for(pdist.seed_index(4, rank), extra=1)
    xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
    u_tgt = dmk.eval(xd, torch.as_tensor(f + 0.1 * rng.standard_normal(f.shape), device="cuda"),
                     eps=1e-8, periodic=True, precision=dmk.FP64)
    out = {}
    for name, prec in (("mixed", dmk.MIXED), ("fp64", dmk.FP64)):
        def fwd_bwd():
            xt = xd.clone().requires_grad_(True)
            ft = fd.clone().requires_grad_(True)
            u = dmk.near_stokeslet(xt, ft, eps=1e-8, periodic=True, precision=prec)
            (0.5 * ((u - u_tgt) ** 2).sum()).backward()
        fwd_bwd()
        torch.cuda.synchronize()
        t = max_over_ranks(sum(timed(fwd_bwd, 2)) / 2 / 1e3)
        # the backward pass alone: one dmk_stokes_eval_adjoint call (plan reused)
        p = dmk.Plan(xd, eps=1e-8, periodic=True, precision=prec)
        p.eval_adjoint(fd, u_tgt)
        torch.cuda.synchronize()
        t_b = max_over_ranks(sum(timed(lambda: p.eval_adjoint(fd, u_tgt), 3)) / 3 / 1e3)
        p.close()
        out[name] = {"ms_per_step": 1e3 * t, "targets_per_s": len(x) / t, "backward_adjoint_ms": 1e3 * t_b}
    out.update(workload="3d-periodic-uniform-loss-gradient", n_points=len(x), eps=1e-8,
               step="plan + forward + backward (grad w.r.t. x and f)",
               speedup_mixed_over_fp64=out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"])
    res["gradient_periodic_3d_eps1e-8"] = out

    # periodic 3D Stokeslet, full sum (components = EWALD): the single-level PSWF
    # Ewald split (near pass on a uniform tree + non-uniform FFT Fourier part)
    ew = {}
    for n, eps in ((200_000, 1e-8), (1_000_000, 1e-6)):
        x, f = wl.periodic_3d(n=n, seed_index=pdist.seed_index(4, rank))
        xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
        ud = torch.empty_like(fd)
        # the autotuner picks the uniform level (points per box) of the split
        ns, tune = dmk.autotune(xd, fd, candidates=(n // 512 + 1, n // 64 + 1, n // 8 + 1), repeats=2, eps=eps,
                                periodic=True, precision=dmk.MIXED, components=dmk.EWALD)
        row = {"autotune_ms_by_points_per_box": tune, "points_per_box": ns}
        for name, prec in (("mixed", dmk.MIXED), ("fp64", dmk.FP64)):
            def step():
                p = dmk.Plan(xd, eps=eps, periodic=True, precision=prec, components=dmk.EWALD, leaf_capacity=ns)
                p.eval(fd, out=ud)
                p.close()
            step()
            torch.cuda.synchronize()
            t = max_over_ranks(sum(timed(step, 2)) / 2 / 1e3)
            p = dmk.Plan(xd, eps=eps, periodic=True, precision=prec, components=dmk.EWALD, leaf_capacity=ns)
            p.eval(fd, out=ud)
            st = p.stats()
            t_eval = max_over_ranks(sum(timed(lambda: p.eval(fd, out=ud), 2)) / 2 / 1e3)
            p.close()
            row[name] = {"ms_per_step": 1e3 * t, "eval_ms": 1e3 * t_eval, "targets_per_s": n / t,
                         "uniform_level": st["max_level"]}
        ew[f"n{n}_eps{eps:g}"] = dict(row, n_points=n, eps=eps)
        del xd, fd, ud
    res["ewald_periodic_3d_full_sum"] = {
        "workload": "3d-periodic-uniform, full periodic Stokeslet sum (near + Fourier part)",
        "step": "plan + eval (components = EWALD)", "runs": ew}

    # linear scaling (Sec. 8): sources and as many separate targets on a
    # perturbed sphere (3D) or circle (2D), N_S = N_T, eps = 1e-6, the paper's
    # leaf capacity; a step = plan (sources and targets) + eval + destroy, MIXED
    sweep = []
    for dim, kern, sizes in ((3, dmk.STOKESLET, (100_000, 250_000, 500_000, 1_000_000, 2_000_000, 4_000_000)),
                             (3, dmk.STRESSLET, (1_000_000,)), (2, dmk.STOKESLET, (1_000_000, 4_000_000))):
        for n in sizes:
            xs, xt, f, g, nrm = wl.linear_scaling(n, dim=dim, seed_index=pdist.seed_index(5, rank))
            xsd, xtd = torch.as_tensor(xs, device="cuda"), torch.as_tensor(xt, device="cuda")
            fd = torch.as_tensor(f, device="cuda") if kern == dmk.STOKESLET else None
            gd = torch.as_tensor(g, device="cuda") if kern == dmk.STRESSLET else None
            nd = torch.as_tensor(nrm, device="cuda") if kern == dmk.STRESSLET else None
            ud = torch.empty((n, dim), dtype=torch.float64, device="cuda")
            levels = [0]

            comp = dmk.ALL                                # the whole DMK sum (near + far field)

            def step():
                p = dmk.Plan(xsd, targets=xtd, eps=1e-6, kernels=kern, precision=dmk.MIXED, components=comp)
                p.eval(fd, gd, nd, out=ud)
                p.close()
            step()
            torch.cuda.synchronize()
            t = max_over_ranks(sum(timed(step, 2)) / 2 / 1e3)
            p = dmk.Plan(xsd, targets=xtd, eps=1e-6, kernels=kern, precision=dmk.MIXED, components=comp)
            p.eval(fd, gd, nd, out=ud)
            st = p.stats()
            t_near = max_over_ranks(sum(timed(lambda: p.eval(fd, gd, nd, out=ud), 2)) / 2 / 1e3)
            p.close()
            sweep.append({"dim": dim, "kernel": "stokeslet" if kern == dmk.STOKESLET else "stresslet",
                          "components": "near + far" if comp == dmk.ALL else "near",
                          "n_sources": n, "n_targets": n, "ms_per_step": 1e3 * t, "eval_ms": 1e3 * t_near,
                          "targets_per_s": n / t, "max_level": st["max_level"], "leaves": st["leaves"],
                          "useful_pairs": st["useful_pairs"]})
            del xsd, xtd, fd, gd, nd, ud
    res["linear_scaling_perturbed_surface_eps1e-6"] = {
        "workload": "perturbed sphere (3D) / circle (2D), separate targets, N_S = N_T", "precision": "mixed",
        "points": sweep}
    return res


# ------------------------------------------------------------------ our arm
def far_flops(stage, fi, n_targets, n_sources, kernels=1):
    """Algorithmic flops (FMA = 2) of one far-field stage of one evaluation, from the
    plan's far-field sizes (p, N1) and the numbers of points and boxes; each
    complex multiply-add counts 8 flops, a real-by-complex one 4."""
    p, n1 = fi["p"], fi["n1"]
    nh = (n1 + 1) // 2
    comps = (3 if kernels & 1 else 0) + (6 if kernels & 2 else 0)
    if stage == "leaf_eval":       # per target: c, b and a contractions of the 3 x p^3 grid
        return n_targets * (2 * (3 * p ** 3 + 3 * p ** 2 + 3 * p) + p ** 2)
    if stage == "leaf_charges":    # per source: the (a, b, c) weight products, then comps x p^3 charges
        return n_sources * (comps * 2 * p ** 3 + (comps // 3) * (p ** 3 + p ** 2))
    if stage == "outgoing":        # per box and component: p^3 -> nh x n1 x n1 in three stages
        return fi["source_boxes"] * comps * (4 * p ** 3 * nh + 8 * p ** 2 * nh * n1 + 8 * p * nh * n1 * n1)
    if stage == "incoming":        # per box and velocity component: the reverse, real part kept
        return fi["target_boxes"] * 3 * (8 * nh * n1 * n1 * p + 8 * nh * n1 * p * p + 8 * nh * p ** 3)
    return None


def run_ours(args):
    import numpy as np
    import torch

    from paper_2509_21471_gb300 import dist as pdist
    world = pdist.world_size()
    rank = pdist.rank()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    pdist.init("nccl")

    from paper_2509_21471_gb300 import dmk, workloads as wl

    barrier = pdist.barrier
    max_over_ranks = pdist.max_over_ranks

    x_np, f_np = wl.clustered_3d(n=args.n, sigma=0.02, seed_index=pdist.seed_index(1))
    N = x_np.shape[0]
    x_h = torch.from_numpy(x_np).pin_memory()
    f_h = torch.from_numpy(f_np).pin_memory()
    u_h = torch.empty((N, 3), dtype=torch.float64).pin_memory()
    x_d = x_h.to("cuda")
    f_d = f_h.to("cuda")
    u_d = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def flush():
        flush_buf.fill_(1.0)

    def timed(fn, k):
        ms = []
        for _ in range(k):
            flush()
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            ms.append(e0.elapsed_time(e1))
        return ms

    # ---- leaf capacity of the full sum: the library's autotuner (plan + eval per candidate)
    tune = None
    if args.leaf_capacity:
        ns = args.leaf_capacity
    else:
        ns, tune = dmk.autotune(x_d, f_d, candidates=(1024, 2048, 3072, 4096, 6144), repeats=2, eps=args.eps,
                                precision=dmk.MIXED, components=dmk.ALL)
        ns = int(max_over_ranks(float(ns)))

    def step(prec):
        p = dmk.Plan(x_d, eps=args.eps, precision=prec, leaf_capacity=ns, components=dmk.ALL)
        p.eval(f_d, out=u_d)
        p.close()

    # ---- warm-up (both precisions: first-use costs of pools, tables and kernels)
    for _ in range(args.warmup):
        step(dmk.MIXED)
    step(dmk.FP64)
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms_mixed = timed(lambda: step(dmk.MIXED), args.steps)
    clocks = sampler.stop()
    t_mixed = max_over_ranks(sum(ms_mixed) / 1e3)
    value = pdist.job_rate(N, args.steps, t_mixed)

    ms_fp64 = timed(lambda: step(dmk.FP64), max(1, args.steps // 2))
    t_fp64 = max_over_ranks(sum(ms_fp64) / 1e3) / len(ms_fp64)

    # ---- evaluation alone (plan reused): stage times, near-field pair rates, far field
    evals = {}
    launches = None
    for name, prec in (("mixed", dmk.MIXED), ("fp64", dmk.FP64)):
        p = dmk.Plan(x_d, eps=args.eps, precision=prec, leaf_capacity=ns, components=dmk.ALL)
        l0 = p.stats()["launches"]
        p.eval(f_d, out=u_d)
        torch.cuda.synchronize()
        st = p.stats()
        if prec == dmk.MIXED:
            # kernels of one step: plan build + one eval (the pair count is not part of a step)
            launches = l0 + (st["launches"] - l0 - 1)
        k = args.steps if prec == dmk.MIXED else max(1, args.steps // 3)
        ms = timed(lambda: p.eval(f_d, out=u_d), k)
        t = max_over_ranks(sum(ms) / len(ms) / 1e3)
        stages = {}
        for _ in range(3 if prec == dmk.MIXED else 1):
            flush()
            torch.cuda.synchronize()
            _, tr = p.eval_traced(f_d, out=u_d)
            for key, v in tr.items():
                stages.setdefault(key, []).append(v)
        stages = {key: float(np.median(v)) for key, v in stages.items()}
        t_near = max_over_ranks(stages["near"] / 1e3)
        fi = p.far_info()
        evals[name] = dict(eval_ms=1e3 * t, stage_ms=stages, far_info=fi,
                           near_ms=1e3 * t_near, issued_pairs=st["issued_pairs"], useful_pairs=st["useful_pairs"],
                           gpairs_issued=st["issued_pairs"] / t_near / 1e9,
                           gpairs_useful=st["useful_pairs"] / t_near / 1e9,
                           leaves=st["leaves"], max_level=st["max_level"], tiles=st["tiles"], leaf_capacity=ns)
        p.close()

    # ---- the near-field pass alone at the paper's leaf capacity (plan + eval, components = NEAR)
    def near_step():
        p = dmk.Plan(x_d, eps=args.eps, precision=dmk.MIXED, leaf_capacity=0, components=dmk.NEAR)
        p.eval(f_d, out=u_d)
        p.close()
    near_step()
    t_near_step = max_over_ranks(sum(timed(near_step, args.steps)) / 1e3) / args.steps
    p = dmk.Plan(x_d, eps=args.eps, precision=dmk.MIXED, leaf_capacity=0, components=dmk.NEAR)
    p.eval(f_d, out=u_d)
    torch.cuda.synchronize()
    st_near = p.stats()
    t_near_only = max_over_ranks(sum(timed(lambda: p.eval(f_d, out=u_d), args.steps)) / args.steps / 1e3)
    p.close()
    near_only = {"ms_per_step": 1e3 * t_near_step, "targets_per_s": N / t_near_step,
                 "near_ms": 1e3 * t_near_only, "leaf_capacity": st_near["leaf_capacity"],
                 "useful_pairs": st_near["useful_pairs"], "issued_pairs": st_near["issued_pairs"],
                 "gpairs_useful": st_near["useful_pairs"] / t_near_only / 1e9}

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    # the forces travel on a second stream while the tree is built from x
    copy_stream = torch.cuda.Stream()

    def e2e_step():
        x_d.copy_(x_h, non_blocking=True)
        with torch.cuda.stream(copy_stream):
            f_d.copy_(f_h, non_blocking=True)
        f_ready = copy_stream.record_event()
        p = dmk.Plan(x_d, eps=args.eps, precision=dmk.MIXED, leaf_capacity=ns, components=dmk.ALL)
        torch.cuda.current_stream().wait_event(f_ready)
        p.eval(f_d, out=u_d)
        p.close()
        u_h.copy_(u_d, non_blocking=True)
    ms_e2e = timed(e2e_step, args.steps)
    t_e2e = max_over_ranks(sum(ms_e2e) / 1e3)
    e2e = {"value": pdist.job_rate(N, args.steps, t_e2e), "unit": "targets/s",
           "h2d_bytes_per_step": int(x_h.numel() * 8 + f_h.numel() * 8), "d2h_bytes_per_step": int(u_h.numel() * 8)}

    # ---- roofline of the dominant kernel: the far-field stage that takes longest
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = N_SM * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    peak_basis = (f"derived: {N_SM} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz "
                  "(max SM clock of MEASURED_PEAKS.json)")
    mx = evals["mixed"]
    kern_of = {"leaf_eval": "k_far_eval_tc (leaf grids at the targets, tcgen05)",
               "leaf_charges": "k_far_weights + k_far_values + k_far_anterp_tc (leaf proxy charges, tcgen05)",
               "outgoing": "k_far_out_fused (outgoing plane waves + kernel contraction)",
               "incoming": "k_far_ev_fused (incoming plane waves to the potential grids)"}
    stage_flops = {k: far_flops(k, mx["far_info"], N, N) for k in kern_of}
    near_tf = None
    if args.eps >= 2e-7:
        c32 = [len(dmk.kernel_table(3, args.eps, w, fp32=True)[2]) for w in (0, 1)]
        # Algorithmic flops (FMA = 2) of the symmetric Stokeslet pass: per unordered
        # pair the geometry, 1/r and both polynomials once (40 + 2(n_g - 1) + 2(n_h - 1),
        # including one application to a force) plus the second application (18);
        # useful_pairs counts ordered pairs, so per useful pair half of that.
        flops_one_side = 40 + 2 * (c32[0] - 1) + 2 * (c32[1] - 1)
        flops_per_pair = (flops_one_side + 18) / 2
        kern_of["near"] = "k_near_sym (symmetric near field, mixed precision)"
        stage_flops["near"] = mx["useful_pairs"] * flops_per_pair
        near_tf = stage_flops["near"] / (mx["stage_ms"]["near"] / 1e3) / 1e12
    dom = max(kern_of, key=lambda k: mx["stage_ms"][k])
    achieved = stage_flops[dom] / (mx["stage_ms"][dom] / 1e3) / 1e12
    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
    # capture of the same recipe at N = 5e5 and the same leaf capacity, scaled by the
    # point count
    traffic_5e5 = TRAFFIC_5E5.get((dom, ns)) if args.eps == 1e-6 else None
    traffic = traffic_5e5 * args.n / 500_000 if traffic_5e5 else None
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))

    def stage_dram(k):
        # DRAM GB/s of a stage against the measured HBM copy bandwidth: the ncu bytes of
        # the N = 5e5 capture at the same leaf capacity, scaled by the point count
        t5 = TRAFFIC_5E5.get((k, ns)) if args.eps == 1e-6 else None
        if not t5:
            return {}
        gbs = t5 * args.n / 500_000 / (mx["stage_ms"][k] / 1e3) / 1e9
        return {"dram_gbs": gbs, "hbm_frac": gbs / hbm_peak}

    # the two tcgen05 stages against the TF32 tensor peak: measured bf16 x the nominal
    # TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s dense); algorithmic flops, and the flops the
    # MMAs issue (three split-TF32 products, M padded to 128-row tiles, N to 16 columns)
    tf32_peak = float(peaks.get("bf16_tflops", 1900.0)) * 1.1 / 2.25
    fi = mx["far_info"]

    def stage_tensor(k):
        if k not in ("leaf_charges", "leaf_eval") or not fi["fp32"]:
            return {}
        p_ = fi["p"]
        if k == "leaf_charges":     # per source and group: 128-row tiles of p^2 x NP columns x 2 (FMA) x 3
            issued = N * ((p_ * p_ + 127) // 128 * 128) * ((3 * p_ + 15) // 16 * 16) * 2 * 3
        else:                       # per target: 3p rows of RW columns in 240-column blocks x RW (K) x 2 x 3
            rw = max(16, (p_ + 7) // 8 * 8)
            rb = 256 // rw
            while (rb * rw) % 16:
                rb -= 1
            issued = N * ((3 * p_ + rb - 1) // rb) * rb * rw * rw * 2 * 3
        t = mx["stage_ms"][k] / 1e3
        return {"engine": "tcgen05 kind::tf32, split-TF32 (3 MMAs per product)", "tf32_peak_tflops": tf32_peak,
                "tensor_frac_algorithmic": stage_flops[k] / t / 1e12 / tf32_peak,
                "tensor_frac_issued": issued / t / 1e12 / tf32_peak}

    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "traffic_note": "bytes per launch, ncu capture at N=5e5 (same leaf capacity) scaled by the point count",
                "kernel": kern_of[dom], "stage_ms": mx["stage_ms"][dom], "flops_per_launch": stage_flops[dom],
                "peak_basis": peak_basis, "fp32": bool(mx["far_info"]["fp32"]),
                "hbm_peak_gbs": hbm_peak, "hbm_peak_basis": "hbm_gbs of MEASURED_PEAKS.json (measured copy)",
                "all_stages": {k: {"ms": mx["stage_ms"][k],
                                   "tflops": stage_flops[k] / (mx["stage_ms"][k] / 1e3) / 1e12,
                                   "frac": stage_flops[k] / (mx["stage_ms"][k] / 1e3) / 1e12 / peak_tflops,
                                   **stage_dram(k), **stage_tensor(k)}
                               for k in kern_of}}
    if stage_tensor(dom):           # a tensor-core stage dominates: its own peak
        roofline.update(bound="tensor", peak=tf32_peak, frac=achieved / tf32_peak,
                        peak_basis="bf16_tflops of MEASURED_PEAKS.json x 1.1 / 2.25 (nominal TF32 / bf16)")
    if near_tf is not None:
        roofline["near_field"] = {"kernel": kern_of["near"], "achieved": near_tf, "frac": near_tf / peak_tflops,
                                  "flops_per_useful_pair": flops_per_pair, "flops_one_side": flops_one_side,
                                  "frac_at_one_sided_flops": near_tf * flops_one_side / flops_per_pair / peak_tflops}

    extras = None
    if not args.no_extras:
        extras = run_extras(args, dmk, wl, timed, max_over_ranks, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t1, tn, procs = oracle_timings(args.cpu_sample, args.eps, 256)
        cpu = {"value": args.cpu_sample / tn, "unit": "targets/s", "cores": procs, "kind": "oracle",
               "sample": f"same 8-Gaussian recipe at N={args.cpu_sample} points, leaf capacity 256: the oracle's "
                         f"whole DMK sum (tree, near pass, far field of Sec. 6), numpy with its threaded BLAS on "
                         f"every core, one run: {tn:.2f} s",
               "one_thread": {"value": args.cpu_sample / t1, "unit": "targets/s", "cores": 1, "seconds": t1}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_mixed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 (near pair terms compensated, far-field transforms f32; f64 self term, output)",
                "data": "synthetic", "config": workload_config(args, ns),
                "fp64": {"value": N * world / t_fp64, "unit": "targets/s", "ms_per_step": 1e3 * t_fp64},
                "speedup_mixed_over_fp64": t_fp64 / (t_mixed / args.steps),
                "autotune_ms_by_leaf_capacity": tune, "evaluation": evals, "near_field_pass_alone": near_only,
                "e2e": e2e, "gpu_launches": launches,
                "gpu_launches_note": "our kernels per step (plan + eval); CUB sort/scan kernels not counted",
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "other_workloads": extras}
        print(json.dumps(line), flush=True)
    pdist.finish()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.batched_only > 0:
        run_batched_only(args)
    elif args.ewald_only > 0:
        run_ewald_only(args)
    elif args.sweep:
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
