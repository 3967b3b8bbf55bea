"""Benchmark: BP3 (H1 diffusion) Jacobi-PCG throughput, GDOF/s per CG iteration.

One step = one pass of the whole hot path over one synthetic problem:
geometry setup D from the (device-resident) vertices, load vector of the sine
manufactured solution, matrix-free diagonal, and the solve (every CG iteration
applies the fused G^T B^T D B G kernel).  Each solver form is run to the same
accuracy: a solution within --target-err (1e-10, relative l2) of a reference
solution of the same discrete problem (FP64 CG with an FP64 p-multigrid V-cycle and
the native binary64 operator, to a residual of 1e-13); its outer tolerance is the
loosest of --rtol * 10^(k/2) that achieves this, found before the timed steps and checked on every
warm-up step (tightened while a warm-up step misses the target: the FP32 forms' iteration counts vary
from run to run); `solution_rel_err_max_checked` is the largest error of those steps and the last one.
Forms: the mixed-precision one (FP64 iterative refinement around an FP32
Jacobi-PCG; the headline `value`), the plain FP64 Jacobi-PCG (`fp64_plain`), the
mixed-precision CG with reliable updates (`mixed_reliable`) and FP64 CG preconditioned
with an FP32 p-multigrid V-cycle (`mg_pcg_fp32_vcycle`).  A second BP3 case (p=6 on
32^3 elements, `bp3_p6_n32`) and short runs of the 512-problem batch (`batch`) and of
the served stream (`serve`) ride on the same line.
value = N * (CG iterations) / step time, summed over ranks (independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import fem_inputs as FI  # noqa: E402

METRIC = "BP3 GDOF/s per CG iter (FP64 vs mixed+refine)"
UNIT = "GDOF/s"


def workload_name(p, n, q, stop="solution within 1e-10 (relative l2) of a reference solve"):
    N = (p * n + 1) ** 3
    return (f"BP3 diffusion, p={p}, q={q}, {n}^3 perturbed trilinear hexes (+-0.1h), N={N} DOFs, "
            f"sine manufactured RHS, homogeneous Dirichlet, {stop}")


def flops_per_elem(n, q, form):
    """Algorithmic flops of one element's sum-factorised action (standard 3-stage
    contractions forward and transposed, plus the pointwise D)."""
    if form == "mass":
        return 4 * n * q * (n * n + n * q + q * q) + q ** 3
    return 2 * (4 * n ** 3 * q + 6 * n * n * q * q + 6 * n * q ** 3) + 15 * q ** 3


def bytes_per_elem(n, q, form, p, nelem_per_dim, word=8):
    """Algorithmic HBM bytes of one action per element: D, the element->DOF map and
    x/y once per global DOF (word = 8 for FP64, 4 for FP32 data)."""
    ncomp = 6 if form == "diffusion" else 1
    N = (p * nelem_per_dim + 1) ** 3
    E = nelem_per_dim ** 3
    return word * ncomp * q ** 3 + 4 * n ** 3 + 2.0 * word * N / E


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # samples go to BENCH_CLOCK_DIR if set (to keep them), else to the temporary directory
        out = os.environ.get("BENCH_CLOCK_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smmax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smmax), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def reduce_max_sum(t, work, dist=None, device="cpu"):
    """Whole-job aggregation over independent replicas: the slowest rank's time and the
    total work of all ranks (one all-reduce each; no data-path collective)."""
    if dist is None:
        return float(t), float(work)
    import torch
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    ww = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(ww, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(ww[0])


# nominal FP64 rate of the B300 (no FP64 tensor-core path); the FP64 pipe bounds this kernel
FP64_PEAK_GFLOPS = 1250.0
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture) of the
# current apply kernels on the default workload: captured at 40^3 elements (412.9 / 413.0 MB FP32
# variants 1 / 2, 413.0 MB variant 1 with (d, A d) fused -- re-taken with the packed-FMA build, same
# bytes --, 795.3 MB double-float in packed pairs with its exponent-range test: the algorithmic
# bytes, y read once for the atomics) and scaled to 64^3 by elements (D, map) and DOFs (x, y).
# Only reported when that kernel is timed.
NCU_TRAFFIC_P4_N64 = {"f32_v1": 1.6910e9, "f32_v2": 1.6916e9, "f32dot_v1": 1.6914e9, "df": 3.2589e9}
# ceiling of the double-float FP64 action: 12 FP32-pipe instructions per FP64-accurate
# multiply-add (exact product by FMA, TwoSum accumulation) on 128 FP32 lanes/SM x 148 SMs
# at 2.032 GHz, 2 flops per multiply-add
DF_PEAK_GFLOPS = 2 * 128 * 148 * 2.032 / 12


# ----------------------------------------------------------------------------- oracle arm

def oracle_sample(p, n_sample, seed=0):
    """One bounded sample of the workload on the CPU oracle: same p, form, mesh recipe
    and solver, on n_sample^3 elements.  Returns (DOF-iterations, seconds, iterations)."""
    import oracle as O
    t0 = time.perf_counter()
    mesh = O.HexGridMesh(n_sample, n_sample, n_sample, FI.perturbed_cube_vertices(n_sample, n_sample, n_sample,
                                                                                   seed=seed))
    prob = O.Problem(mesh, p, None, O.DIFFUSION)
    b = prob.sine_rhs()
    x, it, res = prob.solve(b, rtol=1e-10)
    dt = time.perf_counter() - t0
    return prob.N * it, dt, it


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return 1


def run_reference(args, rank, world):
    """The oracle as it stands, on this host's cores, on a bounded sample of the BP3
    workload (same p, recipe and solver on --oracle-n^3 elements instead of --n^3)."""
    if rank != 0:
        return 0
    p, n_s = args.p, args.oracle_n
    for _ in range(args.warmup):
        oracle_sample(p, n_s)
    tot_dofit, tot_t, its = 0, 0.0, []
    for _ in range(args.steps):
        d, t, it = oracle_sample(p, n_s)
        tot_dofit += d
        tot_t += t
        its.append(it)
    value = tot_dofit / tot_t / 1e9
    sample = (f"oracle (CSR assembly by quadrature + Jacobi PCG to 1e-10, numpy/scipy with their default thread "
              f"pools) on {n_s}^3 elements, p={p}, N={(p * n_s + 1) ** 3}, a bounded sample of the {args.n}^3 "
              f"workload; timed: assembly, load vector, solve")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(p, n_s, p + 2, "Jacobi PCG to a 1e-10 residual")
                                   + f" (CPU sample of the {args.n}^3 workload)",
                       "full_workload": workload_name(p, args.n, p + 2), "sample": sample},
            "iterations": its,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle", "sample": sample,
                             "host_nproc": os.cpu_count(), "host_cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm

def bp3_case(args, p, n, rank, world, dist, steps, forms, with_e2e, with_roofline=True):
    """Time the BP3 sine problem (p, n^3 elements) for the solver forms in `forms` ("mixed",
    "fp64", "reliable", "mg") on one device.  Each form's outer tolerance is first tightened from
    --rtol until its solution is within --target-err (relative l2) of a reference solution of the
    same discrete problem (see reference_solution), so that the forms are compared at equal
    accuracy; then `steps` steps are timed.  Returns {form: results} and the reference's stats."""
    import torch

    import paper_2402_15940_b300 as F

    local = int(os.environ.get("LOCAL_RANK", "0"))
    verts_np = FI.perturbed_cube_vertices(n, n, n, seed=rank)
    op = F.Operator(n, n, n, verts_np, p, form="diffusion")
    q, N, E = op.q, op.N, op.E
    op.set_essential(op.boundary_dofs())
    op.set_cg_mode(args.cg_mode)
    if args.f32_variant >= 0:   # pin the kernels (e.g. under a profiler, whose timing misleads the autotuner)
        op.set_f32_variant(args.f32_variant)
    if args.f64_variant >= 0:
        op.set_f64_variant(args.f64_variant)
    op.set_fused_dot(args.fused_dot)
    verts = torch.from_numpy(verts_np).cuda()
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    scale = 3 * math.pi ** 2

    def barrier():
        if dist is not None:
            dist.barrier()

    def aggregate(t, work):
        return reduce_max_sum(t, work, dist, device="cuda")

    mg = {}

    def solve(prec, rtol):
        if prec == "fp64":
            _, st = op.solve(b, x, rtol=rtol, maxit=args.maxit)
            return st["iterations"], st
        if prec == "mg":
            _, st = mg["mg"].solve(b, x, rtol=rtol, maxit=args.maxit)
            return st["iterations"], st
        if prec == "reliable":
            _, st = op.solve_reliable(b, x, rtol=rtol, delta=args.delta)
            return st["inner_iterations"], st
        _, st = op.solve_refined(b, x, rtol=rtol, inner_rtol=args.inner_rtol)
        return st["inner_iterations"], st

    def step(prec, rtol):
        op.set_vertices(verts)          # D from the trilinear map (a1)
        if prec == "mg":
            if "mg" not in mg:
                mg["mg"] = F.Multigrid(op, smooth_degree=2, coarse_degree=24, precision="fp32")
            else:
                mg["mg"].update()       # every level follows the mesh: D, diagonals, eigenvalue bounds
        op.rhs_sine(scale, out=b)       # load vector (a11)
        x.zero_()
        return solve(prec, rtol)        # diagonal (a10) + PCG (a9; a2-a8 in every iteration)

    def reference_solution():
        """The same discrete problem solved by another solver in native FP64: CG preconditioned
        by an FP64 p-multigrid V-cycle, with the DFMA (binary64) operator action, to a relative
        residual of --ref-rtol.  Its own FP64 residual b - A x_ref is reported beside it."""
        rop = F.Operator(n, n, n, verts_np, p, form="diffusion")
        rop.set_essential(rop.boundary_dofs())
        rop.set_f64_variant(0)
        rmg = F.Multigrid(rop, smooth_degree=2, coarse_degree=24, precision="fp64")
        rb = rop.rhs_sine(scale)
        xr, st = rmg.solve(rb, rtol=args.ref_rtol, maxit=500)
        res = torch.linalg.norm(rb - rop.apply(xr)) / torch.linalg.norm(rb)
        info = {"solver": f"FP64 CG + FP64 p-multigrid V-cycle, native binary64 (DFMA) operator, rtol "
                          f"{args.ref_rtol}", "iterations": st["iterations"], "true_rel_residual": float(res)}
        del rmg, rop
        return xr, info

    xref, ref_info = reference_solution() if args.target_err > 0 else (None, None)

    def sol_err():
        if xref is None:
            return None
        return float(torch.linalg.norm(x - xref) / torch.linalg.norm(xref))

    def calibrate(prec):
        """The loosest outer tolerance, of --rtol * 10^(k/2) for k = --rtol-search, ..., 1, 0, -1, ...,
        whose solution is within --target-err of the reference (each form at the accuracy the
        target asks for, no tighter); these solves also warm the form up."""
        if xref is None:
            step(prec, args.rtol)
            return args.rtol, []
        tried = []
        k = args.rtol_search
        while True:
            rt = args.rtol * 10.0 ** (k / 2.0)
            step(prec, rt)
            e = sol_err()
            tried.append({"rtol": rt, "solution_rel_err": e})
            if e <= args.target_err or k <= -8:
                return rt, tried
            k -= 1

    def timed(prec):
        rtol, tried = calibrate(prec)
        # the warm-up steps also check the accuracy at that tolerance: the FP32 forms' iteration
        # counts vary from run to run (the order of the FP32 scatter's atomic additions), so a
        # tolerance that met the target once can miss it; then it is tightened one step (10^-1/2)
        # and the warm-up repeated
        checked = []
        for _ in range(4):
            errs = []
            for _ in range(args.warmup):
                step(prec, rtol)
                errs.append(sol_err())
            checked += errs
            if xref is None or not errs or max(errs) <= args.target_err:
                break
            rtol /= 10.0 ** 0.5
            tried.append({"rtol": rtol, "tightened_after_warmup_errors": errs})
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        l0 = F.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its, stats = [], []
        with ClockSampler(local) as clk:
            ev0.record()
            for _ in range(steps):
                it, st = step(prec, rtol)
                its.append(it)
                stats.append(st)
            ev1.record()
            torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches = F.launch_count() - l0
        t, work = aggregate(ev0.elapsed_time(ev1) / 1e3, N * sum(its))
        return {"value": work / t / 1e9, "ms_per_step": 1e3 * t / steps, "iterations_per_step": its,
                "gpu_launches": launches, "clocks": clk.summary(), "stats": stats[-1], "rtol": rtol,
                "solution_rel_err": sol_err(),
                "solution_rel_err_max_checked": max([e for e in checked + [sol_err()] if e is not None], default=None),
                "rtol_search": tried}

    def kernel_time(prec, reps=20):
        if prec == "fp64":
            xr = torch.from_numpy(FI.uniform_vector(N, seed=1)).cuda()
            fn = lambda out: op.apply(xr, out=out)  # noqa: E731
            yr = torch.empty_like(xr)
        else:
            xr = torch.from_numpy(FI.uniform_vector(N, seed=1).astype(np.float32)).cuda()
            if args.fused_dot:   # the build the CG loop runs: the action with (d, A d) fused
                xax = torch.empty(1, dtype=torch.float64, device="cuda")
                fn = lambda out: op.apply_f32_dot(xr, out=out, xax=xax)  # noqa: E731
            else:
                fn = lambda out: op.apply_f32(xr, out=out)  # noqa: E731
            yr = torch.empty_like(xr)
        for _ in range(3):
            fn(yr)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        k0.record()
        for _ in range(reps):
            fn(yr)
        k1.record()
        torch.cuda.synchronize()
        return k0.elapsed_time(k1) / 1e3 / reps

    def e2e(prec, rtol, k):
        vh = torch.from_numpy(verts_np).pin_memory().numpy()
        bh = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        op.set_vertices(verts)
        op.rhs_sine(scale, out=b)
        bh[:] = b.cpu().numpy()
        xh = torch.zeros(N, dtype=torch.float64).pin_memory().numpy()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        its = 0
        for _ in range(k):
            op.set_vertices(vh)
            xh[:] = 0.0
            if prec == "fp64":
                _, st = op.solve_host(bh, xh, rtol=rtol, maxit=args.maxit)
                its += st["iterations"]
            else:
                _, st = op.solve_refined_host(bh, xh, rtol=rtol, inner_rtol=args.inner_rtol)
                its += st["inner_iterations"]
        torch.cuda.synchronize()
        te, work = aggregate(time.perf_counter() - t0, N * its)
        return {"value": work / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(vh.nbytes + 2 * bh.nbytes),
                "d2h_bytes_per_step": int(xh.nbytes), "ms_per_step": 1e3 * te / k, "steps": k}

    hbm_peak, hbm_src = peaks()
    results = {}
    for prec in forms:
        r = timed(prec)
        results[prec] = r
        if prec not in ("mixed", "fp64") or not with_roofline:
            continue
        t_apply = kernel_time(prec)
        if prec == "fp64":
            fl = flops_per_elem(p + 1, q, "diffusion") * E
            ach = fl / t_apply / 1e9
            v64, vname = op.f64_variant()
            if v64 in (1, 2):   # double-float (full- or half-size blocks)
                traffic = args.traffic_fp64
                if traffic is None and (p, n) == (4, 64):
                    traffic = NCU_TRAFFIC_P4_N64["df"]
                r["roofline"] = {"bound": "alu", "achieved": ach, "peak": DF_PEAK_GFLOPS, "unit": "GFLOP/s",
                                 "frac": ach / DF_PEAK_GFLOPS, "traffic": traffic,
                                 "kernel": f"pa_apply_df<{p},{q},diffusion> ({vname}, autotuned)",
                                 "apply_ms": 1e3 * t_apply,
                                 "peak_note": "FP64-accurate flops at the FP32 pipe's rate / 12 instructions per "
                                              "multiply-add (128 lanes x 148 SMs x 2.032 GHz; derived)",
                                 "vs_fp64_pipe_peak": ach / FP64_PEAK_GFLOPS}
            else:
                r["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                                 "frac": ach / FP64_PEAK_GFLOPS, "traffic": args.traffic_fp64,
                                 "kernel": f"pa_apply<double,{p},{q},diffusion> ({vname}, autotuned)",
                                 "apply_ms": 1e3 * t_apply,
                                 "peak_note": "FP64 pipe: nominal 1.25 TFLOP/s (2 DFMA/clk/SM x 148 SMs)"}
            op.set_f64_variant(0)           # the DFMA kernel on the same input, for comparison
            t_dfma = kernel_time(prec)
            op.set_f64_variant(args.f64_variant)   # back to the measured (or pinned) choice
            r["dfma_kernel"] = {"kernel": f"pa_apply<double,{p},{q},diffusion>", "apply_ms": 1e3 * t_dfma,
                                "achieved": fl / t_dfma / 1e9, "unit": "GFLOP/s",
                                "frac_of_fp64_pipe": fl / t_dfma / 1e9 / FP64_PEAK_GFLOPS}
            r["arithmetic"] = ("FP64-accurate double-float on the FP32 pipe (autotuned)" if v64 in (1, 2) else
                               "native binary64 (DFMA, autotuned)")
        else:
            by = bytes_per_elem(p + 1, q, "diffusion", p, n, word=4) * E
            ach = by / t_apply / 1e9
            fl = flops_per_elem(p + 1, q, "diffusion") * E
            traffic = args.traffic_fp32
            if traffic is None and (p, n) == (4, 64):
                traffic = NCU_TRAFFIC_P4_N64.get(f"f32{'dot' if args.fused_dot else ''}_v{op.f32_variant()[0]}")
            r["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                             "frac": ach / hbm_peak, "traffic": traffic,
                             "kernel": f"pa_apply_f32_tma<{p},{q},diffusion> variant {op.f32_variant()[0]} "
                                       f"({op.f32_variant()[1]}, autotuned)"
                                       + (", (d, A d) fused; timed with its slot collection" if args.fused_dot else ""),
                             "apply_ms": 1e3 * t_apply,
                             "peak_note": f"HBM copy bandwidth ({hbm_src})",
                             "frac_of_nominal_8tbs": ach / 8000.0,
                             "fp32_tflops": fl / t_apply / 1e12}
        r["apply_gdofs"] = N / t_apply / 1e9
        if with_e2e:
            # the headline form end to end every step; the FP64 form on a few steps (its solves are long)
            k = steps if prec == "mixed" else min(steps, 3)
            r["e2e"] = e2e(prec, r["rtol"], k)
    del op, mg
    torch.cuda.empty_cache()
    return results, ref_info, (N, E, q)


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_cpu_baseline(p, n_s):
    """The oracle as it stands on this host: once limited to one thread and once with its
    libraries' thread pools opened to every core (numpy's BLAS parallelises the element
    matrices; scipy's sparse products stay on one thread)."""
    out = {}
    try:
        from threadpoolctl import threadpool_limits
    except Exception:
        threadpool_limits = None
    for label, lim in (("single_thread", 1), ("all_cores", os.cpu_count() or 1)):
        if threadpool_limits is not None:
            with threadpool_limits(limits=lim):
                th = cpu_threads()
                d, t, it = oracle_sample(p, n_s)
        else:
            d, t, it = oracle_sample(p, n_s)
            th = cpu_threads()
        out[label] = {"value": d / t / 1e9, "seconds": t, "threads": th, "iterations": it}
    return out


def run_ours(args, rank, world, dist):
    import torch

    import paper_2402_15940_b300 as F

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    p, n = args.p, args.n
    forms = [f for f in ("mg", "reliable", "mixed", "fp64")
             if (f != "mg" or args.multigrid) and (f != "reliable" or args.reliable)
             and (f not in ("mixed", "fp64") or args.precision in (f, "both"))]
    results, ref_info, (N, E, q) = bp3_case(args, p, n, rank, world, dist, args.steps, forms,
                                            with_e2e=not args.no_e2e)
    second = None
    if args.p2 > 0:
        k2 = min(args.steps, args.steps2)
        res2, ref2, (N2, E2, q2) = bp3_case(args, args.p2, args.n2, rank, world, dist, k2,
                                            [f for f in ("mixed", "fp64") if f in forms], with_e2e=False)
        second = {"workload": workload_name(args.p2, args.n2, q2), "steps": k2, "reference": ref2}
        for f, r in res2.items():
            second[f] = {k: r.get(k) for k in ("value", "ms_per_step", "iterations_per_step", "rtol",
                                                 "solution_rel_err", "solution_rel_err_max_checked", "roofline",
                                                 "apply_gdofs", "gpu_launches", "clocks", "arithmetic")}
        if "mixed" in res2 and "fp64" in res2:
            second["time_to_solution_speedup_vs_fp64"] = res2["fp64"]["ms_per_step"] / res2["mixed"]["ms_per_step"]

    extras = {}
    if args.extras and world == 1:
        # the operator sweep at its largest size (~3e7 DOFs per order and form); first, so that its
        # operators' variant choices are not the ones timed while the served stream kept the GPU busy
        extras["sweep"] = run_sweep(args, rank, world, dist, targets=(3e7,), quiet=True)
        extras["batch"] = run_batch(args, rank, world, dist, steps=min(args.steps, 2), warmup=1, quiet=True)
        extras["serve"] = run_serve(args, rank, world, dist, rates=[float(args.serve_rate)], quiet=True,
                                    solver="jacobi")
        # the same stream with the p-multigrid preconditioner for the large diffusion requests
        extras["serve_pmg"] = run_serve(args, rank, world, dist, rates=[float(args.serve_rate)], quiet=True,
                                        solver="auto")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_cpu_baseline(p, args.oracle_n)
        allc = cb["all_cores"]
        cpu = {"value": allc["value"], "unit": UNIT, "cores": allc["threads"], "kind": "oracle",
               "sample": f"oracle CSR assembly + Jacobi PCG to 1e-10 on {args.oracle_n}^3 elements, p={p}, "
                         f"N={(p * args.oracle_n + 1) ** 3}, {allc['iterations']} iterations, "
                         f"{allc['seconds']:.1f} s with the libraries' thread pools opened to all cores",
               "single_thread": cb["single_thread"], "host_nproc": os.cpu_count(), "host_cpu": cpu_model()}

    if rank == 0:
        head = results.get("mixed") or results["fp64"]
        mixed = "mixed" in results
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64 (FP32 operator and inner CG, FP64 refinement residual/dots/scalars/setup)"
                         if mixed else "f64",
                "data": "synthetic",
                "config": {"workload": workload_name(p, n, q),
                           "precision": "mixed+refine" if mixed else "fp64",
                           "solver": (f"FP64 iterative refinement around FP32 Jacobi-PCG (inner rtol "
                                      f"{args.inner_rtol}), outer rtol {head['rtol']:.3g}: the loosest of "
                                      f"{args.rtol:g}*10^(k/2) whose solution is within {args.target_err:g} of the "
                                      f"reference solution") if mixed else f"FP64 Jacobi-PCG to rtol {head['rtol']:.3g}",
                           "accuracy_target": {"solution_rel_err": args.target_err, "reference": ref_info},
                           "cg_loop": args.cg_mode,
                           "l2": "inputs larger than L2 (D alone is %.2f GB)" % (E * 6 * q ** 3 * 8 / 1e9),
                           "parallelism": "independent replicas, one per GPU" if world > 1 else "single GPU"},
                "iterations_per_step": head["iterations_per_step"], "roofline": head["roofline"],
                "solution_rel_err": head["solution_rel_err"],
                "solution_rel_err_max_checked": head.get("solution_rel_err_max_checked"),
                "cpu_baseline": cpu, "e2e": head.get("e2e"), "gpu_launches": head["gpu_launches"],
                "clocks": head["clocks"]}
        if mixed:
            line["refine_stats"] = head["stats"]
        if "mg" in results:
            m = results["mg"]
            line["mg_pcg_fp32_vcycle"] = {
                "solver": "FP64 CG preconditioned by a p-multigrid V-cycle (p=4,2,1; Chebyshev-Jacobi degree 2, "
                          "coarsest degree 24) run in FP32; set-up (levels' D, diagonals, eigenvalue bounds) "
                          "inside every step",
                "ms_per_step": m["ms_per_step"], "iterations_per_step": m["iterations_per_step"],
                "gdofs_per_cg_iter": m["value"], "gpu_launches": m["gpu_launches"], "rtol": m["rtol"],
                "solution_rel_err": m["solution_rel_err"],
                "solution_rel_err_max_checked": m.get("solution_rel_err_max_checked")}
            if "fp64" in results:
                line["mg_pcg_fp32_vcycle"]["time_to_solution_speedup_vs_fp64"] = (
                    results["fp64"]["ms_per_step"] / m["ms_per_step"])
        if "reliable" in results:
            m = results["reliable"]
            line["mixed_reliable"] = {
                "solver": f"one FP32 Jacobi-PCG recurrence, residual replaced by the FP64 residual each time it "
                          f"falls by {args.delta} (reliable updates; direction and scalars kept)",
                "ms_per_step": m["ms_per_step"], "iterations_per_step": m["iterations_per_step"],
                "gdofs_per_cg_iter": m["value"], "gpu_launches": m["gpu_launches"],
                "replacements": m["stats"]["outer_iterations"], "rel_residual": m["stats"]["rel_residual"],
                "rtol": m["rtol"], "solution_rel_err": m["solution_rel_err"],
                "solution_rel_err_max_checked": m.get("solution_rel_err_max_checked")}
            if "fp64" in results:
                line["mixed_reliable"]["time_to_solution_speedup_vs_fp64"] = (
                    results["fp64"]["ms_per_step"] / m["ms_per_step"])
        if mixed and "fp64" in results:
            f64 = results["fp64"]
            line["fp64_plain"] = {k: f64.get(k) for k in ("value", "ms_per_step", "iterations_per_step", "roofline",
                                                           "dfma_kernel", "e2e", "apply_gdofs", "gpu_launches",
                                                           "clocks", "rtol", "solution_rel_err",
                                                           "solution_rel_err_max_checked", "arithmetic")}
            line["time_to_solution_speedup_vs_fp64"] = f64["ms_per_step"] / head["ms_per_step"]
            line["speedup_note"] = "both forms at solution error <= %g against the reference" % args.target_err
        if second is not None:
            line["bp3_p%d_n%d" % (args.p2, args.n2)] = second
        for k, v in extras.items():
            line[k] = v
        print(json.dumps(line), flush=True)
    return 0


def run_batch(args, rank, world, dist, steps=None, warmup=None, quiet=False):
    """512 independent problems (mass or diffusion with probability 1/2, p uniform in
    1..6, elements per direction uniform in 2..24, seeded perturbed cubes, random nodal
    right-hand sides with zero boundary rows for diffusion) solved together by FP64
    Jacobi-PCG to 1e-10 in one graph-driven batch.  One step = one batched solve
    (diagonal + PCG); the batch set-up (maps, D) is timed separately.  With quiet=True the
    line is returned (for the default run's extra key) instead of printed."""
    import torch

    import paper_2402_15940_b300 as F

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    mix = FI.problem_mix(args.batch_count, seed=rank)
    probs = [{"n": m["n"], "p": m["p"], "form": m["form"],
              "vertices": FI.perturbed_cube_vertices(*m["n"], seed=m["mesh_seed"])} for m in mix]
    t0 = time.perf_counter()
    bt = F.Batch(probs)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    bh = FI.uniform_vector(bt.N, seed=11 + rank)
    for i, pr in enumerate(probs):
        if pr["form"] == "diffusion":
            nx, ny, nz = pr["n"]
            Nx, Ny, Nz = pr["p"] * nx + 1, pr["p"] * ny + 1, pr["p"] * nz + 1
            g = np.arange(Nx * Ny * Nz)
            gx, gy, gz = g % Nx, (g // Nx) % Ny, g // (Nx * Ny)
            on = (gx == 0) | (gy == 0) | (gz == 0) | (gx == Nx - 1) | (gy == Ny - 1) | (gz == Nz - 1)
            bh[bt.offsets[i] + g[on]] = 0.0
    b = torch.from_numpy(bh).cuda()
    x = torch.zeros(bt.N, dtype=torch.float64, device="cuda")

    def step():
        x.zero_()
        _, st = bt.solve(b, x, rtol=args.rtol, maxit=args.maxit)
        return st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    l0 = F.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dofit, maxits = 0.0, []
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(steps):
            st = step()
            dofit += st["dof_iterations"]
            maxits.append(int(st["max_iterations"]))
        ev1.record()
        torch.cuda.synchronize()
    t, work = reduce_max_sum(ev0.elapsed_time(ev1) / 1e3, dofit, dist, device="cuda")
    launches64 = F.launch_count() - l0

    # the same batch by batched mixed-precision refinement (FP32 corrections, FP64 residuals)
    def step_refined():
        x.zero_()
        _, st = bt.solve_refined(b, x, rtol=args.rtol, inner_rtol=args.inner_rtol)
        return st

    for _ in range(warmup):
        step_refined()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    l1 = F.launch_count()
    dofit32, maxin, outer = 0.0, [], []
    with ClockSampler(local) as clk32:
        ev0.record()
        for _ in range(steps):
            st = step_refined()
            dofit32 += st["dof_iterations"]
            maxin.append(int(st["max_inner_iterations"]))
            outer.append(int(st["outer_iterations"]))
        ev1.record()
        torch.cuda.synchronize()
    t32, work32 = reduce_max_sum(ev0.elapsed_time(ev1) / 1e3, dofit32, dist, device="cuda")

    # and by batched reliable updates (per-problem FP32 recurrences, FP64 residual replacement)
    def step_reliable():
        x.zero_()
        _, st = bt.solve_reliable(b, x, rtol=args.rtol, delta=args.delta)
        return st

    for _ in range(warmup):
        step_reliable()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    l2 = F.launch_count()
    dofitr, maxr, repl = 0.0, [], []
    with ClockSampler(local) as clkr:
        ev0.record()
        for _ in range(steps):
            st = step_reliable()
            dofitr += st["dof_iterations"]
            maxr.append(int(st["max_inner_iterations"]))
            repl.append(int(st["outer_iterations"]))
        ev1.record()
        torch.cuda.synchronize()
    tr, workr = reduce_max_sum(ev0.elapsed_time(ev1) / 1e3, dofitr, dist, device="cuda")
    reliable = {"solver": "batched FP32 Jacobi-PCG recurrences with FP64 residual replacement each time they "
                          f"fall by {args.delta} (reliable updates), one CUDA-graph loop per segment",
                "ms_per_step": 1e3 * tr / steps, "solves_per_s": args.batch_count * world * steps / tr,
                "gdofs_per_fp32_iter": workr / tr / 1e9, "max_inner_iterations_per_step": maxr,
                "replacements_per_step": repl, "time_to_solution_speedup_vs_fp64": t / tr,
                "gpu_launches": F.launch_count() - l2, "clocks": clkr.summary()}
    refined = {"solver": "FP64 iterative refinement (per-problem FP64 residual and stop) around batched FP32 "
                         f"Jacobi-PCG corrections (inner rtol {args.inner_rtol}), one CUDA-graph loop per step",
               "ms_per_step": 1e3 * t32 / steps, "solves_per_s": args.batch_count * world * steps / t32,
               "gdofs_per_fp32_iter": work32 / t32 / 1e9, "max_inner_iterations_per_step": maxin,
               "outer_iterations_per_step": outer, "time_to_solution_speedup_vs_fp64": t / t32,
               "gpu_launches": F.launch_count() - l1, "clocks": clk32.summary()}
    if rank == 0:
        line = {"metric": "batched BP1/BP3 solves: GDOF/s per CG iter", "value": work / t / 1e9, "unit": UNIT,
                "n_gpus": world, "steps": steps, "warmup": warmup,
                "ms_per_step": 1e3 * t / steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{args.batch_count} independent problems, form mass|diffusion (p=0.5), "
                                       "p~U{1..6}, n_d~U{2..24}, perturbed cubes, random nodal RHS, "
                                       "FP64 Jacobi-PCG to 1e-10, one CUDA-graph batch",
                           "total_dofs": bt.N, "groups": bt.groups},
                "solves_per_s": args.batch_count * world * steps / t,
                "max_iterations_per_step": maxits, "setup_s": setup_s,
                "gpu_launches": launches64, "clocks": clk.summary(), "mixed_refined": refined,
                "mixed_reliable": reliable,
                # the autotuner's picks per (p, form) group: FP64 action (0 DFMA, 1 double-float,
                # 2 double-float in half-size tiles) and the FP32 tile's elements per block
                "autotune_picks": [{**g, "f64_kernel": F.load_library().fepa_f64_variant_name(g["f64_variant"]).decode()}
                                   for g in bt.group_info()]}
        if quiet:
            return line
        print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, rank, world, dist, targets=(1e5, 1e6, 3e7), quiet=False):
    """Operator-action sweep (BP1 mass and BP3 diffusion, p = 1..8, q = p+2, seeded perturbed
    cubes, x ~ U[-1, 1]) at about 1e5, 1e6 and 3e7 DOFs (targets): single-application GDOF/s of
    the FP64-accurate action (autotuned kernel) and of the FP32 action, and GDOF/s per Jacobi-PCG
    iteration (FP64, all boundary DOFs essential for diffusion), each against its roofline.
    quiet: return the line (rank 0) instead of printing it."""
    import torch

    import paper_2402_15940_b300 as F

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    hbm_peak, hbm_src = peaks()

    def ev_time(fn, reps):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    rows = []
    t_start = time.perf_counter()
    for p in range(1, 9):
        for form in ("mass", "diffusion"):
            for target in targets:
                n = max(1, int(round((target ** (1.0 / 3.0) - 1) / p)))
                op = F.Operator(n, n, n, FI.perturbed_cube_vertices(n, n, n, seed=rank), p, form=form)
                q, N, E = op.q, op.N, op.E
                x = torch.from_numpy(FI.uniform_vector(N, seed=1)).cuda()
                y = torch.empty_like(x)
                t64 = ev_time(lambda: op.apply(x, out=y), 20)
                x32, y32 = x.float(), torch.empty(N, dtype=torch.float32, device="cuda")
                t32 = ev_time(lambda: op.apply_f32(x32, out=y32), 20)
                v64 = op.f64_variant()[0]
                fl = flops_per_elem(p + 1, q, form) * E
                by64 = bytes_per_elem(p + 1, q, form, p, n, word=8) * E
                by32 = bytes_per_elem(p + 1, q, form, p, n, word=4) * E
                alu_peak = DF_PEAK_GFLOPS if v64 in (1, 2) else FP64_PEAK_GFLOPS
                # roofline of the FP64-accurate action: the slower of its ALU ceiling and HBM
                roof64 = min(alu_peak * 1e9 / (fl / E), hbm_peak * 1e9 / (by64 / E)) * N / E
                if form == "diffusion":
                    op.set_essential(op.boundary_dofs())
                b = op.rhs_sine(1.0)
                xs = torch.zeros(N, dtype=torch.float64, device="cuda")
                it_lo, it_hi = 10, 60
                t_lo = ev_time(lambda: op.iterations(b, xs.zero_(), it_lo), 1)
                t_hi = ev_time(lambda: op.iterations(b, xs.zero_(), it_hi), 1)
                t_it = max(t_hi - t_lo, 1e-9) / (it_hi - it_lo)
                rows.append({
                    "p": p, "form": form, "n": n, "ndofs": N,
                    "fp64_action": {"kernel": op.f64_variant()[1], "ms": 1e3 * t64, "gdofs": N / t64 / 1e9,
                                    "gflops": fl / t64 / 1e9, "frac_alu": fl / t64 / 1e9 / alu_peak,
                                    "gbs": by64 / t64 / 1e9, "frac_hbm": by64 / t64 / 1e9 / hbm_peak,
                                    "frac_roofline": (N / t64) / roof64},
                    "fp32_action": {"variant": op.f32_variant()[0], "ms": 1e3 * t32, "gdofs": N / t32 / 1e9,
                                    "gbs": by32 / t32 / 1e9, "frac_hbm": by32 / t32 / 1e9 / hbm_peak},
                    "fp64_cg_iteration": {"ms": 1e3 * t_it, "gdofs": N / t_it / 1e9}})
                del op, x, y, x32, y32, b, xs
                torch.cuda.empty_cache()
    if rank == 0:
        big = [r for r in rows if r["p"] == 4 and r["form"] == "diffusion"][-1]
        line = {"metric": "BP1/BP3 operator sweep: GDOF/s per FP64-accurate application", "value":
                big["fp64_action"]["gdofs"], "unit": UNIT, "n_gpus": world, "steps": 20, "warmup": 3,
                "ms_per_step": big["fp64_action"]["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 (double-float or DFMA, autotuned) | f32", "data": "synthetic",
                "config": {"workload": "p = 1..8, mass and diffusion, q = p+2, perturbed cubes at ~"
                                       + ", ".join("%.0e" % t for t in targets)
                                       + " DOFs, x ~ U[-1,1]; value = diffusion p=4 at the largest size",
                           "peaks": {"hbm_gbs": hbm_peak, "hbm_source": hbm_src, "df_gflops": DF_PEAK_GFLOPS,
                                     "fp64_gflops": FP64_PEAK_GFLOPS}},
                "sweep": rows, "wall_s": time.perf_counter() - t_start}
        if quiet:
            return line
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank, world, dist, rates=None, quiet=False, solver=None):
    """Served solve stream: for each arrival rate, `--requests` requests (mass or
    diffusion, p uniform in 1..8, DOFs log-uniform in 1e3..5e6, FP64 or mixed with
    refinement to 1e-10, seeded perturbed cubes, sine RHS) arrive as a Poisson process
    and are served with continuous batching under an HBM budget.  solver "jacobi": every
    request by Jacobi-PCG (mixed: FP32 Jacobi-PCG in FP64 refinement); "auto": diffusion
    requests of at least --pmg-min-dofs DOFs by CG with the p-multigrid V-cycle (FP64, or
    FP32 for the mixed ones)."""
    solver = args.serve_solver if solver is None else solver
    import torch

    from paper_2402_15940_b300 import launch_count
    from paper_2402_15940_b300.serve import GpuExecutor, Request, Server, poisson_arrivals

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # the requests' meshes are their own input data: generated before the timed region (as the
    # batch's are), so the served time covers building the ops from them, not drawing them
    spec0 = FI.serve_requests(args.requests, seed=100 * rank)
    meshes = {(tuple(s["n"]), s["mesh_seed"]): FI.perturbed_cube_vertices(*s["n"], seed=s["mesh_seed"])
              for s in spec0}
    vf = lambda n, seed: meshes[(tuple(n), seed)]  # noqa: E731
    rates = [float(r) for r in args.rates.split(",")] if rates is None else rates
    per_rate = []
    l0 = launch_count()
    with ClockSampler(local) as clk:
        for k, rate in enumerate(rates):
            spec = FI.serve_requests(args.requests, seed=100 * rank)   # same requests at every rate
            reqs = [Request(rid=i, form=s["form"], p=s["p"], n=s["n"], mesh_seed=s["mesh_seed"],
                            precision=s["precision"]) for i, s in enumerate(spec)]
            poisson_arrivals(reqs, rate=rate, seed=k)
            srv = Server(GpuExecutor(vf, priorities=args.serve_priorities, async_start=args.serve_async,
                                     workers=args.serve_workers),
                         hbm_budget=args.hbm_budget, tick_iters=args.tick_iters, policy=args.serve_policy,
                         solver=solver, pmg_min_dofs=args.pmg_min_dofs,
                         tick_seconds=args.tick_seconds if args.tick_seconds > 0 else None)
            srv.run(reqs)
            rep = srv.report()
            rep["rate"] = rate
            per_rate.append(rep)
    if rank == 0:
        top = max(per_rate, key=lambda r: r["solves_per_s"])
        line = {"metric": "served solves/s, p50/p99 latency", "value": top["solves_per_s"], "unit": "solves/s",
                "n_gpus": world, "steps": len(rates), "warmup": 0, "ms_per_step": 1e3 * top["makespan_s"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 | f32+f64",
                "data": "synthetic",
                "config": {"workload": f"{args.requests} requests per rate, Poisson arrivals, mass|diffusion, "
                                       "p~U{1..8}, DOFs log-uniform 1e3..5e6, FP64 or mixed+refine (1/2 each) "
                                       "to 1e-10, continuous batching; meshes generated before the timed region",
                           "hbm_budget_bytes": args.hbm_budget,
                           "solver": ("Jacobi-PCG (mixed: FP32 Jacobi-PCG in FP64 refinement)" if solver == "jacobi"
                                      else f"diffusion requests of >= {args.pmg_min_dofs} DOFs: FP64 CG with the "
                                           "p-multigrid V-cycle (FP32 V-cycle for the mixed ones); others Jacobi-PCG"),
                           "tick_iters": args.tick_iters, "policy": args.serve_policy,
                           "stream_priorities": args.serve_priorities, "async_start": args.serve_async,
                           "creation_workers": args.serve_workers,
                           "tick_seconds": args.tick_seconds},
                "per_rate": per_rate, "gpu_launches": launch_count() - l0, "clocks": clk.summary()}
        if quiet:
            return line
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--oracle-n", type=int, default=12)
    ap.add_argument("--precision", choices=["mixed", "fp64", "both"], default="both")
    ap.add_argument("--cg-mode", choices=["graph", "stream"], default="graph",
                    help="graph: CG loop in one CUDA graph (default); stream: plain launches (for profiling)")
    ap.add_argument("--inner-rtol", type=float, default=1e-4)
    ap.add_argument("--delta", type=float, default=0.03, help="reliable-update replacement factor")
    ap.add_argument("--f32-variant", type=int, default=-1, help="pin the FP32 action's launch shape (-1: autotune)")
    ap.add_argument("--f64-variant", type=int, default=-1, help="pin the FP64 action (0 DFMA, 1 double-float)")
    ap.add_argument("--no-reliable", dest="reliable", action="store_false",
                    help="skip the reliable-update mixed solve")
    ap.add_argument("--no-multigrid", dest="multigrid", action="store_false",
                    help="skip the p-multigrid preconditioned form")
    ap.add_argument("--traffic-fp64", type=float, default=None, help="DRAM bytes per FP64 apply launch (ncu)")
    ap.add_argument("--traffic-fp32", type=float, default=None, help="DRAM bytes per FP32 apply launch (ncu)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fused-dot", dest="fused_dot", action="store_false",
                    help="FP32 CG: (d, A d) by a separate pass instead of from the action kernel")
    ap.add_argument("--workload", choices=["bp3", "batch", "serve", "sweep"], default="bp3")
    ap.add_argument("--rates", default="10,100,1000,5000")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--hbm-budget", type=float, default=150e9)
    ap.add_argument("--tick-iters", type=int, default=32)
    ap.add_argument("--tick-seconds", type=float, default=2e-3,
                    help="serve: estimated GPU time per advance of a request (0: always --tick-iters)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--target-err", type=float, default=1e-10,
                    help="solution error (relative l2, against the reference solve) every BP3 form is run to; "
                         "0: stop at --rtol without a reference")
    ap.add_argument("--ref-rtol", type=float, default=1e-13, help="relative residual of the reference solve")
    ap.add_argument("--rtol-search", type=int, default=6,
                    help="the tolerance search starts at --rtol * 10^(k/2) with this k and tightens by sqrt(10)")
    ap.add_argument("--p2", type=int, default=6, help="second BP3 case: order (0 skips it)")
    ap.add_argument("--n2", type=int, default=32, help="second BP3 case: elements per direction")
    ap.add_argument("--steps2", type=int, default=5, help="second BP3 case: at most this many timed steps")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the short batch and serve runs of the default line")
    ap.add_argument("--serve-rate", type=float, default=1000.0, help="arrival rate of the default line's serve run")
    ap.add_argument("--serve-solver", choices=["jacobi", "auto"], default="jacobi",
                    help="--workload serve: Jacobi-PCG for every request, or p-multigrid CG for large diffusion ones")
    ap.add_argument("--pmg-min-dofs", type=int, default=50000,
                    help="smallest diffusion request solved with the p-multigrid preconditioner (--serve-solver auto)")
    ap.add_argument("--serve-policy", choices=["fifo", "sjf"], default="fifo",
                    help="admission order of waiting requests (arrival order, or least estimated work first)")
    ap.add_argument("--serve-workers", type=int, default=2,
                    help="host threads that build the requests' ops (with asynchronous start)")
    ap.add_argument("--serve-sync-start", dest="serve_async", action="store_false",
                    help="build each request's op on the scheduler thread (default: on a worker thread)")
    ap.add_argument("--no-serve-priorities", dest="serve_priorities", action="store_false",
                    help="every request on a normal-priority stream (default: short requests on high-priority ones)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        if args.workload == "batch":
            return run_batch(args, rank, world, dist)
        if args.workload == "serve":
            return run_serve(args, rank, world, dist)
        if args.workload == "sweep":
            return run_sweep(args, rank, world, dist)
        return run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
