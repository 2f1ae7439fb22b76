"""Benchmark: gamma-solves/s of the convex clustering path on one B300.

One step = the whole hot path on one synthetic problem: build the exact
symmetrized kNN graph with Gaussian weights (ccm_build_graph) and solve the
warm-started gamma path to KKT <= 1e-6 and relative gap <= 1e-6 with labels
(ccm_solve_path). Default workload: the largest single-GPU one, a
100-component Gaussian mixture with n = 200,000 points in d = 50, k = 10,
phi = 0.5, 30 gammas in [1e-3, 1e2] (`--workload` selects another).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {ccm,reference}]

Prints one JSON line (rank 0). Under torchrun every rank solves its own
seeded problem (replicas: the path has no exchange step), so scaling is weak
and `value` sums the ranks' gamma-solves over the slowest rank's time.
`--impl reference` times the CPU oracle (plain float64 numpy/scipy) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "gmm200k_d50"
NOMINAL_HBM_GBS = 7700.0   # B300 HBM3e nominal bandwidth, for the second roofline denominator
TOL = 1e-6          # metric threshold on KKT and relative gap
SOLVE_TOL = 2e-7    # solver stop: tighter, so X is within 1e-6 of the oracle
METRIC = "gamma-solves/s at KKT<=1e-6 (graph build + path solve)"


def operator_kernel(d, precision="mixed"):
    """Name of the Newton-CG operator kernel the grid engine launches for rows of
    d features (the same dispatch as the library: rows of up to 16 quads use the
    register form, halved to two quads per lane from 8 lanes; longer rows the
    shared-memory ring form)."""
    tc = "float" if precision == "mixed" else "double"
    nq = -(-d // 4)
    if nq <= 16:
        lanes = 1
        while lanes < nq:
            lanes *= 2
        lanes, quads = (lanes // 2, 2) if lanes >= 8 else (lanes, 1)
        return f"k_cg_matvec<{lanes}, {quads}, {tc}>"
    return f"k_cg_matvec_ring<{-(-nq // 32)}, {tc}, 4>"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one operator
# launch from an ncu capture of the current kernel on the workload, per launch;
# every launch of the n = 200,000, phi = 0.5 path has every edge outside the
# ball, so one launch stands for all of them (profiles/k_cg_matvec_gmm200k_d50.md).
OPERATOR_TRAFFIC = {("gmm200k_d50", "mixed"): 628177920 + 42105088}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(",") for ln in self.f.read().splitlines() if ln.strip()]
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax = max(smax, float(r[1]))
                for nm, v in zip(names, r[3:7]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(seed, workload=None):
    A, _, wl = synth.make_workload(workload or WORKLOAD, seed)
    gam = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    return A, wl, gam


# Bounded samples of each recipe for the CPU oracle (points, gammas from the
# start of the grid; None = all), sized for about 5-15 s on one core so that the
# reference arm's 25 default driver steps end within a few minutes: the
# n = 200,000 recipe at phi = 0.5 barely fuses and the oracle solves 3,000 of its
# points over all 30 gammas in about 6 s; with phi = 1/median it fuses and 500
# points take about 11 s; on the MNIST-shaped recipe the 25th gamma alone takes
# about 45 s at 300 points, so that sample stops after 24.
ORACLE_SAMPLE = {"gmm200k_d50": (3000, None), "gmm200k_d50_medphi": (500, None),
                 "mnist10k_d784": (300, 24)}


def run_oracle_sample(seed):
    """CPU oracle on a bounded, fixed sample of the bench workload's recipe (the
    same work every call). Returns (gamma-solves/s, description, BLAS threads)."""
    import contextlib
    try:
        from threadpoolctl import threadpool_limits
        limit = threadpool_limits(limits=1)
        threads = 1
    except ImportError:             # not installed: BLAS keeps its default threads
        limit = contextlib.nullcontext()
        threads = os.cpu_count() or 1

    from oracle import graph as og
    from oracle import ssnal as osn
    n_s, n_gamma = ORACLE_SAMPLE.get(WORKLOAD, (500, None))
    A, _, wl = synth.make_workload(WORKLOAD, seed, n=min(n_s, synth.WORKLOADS[WORKLOAD].n))
    gam = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    gam_s = gam[:n_gamma] if n_gamma else gam
    with limit:
        t0 = time.perf_counter()
        edges, w, _ = og.build_graph(A, wl.k, wl.phi)
        X = U = None
        sigma = 1.0
        for g in gam_s:
            # same penalty cap as the library's default for q = 2; iteration caps
            # keep one gamma bounded
            X, U, sigma, _ = osn.solve(A, edges, w, g, X, U, sigma, tol=TOL, sigma_max=10.0,
                                       max_outer=100, max_newton=30)
        el = time.perf_counter() - t0
    done = len(gam_s)
    return done / el, (f"oracle graph + SSNAL path on n={A.shape[0]} points of the {WORKLOAD} "
                       f"recipe (d={A.shape[1]}, k={wl.k}), first {done} of {len(gam)} gammas, "
                       f"tol 1e-6, {el:.1f} s, BLAS threads {threads}"), threads


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        run_oracle_sample(0)
    desc = ""
    t_all = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        v, desc, thr = run_oracle_sample(0)
        t_all += time.perf_counter() - t0
        vals.append(v)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "gamma-solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * t_all / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "gamma-solves/s", "cores": thr,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "gamma-solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def job_rate(ms_local, units_per_rank, dist=None, device="cpu"):
    """Whole-job throughput of a replicated run: every rank processed
    `units_per_rank` units in its own `ms_local` milliseconds; the job took the
    slowest rank's time (MAX over ranks). Returns (units per second, job ms)."""
    import torch
    ms = float(ms_local)
    world = 1
    if dist is not None and dist.is_initialized():
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        world = dist.get_world_size()
    return world * units_per_rank / (ms / 1000.0), ms


def _time(fn, stream, reps=1):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def form_batched(args):
    """Batched form: 256 independent problems (n ~ U{500..5000}, d = 16) in one
    persistent launch, against a loop of plain ccm_solve_path calls (grid
    engine) on the same GPU, same tolerance."""
    import torch
    import paper_2501_15964_b300 as ccm
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    probs = synth.batched_problems(0, count=args.batch)
    gam = probs[0]["gammas"]
    dev = []
    for p in probs:
        A = torch.tensor(p["A"], device="cuda")
        E, w, _ = ccm.build_graph(A, p["k"], p["phi"])
        dev.append(dict(A=A, edges=E, w=w))
    T = len(gam)
    for _ in range(max(1, args.warmup)):
        ccm.solve_path_batched(dev, gam, tol=SOLVE_TOL)
    ms_b, (Xs, Ls, st) = _time(lambda: ccm.solve_path_batched(dev, gam, tol=SOLVE_TOL), stream,
                               args.steps)
    flat = [s for ps in st for s in ps]
    nloop = min(args.loop, len(dev))

    shape = ccm.last_profile()
    shape = {"lanes": shape["block_lanes"], "quads_per_lane": shape["block_quads"]}

    def loop():  # each problem with the engine ccm_solve_path picks by itself (AUTO)
        for p in dev[:nloop]:
            ccm.solve_path(p["A"], p["edges"], p["w"], gam, tol=SOLVE_TOL, engine=0)
    loop()
    ms_l, _ = _time(loop, stream, 1)
    ms_sub, _ = _time(lambda: ccm.solve_path_batched(dev[:nloop], gam, tol=SOLVE_TOL), stream, 1)
    line = {"form": "batched", "metric": "gamma-solves/s, batched vs loop of plain solves",
            "unit": "gamma-solves/s", "problems": len(dev), "gammas": T, "tol": SOLVE_TOL,
            "batched_value": len(dev) * T / (ms_b / 1000), "batched_ms": ms_b,
            "loop_problems": nloop, "loop_value": nloop * T / (ms_l / 1000), "loop_ms": ms_l,
            "batched_same_subset_value": nloop * T / (ms_sub / 1000),
            "speedup_same_subset": ms_l / ms_sub, "autotuned_shape": shape,
            "max_kkt": max(s["kkt"] for s in flat), "max_gap": max(s["gap"] for s in flat),
            "not_converged": sum(1 for s in flat if s["status"] != 0)}
    print(json.dumps(line), flush=True)
    return 0


def form_vjp(args):
    """Adjoint form: dL/dA and dL/dw of sum_t ||X*(gamma_t) - T||^2 on the
    n = 20,000, d = 64 workload, against two plain path solves (the cost of
    one central-difference direction)."""
    import torch
    import paper_2501_15964_b300 as ccm
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    A, _, wl = synth.make_workload("gmm20k_d64", 0)
    gam = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    T = torch.tensor(synth.adjoint_target(0, A.shape[0], A.shape[1]), device="cuda")
    At = torch.tensor(A, device="cuda")
    E, w, _ = ccm.build_graph(At, wl.k, wl.phi)
    X, _, _, st = ccm.solve_path(At, E, w, gam, tol=SOLVE_TOL)
    G = 2.0 * (X - T)
    ccm.path_vjp(At, E, w, gam, X, G)
    ms_s, _ = _time(lambda: ccm.solve_path(At, E, w, gam, tol=SOLVE_TOL), stream, args.steps)
    ms_v, _ = _time(lambda: ccm.path_vjp(At, E, w, gam, X, G), stream, args.steps)
    line = {"form": "adjoint", "metric": "VJP time vs two plain path solves", "unit": "ms",
            "workload": "gmm20k_d64", "n": int(A.shape[0]), "d": int(A.shape[1]),
            "edges": int(E.shape[0]), "gammas": len(gam), "path_solve_ms": ms_s,
            "vjp_ms": ms_v, "two_solves_over_vjp": 2 * ms_s / ms_v,
            "clusters": [s["n_clusters"] for s in st]}
    print(json.dumps(line), flush=True)
    return 0


def form_admm(args):
    """ADMM and fast AMA (the paper's other two solvers) against SSNAL on the
    same GPU, grid engine, same tolerance: the n = 200, d = 2 workload (20 gammas)."""
    import torch
    import paper_2501_15964_b300 as ccm
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    A, _, wl = synth.make_workload("gmm200_d2", 0)
    gam = synth.gamma_grid(wl.gamma_lo, wl.gamma_hi, wl.n_gamma)
    At = torch.tensor(A, device="cuda")
    E, w, _ = ccm.build_graph(At, wl.k, wl.phi)
    runs = {}
    for name, fn in (("ssnal", ccm.solve_path), ("admm", ccm.solve_path_admm),
                     ("ama", ccm.solve_path_ama)):
        fn(At, E, w, gam, tol=SOLVE_TOL, engine=1)
        ms, (_, _, _, st) = _time(lambda: fn(At, E, w, gam, tol=SOLVE_TOL, engine=1), stream,
                                  args.steps)
        runs[name] = {"ms": ms, "value": len(gam) / (ms / 1000.0),
                      "iterations": sum(s["outer"] for s in st), "cg": sum(s["cg"] for s in st),
                      "max_kkt": max(s["kkt"] for s in st), "max_gap": max(s["gap"] for s in st),
                      "not_converged": sum(1 for s in st if s["status"] != 0)}
    line = {"form": "admm", "metric": "gamma-solves/s, SSNAL vs ADMM vs fast AMA (grid engine)",
            "unit": "gamma-solves/s", "workload": "gmm200_d2", "gammas": len(gam),
            "tol": SOLVE_TOL, "ssnal": runs["ssnal"], "admm": runs["admm"], "ama": runs["ama"],
            "ssnal_over_admm": runs["admm"]["ms"] / runs["ssnal"]["ms"],
            "ssnal_over_ama": runs["ama"]["ms"] / runs["ssnal"]["ms"]}
    print(json.dumps(line), flush=True)
    return 0


def form_qnorm(args):
    """Model CCM with q = 1 (l1 norm on x_i - x_j) and q = inf (max norm) against
    q = 2 on the bench workload: graph build + path, same tolerance,
    device-resident."""
    import torch
    import paper_2501_15964_b300 as ccm
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    A, wl, gam = make_problem(0, args.workload)
    if args.n_gamma > 0:
        gam = gam[: args.n_gamma]
    At = torch.tensor(A, device="cuda")
    out = {}
    for q in args.qs.split(","):
        def step():
            E, w, _ = ccm.build_graph(At, wl.k, wl.phi)
            kw = {"sigma_max": args.sigma_max} if args.sigma_max > 0 else {}
            return ccm.solve_path(At, E, w, gam, q=q, tol=SOLVE_TOL, **kw)
        if args.warmup > 0:
            step()
        ms, (_, _, _, st) = _time(step, stream, args.steps)
        out[f"q{q}"] = {"value": len(gam) / (ms / 1000.0), "ms": ms,
                        "newton": sum(s["newton"] for s in st), "cg": sum(s["cg"] for s in st),
                        "max_kkt": max(s["kkt"] for s in st), "max_gap": max(s["gap"] for s in st),
                        "not_converged": sum(1 for s in st if s["status"] != 0),
                        "clusters_last_gamma": st[-1]["n_clusters"],
                        "newton_per_gamma": [s["newton"] for s in st],
                        "cg_per_gamma": [s["cg"] for s in st]}
        print(json.dumps({"form": "qnorm", "workload": args.workload, "q": q, **out[f"q{q}"]}),
              flush=True)
    line = {"form": "qnorm", "metric": "gamma-solves/s for q = " + args.qs + " (graph build + path)",
            "unit": "gamma-solves/s", "workload": args.workload, "gammas": len(gam),
            "tol": SOLVE_TOL, "sigma_max": args.sigma_max if args.sigma_max > 0 else "default",
            **out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ccm", choices=["ccm", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS),
                    help="synthetic workload (default: the MNIST-shaped one)")
    ap.add_argument("--n-gamma", type=int, default=0,
                    help="solve only the first N gammas of the path (profiling runs)")
    ap.add_argument("--sigma-max", type=float, default=0.0,
                    help="penalty cap passed to the solver in the qnorm form (0: library default)")
    ap.add_argument("--qs", default="2,1,inf",
                    help="comma-separated q values of the qnorm form (1, 2, inf)")
    ap.add_argument("--gamma-from", type=int, default=0,
                    help="start the path at this index of the gamma grid, cold (profiling runs)")
    ap.add_argument("--form", default="path",
                    choices=["path", "batched", "adjoint", "admm", "qnorm"],
                    help="path (default, the JSON contract line), or the batched, adjoint, "
                         "ADMM / fast AMA or q-norm (q = 2, 1, inf) comparison")
    ap.add_argument("--batch", type=int, default=256, help="problems in the batched form")
    ap.add_argument("--loop", type=int, default=32,
                    help="problems solved one by one for the batched comparison")
    args = ap.parse_args()
    globals()["WORKLOAD"] = args.workload
    if args.form == "batched":
        return form_batched(args)
    if args.form == "adjoint":
        return form_vjp(args)
    if args.form == "admm":
        return form_admm(args)
    if args.form == "qnorm":
        return form_qnorm(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    import paper_2501_15964_b300 as ccm

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    prec = 1 if args.precision == "mixed" else 0
    A, wl, gam = make_problem(rank)
    gam = gam[args.gamma_from:]
    if args.n_gamma > 0:
        gam = gam[: args.n_gamma]
    T = len(gam)
    dev = torch.device("cuda", local)
    A_dev = torch.tensor(A, device=dev)
    A_host = torch.tensor(A).pin_memory()
    stream = torch.cuda.current_stream()

    def step(A_in, X_out=None, labels_host=None):
        E, w, _ = ccm.build_graph(A_in, wl.k, wl.phi)
        X, lab, _, stats = ccm.solve_path(A_in, E, w, gam, tol=SOLVE_TOL, precision=prec,
                                          profile=1, X_out=X_out, labels_host=labels_host)
        return X, lab, stats, E

    for _ in range(args.warmup):
        step(A_dev)
    barrier()

    # device-resident timed region
    l0 = ccm.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    mv_ms = mv_bytes = mv_n = 0.0
    stats_all = []
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            X, lab, stats, E = step(A_dev)
            p = ccm.last_profile()
            mv_ms += p["matvec_ms_total"]
            mv_bytes += p["matvec_bytes_total"]
            mv_n += p["matvec_launches"]
            stats_all.append(stats)
        ev1.record(stream)
        barrier()
    launches = ccm.launch_count() - l0
    value, ms = job_rate(ev0.elapsed_time(ev1), T * args.steps, dist, dev)

    # end-to-end through the public API with host buffers: pinned host A -> device,
    # full path with X and labels written to pinned host memory by the library
    # (each gamma's X is copied out while the next gamma solves)
    X_host = torch.empty((T, A.shape[0], A.shape[1]), dtype=torch.float64).pin_memory()
    L_host = torch.empty((T, A.shape[0]), dtype=torch.int32).pin_memory()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        A_in = A_host.to(dev, non_blocking=True)
        step(A_in, X_out=X_host, labels_host=L_host)
    e1.record(stream)
    barrier()
    e2e, ems = job_rate(e0.elapsed_time(e1), T * args.steps, dist, dev)

    if rank == 0:
        peak, peak_kind = _peaks()
        achieved = (mv_bytes / 1e9) / (mv_ms / 1000.0) if mv_ms > 0 else None
        flat = [s for st in stats_all for s in st]
        line = {
            "metric": METRIC, "value": value, "unit": "gamma-solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (CG operator f32)" if prec == 1 else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": int(A.shape[0]), "d": int(A.shape[1]),
                       "k": wl.k, "phi": (wl.phi if wl.phi > 0 else "1/median"), "gammas": T, "tol": SOLVE_TOL,
                       "edges": int(E.shape[0]),
                       "l2": "inputs larger than L2 (per-step working set > 1 GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": operator_kernel(A.shape[1], args.precision),
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "frac_of_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "launches_timed": int(mv_n),
                         "ms_per_step": mv_ms / args.steps,
                         "traffic": OPERATOR_TRAFFIC.get((WORKLOAD, args.precision)),
                         "algorithmic_bytes_per_launch": (mv_bytes / mv_n) if mv_n else None},
            "e2e": {"value": e2e, "unit": "gamma-solves/s",
                    "h2d_bytes_per_step": int(A.nbytes),
                    "d2h_bytes_per_step": int(X_host.numel() * 8 + L_host.numel() * 4)},
            "gpu_launches": int(launches),
            "solver": {"max_kkt": max(s["kkt"] for s in flat),
                       "max_gap": max(s["gap"] for s in flat),
                       "not_converged": sum(1 for s in flat if s["status"] != 0),
                       "newton_per_step": sum(s["newton"] for s in flat) / args.steps,
                       "cg_per_step": sum(s["cg"] for s in flat) / args.steps,
                       "clusters_last_gamma": flat[-1]["n_clusters"]},
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            v, desc, thr = run_oracle_sample(0)
            line["cpu_baseline"] = {"value": v, "unit": "gamma-solves/s", "cores": thr,
                                    "kind": "oracle", "sample": desc}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
