#!/usr/bin/env python
"""Benchmark of the preconditioned ECS Helmholtz solve (one step = one full solve from x = 0 to a
relative residual of 1e-8, FP64 FGMRES right-preconditioned by one complex64 multigrid cycle on
the complex-scaled-grid operator, theta_a = pi/10, the angle a sweep over pi/17 .. pi/6 picks for
these workloads).  Workloads (seeded, synthetic):

  2d-well-n1025  1025 x 1025 nodes, k^2 = 2(E - V) with a Gaussian well and growth toward the
                 boundary so that k h <= 0.6, ECS at pi/6 beyond |x|, |y| = 0.75, random source
                 on |x|_inf < 0.5; FGMRES(30), V(2,2) omega-Jacobi 0.8 (the headline)
  3d-well-n257   the same in 3D on 257^3 nodes, 7-point stencil, FGMRES(20)
  batch-64       64 independent 2D problems, sizes from {129, 257, 513, 1025}, energies in
                 [0.5, 4], Gaussian sources, solved together (helm_solve_batch)

Prints one JSON line for the chosen workload: value = unknowns solved per second over all
ranks (Mdof/s), with the plain FP64 solve beside it, the dominant kernel class's roofline, the
CPU oracle as a baseline (single-threaded and on all host cores), an end-to-end number through
the public API with host buffers, and the SM clocks sampled during the timed region.  With the
default workload the line also carries the other two workloads, measured the same way in
shorter runs, under "other_configs" (--no-extra skips them).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 2d-well-n1025|3d-well-n257|batch-64] [--no-extra]

Under torchrun every rank solves its own independent problem (seed + rank) or its shard of the
batch: no collective touches the data path.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "preconditioned solve time to rel. residual 1e-8 and Mdof/s, mixed vs FP64; HBM GB/s % peak"
UNIT = "Mdof/s"
SM_COUNT = 152
FP64_FMA_PER_SM_CLK = 2  # GB300: 1.25 TFLOP/s FP64 at 2.07 GHz over 152 SMs = 2 FMA / SM / clock
WORKLOADS = ("2d-well-n1025", "3d-well-n257", "batch-64")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOADS[0], choices=WORKLOADS)
    ap.add_argument("--n", type=int, default=0, help="grid nodes per axis (0 = the workload's own)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="do not attach the other workloads to the line")
    ap.add_argument("--cpu-iters", type=int, default=0, help="oracle iterations in the CPU sample (0 = auto)")
    ap.add_argument("--batch", type=int, default=0, metavar="COUNT",
                    help="batch-64 workload with COUNT problems instead of 64")
    ap.add_argument("--no-tune", action="store_true", help="default kernel choices instead of the autotuned ones")
    ap.add_argument("--gs", default="dcgs2", choices=["dcgs2", "df", "fp64"],
                    help="Arnoldi arithmetic of the mixed solve (see helm_gs_arith)")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="ITERS",
                    help="profiling case: build the workload's problem and run one solve capped at ITERS "
                         "iterations, nothing else (keeps the launch count small enough for ncu)")
    ap.add_argument("--ncu-precond", type=int, default=0, metavar="CALLS",
                    help="profiling case: build the workload's hierarchy only (no Krylov workspace) and run CALLS "
                         "preconditioner applications (one complex64 cycle each), nothing else")
    ap.add_argument("--cpu-leg", default=None, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def dist_env():
    from paper_1012_4307_gb300.distributed import rank_env
    return rank_env()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def problem(workload, n=0, seed_offset=0):
    from paper_1012_4307_gb300 import workloads as W
    if workload == "2d-well-n1025":
        return W.config_2d_well(n or 1025, seed=1 + seed_offset)
    if workload == "3d-well-n257":
        return W.config_3d_well(n or 257, seed=2 + seed_offset)
    raise ValueError(workload)


# ---------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for r in csv.reader(fh):
                if len(r) >= 9:
                    rows.append([c.strip() for c in r])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------- CPU oracle
def oracle_iterations(name):
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")) as fh:
            d = json.load(fh)
        return d[name]["iterations"]
    except (OSError, KeyError, ValueError):
        return None


def cpu_leg_main(spec):
    """Child process of the CPU baseline (no CUDA): times the oracle's FP64 FGMRES(restart) with
    its FP64 cycle for spec["iters"] iterations on the workload's full problem and prints
    {"sec_per_iter", "iterations", "seconds", "threads"}.  The oracle build (single-threaded or
    all cores) comes from HELM_ORACLE_OPENMP in the environment."""
    from oracle import oracle as O
    from paper_1012_4307_gb300 import workloads as W
    O.build()
    if spec.get("batch_n"):
        P = W.Problem("b", 2, spec["batch_n"], W.k2_well_growth(2, spec["batch_n"], E=2.0),
                      W.gaussian_source(2, spec["batch_n"], 0.05, 3), coarsest_n=17, restart=30, tol=1e-8,
                      theta_a=W.WELL_THETA_A)
    else:
        P = problem(spec["workload"], spec.get("n", 0))
    z = O.axes(P.dim, P.n, theta=P.theta, r0lo=-P.r0, r0hi=P.r0)
    A, M = O.helmholtz_ops(z, P.k2, pc=P.pc, theta_a=P.theta_a)
    mg = O.MG(M, P.coarsest_n, P.nu1, P.nu2, P.omega, P.smoother)
    t0 = time.perf_counter()
    x, st = O.fgmres(A, mg, P.f, tol=spec["tol"], restart=P.restart, maxit=spec["iters"])
    dt = time.perf_counter() - t0
    print(json.dumps({"sec_per_iter": dt / max(st["iterations"], 1), "iterations": st["iterations"], "seconds": dt,
                      "threads": O.threads()}), flush=True)


def run_cpu_leg(spec, all_cores):
    """Runs cpu_leg_main in a fresh CPU-only process (spawned, so no CUDA state is inherited)."""
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    env["HELM_ORACLE_OPENMP"] = "1" if all_cores else "0"
    if all_cores:
        env["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    else:
        env.pop("OMP_NUM_THREADS", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", json.dumps(spec)], env=env,
                       capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("CPU oracle leg failed: %s" % r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(P, tol, iters, iterations_needed, source, single=True, full_solve=False):
    """The oracle (plain C, FP64 FGMRES with its FP64 cycle) timed on the host: on all cores, a
    complete solve to tol (full_solve) or a bounded sample of iters iterations projected to
    iterations_needed; and (single) one core, a sample of iters iterations projected."""
    spec = {"workload": "3d-well-n257" if P.dim == 3 else "2d-well-n1025", "n": P.n, "tol": tol}
    allc = run_cpu_leg(dict(spec, iters=5000 if full_solve else iters), all_cores=True)
    if full_solve:
        solve_all = allc["seconds"]
        what = "one complete FGMRES(%d) solve to %.0e (%d iterations)" % (P.restart, tol, allc["iterations"])
    else:
        solve_all = allc["sec_per_iter"] * iterations_needed
        what = ("%d FGMRES(%d) iterations, %.1f s, projected to the %d iterations of a full solve (%s)"
                % (allc["iterations"], P.restart, allc["seconds"], iterations_needed, source))
    out = {"value": P.unknowns / solve_all / 1e6, "unit": UNIT, "cores": allc["threads"], "kind": "oracle",
           "projected": not full_solve,
           "sample": "plain C FP64 oracle (FP64 V(%d,%d) CSG cycle, OpenMP over independent node loops, serial "
                     "reductions) on the full %s problem on %d host cores: %s"
                     % (P.nu1, P.nu2, P.name, allc["threads"], what),
           "seconds_per_iteration": allc["sec_per_iter"], "solve_s": solve_all}
    if single:
        one = run_cpu_leg(dict(spec, iters=iters), all_cores=False)
        solve_one = one["sec_per_iter"] * iterations_needed
        out["single_core"] = {"value": P.unknowns / solve_one / 1e6, "cores": 1, "projected": True,
                              "seconds_per_iteration": one["sec_per_iter"], "projected_solve_s": solve_one,
                              "sample": "%d iterations, %.1f s on one core, projected to %d iterations"
                                        % (one["iterations"], one["seconds"], iterations_needed)}
    return out


# ---------------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm is the CPU oracle (the paper ships no code), on all host cores.  For the
    2D workloads every timed step is one complete oracle solve to the tolerance (measured, not
    projected); warm-up steps run a 2-iteration sample.  The 3D workload (about 2.4 s per oracle
    iteration even on all cores) times a one-iteration sample per step, projected to the FP64 GPU
    solve's iteration count."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    wl = args.workload
    if wl == "batch-64" or args.batch:
        print(json.dumps({"impl": "reference", "unavailable": "the batch workload has no oracle arm: its problems "
                          "are independent single solves, each covered by the 2d-well arm"}), flush=True)
        return
    P = problem(wl, args.n)
    full = P.dim == 2
    secs, its, threads = [], [], 1
    for s in range(args.warmup + args.steps):
        timed = s >= args.warmup
        iters = 5000 if (full and timed) else (2 if P.dim == 2 else 1)
        r = run_cpu_leg({"workload": wl, "n": P.n, "tol": args.tol, "iters": iters}, all_cores=True)
        threads = r["threads"]
        if timed:
            secs.append(r["seconds"] if full else r["sec_per_iter"])
            its.append(r["iterations"])
    if full:
        solve_s = statistics.mean(secs)
        sample = ("each timed step: one complete FGMRES(%d) solve of the plain C FP64 oracle (FP64 V(2,2) CSG "
                  "cycle) to %.0e on the full problem, %d iterations, on %d host cores (OpenMP over independent "
                  "node loops, serial reductions); warm-up steps: 2-iteration samples" % (P.restart, args.tol, its[-1],
                                                                                         threads))
        projected = False
    else:
        it_needed = oracle_iterations(P.name) or 31
        solve_s = statistics.mean(secs) * it_needed
        sample = ("each step: one FGMRES(%d) iteration of the plain C FP64 oracle on the full problem on %d host "
                  "cores, projected to %d iterations" % (P.restart, threads, it_needed))
        projected = True
    value = P.unknowns / solve_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": solve_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": P.name, "unknowns": P.unknowns,
                       "solver": "FGMRES(%d), FP64 V(2,2) CSG cycle, theta_a=pi/%.3g" % (P.restart, math.pi / P.theta_a),
                       "tol": args.tol},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "projected": projected,
                             "sample": sample}}
    print(json.dumps(line), flush=True)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant
# kernels, from the ncu captures summarised under profiles/.  Reported only while the kernel's
# source file is the one that was captured (same SHA-1); otherwise null.
NCU_TRAFFIC = {
    ("2d-well-n1025", "update_norm"): dict(kernel="k_update2_pair", source="paper_1012_4307_gb300/csrc/kernels_gs_df.cu",
                                           sha1="093841d405022c73eadc49970ff88b158dc8bcf7", bytes=314093312,
                                           launch="basis slot j = 15, the mean over a restart cycle being 14.5",
                                           profile="profiles/gram_schmidt_dcgs2_kernels_n1025.md"),
    ("2d-well-n1025", "mdot"): dict(kernel="k_mdot2_pair", source="paper_1012_4307_gb300/csrc/kernels_gs_df.cu",
                                    sha1="093841d405022c73eadc49970ff88b158dc8bcf7", bytes=290221312,
                                    launch="basis slot j = 15, the mean over a restart cycle being 14.5",
                                    profile="profiles/gram_schmidt_dcgs2_kernels_n1025.md"),
    # captured at 161^3 (whose basis vectors, 67 MB each, also stream from DRAM: traffic 0.98 x the
    # algorithmic bytes) and scaled to 257^3 by the node count
    ("3d-well-n257", "update_norm"): dict(kernel="k_update2_pair", source="paper_1012_4307_gb300/csrc/kernels_gs_df.cu",
                                          sha1="093841d405022c73eadc49970ff88b158dc8bcf7", bytes=3871945711,
                                          launch="basis slot j = 10 of FGMRES(20), captured at 161^3 and scaled by "
                                                 "the node count",
                                          profile="profiles/update_pass_3d_well_n161.md"),
}


def ncu_traffic(workload, kernel_class):
    import hashlib
    t = NCU_TRAFFIC.get((workload, kernel_class))
    if not t:
        return None, "no ncu capture of this kernel class on this workload"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), t["source"])
    with open(path, "rb") as fh:
        if hashlib.sha1(fh.read()).hexdigest() != t["sha1"]:
            return None, "kernel changed since the ncu capture in %s" % t["profile"]
    return t["bytes"], "%s, one launch at %s (%s)" % (t["kernel"], t["launch"], t["profile"])


GS_NAMES = {"dcgs2": "double-FP32 delayed CGS2 on float-pair vectors",
            "df": "double-FP32 CGS + DGKS on float-pair vectors",
            "fp64": "IEEE FP64 CGS + DGKS"}


def roofline_from_profile(prof, peaks, peak_src, sm_max, workload=""):
    """Roofline of the dominant kernel class of one profiled solve (eager launches, one event
    pair each): achieved = algorithmic bytes (or FP64 flops) per launch / mean launch time."""
    dname, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    fp64_peak_tflops = 2 * FP64_FMA_PER_SM_CLK * SM_COUNT * sm_max * 1e6 / 1e12
    avg_s = d["ms"] / max(d["launches"], 1) / 1e3
    gbs = d["bytes"] / max(d["launches"], 1) / avg_s / 1e9
    tfs = d["flops"] / max(d["launches"], 1) / avg_s / 1e12
    hbm = peaks.get("hbm_gbs", 6800.0)
    eager_ms = sum(v["ms"] for v in prof.values())
    if d["flops"] > 0 and d["flops"] / max(d["bytes"], 1) > fp64_peak_tflops * 1e3 / hbm:
        roof = {"bound": "alu", "achieved": tfs, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": tfs / fp64_peak_tflops,
                "peak_source": "FP64 FMA units: 2 per SM per clock x 152 SMs x %.0f MHz" % sm_max,
                "hbm_gbs_achieved": gbs, "hbm_frac": gbs / hbm}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "peak_source": "%s hbm_gbs (%s)" % (peak_src, "of measured" if peak_src == "measured" else "of fallback")}
    traffic, traffic_note = ncu_traffic(workload, dname)
    roof.update({"traffic": traffic, "traffic_note": traffic_note, "kernel_class": dname,
                 "launches_per_solve": d["launches"], "avg_launch_us": avg_s * 1e6,
                 "algorithmic_bytes_per_launch": d["bytes"] / max(d["launches"], 1),
                 "profile_schedule": "eager: graphs and the side stream off, one CUDA event pair per launch on "
                                     "the library's stream",
                 "share_of_eager_solve": d["ms"] / max(eager_ms, 1e-9), "eager_solve_ms": eager_ms})
    return roof


def breakdown_from_profile(prof, hbm):
    out = {}
    for k, v in prof.items():
        if not v["launches"]:
            continue
        e = {"launches": v["launches"], "ms": round(v["ms"], 4)}
        if v["ms"] > 0:
            e["GB/s"] = round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1)
            e["frac"] = round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm, 4)
            if abs(v["bytes_pass"] - v["bytes"]) > 1e-6 * max(v["bytes"], 1.0):
                # temporally blocked kernels: the same work counted sweep by sweep (may exceed 1)
                e["GB/s_per_pass"] = round(v["bytes_pass"] / (v["ms"] / 1e3) / 1e9, 1)
                e["frac_per_pass"] = round(v["bytes_pass"] / (v["ms"] / 1e3) / 1e9 / hbm, 4)
        out[k] = e
    return out


def run_single(args, workload, steps, warmup, extra=False):
    """One workload solved repeatedly by krylov_solve; returns the JSON line (dict) on rank 0."""
    import torch
    import torch.distributed as dist

    from paper_1012_4307_gb300 import helm

    world, rank, local = dist_env()
    peaks, peak_src = load_peaks()
    P = problem(workload, 0 if extra else args.n, seed_offset=rank)
    k2 = torch.from_numpy(P.k2).cuda()
    stream = torch.cuda.current_stream()
    mg = helm.MGParams(kind="csg", theta_a=P.theta_a, nu1=P.nu1, nu2=P.nu2, omega=P.omega, coarsest_n=P.coarsest_n,
                       prec="c64", gs=args.gs)
    n = [P.n] * P.dim
    h = helm.helm_create(P.dim, n, k2, theta=P.theta, mg=mg)
    f = torch.from_numpy(P.f).cuda()
    x = torch.zeros_like(f)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    # kernel choices of the cycle: autotuned once per library build and grid (JSON cache beside
    # the library); a profiling case only installs a stored choice, so that it launches no
    # tuning runs of its own
    tuning, tune_ms = None, None
    if not args.no_tune:
        if args.ncu_case or args.ncu_precond:
            tuning = helm.cached_tuning(h, "c64")
            if tuning:
                helm.helm_set_tuning(h, tuning)
        else:
            tuning, tune_ms = helm.helm_autotune(h, "c64", reps=25, cache=helm.default_tuning_cache())

    def solve(handle, out):
        out.zero_()
        return helm.krylov_solve(handle, f, out, tol=args.tol, restart=P.restart, maxit=5000)

    if args.ncu_case:
        x.zero_()
        _, st = helm.krylov_solve(h, f, x, tol=args.tol, restart=P.restart, maxit=args.ncu_case,
                                  raise_on_noconv=False)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": P.name, "iterations": st.iterations, "rel_res": st.rel_res}), flush=True)
        return None
    if args.ncu_precond:
        for _ in range(args.ncu_precond):
            helm.mg_precondition(h, f, torch.complex64)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_precond": P.name, "calls": args.ncu_precond,
                          "device_bytes": torch.cuda.memory_allocated()}), flush=True)
        return None

    for _ in range(warmup):
        solve(h, x)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    st = None
    for _ in range(steps):
        flush.fill_(1)
        e0.record(stream)
        _, st = solve(h, x)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = total_ms / steps
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * P.unknowns / (ms_max / 1e3) / 1e6

    # launches per solve and the dominant kernel class, from one profiled solve
    helm.helm_profile(h, True)
    solve(h, x)
    prof = helm.helm_profile_read(h)
    helm.helm_profile(h, False)
    launches = sum(v["launches"] for v in prof.values())
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roof = roofline_from_profile(prof, peaks, peak_src, sm_max, P.name)
    breakdown = breakdown_from_profile(prof, peaks.get("hbm_gbs", 6800.0))

    # plain FP64 method on the same problem (FP64 cycle, FP64 Gram-Schmidt), and the mixed
    # method with FP64 Gram-Schmidt; error of the mixed solution against the FP64 one
    def timed_variant(prec, gs, reps=2):
        mgv = helm.MGParams(kind="csg", theta_a=P.theta_a, nu1=P.nu1, nu2=P.nu2, omega=P.omega,
                            coarsest_n=P.coarsest_n, prec=prec, gs=gs)
        hv = helm.helm_create(P.dim, n, k2, theta=P.theta, mg=mgv)
        xv = torch.zeros_like(f)
        solve(hv, xv)
        tt, stv = 0.0, None
        for _ in range(reps):
            flush.fill_(2)
            e0.record(stream)
            _, stv = solve(hv, xv)
            e1.record(stream)
            e1.synchronize()
            tt += e0.elapsed_time(e1)
        hv.close()
        msv = tt / reps
        return xv, {"ms_per_solve": msv, "iterations": stv.iterations, "rel_res": stv.rel_res,
                    "value": P.unknowns / (msv / 1e3) / 1e6, "speedup_of_headline": msv / ms}

    fp64 = mixed_fp64gs = None
    if not args.no_fp64 and rank == 0:
        x64, fp64 = timed_variant("c128", "fp64", reps=1 if extra else 2)
        fp64["mixed_vs_fp64_rel_l2"] = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
        del x64
        if not extra:
            _, mixed_fp64gs = timed_variant("c64", "fp64", reps=1)

    # end to end through the public API: pinned host rhs -> device, solve, solution -> host
    f_host = torch.from_numpy(P.f).pin_memory()
    x_host = torch.empty_like(f_host).pin_memory()
    e2e_ms = 0.0
    for k in range(steps):
        flush.fill_(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f.copy_(f_host, non_blocking=True)
        x.zero_()
        helm.krylov_solve(h, f, x, tol=args.tol, restart=P.restart, maxit=5000)
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms /= steps
    te = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": world * P.unknowns / (float(te.item()) / 1e3) / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": f_host.numel() * 16, "d2h_bytes_per_step": x_host.numel() * 16,
           "ms_per_step": float(te.item())}
    h.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        it_needed = oracle_iterations(P.name)
        source = "the oracle's own FGMRES iteration count (tests/golden/oracle_iterations.json)"
        if it_needed is None:
            it_needed = fp64["iterations"] if fp64 else st.iterations
            source = "the iteration count of the FP64 GPU solve (no stored oracle count for this workload)"
        if P.dim == 3:
            # about 30 s per single-threaded iteration at 257^3: all cores only, one iteration
            cpu = cpu_baseline(P, args.tol, 1, it_needed, source, single=False)
        else:
            cpu = cpu_baseline(P, args.tol, args.cpu_iters or 6, it_needed, source, full_solve=True)

    if rank != 0:
        return None
    solver = ("FGMRES(%d), FP64 Hessenberg/Givens/true residual/solution; Arnoldi: %s; CSG theta_a=pi/%.3g, "
              "V(2,2) omega-Jacobi 0.8, complex64 cycle" % (P.restart, GS_NAMES[args.gs], math.pi / P.theta_a))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 cycle / f64 outer", "data": "synthetic",
            "config": {"workload": P.name, "unknowns": P.unknowns, "nodes": n, "solver": solver,
                       "tol": args.tol, "ecs_theta": "pi/6", "kh_max": 0.6,
                       "l2": "256 MiB device write before every step, outside the timed events"
                             + ("; every complex128 vector (%.0f MB) exceeds L2" % (P.f.nbytes / 1e6)
                                if P.f.nbytes > 129e6 else ""),
                       "cycle_tuning": tuning, "tuned_ms_per_cycle": tune_ms,
                       "parallelism": "independent problem per rank" if world > 1 else "single GPU"},
            "solve": {"iterations": st.iterations, "restarts": st.restarts, "rel_res": st.rel_res,
                      "ms_per_solve": ms_max, "us_per_iteration": ms_max * 1e3 / max(st.iterations, 1),
                      "reorthogonalizations": st.reorthogonalizations},
            "fp64": fp64, "mixed_fp64_gram_schmidt": mixed_fp64gs, "roofline": roof, "kernels": breakdown,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches * steps,
            "gpu_launches_per_step": launches, "peaks": peak_src}


# ---------------------------------------------------------------------------------- batch
def run_batch(args, count, steps, warmup, extra=False):
    """count problems solved together by helm_solve_batch, against the same problems solved one
    after another by krylov_solve.  Under torchrun the problems are sharded over the ranks by
    longest processing time (no data exchange); the job's time is the slowest rank's."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1012_4307_gb300 import distributed as D
    from paper_1012_4307_gb300 import helm
    from paper_1012_4307_gb300 import workloads as W

    world, rank, local = D.rank_env()
    peaks, peak_src = load_peaks()
    all_probs = W.config_batch(count=count)
    shard = D.lpt_partition([D.solve_cost(P.n) for P in all_probs], world)[rank]
    probs = [all_probs[i] for i in shard]
    mg = helm.MGParams(kind="csg", theta_a=probs[0].theta_a, prec="c64", gs=args.gs, coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    # every problem's right-hand side and solution as a view into one device buffer each, so that
    # a whole batch moves between host and device in one copy per direction
    sizes = [P.f.size for P in probs]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    rhs_flat = torch.from_numpy(np.concatenate([P.f.ravel() for P in probs])).cuda()
    x_flat = torch.zeros_like(rhs_flat)
    rhs = [rhs_flat[offs[i]:offs[i + 1]].view(P.f.shape) for i, P in enumerate(probs)]
    xs = [x_flat[offs[i]:offs[i + 1]].view(P.f.shape) for i, P in enumerate(probs)]
    if args.ncu_case:
        # profiling case: the stored tunings, one batch solve capped at ncu_case iterations
        for i in range(len(probs)):
            hb = helm.batch_handle(b, i)
            t = helm.cached_tuning(hb, "c64")
            if t:
                helm.helm_set_tuning(hb, t)
        st = helm.helm_solve_batch(b, rhs, xs, tol=args.tol, restart=30, maxit=args.ncu_case, raise_on_noconv=False)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "batch-%d" % count, "engine": helm.helm_batch_get_engine(b),
                          "iterations": [x.iterations for x in st]}), flush=True)
        return None
    tunings = None if args.no_tune else helm.helm_autotune_batch(b, "c64", reps=25, cache=helm.default_tuning_cache())
    unknowns = sum(P.unknowns for P in probs)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def batch_once():
        x_flat.zero_()
        return helm.helm_solve_batch(b, rhs, xs, tol=args.tol, restart=30, maxit=5000)

    for _ in range(max(1, warmup)):
        batch_once()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    tot = 0.0
    stats = None
    for _ in range(steps):
        flush.fill_(1)
        e0.record(stream)
        stats = batch_once()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = D.max_over_ranks(tot / steps, device="cuda")
    unknowns_all = int(D.sum_over_ranks(unknowns, device="cuda"))
    value = unknowns_all / (ms / 1e3) / 1e6

    # kernel classes summed over every problem's handle, from one profiled batch solve
    handles = [helm.batch_handle(b, i) for i in range(len(probs))]
    for hh in handles:
        helm.helm_profile(hh, True)
    batch_once()
    prof = None
    for hh in handles:
        p = helm.helm_profile_read(hh)
        helm.helm_profile(hh, False)
        if prof is None:
            prof = {k: dict(v) for k, v in p.items()}
        else:
            for k, v in p.items():
                for f in v:
                    prof[k][f] += v[f]
    launches = sum(v["launches"] for v in prof.values())
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roof = roofline_from_profile(prof, peaks, peak_src, sm_max, "batch-%d" % count)
    breakdown = breakdown_from_profile(prof, peaks.get("hbm_gbs", 6800.0))

    # end to end: every problem's rhs from pinned host memory (one buffer, one copy), the batch
    # solve, every solution back (one copy)
    f_host = rhs_flat.cpu().pin_memory()
    x_host = torch.empty_like(f_host).pin_memory()
    e2e_ms = 0.0
    for _ in range(steps):
        flush.fill_(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rhs_flat.copy_(f_host, non_blocking=True)
        batch_once()
        x_host.copy_(x_flat, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = D.max_over_ranks(e2e_ms / steps, device="cuda")
    nbytes = f_host.numel() * 16
    e2e = {"value": unknowns_all / (e2e_ms / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms}

    # the same problems one after another through krylov_solve (same settings and tunings)
    seq_ms = None
    if world == 1 and not extra:
        seq_ms = 0.0
        for P, r in zip(probs, rhs):
            h = helm.helm_create(2, [P.n, P.n], torch.from_numpy(P.k2).cuda(), theta=P.theta, mg=mg)
            if tunings:
                helm.helm_set_tuning(h, tunings[helm.tuning_key(h, "c64")])
            x = torch.zeros_like(r)
            helm.krylov_solve(h, r, x, tol=args.tol, restart=30, maxit=5000)
            x.zero_()
            e0.record(stream)
            helm.krylov_solve(h, r, x, tol=args.tol, restart=30, maxit=5000)
            e1.record(stream)
            e1.synchronize()
            seq_ms += e0.elapsed_time(e1)
            h.close()

    # CPU oracle: a sample of iterations per distinct grid size on all cores, projected with
    # each problem's iteration count of the GPU solve
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        per = {}
        for nn in sorted({P.n for P in probs}):
            per[nn] = run_cpu_leg({"batch_n": nn, "tol": args.tol, "iters": 3 if nn <= 513 else 2}, all_cores=True)
        proj = sum(per[P.n]["sec_per_iter"] * s.iterations for P, s in zip(probs, stats))
        cpu = {"value": unknowns / proj / 1e6, "unit": UNIT, "cores": per[max(per)]["threads"], "kind": "oracle",
               "projected": True, "projected_solve_s": proj,
               "sample": "per grid size, 2-3 FGMRES(30) iterations of the plain C FP64 oracle (FP64 V(2,2) CSG cycle) "
                         "on all host cores; each problem projected with its GPU solve's iteration count",
               "seconds_per_iteration_by_n": {str(k): v["sec_per_iter"] for k, v in per.items()}}
    b = None
    if rank != 0:
        return None
    return {"metric": "batched solve throughput (all problems to rel. residual %.0e), Mdof/s" % args.tol,
            "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "c64 cycle / f64 outer", "data": "synthetic",
            "config": {"workload": "batch-%d" % count,
                       "description": "%d 2D well problems, sizes {129,257,513,1025}, E in [0.5,4], Gaussian "
                                      "sources, FGMRES(30), CSG V(2,2) complex64 cycle" % count,
                       "unknowns": unknowns_all, "sizes": [P.n for P in all_probs],
                       "parallelism": "problems sharded over ranks by longest processing time" if world > 1
                       else "single GPU",
                       "l2": "256 MiB device write before every step, outside the timed events",
                       "cycle_tuning": tunings},
            "iterations_rank0": [s.iterations for s in stats], "roofline": roof, "kernels": breakdown,
            "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / ms if seq_ms else None,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches * steps,
            "gpu_launches_per_step": launches, "peaks": peak_src}


# ---------------------------------------------------------------------------------- main
def main():
    args = parse()
    if args.cpu_leg is not None:
        return cpu_leg_main(json.loads(args.cpu_leg))
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1012_4307_gb300 import helm
    helm.load()
    wl = "batch-64" if args.batch else args.workload
    if wl == "batch-64":
        line = run_batch(args, args.batch or 64, args.steps, args.warmup)
    else:
        line = run_single(args, wl, args.steps, args.warmup)
        if (line is not None and wl == WORKLOADS[0] and world == 1 and not args.no_extra and not args.ncu_case
                and not args.ncu_precond):
            # the other workloads, measured the same way in shorter runs
            line["other_configs"] = {
                "3d-well-n257": run_single(args, "3d-well-n257", steps=3, warmup=2, extra=True),
                "batch-64": run_batch(args, 64, steps=2, warmup=1, extra=True),
            }
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
