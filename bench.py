#!/usr/bin/env python
"""Benchmark: preconditioned solve of the 2D ECS Helmholtz well problem (1025 x 1025 nodes,
k^2 = 2(E - V) with a Gaussian well and growth toward the boundary so that k h <= 0.6, ECS at
pi/6 beyond |x|, |y| = 0.75, random source on |x|_inf < 0.5) to a relative residual of 1e-8 with
FGMRES(30), preconditioned by one complex64 V(2,2) multigrid cycle on the complex-scaled-grid
operator (theta_a = pi/14), FP64 outer solver.  One step = one full solve from x = 0.

Prints one JSON line:  value = unknowns solved per second over all ranks (Mdof/s), with the
plain FP64 solve (FP64 cycle) beside it, the dominant kernel's roofline, the CPU oracle as a
baseline, an end-to-end number through the public API with host buffers, and the SM clocks
sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 1025]

Under torchrun every rank solves its own independent problem (seed 1 + rank): the work per GPU
is fixed, so scaling is weak and no collective touches the data path.
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1025)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-iters", type=int, default=0, help="oracle iterations in the CPU sample (0 = auto)")
    ap.add_argument("--batch", type=int, default=0, metavar="COUNT",
                    help="batched workload instead: COUNT independent 2D problems with sizes drawn from "
                         "{129, 257, 513, 1025} and energies in [0.5, 4], solved together (helm_solve_batch)")
    ap.add_argument("--no-tune", action="store_true", help="default kernel choices instead of the autotuned ones")
    ap.add_argument("--gs", default="dcgs2", choices=["dcgs2", "df", "fp64"],
                    help="Arnoldi arithmetic of the headline solve (see helm_gs_arith)")
    ap.add_argument("--ncu-case", type=int, default=0, metavar="ITERS",
                    help="profiling case: build the same problem and run one solve capped at ITERS iterations, "
                         "nothing else (keeps the launch count small enough for ncu)")
    return ap.parse_args()


def dist_env():
    from paper_1012_4307_gb300.distributed import rank_env
    return rank_env()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


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


def oracle_sample(P, iters, tol):
    """Times the CPU oracle's FP64 FGMRES(30) with its FP64 V(2,2) cycle for ``iters``
    iterations on the full problem (single thread); returns seconds per iteration."""
    from oracle import oracle as O
    z = O.axes(P.dim, P.n, theta=P.theta, r0lo=-P.r0, r0hi=P.r0)
    A, M = O.helmholtz_ops(z, P.k2, pc=P.pc, theta_a=P.theta_a)
    t0 = time.perf_counter()
    mg = O.MG(M, P.coarsest_n, P.nu1, P.nu2, P.omega, P.smoother)
    x, st = O.fgmres(A, mg, P.f, tol=tol, restart=P.restart, maxit=iters)
    dt = time.perf_counter() - t0
    return dt / max(st["iterations"], 1), st["iterations"], dt


def cpu_baseline(P, tol, iters, gpu_fp64_iters):
    it_needed = oracle_iterations(P.name)
    source = "oracle FGMRES iteration count (tests/golden/oracle_iterations.json)"
    if it_needed is None:
        it_needed = gpu_fp64_iters
        source = "iteration count of the FP64 GPU solve (no stored oracle count for this workload)"
    per_it, done, dt = oracle_sample(P, iters, tol)
    solve_s = per_it * it_needed
    return {"value": P.unknowns / solve_s / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d FGMRES(30) iterations of the plain C FP64 oracle (FP64 V(2,2) CSG cycle) on the full "
                      "%s problem, %.1f s, scaled to the %d iterations of a full solve (%s)"
                      % (done, P.name, dt, it_needed, source),
            "seconds_per_iteration": per_it, "projected_solve_s": solve_s}


# ---------------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1012_4307_gb300 import workloads as W
    from oracle import oracle as O
    O.build()
    P = W.config_2d_well(args.n, seed=1)
    it_needed = oracle_iterations(P.name)
    iters = 2
    vals = []
    for s in range(args.warmup + args.steps):
        per_it, done, dt = oracle_sample(P, iters, args.tol)
        if s >= args.warmup:
            vals.append(per_it)
    per_it = statistics.mean(vals)
    if it_needed is None:
        it_needed = 1
    solve_s = per_it * it_needed
    value = P.unknowns / solve_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": solve_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": P.name, "unknowns": P.unknowns, "solver": "FGMRES(30), FP64 V(2,2) CSG cycle",
                       "tol": args.tol},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: %d FGMRES(30) iterations of the plain C FP64 oracle on the full "
                                       "problem (single thread), scaled to the %d iterations of a full solve"
                                       % (iters, it_needed)}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------- batch
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant
# kernels, from the ncu captures summarised under profiles/.  Reported only while the kernel's
# source file is the one that was captured (same SHA-1); otherwise null.
NCU_TRAFFIC = {
    "update_norm": dict(kernel="k_update2_pair", source="paper_1012_4307_gb300/csrc/kernels_gs_df.cu",
                        sha1="57192057f858d44ef0ecd41b7097a4cc8973d85f", bytes=314946304,
                        launch="basis slot j = 15, the mean over a restart cycle being 14.5",
                        profile="profiles/gram_schmidt_dcgs2_kernels_n1025.md"),
    "mdot": dict(kernel="k_mdot2_pair", source="paper_1012_4307_gb300/csrc/kernels_gs_df.cu",
                 sha1="57192057f858d44ef0ecd41b7097a4cc8973d85f", bytes=289090816,
                 launch="basis slot j = 15, the mean over a restart cycle being 14.5",
                 profile="profiles/gram_schmidt_dcgs2_kernels_n1025.md"),
}


def ncu_traffic(kernel_class):
    import hashlib
    t = NCU_TRAFFIC.get(kernel_class)
    if not t:
        return None, None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), t["source"])
    with open(path, "rb") as fh:
        if hashlib.sha1(fh.read()).hexdigest() != t["sha1"]:
            return None, "kernel changed since the ncu capture in %s" % t["profile"]
    return t["bytes"], "%s, one launch at %s (%s)" % (t["kernel"], t["launch"], t["profile"])


GS_NAMES = {"dcgs2": "double-FP32 delayed CGS2 on float-pair vectors",
            "df": "double-FP32 CGS + DGKS on float-pair vectors",
            "fp64": "IEEE FP64 CGS + DGKS"}


def run_batch(args):
    """COUNT problems solved together (one host thread, one stream and CUDA-graph-replayed
    FGMRES steps per problem) against the same problems solved one after another.  Under
    torchrun the problems are sharded over the ranks by longest processing time (no data
    exchange); the job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist

    from paper_1012_4307_gb300 import distributed as D
    from paper_1012_4307_gb300 import helm
    from paper_1012_4307_gb300 import workloads as W

    world, rank, local = D.rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    helm.load()
    all_probs = W.config_batch(count=args.batch)
    shard = D.lpt_partition([D.solve_cost(P.n) for P in all_probs], world)[rank]
    probs = [all_probs[i] for i in shard]
    mg = helm.MGParams(kind="csg", prec="c64", gs=args.gs, coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    tunings = None if args.no_tune else helm.helm_autotune_batch(b, "c64", cache=helm.default_tuning_cache())
    rhs = [torch.from_numpy(P.f).cuda() for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    unknowns = sum(P.unknowns for P in probs)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def batch_once():
        for x in xs:
            x.zero_()
        return helm.helm_solve_batch(b, rhs, xs, tol=args.tol, restart=30, maxit=5000)

    for _ in range(max(1, args.warmup)):
        batch_once()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    tot = 0.0
    for _ in range(args.steps):
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
    ms = D.max_over_ranks(tot / args.steps, device="cuda")
    unknowns = int(D.sum_over_ranks(unknowns, device="cuda"))
    # the same problems one after another through krylov_solve (same handles' settings)
    seq_ms = 0.0
    for P, r in (zip(probs, rhs) if world == 1 else []):
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
    line = {"metric": "batched solve throughput (all problems to rel. residual %.0e)" % args.tol,
            "value": unknowns / (ms / 1e3) / 1e6, "unit": "Mdof/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "dtype": "c64 cycle / f64 outer", "data": "synthetic",
            "config": {"workload": "batch of %d 2D well problems, sizes {129,257,513,1025}, E in [0.5,4]" % args.batch,
                       "unknowns": unknowns, "sizes": [P.n for P in all_probs],
                       "parallelism": "problems sharded over ranks by longest processing time" if world > 1 else "single GPU",
                       "l2": "256 MiB device write before every step, outside the timed events",
                       "cycle_tuning": tunings},
            "iterations_rank0": [s.iterations for s in stats],
            "sequential_ms": seq_ms if world == 1 else None,
            "speedup_vs_sequential": seq_ms / ms if world == 1 else None, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch:
        return run_batch(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1012_4307_gb300 import helm
    from paper_1012_4307_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    helm.load()
    peaks, peak_src = load_peaks()

    P = W.config_2d_well(args.n, seed=1 + rank)
    k2 = torch.from_numpy(P.k2).cuda()
    stream = torch.cuda.current_stream()
    mg = helm.MGParams(kind="csg", theta_a=P.theta_a, nu1=P.nu1, nu2=P.nu2, omega=P.omega, coarsest_n=P.coarsest_n,
                       prec="c64", gs=args.gs)
    h = helm.helm_create(2, [P.n, P.n], k2, theta=P.theta, mg=mg)
    f = torch.from_numpy(P.f).cuda()
    x = torch.zeros_like(f)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    # kernel choices of the cycle: autotuned once per library build and grid (JSON cache beside
    # the library); a profiling case only installs a stored choice, so that it launches no
    # tuning runs of its own
    tuning, tune_ms = None, None
    if not args.no_tune:
        if args.ncu_case:
            tuning = helm.cached_tuning(h, "c64")
            if tuning:
                helm.helm_set_tuning(h, tuning)
        else:
            tuning, tune_ms = helm.helm_autotune(h, "c64", reps=10, cache=helm.default_tuning_cache())

    def solve(handle, out):
        out.zero_()
        return helm.krylov_solve(handle, f, out, tol=args.tol, restart=P.restart, maxit=5000)

    if args.ncu_case:
        x.zero_()
        _, st = helm.krylov_solve(h, f, x, tol=args.tol, restart=P.restart, maxit=args.ncu_case,
                                  raise_on_noconv=False)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": P.name, "iterations": st.iterations, "rel_res": st.rel_res}), flush=True)
        return

    for _ in range(args.warmup):
        solve(h, x)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    st = None
    torch.cuda.synchronize()
    for _ in range(args.steps):
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
    ms = total_ms / args.steps
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * P.unknowns / (ms_max / 1e3) / 1e6

    # launches per solve and the dominant kernel, from one profiled solve (events on the library's stream)
    helm.helm_profile(h, True)
    solve(h, x)
    prof = helm.helm_profile_read(h)
    helm.helm_profile(h, False)
    launches = sum(v["launches"] for v in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak_tflops = 2 * FP64_FMA_PER_SM_CLK * SM_COUNT * sm_max * 1e6 / 1e12
    avg_s = d["ms"] / max(d["launches"], 1) / 1e3
    gbs = d["bytes"] / max(d["launches"], 1) / avg_s / 1e9
    tfs = d["flops"] / max(d["launches"], 1) / avg_s / 1e12
    hbm = peaks.get("hbm_gbs", 6800.0)
    if d["flops"] > 0 and d["flops"] / max(d["bytes"], 1) > fp64_peak_tflops * 1e3 / hbm:
        roof = {"bound": "alu", "achieved": tfs, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": tfs / fp64_peak_tflops, "peak_source": "FP64 FMA units: 2 per SM per clock x 152 SMs x %.0f MHz"
                % sm_max, "hbm_gbs_achieved": gbs, "hbm_frac": gbs / hbm}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "peak_source": "%s hbm_gbs" % peak_src}
    traffic, traffic_note = ncu_traffic(dname)
    roof.update({"traffic": traffic, "traffic_note": traffic_note, "kernel_class": dname, "launches_per_solve": d["launches"],
                 "avg_launch_us": avg_s * 1e6, "share_of_solve": d["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9)})
    breakdown = {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                     "GB/s": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None}
                 for k, v in prof.items() if v["launches"]}

    # plain FP64 method on the same problem (FP64 cycle, FP64 Gram-Schmidt), and the mixed
    # method with FP64 Gram-Schmidt; error of the mixed solution against the FP64 one
    def timed_variant(prec, gs, reps=2):
        mgv = helm.MGParams(kind="csg", theta_a=P.theta_a, nu1=P.nu1, nu2=P.nu2, omega=P.omega,
                            coarsest_n=P.coarsest_n, prec=prec, gs=gs)
        hv = helm.helm_create(2, [P.n, P.n], k2, theta=P.theta, mg=mgv)
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
        x64, fp64 = timed_variant("c128", "fp64")
        fp64["mixed_vs_fp64_rel_l2"] = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
        _, mixed_fp64gs = timed_variant("c64", "fp64", reps=1)

    # end to end through the public API: pinned host rhs -> device, solve, solution -> host
    f_host = torch.from_numpy(P.f).pin_memory()
    x_host = torch.empty_like(f_host).pin_memory()
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.fill_(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f.copy_(f_host, non_blocking=True)
        x.zero_()
        helm.krylov_solve(h, f, x, tol=args.tol, restart=P.restart, maxit=5000)
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms /= args.steps
    te = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": world * P.unknowns / (float(te.item()) / 1e3) / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": f_host.numel() * 16, "d2h_bytes_per_step": x_host.numel() * 16,
           "ms_per_step": float(te.item())}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters = args.cpu_iters or 6
        cpu = cpu_baseline(P, args.tol, iters, fp64["iterations"] if fp64 else st.iterations)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64 cycle / f64 outer", "data": "synthetic",
                "config": {"workload": P.name, "unknowns": P.unknowns, "nodes": [P.n, P.n],
                           "solver": "FGMRES(30), FP64 Hessenberg/Givens/true residual/solution; Arnoldi: %s; "
                                     "CSG theta_a=pi/14, V(2,2) omega-Jacobi 0.8, complex64 cycle" % GS_NAMES[args.gs],
                           "tol": args.tol, "ecs_theta": "pi/6", "kh_max": 0.6,
                           "l2": "256 MiB device write before every step, outside the timed events",
                           "cycle_tuning": tuning, "tuned_ms_per_cycle": tune_ms,
                           "parallelism": "independent problem per rank" if world > 1 else "single GPU"},
                "solve": {"iterations": st.iterations, "restarts": st.restarts, "rel_res": st.rel_res,
                          "ms_per_solve": ms_max, "reorthogonalizations": st.reorthogonalizations},
                "fp64": fp64, "mixed_fp64_gram_schmidt": mixed_fp64gs, "roofline": roof, "kernels": breakdown, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "gpu_launches": launches * args.steps, "gpu_launches_per_step": launches,
                "peaks": peak_src}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
