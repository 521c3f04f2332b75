#!/usr/bin/env python3
"""Benchmark: mixed-precision even-odd Wilson solve on a 32^3x64 lattice.

One step = one solve of D x = b to a true residual ||b - D x|| / ||b|| <= 1e-10
(random SU(3) links exp(i 0.3 H) seed 1, kappa = 0.12, antiperiodic in time,
one complex Gaussian right-hand side seed 2), from b in HBM (canonical layout)
to x in HBM: layout conversion in, even-odd preparation, inner BiCGStab in
FP16 storage / FP32 arithmetic under defect correction in double-float
arithmetic (--outer-arith 2, the library default; 1: FP64 true-residual check),
reconstruction, full-D true residual, layout conversion out.  The returned x is
re-checked outside the timed region with the FP64 D (true_resid_fp64_recheck).

value = algorithmic bytes of every hopping-kernel launch of the timed steps
(1536 / 768 / 392 B per output site for FP64 / FP32 / FP16, plus the xpay and
clover operands) divided by the timed wall time: the dslash GB/s the whole
solve sustains.  The roofline block reports the inner-precision hopping
kernel alone (CUDA events around each launch, on its stream).

--impl reference times the FP64 CPU oracle (the only reference: the paper
ships no code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_BENCH = (32, 32, 32, 64)
KAPPA = 0.12
TOL = 1e-10
METRIC = "dslash GB/s (% of HBM peak); solve time to 1e-10 resid, mixed vs FP64"
BYTES_F64 = 1536.0     # algorithmic bytes per eo-dslash output site, FP64 (8 links + in + out)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", default="f16", choices=["f16", "f32"])
    ap.add_argument("--lattice", default=None, help="override lattice, e.g. 16,16,16,32")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--inner-tol", type=float, default=None, help="inner relative tolerance")
    ap.add_argument("--eager", action="store_true", help="host-driven inner loop instead of CUDA graphs")
    ap.add_argument("--outer-arith", type=int, default=2, choices=[0, 1, 2],
                    help="outer loop: 0 FP64; 1 double-float defects, FP64 true-residual check; "
                         "2 double-float defects and check (x returned as the checked iterate)")
    ap.add_argument("--mode", default="solve", choices=["solve", "dslash"],
                    help="solve: the timed mixed-precision solve (default); dslash: the hopping kernel alone")
    ap.add_argument("--workload", default="wilson32",
                    choices=["wilson32", "configs0_8x8x8x8", "errors8", "prop24", "uneven6", "clover48", "grad16",
                             "mg16", "dd16"],
                    help="wilson32: the default timed solve; configs0_8x8x8x8: plain FP64 dslash + solve on 8^4; prop24: 12 point sources on 24^3x48 in one "
                         "batched solve; uneven6: six lattices of uneven size in one batched solve; "
                         "clover48: Wilson-clover 48^3x96, 4 RHS, FP16 inner, with grad_b; "
                         "grad16: FP64 solve + adjoint + link gradient on 16^3x32")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other workloads that the default line reports under `workloads`")
    ap.add_argument("--prec", default="f16", choices=["f64", "f32", "f16", "f64df"], help="precision for --mode dslash")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides per launch for --mode dslash")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("BPP_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


# ----------------------------------------------------------------------------- CPU oracle leg
def cpu_oracle_sample(L, target_s=12.0):
    """The FP64 oracle's D (Eq. 1, plain loops) on sampled sites of the lattice:
    returns (GB/s of eo-dslash-equivalent algorithmic bytes, sites, seconds, threads)."""
    import numpy as np

    import oracle
    import synth
    V = L[0] * L[1] * L[2] * L[3]
    U = synth.random_links(L, seed=1)
    psi = synth.gaussian_spinor(L, seed=2)
    rng = np.random.default_rng(0)
    n = 4096
    total_sites, total_t = 0, 0.0
    while total_t < target_s:
        sites = np.sort(rng.choice(V, size=min(n, V), replace=False))
        t0 = time.perf_counter()
        oracle.apply_D(U, psi, KAPPA, L, (1, 1, 1, -1), sites=sites)
        dt = time.perf_counter() - t0
        total_sites += len(sites)
        total_t += dt
        if dt < 0.5 * target_s:
            n = min(V, n * 4)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return total_sites * BYTES_F64 / total_t / 1e9, total_sites, total_t, threads


OUTER_NAMES = {0: "FP64 defect correction", 1: "defect correction with double-float defects and an FP64 "
                                              "true-residual check",
               2: "defect correction in double-float arithmetic (defects and true-residual check; x returned "
                  "in FP64 and re-checked with the FP64 D)"}


def solve_config(L, inner_name, world=1, outer_arith=2):
    """The benchmark workload as reported in `config` (shared by both arms)."""
    return {"workload": f"Wilson eo-BiCGStab solve, {'x'.join(map(str, L))}, kappa {KAPPA}, 1 Gaussian RHS, "
                        f"{inner_name} inner + {OUTER_NAMES[outer_arith]} to true resid {TOL}",
            "lattice": list(L), "kappa": KAPPA, "tol": TOL, "rhs": 1, "outer_arith": outer_arith,
            "l2": "inputs larger than L2 (links 1.2 GB FP64 / 0.6 GB FP32 / 0.3 GB FP16); no flush",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    L = tuple(int(v) for v in args.lattice.split(",")) if args.lattice else L_BENCH
    times, gbs = [], []
    cores = None
    for step in range(args.warmup + args.steps):
        v, sites, secs, cores = cpu_oracle_sample(L, target_s=4.0)
        if step >= args.warmup:
            times.append(secs)
            gbs.append(v)
    value = statistics.mean(gbs)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": solve_config(L, "f16-storage/f32" if args.inner == "f16" else "f32", 1, args.outer_arith),
           "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                            "sample": "the oracle's FP64 D (Eq. 1, plain C loops, OpenMP) on random site samples of "
                                      "this lattice, ~4 s per step, as the even-odd dslash work of the solve: "
                                      "1536 B per output site (the oracle's full solve would take hours)"},
           "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2111_04457_b300 as bpp
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = tuple(int(v) for v in args.lattice.split(",")) if args.lattice else L_BENCH
    V = L[0] * L[1] * L[2] * L[3]
    inner = bpp.F16 if args.inner == "f16" else bpp.F32

    U = synth.random_links(L, seed=1)
    b_np = synth.gaussian_spinor(L, seed=2)
    g = bpp.Gauge(torch.from_numpy(U).to(dev), L)
    del U
    b = torch.from_numpy(b_np).to(dev)
    x = torch.empty_like(b)
    opts = bpp.solve_opts(inner_prec=inner, inner_tol=args.inner_tol, use_graph=0 if args.eager else 2,
                          outer_arith=args.outer_arith)
    stream = torch.cuda.current_stream()

    # warm-up (also runs the block-size autotuner on first use)
    for _ in range(args.warmup):
        _, st = bpp.solve(g, b, KAPPA, 0.0, TOL, opts, x=x)
    torch.cuda.synchronize()

    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for p in (0, 1, 2, 3):
        bpp.work_read(p, reset=True)
    bpp.launch_count(reset=True)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        _, st = bpp.solve(g, b, KAPPA, 0.0, TOL, opts, x=x)
        stats.append(st[0])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_local = e0.elapsed_time(e1)
    launches = bpp.launch_count()
    work = {p: bpp.work_read(p, reset=True) for p in (0, 1, 2, 3)}
    clk = clocks.stop()
    ms = allreduce_max(ms_local, world, dev)
    hop_bytes = sum(v[1] for v in work.values())
    hop_bytes_all = allreduce_sum(hop_bytes, world, dev)
    value = hop_bytes_all / (ms / 1000.0) / 1e9
    true_res = max(s["true_resid"] for s in stats)
    # the returned x re-checked with the FP64 D of Eq. (1) (a separate kernel
    # path from the solver's own check)
    true_res_fp64 = (torch.linalg.vector_norm(b - bpp.dirac_apply(g, x, KAPPA)) /
                     torch.linalg.vector_norm(b)).item()

    # per-class timing of one more solve of the same workload, host-driven (no
    # graphs, convergence checked every 4 inner iterations, so a few more
    # iterations than the timed solve): every kernel launch bracketed by CUDA
    # events on its stream
    bpp.prof_enable(True)
    for c in CLASS_NAMES:
        bpp.prof_read(c, reset=True)
    bpp.solve(g, b, KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=inner, inner_tol=args.inner_tol, use_graph=0,
                                                    outer_arith=args.outer_arith), x=x)
    torch.cuda.synchronize()
    bpp.prof_enable(False)
    prof = {c: bpp.prof_read(c, reset=False) for c in (0, 1, 2, 3)}
    peak_hbm, peak_kind = measured_peaks()
    budget = step_budget(bpp, peak_hbm)
    alu = _peak_fp64_fp32(dev)
    n_in, ms_in, by_in = prof[inner]
    n64, ms64, by64 = prof[0]
    # the inner-precision hopping kernel: HBM-bound; bytes = 8 links + input and
    # output spinor per site (392 B for FP16), plus the xpay operand that the
    # second hop of each Schur application reads (52 B, half of the launches)
    # and rhat, read by the hop that also forms <rhat, v> (52 B, a quarter)
    inner_gbs = by_in / (ms_in / 1000.0) / 1e9 if ms_in > 0 else None
    roof_inner = {"bound": "hbm", "achieved": inner_gbs, "peak": peak_hbm, "unit": "GB/s",
                  "frac": (inner_gbs / peak_hbm) if inner_gbs else None, "traffic": None,
                  "kernel": "k_hop inner precision", "peak_kind": peak_kind, "launches": n_in,
                  "avg_us": 1000 * ms_in / max(n_in, 1), "share_ms": ms_in,
                  "bytes_counted": "8 links + in + out spinor per site, + the xpay operand of the second Schur hop, "
                                   "+ rhat where that hop also forms <rhat, v>"}
    # FP64 hopping kernel: bound by the FP64 pipe; 1320 flop per output site.
    # With the double-float check the mixed solve launches none; it is then
    # timed inside one host-driven plain FP64 solve of the same system.
    f64_source = "the mixed solve's FP64 true-residual check"
    if n64 == 0 and not args.no_fp64:
        bpp.prof_enable(True)
        bpp.prof_read(0, reset=True)
        bpp.solve(g, b, KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=bpp.F64, use_graph=0), x=x)
        torch.cuda.synchronize()
        bpp.prof_enable(False)
        n64, ms64, by64 = bpp.prof_read(0, reset=True)
        f64_source = "one host-driven plain FP64 solve of the same system"
    f64_flops = n64 * (V // 2) * 1320.0
    f64_tf = f64_flops / (ms64 / 1000.0) / 1e12 if ms64 > 0 else None
    # the FP64 FMA pipe's measured throughput (cuBLAS DGEMM runs on the FP64
    # tensor cores, not on the pipe this kernel uses)
    f64_peak = alu["fp64"]["peak"]
    roof_f64 = {"bound": "alu", "achieved": f64_tf, "peak": f64_peak, "unit": "TFLOP/s",
                "frac": (f64_tf / f64_peak) if f64_tf else None, "traffic": None,
                "kernel": "k_hop FP64", "timed_in": f64_source,
                "peak_kind": alu["fp64"]["peak_kind"],
                "derived_tflops_context": alu["fp64"]["derived_tflops"],
                "dgemm_tflops_context": alu["fp64"]["gemm_tflops"], "flop_per_site": 1320,
                "launches": n64, "avg_us": 1000 * ms64 / max(n64, 1), "share_ms": ms64,
                "hbm_gbs": (by64 / (ms64 / 1000.0) / 1e9) if ms64 > 0 else None}
    # double-float hopping kernel: bound by the FP32 pipe; DF_OPS_PER_SITE FP32
    # operations per output site; peak = FP32 lane operations per second (half
    # the FMA flop rate)
    nd, msd, byd = prof[3]
    df_tops = nd * (V // 2) * DF_OPS_PER_SITE / (msd / 1000.0) / 1e12 if msd > 0 else None
    df_peak = alu["fp32"]["peak"] / 2.0
    roof_df = {"bound": "alu", "achieved": df_tops, "peak": df_peak, "unit": "Tops/s (FP32 lane operations)",
               "frac": (df_tops / df_peak) if df_tops else None, "traffic": None,
               "kernel": "k_hop double-float (even-odd preparation, outer defects)",
               "peak_kind": alu["fp32"]["peak_kind"] + ", / 2 (an FMA is 2 flop, 1 lane operation)",
               "sgemm_tflops_context": alu["fp32"]["gemm_tflops"],
               "ops_per_site": DF_OPS_PER_SITE, "launches": nd, "avg_us": 1000 * msd / max(nd, 1), "share_ms": msd,
               "hbm_gbs": (byd / (msd / 1000.0) / 1e9) if msd > 0 else None}
    # DRAM traffic per launch of the inner hopping kernel, from the committed
    # ncu capture of this workload (a stored figure: null when the capture does
    # not match this lattice and precision)
    try:
        with open(os.path.join(ROOT, "profiles", "k_hop_f16_32x64_in_solve.json")) as f:
            cap = json.load(f)
        if inner == bpp.F16 and list(L) == cap["lattice"]:
            roof_inner["traffic"] = cap["traffic_bytes_per_launch"]
            roof_inner["traffic_source"] = "stored: profiles/k_hop_f16_32x64_in_solve.md (ncu, not this run)"
    except (OSError, KeyError, ValueError):
        pass
    # the dominant kernel of the timed (mixed) solve
    in_step = [roof_inner, roof_df] + ([roof_f64] if f64_source.startswith("the mixed") else [])
    dominant = max(in_step, key=lambda r: r["share_ms"])

    # e2e: host pinned b -> solve (library copies in and out) -> host x
    b_host = torch.from_numpy(b_np).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    for _ in range(1):
        bpp.solve(g, b_host, KAPPA, 0.0, TOL, opts, x=x_host)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        bpp.solve(g, b_host, KAPPA, 0.0, TOL, opts, x=x_host)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = allreduce_max(e0.elapsed_time(e1), world, dev)
    e2e_value = hop_bytes_all / (e2e_ms / 1000.0) / 1e9

    # plain FP64 solve on the same GPU (comparison of the metric's second half)
    fp64_ms = None
    if not args.no_fp64:
        o64 = bpp.solve_opts(inner_prec=bpp.F64)
        bpp.solve(g, b, KAPPA, 0.0, TOL, o64, x=x)
        torch.cuda.synchronize()
        e0.record(stream)
        _, st64 = bpp.solve(g, b, KAPPA, 0.0, TOL, o64, x=x)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = e0.elapsed_time(e1)
    native_outer_ms = None
    if not args.no_fp64:
        on = bpp.solve_opts(inner_prec=inner, inner_tol=args.inner_tol, use_graph=0 if args.eager else 2, outer_df64=False)
        bpp.solve(g, b, KAPPA, 0.0, TOL, on, x=x)
        torch.cuda.synchronize()
        e0.record(stream)
        bpp.solve(g, b, KAPPA, 0.0, TOL, on, x=x)
        e1.record(stream)
        torch.cuda.synchronize()
        native_outer_ms = e0.elapsed_time(e1)
    # the same solve with the true-residual check in FP64 arithmetic
    fp64_check_ms = None
    if args.outer_arith == 2:
        oc = bpp.solve_opts(inner_prec=inner, inner_tol=args.inner_tol, use_graph=0 if args.eager else 2,
                            outer_arith=1)
        for _ in range(3):
            bpp.solve(g, b, KAPPA, 0.0, TOL, oc, x=x)
        torch.cuda.synchronize()
        e0.record(stream)
        bpp.solve(g, b, KAPPA, 0.0, TOL, oc, x=x)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_check_ms = e0.elapsed_time(e1)
    f32_ms = None
    if inner != bpp.F32:
        o32 = bpp.solve_opts(inner_prec=bpp.F32)
        bpp.solve(g, b, KAPPA, 0.0, TOL, o32, x=x)
        torch.cuda.synchronize()
        e0.record(stream)
        bpp.solve(g, b, KAPPA, 0.0, TOL, o32, x=x)
        e1.record(stream)
        torch.cuda.synchronize()
        f32_ms = e0.elapsed_time(e1)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, sites, secs, cores = cpu_oracle_sample(L, target_s=12.0)
        cpu = {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle D (Eq. 1, plain C loops, OpenMP) on {sites} random sites of the "
                         f"{L[0]}x{L[1]}x{L[2]}x{L[3]} lattice in {secs:.1f} s; 1536 B per output site"}

    workloads = None
    if not args.no_workloads and args.lattice is None and world == 1:
        workloads = {}
        del g
        torch.cuda.synchronize()
        bpp.release_workspace()
        for name in WORKLOADS:
            steps = 2 if name == "clover48" else 5
            workloads[name] = workload_results(name, dev, steps, 3)
            torch.cuda.synchronize()
            bpp.release_workspace()

    if rank != 0:
        return
    ms_step = ms / args.steps
    inner_name = "f16-storage/f32" if inner == bpp.F16 else "f32"
    inner_tol = opts.inner_tol
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"{inner_name} inner, {'double-float' if args.outer_arith == 2 else 'f64'} outer", "data": "synthetic",
        "config": solve_config(L, inner_name, world, args.outer_arith),
        "solve_ms": ms_step,
        "solve_ms_fp64": fp64_ms,
        "solve_ms_f32_inner": f32_ms,
        "solve_ms_fp64_outer_defects": native_outer_ms,
        "speedup_vs_fp64": (fp64_ms / ms_step) if fp64_ms else None,
        "true_resid": true_res,
        "true_resid_fp64_recheck": true_res_fp64,
        "outer_arith": args.outer_arith,
        "solve_ms_fp64_check": fp64_check_ms,
        "inner_tol": inner_tol,
        "graphs": not args.eager,
        "inner_iters": stats[-1]["inner_iters"], "outer_iters": stats[-1]["outer_iters"],
        "hop_launches_per_step": {["f64", "f32", "f16", "f64df"][p]: work[p][0] / args.steps for p in work},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": V * 12 * 16,
                "d2h_bytes_per_step": V * 12 * 16, "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": launches,
        "roofline": dominant,
        "roofline_inner": roof_inner,
        "roofline_fp64": roof_f64,
        "roofline_f64df": roof_df,
        "roofline_timing": "CUDA events around each kernel launch of one extra host-driven solve of the same workload",
        "step_budget": budget,
        "alu_peaks": alu,
        "cpu_baseline": cpu,
        "workloads": workloads,
    }
    print(json.dumps(out), flush=True)


def run_dslash(args, rank, world):
    """The even-odd hopping kernel alone through bpp_dslash (EVEN output from an
    ODD half field), CUDA events around each hopping launch."""
    import torch

    import paper_2111_04457_b300 as bpp
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = tuple(int(v) for v in args.lattice.split(",")) if args.lattice else L_BENCH
    prec = {"f64": bpp.F64, "f32": bpp.F32, "f16": bpp.F16, "f64df": bpp.F64DF}[args.prec]
    g = bpp.Gauge(torch.from_numpy(synth.random_links(L, seed=1)).to(dev), L)
    Vh = L[0] * L[1] * L[2] * L[3] // 2
    dt = torch.complex128 if prec in (bpp.F64, bpp.F64DF) else torch.complex64
    psi = torch.from_numpy(synth.gaussian_spinor(L, seed=2, nrhs=args.nrhs)[:, :Vh]).to(device=dev, dtype=dt)
    for _ in range(args.warmup):
        bpp.dslash(g, psi, KAPPA, bpp.EVEN, prec)
    torch.cuda.synchronize()
    bpp.prof_enable(True)
    bpp.prof_read(prec, reset=True)
    barrier(world)
    for _ in range(args.steps):
        bpp.dslash(g, psi, KAPPA, bpp.EVEN, prec)
    torch.cuda.synchronize()
    bpp.prof_enable(False)
    n, ms, by = bpp.prof_read(prec, reset=True)
    ms = allreduce_max(ms, world, dev)
    by = allreduce_sum(by, world, dev)
    if rank != 0:
        return
    peak, kind = measured_peaks()
    gbs = by / (ms / 1000.0) / 1e9
    print(json.dumps({"metric": "dslash GB/s (hopping kernel alone)", "value": gbs, "unit": "GB/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / max(n, 1) * world,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
                      "data": "synthetic", "config": {"workload": f"even-odd Wilson hopping term {'x'.join(map(str, L))}",
                                                      "lattice": list(L), "nrhs": args.nrhs},
                      "frac_of_hbm": gbs / peak, "peak_kind": kind,
                      "gsites_per_s": n * Vh * args.nrhs / (ms / 1000.0) / 1e9}),
          flush=True)


def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def _peak_fp64_fp32(dev):
    """FP64 and FP32 FMA-pipe throughput measured in this run by the library's
    synthetic FMA kernel (bpp_fma_peak: independent FMA chains on every SM),
    the peak of the ALU-bound hopping kernels, beside cuBLAS DGEMM / SGEMM
    (TF32 off, 4096^3, 2 N^3 flop, best of 3) and the figure derived from the
    unit counts (148 SMs; 2 FP64 and 128 FP32 FMA lanes per SM and clock) at
    the maximum SM clock, as context.  DGEMM runs on the FP64 tensor cores, a
    different unit from the FP64 FMA pipe the FP64 hop uses."""
    import torch

    import paper_2111_04457_b300 as bpp
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, derived in (("fp64", torch.float64, 148 * 2 * 2 * 2.032e9 / 1e12),
                                  ("fp32", torch.float32, 148 * 128 * 2 * 2.032e9 / 1e12)):
            n = 4096
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            tf = 2.0 * n ** 3 / (best / 1e3) / 1e12
            fma = bpp.fma_peak(bpp.F64 if name == "fp64" else bpp.F32)
            out[name] = {"fma_pipe_tflops": fma, "gemm_tflops": tf, "derived_tflops": derived,
                         "peak": fma, "peak_kind": "measured: bpp_fma_peak (FMA pipe, synthetic FMA chains)"}
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


# Double-float (FP32 hi + lo) operations the even-odd hopping kernel performs
# per output site, counted from the df64 algorithm as written (df add 8 FP32
# operations, TwoProd with cross terms 4, lazy accumulation 8, renormalisation
# 3): per hop 12 df adds (projection) + 12 outputs x (6 products + 5 lazy adds
# + 1 renormalisation) + 24 df adds (reconstruction) = 1092; 8 hops; + the -kappa
# scaling (24 df products of 7) and the normalised stores (24 x 3).
DF_OPS_PER_SITE = 8 * (12 * 8 + 12 * (6 * 4 + 5 * 8 + 3) + 24 * 8) + 24 * 7 + 24 * 3

CLASS_NAMES = {0: "hop_f64", 1: "hop_f32", 2: "hop_f16", 3: "hop_f64df", 4: "krylov_vector",
               5: "outer_vector", 6: "layout", 7: "control", 8: "clover", 9: "force"}


def step_budget(bpp, peak_hbm):
    """Per kernel class of one profiled solve: launches, ms, share of the GPU
    time, algorithmic GB/s and its fraction of the HBM peak."""
    rows, total = {}, 0.0
    for c, name in CLASS_NAMES.items():
        n, ms, by = bpp.prof_read(c, reset=True)
        if n == 0:
            continue
        total += ms
        rows[name] = {"launches": n, "ms": ms, "bytes": by,
                      "gbs": (by / (ms / 1e3) / 1e9) if (ms > 0 and by > 0) else None}
    for r in rows.values():
        r["share"] = r["ms"] / total if total > 0 else None
        r["frac_hbm"] = (r["gbs"] / peak_hbm) if r["gbs"] else None
    return {"classes": rows, "gpu_ms": total}


def workload_results(name, dev, steps, warm):
    """One of the other workloads (batched, clover, gradient, plain FP64), timed
    with CUDA events on the current stream: ms per step, algorithmic GB/s of the
    hopping kernels, true residuals, and the oracle's CPU time where it is
    feasible."""
    import numpy as np
    import torch

    import paper_2111_04457_b300 as bpp
    import synth
    from paper_2111_04457_b300.autograd import solve_fn
    stream = torch.cuda.current_stream()
    out = {}

    def work_bytes(reset=True):
        return sum(bpp.work_read(p, reset=reset)[1] for p in (0, 1, 2, 3))

    if name == "configs0_8x8x8x8":
        L = (8, 8, 8, 8)
        U_np = synth.random_links(L, seed=1)
        b_np = synth.gaussian_spinor(L, seed=2)
        g = bpp.Gauge(torch.from_numpy(U_np).to(dev), L)
        b = torch.from_numpy(b_np).to(dev)
        V = L[0] * L[1] * L[2] * L[3]
        par = (np.indices(L[::-1]).sum(axis=0).ravel()) & 1        # parity of lexicographic sites
        be, bo = b[torch.from_numpy(np.flatnonzero(par == 0)).to(dev)], b[torch.from_numpy(np.flatnonzero(par == 1)).to(dev)]
        ms_d, out_e = _timed(lambda: bpp.dslash(g, bo, KAPPA, bpp.EVEN, bpp.F64), 50, 5, stream)
        # bhat = b_e - D_eo b_o = b_e - (-kappa H_eo b_o); the library stops on the
        # full-D residual = Schur residual x ||bhat|| / ||b||
        bhat_n = torch.linalg.vector_norm(be - out_e).item()
        tol = 1e-12 * bhat_n / torch.linalg.vector_norm(b).item()
        o = bpp.solve_opts(inner_prec=bpp.F64)
        work_bytes()
        ms, st = _timed(lambda: bpp.solve(g, b, KAPPA, 0.0, tol, o)[1], steps, warm, stream)
        by = work_bytes() / (steps + warm)
        import oracle
        t0 = time.perf_counter()
        oracle.solve(U_np, b_np, KAPPA, L, tol=1e-12)
        cpu_s = time.perf_counter() - t0
        out = {"workload": "plain FP64 on 8^4: one dslash, then FP64 even-odd BiCGStab to Schur residual 1e-12",
               "dslash_ms": ms_d, "dslash_gbs": (V // 2) * BYTES_F64 / (ms_d / 1e3) / 1e9,
               "dslash_note": "8^4 fits in L2: an L2 figure, not an HBM one",
               "ms_per_step": ms, "gbs": by / (ms / 1e3) / 1e9, "true_resid": st[0]["true_resid"],
               "schur_resid_target": 1e-12, "inner_iters": st[0]["inner_iters"],
               "oracle_solve_s": cpu_s, "oracle_threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}
    elif name == "prop24":
        L = (24, 24, 24, 48)
        g = bpp.Gauge(torch.from_numpy(synth.random_links(L, seed=1)).to(dev), L)
        b = torch.from_numpy(np.stack([synth.point_source(L, i) for i in range(12)])).to(dev)
        x = torch.empty_like(b)
        o = bpp.solve_opts(inner_prec=bpp.F32)
        work_bytes()
        ms, st = _timed(lambda: bpp.solve(g, b, KAPPA, 0.0, TOL, o, x=x)[1], steps, warm, stream)
        by = work_bytes() / (steps + warm)
        xs = torch.empty_like(b[0])
        ms1, _ = _timed(lambda: [bpp.solve(g, b[i], KAPPA, 0.0, TOL, o, x=xs) for i in range(12)], 1, warm, stream)
        # the batched FP32 hop alone (12 sources, plain epilogue): algorithmic
        # bytes per site and source (links counted once per launch) and time
        Vh = L[0] * L[1] * L[2] * L[3] // 2
        bh = b[:, :Vh].to(torch.complex64).contiguous()
        bpp.dslash(g, bh, KAPPA, bpp.EVEN, bpp.F32)
        torch.cuda.synchronize()
        bpp.prof_enable(True)
        bpp.prof_read(1, reset=True)
        for _ in range(10):
            bpp.dslash(g, bh, KAPPA, bpp.EVEN, bpp.F32)
        torch.cuda.synchronize()
        bpp.prof_enable(False)
        n32, ms32, by32 = bpp.prof_read(1, reset=True)
        # where the time goes: one host-driven batched solve and one
        # host-driven single-source solve, every launch timed
        peak_hbm, _ = measured_peaks()
        budgets = {}
        for key, bb, xx in (("batched_12", b, x), ("single_source", b[0], xs)):
            bpp.prof_enable(True)
            for c in CLASS_NAMES:
                bpp.prof_read(c, reset=True)
            bpp.solve(g, bb, KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=bpp.F32, use_graph=0), x=xx)
            torch.cuda.synchronize()
            bpp.prof_enable(False)
            budgets[key] = step_budget(bpp, peak_hbm)
        out = {"workload": "12 spin-colour point sources on 24^3x48, one batched solve (FP32 inner, double-float outer) "
                           "to true resid 1e-10",
               "ms_per_step": ms, "gbs": by / (ms / 1e3) / 1e9, "ms_per_rhs": ms / 12,
               "fp32_hop_12_sources_us": 1000 * ms32 / max(n32, 1),
               "fp32_hop_bytes_per_site_rhs": by32 / max(n32, 1) / (Vh * 12),
               "fp32_hop_12_sources_gbs": by32 / (ms32 / 1e3) / 1e9 if ms32 > 0 else None,
               "ms_12_sequential_single_rhs": ms1, "batching_speedup": ms1 / ms,
               "true_resid_max": max(s["true_resid"] for s in st), "step_budgets": budgets}
    elif name == "uneven6":
        lats = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (16, 16, 16, 32), (20, 20, 20, 40), (24, 24, 24, 48)]
        kap = synth.uniform_kappas(len(lats), seed=4)
        gs = [bpp.Gauge(torch.from_numpy(synth.random_links(L, seed=1)).to(dev), L) for L in lats]
        bs = [torch.from_numpy(synth.gaussian_spinor(L, seed=2 + i)).to(dev) for i, L in enumerate(lats)]
        xs = [torch.empty_like(b) for b in bs]
        o = bpp.solve_opts(inner_prec=bpp.F32)
        work_bytes()
        ms, st = _timed(lambda: bpp.solve_batch(gs, bs, kap, TOL, o, xs=xs)[1], steps, warm, stream)
        by = work_bytes() / (steps + warm)
        ms1, _ = _timed(lambda: [bpp.solve(gs[i], bs[i], kap[i], 0.0, TOL, o, x=xs[i]) for i in range(6)], 1, warm,
                        stream)
        out = {"workload": "6 lattices 8^4 12^4 16^4 16^3x32 20^3x40 24^3x48 (1204992 sites), kappa U[0.10,0.12], "
                           "one batched solve (FP32 inner, double-float outer) to true resid 1e-10",
               "ms_per_step": ms, "gbs": by / (ms / 1e3) / 1e9, "ms_6_sequential": ms1, "batching_speedup": ms1 / ms,
               "true_resid_max": max(s["true_resid"] for s in st)}
    elif name == "clover48":
        L = (48, 48, 48, 96)
        csw = 1.0
        g = bpp.Gauge(torch.from_numpy(synth.random_links(L, seed=1)).to(dev), L)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.clover_build(KAPPA, csw)
        torch.cuda.synchronize()
        build_ms = 1000 * (time.perf_counter() - t0)
        b = torch.from_numpy(synth.gaussian_spinor(L, seed=2, nrhs=4)).to(dev)
        eta = torch.from_numpy(synth.gaussian_spinor(L, seed=3, nrhs=4)).to(dev)

        def step():
            bb = b.clone().requires_grad_(True)
            xx = solve_fn(None, bb, L, KAPPA, csw=csw, tol=TOL, inner_prec=bpp.F16, gauge=g)
            torch.vdot(eta.reshape(-1), xx.reshape(-1)).real.backward()
            return xx.detach(), bb.grad
        work_bytes()
        ms, (xx, lam) = _timed(step, steps, warm, stream)
        by = work_bytes() / (steps + warm)
        res_x = max((torch.linalg.vector_norm(b[r] - bpp.dirac_apply(g, xx[r], KAPPA, csw)) /
                     torch.linalg.vector_norm(b[r])).item() for r in range(4))
        res_l = max((torch.linalg.vector_norm(eta[r] - bpp.dirac_apply(g, lam[r], KAPPA, csw, dagger=True)) /
                     torch.linalg.vector_norm(eta[r])).item() for r in range(4))
        out = {"workload": "Wilson-clover c_SW=1 48^3x96, 4 Gaussian RHS: forward solve + adjoint solve for grad_b "
                           "(FP16-storage inner, double-float outer, true resid 1e-10)",
               "ms_per_step": ms, "gbs": by / (ms / 1e3) / 1e9, "clover_build_ms": build_ms,
               "true_resid_max": res_x, "adjoint_true_resid_max": res_l}
        del g, b, eta, xx, lam
    elif name == "grad16":
        L = (16, 16, 16, 32)
        U_np = synth.random_links(L, seed=1)
        b_np, eta_np = synth.gaussian_spinor(L, seed=2), synth.gaussian_spinor(L, seed=3)
        U = torch.from_numpy(U_np).to(dev)
        b = torch.from_numpy(b_np).to(dev)
        eta = torch.from_numpy(eta_np).to(dev)
        g = bpp.Gauge(U, L)

        def step():
            UU = U.clone().requires_grad_(True)
            bb = b.clone().requires_grad_(True)
            xx = solve_fn(UU, bb, L, KAPPA, tol=1e-12, inner_prec=bpp.F64, gauge=g)
            torch.vdot(eta.reshape(-1), xx.reshape(-1)).real.backward()
            return UU.grad
        work_bytes()
        ms, gU = _timed(step, steps, warm, stream)
        by = work_bytes() / (steps + warm)
        # per-class time of one more step (the link-gradient kernel is class 9)
        bpp.prof_enable(True)
        for c in CLASS_NAMES:
            bpp.prof_read(c, reset=True)
        step()
        torch.cuda.synchronize()
        bpp.prof_enable(False)
        budget = step_budget(bpp, measured_peaks()[0])
        import oracle
        t0 = time.perf_counter()
        x_o = oracle.solve(U_np, b_np, KAPPA, L, tol=1e-12)
        lam_o = oracle.solve(U_np, eta_np, KAPPA, L, tol=1e-12, dagger=True)
        G_o = oracle.link_gradient(x_o, lam_o, KAPPA, L)
        cpu_s = time.perf_counter() - t0
        err = float(np.linalg.norm(gU.cpu().numpy() - G_o) / np.linalg.norm(G_o))
        out = {"workload": "L = Re<eta, D^-1 b> on 16^3x32 FP64: forward solve, adjoint solve, recomputed x, "
                           "link-gradient kernel",
               "ms_per_step": ms, "gbs": by / (ms / 1e3) / 1e9, "grad_U_rel_err_vs_oracle": err,
               "force_kernel_ms": budget["classes"].get("force", {}).get("ms"), "step_budget": budget,
               "oracle_s": cpu_s, "oracle_threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}
    elif name == "mg16":
        # multigrid-preconditioned GCR (FP32, FP64 defect correction) against
        # the lexical BiCGStab with the same outer loop, 16^3x32, kappa 0.12
        L = (16, 16, 16, 32)
        g = bpp.Gauge(torch.from_numpy(synth.random_links(L, seed=1)).to(dev), L)
        b = torch.from_numpy(synth.gaussian_spinor(L, seed=2)).to(dev)
        vecs = torch.from_numpy(np.stack([synth.gaussian_spinor(L, seed=60 + k) for k in range(6)])).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mg = bpp.Multigrid(g, KAPPA, vecs, (4, 4, 4, 4), refine=1)
        torch.cuda.synchronize()
        setup_ms = 1000 * (time.perf_counter() - t0)
        o = bpp.solve_opts(max_inner=200)
        ms, st = _timed(lambda: mg.solve(b, TOL, o)[1], steps, warm, stream)
        ol = bpp.solve_opts(inner_prec=bpp.F32)
        ms_l, st_l = _timed(lambda: bpp.solve_lex(g, b, KAPPA, 0.0, TOL, bpp.LEX_D, ol)[1], steps, warm, stream)
        oe = bpp.solve_opts(inner_prec=bpp.F32)
        ms_e, st_e = _timed(lambda: bpp.solve(g, b, KAPPA, 0.0, TOL, oe)[1], steps, warm, stream)
        del mg
        # near the critical kappa of smoother links (exp(i 0.1 H)): the regime
        # where the coarse correction pays in iterations (one timed solve each)
        U1 = torch.from_numpy(synth.random_links(L, seed=1, eps=0.1)).to(dev)
        g1 = bpp.Gauge(U1, L)
        kc = 0.127
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mg1 = bpp.Multigrid(g1, kc, vecs, (4, 4, 4, 4), refine=3)
        torch.cuda.synchronize()
        setup1 = 1000 * (time.perf_counter() - t0)
        ms1, st1 = _timed(lambda: mg1.solve(b, TOL, o)[1], 1, 1, stream)
        ms1e, st1e = _timed(lambda: bpp.solve(g1, b, kc, 0.0, TOL, oe)[1], 1, 3, stream)
        del mg1, g1, U1
        out = {"workload": "16^3x32 Wilson, one Gaussian RHS: two-level multigrid (4^4 blocks, 6 near-null vectors "
                           "refined by inverse iteration) preconditioning flexible GCR in FP32 under FP64 defect "
                           "correction, against lexical and even-odd BiCGStab (FP32 inner); at kappa 0.12 (links "
                           "exp(i 0.3 H)) and near the critical kappa (links exp(i 0.1 H), kappa 0.127)",
               "ms_per_step": ms, "gbs": 0.0, "setup_ms": setup_ms, "gcr_iters": st[0]["inner_iters"],
               "true_resid": st[0]["true_resid"], "lex_bicgstab_ms": ms_l,
               "lex_bicgstab_iters": st_l[0]["inner_iters"], "lex_true_resid": st_l[0]["true_resid"],
               "eo_bicgstab_ms": ms_e, "eo_bicgstab_iters": st_e[0]["inner_iters"],
               "near_critical": {"kappa": kc, "link_eps": 0.1, "mg_setup_ms": setup1, "mg_ms": ms1,
                                 "mg_gcr_iters": st1[0]["inner_iters"], "mg_true_resid": st1[0]["true_resid"],
                                 "eo_bicgstab_ms": ms1e, "eo_bicgstab_iters": st1e[0]["inner_iters"],
                                 "eo_true_resid": st1e[0]["true_resid"]}}
    elif name == "dd16":
        # the decomposed FP64 solve (slabs in x4 on this GPU) against the
        # undecomposed FP64 solve, 16^3x32
        L = (16, 16, 16, 32)
        U = torch.from_numpy(synth.random_links(L, seed=1)).to(dev)
        g = bpp.Gauge(U, L)
        b = torch.from_numpy(synth.gaussian_spinor(L, seed=2)).to(dev)
        o = bpp.solve_opts(inner_prec=bpp.F64, use_graph=0)
        ms0, st0 = _timed(lambda: bpp.solve(g, b, KAPPA, 0.0, TOL, o)[1], steps, warm, stream)
        out = {"workload": "16^3x32 Wilson FP64 even-odd BiCGStab to 1e-10: decomposition into 2 and 4 slabs in x4 "
                           "(faces exchanged by device copies, per-slab reductions summed across slabs) against the "
                           "undecomposed host-driven solve",
               "ms_per_step": ms0, "gbs": 0.0, "undecomposed_ms": ms0, "undecomposed_iters": st0[0]["inner_iters"]}
        for nd in (2, 4):
            dd = bpp.DomainDecomposition(U, L, nd)
            msd, std = _timed(lambda: dd.solve(b, KAPPA, TOL)[1], steps, warm, stream)
            out[f"slabs{nd}_ms"] = msd
            out[f"slabs{nd}_iters"] = std[0]["inner_iters"]
            out[f"slabs{nd}_true_resid"] = std[0]["true_resid"]
            del dd
    elif name == "errors8":
        # each result's error against the FP64 oracle, per precision, on 8^4
        # (the oracle computes every site): the hopping term of Eq. (1) and
        # the solution x of the mixed-precision solves (true residual 1e-10)
        import oracle
        L = (8, 8, 8, 8)
        U_np = synth.random_links(L, seed=1)
        g = bpp.Gauge(torch.from_numpy(U_np).to(dev), L)
        psi = synth.gaussian_spinor(L, seed=2)
        Vh = 2048
        half = psi[oracle.parity_sites(L, 1)]
        ref = oracle.hop_eo(U_np, half, KAPPA, L, 0)

        def rel(a, b):
            return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
        errs = {}
        for nm, pr in (("f64", bpp.F64), ("f64df", bpp.F64DF), ("f32", bpp.F32), ("f16", bpp.F16)):
            dt = torch.complex128 if pr in (bpp.F64, bpp.F64DF) else torch.complex64
            o_ = bpp.dslash(g, torch.from_numpy(half).to(device=dev, dtype=dt), KAPPA, bpp.EVEN, pr)
            errs["dslash_" + nm] = rel(o_.cpu().numpy().astype(np.complex128), ref)
        x_ref = oracle.solve(U_np, psi, KAPPA, L, tol=1e-13)
        for nm, pr in (("f64", bpp.F64), ("f32", bpp.F32), ("f16", bpp.F16)):
            x_, st_ = bpp.solve(g, torch.from_numpy(psi).to(dev), KAPPA, 0.0, TOL, bpp.solve_opts(inner_prec=pr))
            xn = x_.cpu().numpy()
            errs["solve_x_" + nm + "_inner"] = rel(xn, x_ref)
            errs["solve_true_resid_" + nm + "_inner"] = oracle.true_residual(U_np, psi, xn, KAPPA, L)
        out = {"workload": "errors against the FP64 oracle on 8^4 (seed-1 links, kappa 0.12): the even-odd "
                           "hopping term per precision (norm-relative, inputs in the precision's canonical type), "
                           "and the solution x of solves to true residual 1e-10 per inner precision",
               "ms_per_step": 0.0, "gbs": 0.0, **errs}
    torch.cuda.synchronize()
    out["steps"], out["warmup"] = steps, warm
    return out


WORKLOADS = ["configs0_8x8x8x8", "errors8", "prop24", "uneven6", "grad16", "mg16", "dd16", "clover48"]


def run_workload(args, rank, world):
    """One of the other workloads as its own JSON line."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    r = workload_results(args.workload, dev, args.steps, max(args.warmup, 3))
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": r["gbs"], "unit": "GB/s", "n_gpus": world, "steps": r["steps"],
                          "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "data": "synthetic",
                          "config": {"workload": r["workload"]}, "result": r}), flush=True)


def main():
    args = parse()
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.mode == "dslash":
        run_dslash(args, rank, world)
    elif args.workload != "wilson32":
        run_workload(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
