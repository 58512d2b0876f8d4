"""Benchmark of the explicit finite-volume step (arXiv 2006.01748) on GB300.

Metric: cell-updates/s of the fused FP32 (+Kahan) forward step, next to the
plain FP64 step on the same grid, the % of the measured HBM roofline, and
the adjoint / forward time ratio.

Workload (one bench step): the 8192 x 8192 heterogeneous tissue
(lambda in [0.01, 1], delta=12.5, rho=1, D=4e-5, c=70, disk r=0.1), 5000
explicit Euler steps of the fused FP32 + Kahan kernel with the tuned
temporal-blocking depth, then the FP64 diagnostics of the final state.
Inputs are synthetic and seeded; the 4 GB working set is larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own instance (weak scaling,
no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s FP32 fused vs FP64 plain, % HBM roofline; adjoint/forward time"
BYTES_PER_CELL_PASS = {"fp32_kahan": 60, "fp32": 36, "fp64": 72}
# The method's FP32 flops per cell-step with each face flux evaluated once
# (an FMA counts 2): tumour faces 2 x 6, acid faces 2 x 7, cross-term
# differences and products 4, the two divergences 6, reactions 13, updates
# 3 x 2 (Euler) or 3 x 5 (Kahan).
FLOPS_PER_CELL_STEP = {"fp32": 55, "fp32_kahan": 64}
# The plain FP64 step's arithmetic per cell-step as step64_kernel writes it
# (every face evaluated from both sides, an FMA counts 2): tumour faces
# 4 x 5, their divergence 5, acid diagonal faces 4 x 3, tangential
# differences 6, cross terms 4 x 3, the acid divergence 10, reactions 13,
# Euler updates 3 x 2.
FLOPS_PER_CELL_STEP_FP64 = 84
# nominal HBM3e bandwidth of a GB300 (about 8 TB/s); every HBM fraction is
# reported against the measured copy bandwidth ("frac") and against this
HBM_NOMINAL_GBS = 8000.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=8192)
    ap.add_argument("--time-steps", type=int, default=5000)
    ap.add_argument("--steps-per-pass", type=int, default=0)
    ap.add_argument("--fp64-time-steps", type=int, default=100)
    ap.add_argument("--adjoint-steps", type=int, default=10000)
    ap.add_argument("--ensemble-steps", type=int, default=5000)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 / adjoint / CPU legs")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed plumbing

class Dist:
    """Rank bookkeeping from the torchrun environment.  NCCL when CUDA is
    available, gloo otherwise; used only for the barrier and the max over
    ranks of the timed region (no data-path collective)."""

    def __init__(self, n=None, backend=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            self.device = "cuda" if backend == "nccl" else "cpu"
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, dist):
    import oracle
    from paper_2006_01748_gb300 import inputs
    oracle.build()
    p = inputs.hetero_8192(nx=args.nx, steps=args.time_steps)
    s, a = oracle.setup_for(p)
    # each step: a bounded sample of the workload, 1 explicit step on the full grid
    sample_steps = 1
    U, V, W = p.u0, p.v0, p.w0
    for _ in range(args.warmup):
        U, V, W = oracle.run(s, *a, U, V, W, sample_steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, V, W = oracle.run(s, *a, U, V, W, sample_steps)
    el = time.perf_counter() - t0
    cells = p.cells * sample_steps * args.steps
    value = cells / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(p, args, None),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample_steps} explicit step of the {p.nx}x{p.ny} grid per bench step"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(p, args, T):
    return {"workload": f"hetero_8192: {p.nx}x{p.ny} cells, FP32 fused step with Kahan-compensated state, "
                        f"{args.time_steps} explicit steps per bench step, lambda in [0.01,1], delta=12.5, "
                        f"rho=1, D=4e-5, c=70",
            "cells": p.cells, "time_steps_per_bench_step": args.time_steps, "steps_per_pass": T,
            "l2": "inputs larger than L2 (working set 60 B/cell = %.1f GB)" % (60 * p.cells / 1e9),
            "parallelism": f"{args.gpus} independent instance(s), one per GPU"}


# ---------------------------------------------------------------- our arm

def cpu_baseline_leg(p):
    """The oracle as it stands, one host core, a bounded sample of the same
    workload (3 explicit steps on the full grid)."""
    import oracle
    oracle.build()
    s, a = oracle.setup_for(p)
    n = 3
    t0 = time.perf_counter()
    oracle.run(s, *a, p.u0, p.v0, p.w0, n)
    el = time.perf_counter() - t0
    return {"value": p.cells * n / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} explicit steps of the {p.nx}x{p.ny} grid ({el:.1f} s)"}


def cpu_openmp_leg(p):
    """The same oracle source built with OpenMP over every host core (the row
    loop of its step), a bounded sample of the same workload; a second,
    reported CPU figure beside the one-core baseline.  None without OpenMP."""
    import oracle
    lib = oracle.build_openmp()
    if lib is None:
        return None
    oracle.use_library(lib)
    try:
        s, a = oracle.setup_for(p)
        threads = oracle.threads()
        n = max(3, min(48, 3 * threads))
        oracle.run(s, *a, p.u0, p.v0, p.w0, 1)  # spins up the thread pool
        t0 = time.perf_counter()
        oracle.run(s, *a, p.u0, p.v0, p.w0, n)
        el = time.perf_counter() - t0
    finally:
        oracle.use_library(None)
    return {"value": p.cells * n / el, "unit": "cell-updates/s", "cores": threads, "kind": "oracle (OpenMP build)",
            "sample": f"{n} explicit steps of the {p.nx}x{p.ny} grid ({el:.1f} s)"}


def profiled_traffic(kind: str, T: int, prec: str, chunk: int, cells: int):
    """DRAM bytes per launch of the plan (kind, T, prec) from
    profiles/dram_traffic.txt (one ncu capture per plan on a 4096^2 grid),
    at the captured chunk height nearest to `chunk`, scaled to `cells` by
    the cells processed; None if the plan was not captured."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    best = None
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) < 4 or line.startswith("#"):
                    continue
                if parts[0] != kind or parts[1] != f"T={T}" or parts[2] != prec:
                    continue
                kv = dict(x.split("=") for x in parts[3:] if "=" in x)
                d = abs(int(kv["chunk"]) - chunk)
                if best is None or d < best[0]:
                    best = (d, int(kv["total"]) * cells / int(kv["cells"]))
    except (OSError, KeyError, ValueError):
        return None
    return None if best is None else best[1]


def measured_alu_peaks():
    """FMA rates measured on this GPU by the library's probe (flop/s):
    FP64, FP32 scalar, FP32 packed pairs."""
    from paper_2006_01748_gb300 import gg
    out = {}
    for name, kind, iters in (("fp64", 0, 20000), ("fp32", 1, 1000000), ("fp32x2", 2, 500000)):
        best = 0.0
        for _ in range(2):
            rc, f = gg.gg_probe_fma_rate(kind, iters, 4)
            if rc == gg.GG_OK:
                best = max(best, f)
        out[name] = best / 1e12
    return out


def error_leg():
    """Measured relative max-norm errors against the FP64 oracle, outside the
    timed region: the bench tissue's generator at 512 x 512 (same parameters,
    grid-independent fields) for 5000 steps in each precision, per field; and
    the adjoint workload's configuration at 128 x 128 for 10^4 steps (twin
    target v-misfit), per gradient."""
    import torch
    import oracle
    from paper_2006_01748_gb300 import gg, inputs

    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))

    out = {}
    q = inputs.hetero_8192(nx=512, steps=5000)
    lib = oracle.build_openmp()
    if lib:
        oracle.use_library(lib)  # same bits as the serial build, faster
    try:
        s, a = oracle.setup_for(q)
        ref = oracle.run(s, *a, q.u0, q.v0, q.w0, q.steps)
    finally:
        oracle.use_library(None)
    fwd = {}
    for prec in ("fp64", "fp32_kahan", "fp32"):
        with gg.GGSim.from_problem(q, precision=prec) as sim:
            sim.step(q.steps)
            got = sim.state()
        fwd[prec] = {f: rel(g, r) for f, g, r in zip("uvw", got, ref)}
    out["forward"] = {"workload": "hetero_8192 generator at 512x512, 5000 steps", **fwd}
    p = inputs.adjoint_2048(nx=128, steps=10000)
    tg = inputs.adjoint_2048(nx=128, steps=10000, target=True)
    s, a = oracle.setup_for(p)
    st, at = oracle.setup_for(tg, dt=s.dt)
    Vs = oracle.run(st, *at, tg.u0, tg.v0, tg.w0, p.steps)[1]
    V = oracle.run(s, *a, p.u0, p.v0, p.w0, p.steps)[1]
    gV = oracle.misfit_grad(V, Vs, s.dx, s.dy)
    z = np.zeros_like(V)
    lam0, ga, gs = oracle.adjoint(s, *a, p.u0, p.v0, p.w0, p.steps, z, gV, z)
    gth, gl1, gl2 = oracle.coefficients_vjp(p.theta, p.lambda1, p.lambda2, *ga)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", dt=s.dt) as sim:
        r = sim.adjoint(p.steps, None, torch.from_numpy(gV.astype(np.float32)).cuda().view(-1), None)
    adj = {k: rel(r[k].cpu().numpy().astype(np.float64), ref) for k, ref in
           (("theta", gth), ("lambda1", gl1), ("lambda2", gl2), ("u0", lam0[0]), ("v0", lam0[1]), ("w0", lam0[2]))}
    for qq, name in enumerate(("delta", "rho", "D", "c")):
        adj[name] = abs(r["scalars"][qq] - gs[qq]) / abs(gs[qq])
    out["adjoint"] = {"workload": "adjoint_2048 configuration at 128x128, 10^4 steps, twin-target v-misfit",
                      "precision": "fp32_kahan", **adj}
    out["metric"] = "max|F_gpu - F_oracle| / max|F_oracle| (rate gradients: relative difference)"
    return out


def timed_steps(sim, n, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    sim.step(n)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def run_ours(args, dist):
    import torch
    from paper_2006_01748_gb300 import build, gg, inputs
    torch.cuda.set_device(dist.local)
    build()
    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream(dev)
    p = inputs.hetero_8192(nx=args.nx, steps=args.time_steps, seed=inputs.SEED_HETERO_8192 + dist.rank)
    sim = gg.GGSim.from_problem(p, precision="fp32_kahan", steps_per_pass=args.steps_per_pass)
    plan = sim.plan()
    T = plan["T"]
    n_inner = args.time_steps
    passes = -(-n_inner // T)
    launches_per_step = passes + 2  # step passes + diagnostics partial/final

    for _ in range(args.warmup):
        sim.step(n_inner)
        rc, _d = gg.gg_diagnostics(sim.handle)
        if rc != gg.GG_OK:
            raise RuntimeError(f"diagnostics failed: {rc} {gg.gg_last_error(sim.handle)}")
    torch.cuda.synchronize()

    # timed region: K bench steps bracketed by barrier + synchronize
    clocks = ClockSampler(dist.local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kev = []
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(n_inner)
        b.record(stream)
        kev.append((a, b))
        gg.gg_diagnostics(sim.handle)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dist.barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = dist.max(ms)
    step_ms = [a.elapsed_time(b) for a, b in kev]
    launch_ms = statistics.mean(step_ms) / passes
    value = p.cells * n_inner * args.steps * dist.world / (ms_max / 1e3)

    peak, peak_kind = measured_peaks()
    if plan["kind"] == "warp":
        kname = "stepw1_kernel<Kahan>" if T == 1 else f"stepw_kernel<T={T},Kahan>"
    elif plan["kind"] == "warp2":
        kname = "stepw2_1_kernel<Kahan>" if T == 1 else f"stepw2_kernel<T={T},Kahan>"
    else:
        kname = f"step32_kernel<T={T},Kahan>"
    alg_bytes = BYTES_PER_CELL_PASS["fp32_kahan"] * p.cells
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    traffic = profiled_traffic(plan["kind"], T, "kahan", plan["by"], p.cells)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "frac_nominal": achieved / HBM_NOMINAL_GBS, "peak_nominal": HBM_NOMINAL_GBS,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": kname, "chunk_rows": plan["by"],
                "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": launch_ms,
                "note": "one launch = one pass of T explicit steps: 60 B/cell of state and tensor traffic",
                # temporally blocked: the same throughput against the roof of the one-step pass
                # (60 B per cell-update at the measured HBM bandwidth)
                "t1_roof_cell_updates_per_s": peak * 1e9 / 60, "value_over_t1_roof": value / dist.world / (peak * 1e9 / 60)}

    # the same step seen from the FP32 units: the method's flops per cell-step
    # (each face flux evaluated once: tumour faces 2 x 6, acid faces 2 x 7 + 4
    # per cell for the cross terms, divergences 6, reactions 13, Kahan updates
    # 3 x 5) against the CUDA-core FP32 peak from unit counts and clock
    # (152 SMs x 128 FP32 lanes x 2 flops per FMA x the SM clock under load)
    sm_ghz = (ck.get("sm_mhz") or 2070.0) / 1e3
    fp32_peak = 152 * 128 * 2 * sm_ghz / 1e3  # TFLOP/s
    flops = FLOPS_PER_CELL_STEP["fp32_kahan"] * value / dist.world / 1e12
    roofline_alu = {"bound": "alu", "achieved": flops, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": flops / fp32_peak, "flops_per_cell_step": FLOPS_PER_CELL_STEP["fp32_kahan"],
                    "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz (the measured FMA-chain rate "
                                 "is in alu_peaks_tflops)" % (sm_ghz * 1e3)}

    extras = {}
    if not args.no_extras:
        # the same step with one step per pass (the HBM-bound configuration)
        for name, prec in (("fp32_kahan_T1", "fp32_kahan"), ("fp32_T1", "fp32")):
            s2 = gg.GGSim.from_problem(p, precision=prec, steps_per_pass=1)
            s2.step(20)
            n2 = 200
            ms2 = timed_steps(s2, n2, stream)
            pl2 = s2.plan()
            s2.close()
            bpc = BYTES_PER_CELL_PASS[prec]
            ach2 = bpc * p.cells / (ms2 / 1e3 / n2) / 1e9
            extras[name] = {"value": p.cells * n2 / (ms2 / 1e3), "unit": "cell-updates/s",
                            "roofline": {"bound": "hbm", "achieved": ach2, "peak": peak, "unit": "GB/s",
                                         "frac": ach2 / peak, "frac_nominal": ach2 / HBM_NOMINAL_GBS,
                                         "kernel": f"{'stepw2_1_kernel' if pl2['kind'] == 'warp2' else 'stepw1_kernel'}"
                                                   f"<{prec}>",
                                         "chunk_rows": pl2["by"],
                                         "traffic": profiled_traffic(pl2["kind"], 1, "kahan" if prec == "fp32_kahan"
                                                                     else "plain", pl2["by"], p.cells)}}
        # plain FP64 step on the same grid (fewer time steps; throughput is per cell-update)
        sim64 = gg.GGSim.from_problem(p, precision="fp64")
        sim64.step(5)
        ms64 = timed_steps(sim64, args.fp64_time_steps, stream)
        sim64.close()
        v64 = p.cells * args.fp64_time_steps / (ms64 / 1e3)
        alu = measured_alu_peaks()
        fl64 = FLOPS_PER_CELL_STEP_FP64 * v64 / 1e12
        extras["fp64_plain"] = {"value": v64, "unit": "cell-updates/s", "time_steps": args.fp64_time_steps,
                                "kernel": "step64_kernel",
                                "roofline": {"bound": "alu", "achieved": fl64, "peak": alu["fp64"],
                                             "unit": "TFLOP/s", "frac": fl64 / alu["fp64"] if alu["fp64"] else None,
                                             "flops_per_cell_step": FLOPS_PER_CELL_STEP_FP64,
                                             "peak_kind": "measured: FP64 FMA chains (gg_probe_fma_rate)"},
                                "hbm_frac": 72 * p.cells / (ms64 / 1e3 / args.fp64_time_steps) / 1e9 / peak,
                                "hbm_frac_nominal": 72 * p.cells / (ms64 / 1e3 / args.fp64_time_steps) / 1e9
                                                    / HBM_NOMINAL_GBS,
                                "fp32_over_fp64": value / dist.world / v64}
        extras["alu_peaks_tflops"] = {**alu, "how": "gg_probe_fma_rate: 8 independent FMA chains per thread, "
                                                    "4 waves of 256-thread CTAs, CUDA events"}
        # adjoint / forward on the 2048 x 2048 adjoint workload (10^4 steps,
        # sqrt(N) checkpointing): the forward solve as gg_step runs it (tuned
        # plan), and the whole gg_adjoint call (its own forward pass, the
        # recomputation of every segment, the reverse sweep)
        pa = inputs.adjoint_2048(steps=args.adjoint_steps)
        simf = gg.GGSim.from_problem(pa, precision="fp32_kahan")
        simf.step(48)
        fwd_ms = timed_steps(simf, pa.steps, stream)
        fwd_plan = simf.plan()
        Vn = torch.empty(pa.cells, dtype=torch.float32, device=dev)
        simf.read("v", out=Vn)
        simf.close()
        simt = gg.GGSim.from_problem(pa, precision="fp32_kahan", steps_per_pass=1)
        simt.step(48)
        fwd1_ms = timed_steps(simt, pa.steps, stream)
        simt.close()
        sima = gg.GGSim.from_problem(pa, precision="fp32_kahan")
        dLdv = (Vn / pa.cells).contiguous()
        # the first call allocates the adjoint workspace (checkpoints, stash),
        # which later calls on the same simulation reuse; time the second call
        sima.adjoint(pa.steps, None, dLdv, None, outputs=("theta", "lambda1", "lambda2"))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sima.adjoint(pa.steps, None, dLdv, None, outputs=("theta", "lambda1", "lambda2"))
        b.record(stream)
        torch.cuda.synchronize()
        adj_ms = a.elapsed_time(b)
        sima.close()
        extras["adjoint"] = {"workload": f"adjoint_2048: {pa.nx}x{pa.ny}, {pa.steps} steps, sqrt(N) checkpoints",
                             "forward_plan": fwd_plan, "forward_ms": fwd_ms, "forward_T1_ms": fwd1_ms,
                             "adjoint_ms": adj_ms,
                             "adjoint_over_forward": adj_ms / fwd_ms, "adjoint_over_forward_T1": adj_ms / fwd1_ms}
        # batched ensemble: 256 uneven instances, one persistent graph-captured launch
        specs = inputs.ensemble_specs(256)
        probs = [inputs.ensemble_instance(k, specs[k], steps=args.ensemble_steps) for k in range(256)]
        with gg.GGBatch(probs) as bt:
            tuned = bt.autotune(trial_steps=8)
            bt.step(args.ensemble_steps)  # captures the graph and warms up
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bt.step(args.ensemble_steps)
            b.record(stream)
            torch.cuda.synchronize()
            ens_ms = a.elapsed_time(b)
            info = bt.launch_info()
            # the persistent cooperative kernel (the passes of a step in one
            # launch, a grid barrier between them), at its own best depth and
            # chunk height, beside the tuned launch mode
            best = None
            for T in (2, 3, 4):
                for chunk in (32, 64):
                    bt.set_plan("persistent", T, chunk)
                    bt.step(12 * T)  # captures the graph
                    torch.cuda.synchronize()
                    a.record(stream)
                    bt.step(48 * T)
                    b.record(stream)
                    torch.cuda.synchronize()
                    per_step = a.elapsed_time(b) / (48 * T)
                    if best is None or per_step < best[0]:
                        best = (per_step, T, chunk)
            bt.set_plan("persistent", best[1], best[2])
            bt.step(args.ensemble_steps)
            torch.cuda.synchronize()
            a.record(stream)
            bt.step(args.ensemble_steps)
            b.record(stream)
            torch.cuda.synchronize()
            pers_ms = a.elapsed_time(b)
            pinfo = bt.launch_info()
        ens_cells = sum(q.cells for q in probs)
        extras["ensemble"] = {"workload": f"256 instances, grids from {{128..1024}}^2, {args.ensemble_steps} steps",
                              "cells": ens_cells, "value": ens_cells * args.ensemble_steps / (ens_ms / 1e3),
                              "unit": "cell-updates/s", "plan": tuned, "graph": info["graph"], "ctas": info["ctas"],
                              "hbm_frac": 60 * ens_cells * args.ensemble_steps / tuned["T"] / (ens_ms / 1e3) / 1e9 / peak,
                              "hbm_frac_nominal": 60 * ens_cells * args.ensemble_steps / tuned["T"] / (ens_ms / 1e3)
                                                  / 1e9 / HBM_NOMINAL_GBS,
                              "persistent": {"value": ens_cells * args.ensemble_steps / (pers_ms / 1e3),
                                             "unit": "cell-updates/s", "mode": pinfo["mode"], "T": best[1],
                                             "chunk_rows": best[2], "graph": pinfo["graph"], "ctas": pinfo["ctas"],
                                             "hbm_frac": 60 * ens_cells * args.ensemble_steps / best[1]
                                                         / (pers_ms / 1e3) / 1e9 / peak,
                                             "note": "one cooperative launch per step, a bounded grid barrier "
                                                     "between its passes; best of T in 2..4, chunks 32/64"}}
        # measured per-field / per-gradient errors against the FP64 oracle (outside the timed region)
        if dist.rank == 0:
            extras["errors"] = error_leg()

    # end to end through the public API with host buffers in pinned memory:
    # every step creates the simulation from the host arrays (H2D: tensor
    # angles and eigenvalues, initial state, FP64), advances it, reads the
    # three fields back (D2H, FP32) and destroys it
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hp = dataclasses.replace(p, theta=pinned(p.theta), lambda1=pinned(p.lambda1), lambda2=pinned(p.lambda2),
                             u0=pinned(p.u0), v0=pinned(p.v0), w0=pinned(p.w0))
    outs = [pinned(np.empty((p.ny, p.nx), dtype=np.float32)) for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s3 = gg.GGSim.from_problem(hp, precision="fp32_kahan", steps_per_pass=args.steps_per_pass)
        s3.step(n_inner)
        for f, o in zip(("u", "v", "w"), outs):
            s3.read(f, out=o)
        s3.close()
    torch.cuda.synchronize()
    e2e_el = (time.perf_counter() - t0) / args.steps
    e2e = {"value": p.cells * n_inner / e2e_el, "unit": "cell-updates/s",
           "h2d_bytes_per_step": 6 * 8 * p.cells, "d2h_bytes_per_step": 3 * 4 * p.cells,
           "host_buffers": "pinned", "steps": args.steps}

    if dist.rank == 0:
        cpu = cpu_baseline_leg(p) if (not args.no_extras and dist.world == 1) else None
        cpu_omp = cpu_openmp_leg(p) if (not args.no_extras and dist.world == 1) else None
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(p, args, T), "roofline": roofline, "roofline_alu": roofline_alu,
            "cpu_baseline": cpu,
            "cpu_baseline_omp": cpu_omp, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": ck, **extras,
        }
        print(json.dumps(line), flush=True)
    sim.close()


def main():
    args = parse()
    if args.impl == "reference":
        # the oracle runs on rank 0 only; other ranks exit without work and
        # without joining a process group
        if int(os.environ.get("RANK", "0")) != 0:
            return
        os.environ["WORLD_SIZE"] = "1"
        run_reference(args, Dist())
        return
    dist = Dist()
    try:
        run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
