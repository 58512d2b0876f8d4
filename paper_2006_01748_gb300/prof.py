"""Small, self-contained runs of single kernels, for profilers.

    python -m paper_2006_01748_gb300.prof step --nx 4096 --kind warp2 --T 4 --chunk 128
        3 passes of the FP32 step with that plan on the heterogeneous tissue
        (capture the third: ``ncu --clock-control none -k regex:stepw -s 2 -c 1 ...``)
    python -m paper_2006_01748_gb300.prof step --nx 4096 --fp64 --passes 3
        3 steps of the plain FP64 kernel on the same tissue
    python -m paper_2006_01748_gb300.prof plans --nx 4096
        3 passes of each warp plan, one and two columns per lane (T = 1..4,
        chunks 64/128/256, Kahan) and of the plain FP32 T = 1 plans, one line
        per plan on stdout
    python -m paper_2006_01748_gb300.prof adjoint --nx 2048 --steps 20 --kind warp2 --T 4 --chunk 42
        one gg_adjoint call on the adjoint workload (forward plan fixed, no tuning)
    python -m paper_2006_01748_gb300.prof batch --scale 1 --steps 6 [--mode passes2 --T 3 --chunk 56]
        the 256-instance ensemble, tuned (or with the given plan), a few steps

Each run synchronises and prints what it ran; nothing is timed here (time
with CUDA events in bench.py, profile with ncu around these commands).
"""
from __future__ import annotations

import argparse


def _step(args):
    import torch
    from . import build, gg, inputs
    build()
    p = inputs.hetero_8192(nx=args.nx)
    if args.fp64:
        with gg.GGSim.from_problem(p, precision="fp64") as sim:
            sim.step(args.passes)
            torch.cuda.synchronize()
        print(f"step fp64 cells={p.cells} steps={args.passes}", flush=True)
        return
    prec = "fp32_kahan" if not args.plain else "fp32"
    with gg.GGSim.from_problem(p, precision=prec, steps_per_pass=1) as sim:
        sim.set_plan(args.kind, args.T, chunk=args.chunk)
        sim.step(args.passes * args.T)
        torch.cuda.synchronize()
        print(f"step {args.kind} T={args.T} {'plain' if args.plain else 'kahan'} chunk={sim.plan()['by']} "
              f"cells={p.cells} passes={args.passes}", flush=True)


def _plans(args):
    import torch
    from . import build, gg, inputs
    build()
    p = inputs.hetero_8192(nx=args.nx)
    plans = [("warp", T, "fp32_kahan", c) for T in (1, 2, 3, 4) for c in (64, 128, 256)]
    plans += [("warp2", T, "fp32_kahan", c) for T in (1, 2, 3, 4) for c in (64, 128, 256)]
    plans += [("warp", 1, "fp32", 64), ("warp", 1, "fp32", 128), ("warp2", 1, "fp32", 64), ("warp2", 1, "fp32", 128)]
    for kind, T, prec, chunk in plans:
        with gg.GGSim.from_problem(p, precision=prec, steps_per_pass=1) as sim:
            sim.set_plan(kind, T, chunk=chunk)
            sim.step(3 * T)
            torch.cuda.synchronize()
            print(f"config {kind} T={T} {'kahan' if prec == 'fp32_kahan' else 'plain'} chunk={chunk} "
                  f"cells={p.cells}", flush=True)


def _adjoint(args):
    import torch
    from . import build, gg, inputs
    build()
    p = inputs.adjoint_2048(nx=args.nx, steps=args.steps)
    # a fixed plan (the autotuner's choice at 2048^2), so that no tuning launches run
    with gg.GGSim.from_problem(p, precision="fp32_kahan", steps_per_pass=1) as sim:
        sim.set_plan(args.kind, args.T, chunk=args.chunk)
        t = torch.full((p.cells,), 1.0 / p.cells, dtype=torch.float32, device="cuda")
        r = sim.adjoint(args.steps, None, t, t, outputs=("theta",))
        torch.cuda.synchronize()
        print(f"adjoint {p.nx}x{p.ny} steps={args.steps} scalars={list(r['scalars'])}", flush=True)


def _batch(args):
    import torch
    from . import build, gg, inputs
    build()
    specs = inputs.ensemble_specs(256)
    probs = [inputs.ensemble_instance(k, specs[k], scale=args.scale) for k in range(256)]
    with gg.GGBatch(probs) as b:
        if args.mode:
            b.set_plan(args.mode, args.T, chunk=args.chunk)  # a fixed plan: no tuning launches
            tuned = dict(mode=args.mode, T=args.T, by=args.chunk)
        else:
            tuned = b.autotune(trial_steps=4)
        b.step(args.steps)
        torch.cuda.synchronize()
        print(f"batch plan={tuned} steps={args.steps} info={b.launch_info()}", flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2006_01748_gb300.prof")
    sub = ap.add_subparsers(dest="cmd", required=True)
    s = sub.add_parser("step")
    s.add_argument("--nx", type=int, default=4096)
    s.add_argument("--kind", default="warp", choices=["warp", "warp2", "smem"])
    s.add_argument("--T", type=int, default=1)
    s.add_argument("--chunk", type=int, default=0)
    s.add_argument("--passes", type=int, default=3)
    s.add_argument("--plain", action="store_true")
    s.add_argument("--fp64", action="store_true", help="plain FP64 steps (one kernel launch each)")
    s.set_defaults(fn=_step)
    s = sub.add_parser("plans")
    s.add_argument("--nx", type=int, default=4096)
    s.set_defaults(fn=_plans)
    s = sub.add_parser("adjoint")
    s.add_argument("--nx", type=int, default=2048)
    s.add_argument("--steps", type=int, default=20)
    s.add_argument("--kind", default="warp2", choices=["warp", "warp2"])
    s.add_argument("--T", type=int, default=4)
    s.add_argument("--chunk", type=int, default=42)
    s.set_defaults(fn=_adjoint)
    s = sub.add_parser("batch")
    s.add_argument("--scale", type=int, default=1)
    s.add_argument("--steps", type=int, default=6)
    s.add_argument("--mode", default="", choices=["", "persistent", "passes", "passes2"])
    s.add_argument("--T", type=int, default=4)
    s.add_argument("--chunk", type=int, default=128)
    s.set_defaults(fn=_batch)
    args = ap.parse_args(argv)
    args.fn(args)


if __name__ == "__main__":
    main()
