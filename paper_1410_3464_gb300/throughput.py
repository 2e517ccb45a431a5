"""Throughput of the FP32 path on the large-lattice and batched workloads.

    python -m paper_1410_3464_gb300.throughput --workload large --steps 300
        porous discs 4096x2048 (seed 4), one simulation.  At this size the
        seeded scenes with all reactions leave the EOS domain after a few
        hundred to a few thousand steps (seed 4 lasts longest, past 2,250
        steps), so the run is a throughput measurement of 390 steps, not a
        long simulation
    python -m paper_1410_3464_gb300.throughput --workload plain --steps 2000
        the plain-method scene (128x64, one grain, one bubble, 2 species), FP64
    python -m paper_1410_3464_gb300.throughput --workload porous-fp64 --steps 300
        porous discs 1024x512 (seed 1) on the FP64 path
    python -m paper_1410_3464_gb300.throughput --workload batch --instances 256 --steps 300
        independent porous geometries (seed 4), sides log-uniform 128-1024
        (multiples of 16), porosity U[0.4, 0.8], rates log-uniform 1e-6-1e-1,
        stepped together as one batch (one launch per kernel per step over the
        packed tile list, CUDA graphs of up to 32 steps)
    python -m paper_1410_3464_gb300.throughput --workload batch --variants [--trials 5]
        every bulk-kernel variant (tile shape, nodes per thread, staging)
        fixed in turn on the workload (large, batch, or porous: 1024x512 seed
        1 with L2 flushed before every step): median over --trials profiled
        steps of the bulk kernel's and the whole step's CUDA-event time

The large-lattice and batch working sets exceed the 129 MB L2 by an order of
magnitude, so no flush is needed between steps; the plain scene (3.7 MB in
FP64) lives in L2 and is launch-bound, and its figure is MLUPS only.  The step count is timed with CUDA events on the
library stream after the variant autotuning and a warm-up; the JSON line
gives MLUPS over all nodes, the algorithmic bytes of the bulk kernel (fluid
nodes x 144 B + liquid nodes x 120 B + 2 B per node for FP32 with three
species) per step, the achieved GB/s of the whole step against the measured
HBM bandwidth, and the chosen kernel variant.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import inputs, pslbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STAGING_NAMES = {0: "plain loads", 1: "tma 2-stage", 2: "tma d2q9-box"}


def peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def step_bytes(types, ns, fs=4, gs=4):
    n_fluid = int((types <= 1).sum())
    n_liq = int((types == 0).sum())
    return n_fluid * 36 * fs + n_liq * 10 * ns * gs + 2 * types.size, n_fluid, n_liq


def timed(run_steps, steps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        a.record(stream)
        run_steps(steps)
        b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) * 1e-3


def large(args, precision=pslbm.FP32, scene=None, name=None):
    import torch
    stream = torch.cuda.ExternalStream(pslbm.get_stream())
    t0 = time.time()
    sc = scene if scene is not None else inputs.porous_discs(nx=args.nx, ny=args.ny, seed=args.seed)
    gen_s = time.time() - t0
    fs = 8 if precision == pslbm.FP64 else 4
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as s:
        s.step(90)                       # autotuning (up to 10 variants x 4 steps, twice) and warm-up
        s.sync()
        el = timed(s.step, args.steps, stream)
        s.sync()
        types = s.read(pslbm.F_TYPE)["type"]
        tx, ty, _ = s.tile_shape()
        staged = s.staging()[0]
    nbytes, nf, nl = step_bytes(types, sc["params"]["n_species"], fs=fs, gs=fs)
    N = types.size
    pk, src = peak_gbs()
    gbs = nbytes * args.steps / el / 1e9
    return dict(workload=name or f"porous discs {args.nx}x{args.ny} (seed {args.seed}), FP32, one simulation",
                nodes=N, fluid_nodes=nf, liquid_nodes=nl, steps=args.steps, seconds=el,
                mlups=N * args.steps / el / 1e6, ms_per_step=1e3 * el / args.steps,
                bulk_bytes_per_step=nbytes, step_gbs=gbs, peak_gbs=pk, peak_source=src, frac_of_peak=gbs / pk,
                tile=f"{tx}x{ty}", staging=STAGING_NAMES[staged], scene_generation_s=gen_s)


def batch(args):
    import torch
    stream = torch.cuda.ExternalStream(pslbm.get_stream())
    reqs = inputs.request_stream(args.instances, seed=args.seed, size_range=(128, 1024),
                                 budget_range=(1000, 10000), rate_range=(1e-6, 1e-1),
                                 porosity_range=(0.4, 0.8), stop_fraction=0.0)
    t0 = time.time()
    scenes = [inputs.request_scene(r) for r in reqs]
    gen_s = time.time() - t0
    sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                             precision=pslbm.FP32) for sc in scenes]
    b = pslbm.Batch(sims)
    b.step(90)                           # autotuning (up to 10 variants x 4 steps, twice) and warm-up
    b.sync()
    el = timed(b.step, args.steps, stream)
    b.sync()
    tx, ty, _ = b.tile_shape()
    staged = b.staging()[0]
    b.close()
    nbytes = nf = nl = N = 0
    for s, sc in zip(sims, scenes):
        t = s.read(pslbm.F_TYPE)["type"]
        bb, f, l = step_bytes(t, sc["params"]["n_species"])
        nbytes += bb
        nf += f
        nl += l
        N += t.size
        s.close()
    pk, src = peak_gbs()
    gbs = nbytes * args.steps / el / 1e9
    sides = np.array([(r["nx"], r["ny"]) for r in reqs])
    return dict(workload=(f"{args.instances} porous geometries (seed {args.seed}), sides log-uniform 128-1024, "
                          f"porosity U[0.4,0.8], rates log-uniform 1e-6-1e-1, FP32, one batch"),
                instances=args.instances, nodes=N, fluid_nodes=nf, liquid_nodes=nl,
                mean_nodes_per_instance=N / args.instances, min_side=int(sides.min()), max_side=int(sides.max()),
                steps=args.steps, seconds=el, mlups=N * args.steps / el / 1e6, ms_per_step=1e3 * el / args.steps,
                bulk_bytes_per_step=nbytes, step_gbs=gbs, peak_gbs=pk, peak_source=src, frac_of_peak=gbs / pk,
                tile=f"{tx}x{ty}", staging=STAGING_NAMES[staged], scene_generation_s=gen_s)


# Bulk-kernel variants: (tile shape, staging); the two-node shapes (16x32,
# 32x16) have no staging 1.
VARIANTS = [((16, 16), 0), ((16, 16), 1), ((16, 16), 2), ((32, 8), 0), ((32, 8), 1), ((32, 8), 2),
            ((16, 32), 0), ((16, 32), 2), ((32, 16), 0), ((32, 16), 2)]


def variants(args):
    import statistics
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if args.workload == "porous" else None

    def time_one(obj):
        obj.step(2)
        ts = []
        for _ in range(args.trials + 1):
            if flush is not None:
                flush.zero_()
            ts.append(obj.profile_step(1))
        ts = ts[1:]
        return dict(bulk_ms=statistics.median(t[0]["bulk"] for t in ts),
                    step_ms=statistics.median(t[1] for t in ts))

    def name(shape, sg):
        npt = shape[0] * shape[1] // 256
        return f"{shape[0]}x{shape[1]} ({npt} node{'s' if npt > 1 else ''}/thread), {STAGING_NAMES[sg]}"

    res = {}
    if args.workload == "batch":
        reqs = inputs.request_stream(args.instances, seed=args.seed, size_range=(128, 1024),
                                     budget_range=(1000, 10000), rate_range=(1e-6, 1e-1),
                                     porosity_range=(0.4, 0.8), stop_fraction=0.0)
        sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                                 precision=pslbm.FP32) for sc in (inputs.request_scene(r) for r in reqs)]
        for shape, sg in VARIANTS:
            b = pslbm.Batch(sims, *shape)
            if sg and not b.staging()[1]:
                b.close()
                continue
            b.set_staging(sg)
            res[name(shape, sg)] = time_one(b)
            b.close()
        for s in sims:
            s.close()
        what = f"{args.instances} porous geometries (seed {args.seed}), FP32, one batch"
    else:
        if args.workload == "porous":
            args.nx, args.ny, args.seed = 1024, 512, 1
        sc = inputs.porous_discs(nx=args.nx, ny=args.ny, seed=args.seed)
        with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                              precision=pslbm.FP32) as s:
            for shape, sg in VARIANTS:
                if sg and not s.staging()[1]:
                    continue
                s.set_staging(-1)
                s.set_tile_shape(*shape)
                s.set_staging(sg)
                res[name(shape, sg)] = time_one(s)
        what = f"porous discs {args.nx}x{args.ny} (seed {args.seed}), FP32, one simulation" + (
            ", L2 flushed before every step" if flush is not None else "")
    best = min(res, key=lambda k: res[k]["bulk_ms"])
    return dict(workload=what, trials=args.trials, unit="ms (CUDA events, median)", variants=res, fastest=best)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", choices=["large", "batch", "plain", "porous-fp64", "porous"], default="large")
    ap.add_argument("--variants", action="store_true", help="time every bulk-kernel variant (large, batch, porous)")
    ap.add_argument("--trials", type=int, default=5)
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--steps", type=int, default=300)
    args = ap.parse_args(argv)
    if args.seed is None:
        args.seed = 4
    if args.variants:
        if args.workload not in ("large", "batch", "porous"):
            raise SystemExit("--variants: workload large, batch or porous")
        print(json.dumps(variants(args)), flush=True)
        return
    if args.workload == "porous":
        raise SystemExit("--workload porous is for --variants (the bench times this lattice)")
    if args.workload == "large":
        out = large(args)
    elif args.workload == "batch":
        out = batch(args)
    elif args.workload == "plain":
        out = large(args, precision=pslbm.FP64, scene=inputs.bubble_grain(),
                    name="plain-method scene 128x64 (one D(s) grain r=12, one bubble r=10, species A, B), FP64")
    else:
        out = large(args, precision=pslbm.FP64, scene=inputs.porous_discs(nx=1024, ny=512, seed=1),
                    name="porous discs 1024x512 (seed 1), FP64, one simulation")
    out["precision"] = "fp64" if args.workload in ("plain", "porous-fp64") else "fp32"
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
