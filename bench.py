#!/usr/bin/env python
"""Throughput benchmark of the reactive two-phase LBM step on GB300.

Workload: the porous-medium reactive two-phase lattice (1024x512, seeded
overlapping D(s) discs of radius 8-24 at porosity 0.6, liquid inflow from an
inlet reservoir, phase-following outlet reservoir, seeded gas slugs in the
pores, species B, E, F transported and A derived, R1-R4), FP32 compute with
shifted FP32 storage.  One step is one pass
of the whole hot path: the fused bulk kernel, the VOP kernel and the
amendment kernel.

Prints one JSON line (rank 0).  Metric: MLUPS (all lattice nodes x steps / s,
whole job).  L2 is flushed (256 MiB write) before every timed step; each step
is timed with CUDA events on the library stream.

--impl reference times the CPU oracle on a bounded sample of the same
workload (256x128, same generator) on the host cores.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(nx=1024, ny=512, seed=1)
SAMPLE = dict(nx=256, ny=128, seed=1)
WORKLOAD_NAME = ("porous discs 1024x512 (radii 8-24, porosity 0.6, seed 1), pressure-driven liquid inflow "
                 "(inlet 1% over coexistence, phase-following outlet), seeded gas slugs in the pores, "
                 "species B,E,F transported + A derived, R1-R4 (k1=1e-5, k3=1e-1, k2=1e-3, k4=1e-3)")
PROFILE_JSON = os.path.join(ROOT, "profiles", "k_bulk_porous1024x512_fp32.json")
STAGING_NAMES = {0: "plain loads", 1: "tma 2-stage", 2: "tma 1-stage"}
KERNEL_NAMES = {0: "k_bulk", 1: "k_bulk_tma<2 stages>", 2: "k_bulk_tma<1 stage>"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp32_f16", "fp32_bf16"], default="fp32")
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU oracle baseline and e2e legs")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle

def oracle_run(seconds_budget, max_steps=None, warmup=1):
    """Time the CPU oracle on the bounded sample; returns (MLUPS, steps, seconds)."""
    from oracle import lbm
    from paper_1410_3464_gb300 import inputs
    sc = inputs.porous_discs(**SAMPLE)
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    for _ in range(warmup):
        L.step()
    n = 0
    t0 = time.perf_counter()
    while True:
        L.step()
        n += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and n >= max_steps) or (max_steps is None and el >= seconds_budget):
            break
    nodes = SAMPLE["nx"] * SAMPLE["ny"]
    return nodes * n / el / 1e6, n, el


def sample_desc(n, el):
    return (f"CPU oracle (numpy FP64, one thread) on the same generator at {SAMPLE['nx']}x{SAMPLE['ny']} "
            f"(seed {SAMPLE['seed']}): {n} steps in {el:.1f} s")


# ------------------------------------------------------------------ arms

def reference_arm(args):
    from paper_1410_3464_gb300 import replicas
    ws, rank, _ = replicas.env()
    if rank != 0:
        return 0
    mlups_w, _, _ = oracle_run(0, max_steps=max(1, args.warmup), warmup=0)
    mlups, n, el = oracle_run(0, max_steps=args.steps, warmup=0)
    line = {"metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_NAME, "sample": f"{SAMPLE['nx']}x{SAMPLE['ny']}"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": sample_desc(n, el)},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def ours_arm(args):
    import torch

    from paper_1410_3464_gb300 import inputs, profile_case, pslbm, replicas

    ws, rank, local = replicas.env()
    replicas.init(ws)
    torch.cuda.set_device(local)
    prec = {"fp32": pslbm.FP32, "fp64": pslbm.FP64, "fp32_f16": pslbm.FP32_SOLUTE_F16,
            "fp32_bf16": pslbm.FP32_SOLUTE_BF16}[args.precision]
    fs = 8 if prec == pslbm.FP64 else 4
    gs = {pslbm.FP64: 8, pslbm.FP32: 4}.get(prec, 2)
    sc = inputs.porous_discs(**WORKLOAD)
    N = WORKLOAD["nx"] * WORKLOAD["ny"]
    ns = sc["params"]["n_species"]

    stream = torch.cuda.ExternalStream(pslbm.get_stream())
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    sim = pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"], precision=prec)
    # kernel variant (tile shape x staging) chosen under the timed loop's own
    # conditions (L2 flushed before every step): a few steps of each
    trials = {}
    stagings = [0, 1, 2] if sim.staging()[1] else [0]
    with torch.cuda.stream(stream):
        for shape in ((16, 16), (32, 8)):
            for sg in stagings:
                sim.set_tile_shape(*shape)
                sim.set_staging(sg)
                ts = []
                for _ in range(5):
                    flush.zero_()
                    ts.append(sim.profile_step(1)[1])
                trials[(shape, sg)] = statistics.median(ts[1:])
        torch.cuda.synchronize()
    best = min(trials, key=trials.get)
    sim.set_tile_shape(*best[0])
    sim.set_staging(best[1])
    t = sim.read(pslbm.F_TYPE)["type"]
    n_fluid = int((t <= 1).sum())
    n_liq = int((t == 0).sum())

    replicas.barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    kern = {"bulk": [], "vop": [], "amend": []}
    tot = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            k, total = sim.profile_step(1)
            for key in kern:
                kern[key].append(k[key])
            tot.append(total)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sim.sync()
    replicas.barrier(ws)
    my_ms = replicas.max_over_ranks(float(sum(tot)), ws)
    value = replicas.whole_job_rate(N * args.steps, ws, my_ms * 1e-3) / 1e6
    bulk_ms = statistics.mean(kern["bulk"])
    bytes_per_launch = n_fluid * 36 * fs + n_liq * 10 * ns * gs + 2 * N
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = bytes_per_launch / (bulk_ms * 1e-3) / 1e9
    tshape = sim.tile_shape()
    staged = sim.staging()[0]
    variant = f"{tshape[0]}x{tshape[1]} {STAGING_NAMES[staged]}"
    traffic = None
    if os.path.exists(PROFILE_JSON) and prec == pslbm.FP32:
        # DRAM bytes per launch from an ncu capture of the same kernel variant
        # built from the same sources (null otherwise)
        pj = json.load(open(PROFILE_JSON))
        if pj.get("source_hash") == profile_case.kernel_source_hash():
            traffic = pj.get("traffic_per_launch", {}).get(variant)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": KERNEL_NAMES[staged], "bytes_per_launch": bytes_per_launch,
                "kernel_ms": bulk_ms, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "kernel_share": bulk_ms / statistics.mean(tot)}

    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": my_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "fp32", "fp64": "f64", "fp32_f16": "fp32 (f16 solute storage)",
                      "fp32_bf16": "fp32 (bf16 solute storage)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "nx": WORKLOAD["nx"], "ny": WORKLOAD["ny"],
                       "fluid_nodes": n_fluid, "liquid_nodes": n_liq, "precision": args.precision,
                       "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"replicas x{ws}",
                       "tile": f"{tshape[0]}x{tshape[1]}", "staging": STAGING_NAMES[staged],
                       "variant_trials_ms": {f"{k[0][0]}x{k[0][1]} {STAGING_NAMES[k[1]]}": v
                                             for k, v in sorted(trials.items())}},
            "roofline": roofline,
            "kernel_ms": {k: statistics.mean(v) for k, v in kern.items()},
            "gpu_launches": 3 * args.steps}
    if clk:
        line["clocks"] = clk

    if not args.skip_cpu:
        # end to end through the C ABI with host buffers: create (host->device
        # copy of the scene), then every step a step call and a read of that
        # step's budget to the host, then a read of all fields
        replicas.barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2 = pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                                precision=prec)
        mon_bytes = 0
        for _ in range(args.steps):
            sim2.step(1)
            sim2.monitor()              # the step's result: step count, max rho_1, status
            mon_bytes += 64
        out = sim2.read(pslbm.F_RHO1 | pslbm.F_RHO2 | pslbm.F_UX | pslbm.F_UY | pslbm.F_CONC | pslbm.F_TYPE |
                        pslbm.F_VOL | pslbm.F_BUDGET)
        el = time.perf_counter() - t0
        sim2.close()
        h2d = sc["mask"].nbytes + sc["rho1"].nbytes + sc["rho2"].nbytes + sc["conc"].nbytes
        d2h = sum(v.nbytes for v in out.values()) + mon_bytes
        e2e_val = replicas.whole_job_rate(N * args.steps, ws, replicas.max_over_ranks(el, ws)) / 1e6
        line["e2e"] = {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                       "d2h_bytes_per_step": d2h / args.steps,
                       "note": "scene copied at create; each step's monitor (step count, max rho_1, status) "
                               "read to the host; all fields and the budget read after the last step"}
        if rank == 0:
            mlups, n, elc = oracle_run(10.0)
            line["cpu_baseline"] = {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                                    "sample": sample_desc(n, elc)}
    sim.close()
    replicas.finish(ws)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
