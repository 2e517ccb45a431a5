#!/usr/bin/env python
"""Throughput benchmark of the reactive two-phase LBM step on GB300.

Workloads (--workload):
  batch (default)  256 independent porous geometries stepped together as one
                   batch: sides log-uniform 128-1024 (multiples of 16),
                   porosity U[0.4, 0.8], reaction rates log-uniform 1e-6-1e-1,
                   seeded gas bubbles, inlet/outlet reservoirs, species B, E, F
                   transported and A derived, FP32 (48.5 M nodes, 14.6 GB of
                   device state, far larger than L2).  With N ranks the trace
                   holds 256 N requests and every rank takes its own 256.
  porous           one porous lattice 1024x512 (seed 1), the same physics; its
                   state (about 150 MB) is near the L2 size, so L2 is flushed
                   (256 MiB write) before every timed step.
  large            one porous lattice 4096x2048 (seed 4).

One step is one pass of the whole hot path: the fused bulk kernel, the VOP
kernel and the amendment kernel, over every node of every member.  Each timed
step is bracketed per kernel by CUDA events on the library stream.  Prints one
JSON line (rank 0).  Metric: MLUPS (all lattice nodes x steps / s, whole job).

--impl reference times the CPU oracle (plain numpy FP64) on the host cores on a
bounded sample of the same workload: small members of the same request trace,
one per worker process, each advanced --warmup + --steps oracle steps.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

BATCH = dict(instances=256, seed=4, size_range=(128, 1024), budget_range=(1000, 10000), rate_range=(1e-6, 1e-1),
             porosity_range=(0.4, 0.8))
SINGLES = {"porous": dict(nx=1024, ny=512, seed=1), "large": dict(nx=4096, ny=2048, seed=4)}
PHYSICS = ("pressure-driven liquid inflow (inlet reservoir over coexistence, phase-following outlet), seeded gas "
           "bubbles in the pores, species B,E,F transported + A derived, R1-R4")
WORKLOAD_NAMES = {
    "batch": ("256 porous geometries in one batch (request trace seed 4): sides log-uniform 128-1024 (multiples of "
              "16), porosity U[0.4,0.8], rates k1,k3,k2,k4 log-uniform 1e-6-1e-1 (k1 capped at 1e-4), " + PHYSICS),
    "porous": "porous discs 1024x512 (radii 8-24, porosity 0.6, seed 1), " + PHYSICS + " (k1=1e-5, k3=1e-1, k2=k4=1e-3)",
    "large": "porous discs 4096x2048 (radii 8-24, porosity 0.6, seed 4), " + PHYSICS + " (k1=1e-5, k3=1e-1, k2=k4=1e-3)",
}
# oracle sample: members of the same trace with both sides at most this long
SAMPLE_SIDE = 256
STAGING_NAMES = {0: "plain loads", 1: "tma 2-stage", 2: "tma d2q9-box"}
PROFILE_TAGS = {"batch": "batch256", "porous": "porous1024x512", "large": "porous4096x2048"}
KERNEL_NAMES = {0: "k_bulk", 1: "k_bulk_tma<D2Q9+D2Q5 boxes>", 2: "k_bulk_tma<D2Q9 box, 3 blocks>"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["batch", "porous", "large"], default="batch")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp32_f16", "fp32_bf16"], default="fp32")
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU oracle baseline and the e2e leg")
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


# ------------------------------------------------------------------ workloads

def batch_requests(rank=0, world=1):
    from paper_1410_3464_gb300 import inputs, replicas
    reqs = inputs.request_stream(BATCH["instances"] * world, seed=BATCH["seed"], size_range=BATCH["size_range"],
                                 budget_range=BATCH["budget_range"], rate_range=BATCH["rate_range"],
                                 porosity_range=BATCH["porosity_range"], stop_fraction=0.0)
    return replicas.share(reqs, rank, world)


def oracle_sample(workload, count):
    """The bounded CPU sample of a workload: `count` scene descriptions the
    oracle workers build themselves."""
    if workload == "batch":
        small = [r for r in batch_requests() if r["nx"] <= SAMPLE_SIDE and r["ny"] <= SAMPLE_SIDE]
        return [("request", r) for r in small[:count]]
    seed = SINGLES[workload]["seed"]
    return [("porous", dict(nx=256, ny=128, seed=seed))] * count


def _build_scene(desc):
    from paper_1410_3464_gb300 import inputs
    kind, d = desc
    return inputs.request_scene(d) if kind == "request" else inputs.porous_discs(**d)


def _oracle_worker(desc, warmup, steps, seconds):
    """One oracle process: build the scene, run `warmup` steps, then `steps`
    timed steps (or as many as fit in `seconds` when steps is None).
    Returns (nodes, timed steps, elapsed seconds)."""
    from oracle import lbm
    sc = _build_scene(desc)
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    for _ in range(warmup):
        L.step()
    n = 0
    t0 = time.perf_counter()
    while True:
        L.step()
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= seconds):
            break
    return int(sc["mask"].size), n, el


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def oracle_pool_run(workload, workers, warmup, steps, seconds):
    """Run the oracle on `workers` host processes at once (spawned, one numpy
    thread each); returns (MLUPS over all workers, total node-steps, wall s, sample text)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    descs = oracle_sample(workload, workers)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(descs)) as pool:
        res = pool.starmap(_oracle_worker, [(d, warmup, steps, seconds) for d in descs])
    node_steps = sum(nodes * n for nodes, n, _ in res)
    wall = max(el for _, _, el in res)
    sizes = sorted({f"{d[1]['nx']}x{d[1]['ny']}" for d in descs})
    text = (f"CPU oracle (numpy FP64) in {len(descs)} process(es), one per scene, on "
            f"{'members of the same request trace with both sides <= %d' % SAMPLE_SIDE if workload == 'batch' else 'a 256x128 lattice of the same generator'}"
            f" ({', '.join(sizes[:6])}{', ...' if len(sizes) > 6 else ''}): {warmup} warm-up step(s), then "
            f"{min(n for _, n, _ in res)}-{max(n for _, n, _ in res)} timed steps per scene in {wall:.1f} s")
    return node_steps / wall / 1e6, node_steps, wall, text


def cpu_baseline(workload):
    """The oracle on one host core and on all host cores, about 10 s each."""
    ncores = os.cpu_count() or 1
    one, _, _, one_text = oracle_pool_run(workload, 1, 1, None, 10.0)
    allc, _, _, all_text = oracle_pool_run(workload, ncores, 1, None, 10.0)
    return {"value": allc, "unit": "MLUPS", "cores": ncores, "kind": "oracle", "sample": all_text,
            "single_thread": {"value": one, "unit": "MLUPS", "cores": 1, "sample": one_text},
            "cpu_model": cpu_model(), "nproc": ncores}


# ------------------------------------------------------------------ arms

def reference_arm(args):
    from paper_1410_3464_gb300 import replicas
    ws, rank, _ = replicas.env()
    if rank != 0:
        return 0
    ncores = os.cpu_count() or 1
    mlups, node_steps, wall, text = oracle_pool_run(args.workload, ncores, max(1, args.warmup), args.steps, None)
    line = {"metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_NAMES[args.workload], "sample": text},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": ncores, "kind": "oracle", "sample": text,
                             "cpu_model": cpu_model()},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def algorithmic_bytes(types, ns, fs, gs):
    """Bulk-kernel bytes of one step: every population of a fluid node read and
    written once (2 x 18 x fs), every solute population of a liquid node read and
    written once (2 x 5 ns x gs), one type byte read and written per node."""
    n_fluid = int((types <= 1).sum())
    n_liq = int((types == 0).sum())
    return n_fluid * 36 * fs + n_liq * 10 * ns * gs + 2 * types.size, n_fluid, n_liq


def profile_traffic(workload, variant):
    """DRAM bytes per bulk launch from the committed ncu summary of the same
    kernel variant built from the same device sources (None otherwise)."""
    from paper_1410_3464_gb300 import profile_case
    path = os.path.join(ROOT, "profiles", f"k_bulk_{PROFILE_TAGS[workload]}_fp32.json")
    if not os.path.exists(path):
        return None
    pj = json.load(open(path))
    if pj.get("source_hash") != profile_case.kernel_source_hash():
        return None
    return pj.get("traffic_per_launch", {}).get(variant)


# GB300's nominal FP64 rate: 152 SMs x 2.07 GHz x 2 FP64 FMA per clock x 2 flops
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12


def fp64_roofline(workload, variant, kernel_ms):
    """FP64-ALU roofline of the FP64 bulk kernel: the FP64 operations one launch
    executes (ncu count from the committed summary of the same kernel variant
    built from the same sources) per launch time, against the nominal FP64
    rate.  None without a matching summary."""
    from paper_1410_3464_gb300 import profile_case
    path = os.path.join(ROOT, "profiles", f"k_bulk_{PROFILE_TAGS[workload]}_fp64.json")
    if not os.path.exists(path):
        return None
    pj = json.load(open(path))
    if pj.get("source_hash") != profile_case.kernel_source_hash("fp64"):
        return None
    flops = pj.get("fp64_flops_per_launch", {}).get(variant)
    if not flops:
        return None
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "k_bulk<double>", "variant": variant,
            "flops_per_launch": flops, "kernel_ms": kernel_ms,
            "peak_source": "nominal GB300 FP64 rate (152 SMs x 2.07 GHz x 2 FMA/clock x 2 flops)",
            "fp64_pipe_active_pct_ncu": pj.get("fp64_pipe_active_pct", {}).get(variant)}


def ours_arm(args):
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    import torch

    from paper_1410_3464_gb300 import inputs, pslbm, replicas

    ws, rank, local = replicas.env()
    replicas.init(ws)
    torch.cuda.set_device(local)
    prec = {"fp32": pslbm.FP32, "fp64": pslbm.FP64, "fp32_f16": pslbm.FP32_SOLUTE_F16,
            "fp32_bf16": pslbm.FP32_SOLUTE_BF16}[args.precision]
    fs = 8 if prec == pslbm.FP64 else 4
    gs = {pslbm.FP64: 8, pslbm.FP32: 4}.get(prec, 2)
    stream = torch.cuda.ExternalStream(pslbm.get_stream())
    batch = args.workload == "batch"
    if batch:
        scenes = [inputs.request_scene(r) for r in batch_requests(rank, ws)]
    else:
        scenes = [inputs.porous_discs(**SINGLES[args.workload])]
    N = sum(int(sc["mask"].size) for sc in scenes)
    ns = scenes[0]["params"]["n_species"]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda") if args.workload == "porous" else None

    def make_sims(src=None):
        return [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                                 precision=prec) for sc in (src or scenes)]

    def pinned(a):
        """A copy of a host array in pinned (page-locked) memory, as a numpy view
        of a torch tensor that owns the memory (kept alive by the caller)."""
        if a is None:
            return None, None
        t = torch.empty(a.shape, dtype=getattr(torch, a.dtype.name), pin_memory=True)
        v = t.numpy()
        v[...] = a
        return v, t

    sims = make_sims()
    trials = None
    if batch:
        runner = pslbm.Batch(sims)
        runner.step(90)              # variant autotuning (10 variants x 4 steps, twice) and a first warm-up
    else:
        # one lattice: each variant timed for 5 steps under the timed loop's own
        # conditions (L2 flushed before every step for the 1024x512 lattice)
        runner = sims[0]
        trials = {}
        stagings = [0, 1, 2] if runner.staging()[1] else [0]
        with torch.cuda.stream(stream):
            for shape in ((16, 16), (32, 8), (16, 32), (32, 16)):
                for sg in stagings:
                    if sg == 1 and shape[0] * shape[1] > 256:
                        continue     # two nodes per thread: no staging 1
                    runner.set_staging(-1)
                    runner.set_tile_shape(*shape)
                    runner.set_staging(sg)
                    ts = []
                    for _ in range(5):
                        if flush is not None:
                            flush.zero_()
                        ts.append(runner.profile_step(1)[1])
                    trials[(shape, sg)] = statistics.median(ts[1:])
        torch.cuda.synchronize()
        best = min(trials, key=trials.get)
        runner.set_staging(-1)
        runner.set_tile_shape(*best[0])
        runner.set_staging(best[1])
    runner.step(args.warmup)         # warm-up with the chosen variant
    torch.cuda.synchronize()
    tshape = runner.tile_shape()
    staged = runner.staging()[0]

    replicas.barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    kern = {"bulk": [], "vop": [], "amend": []}
    tot = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            if flush is not None:
                flush.zero_()
            k, total = runner.profile_step(1)
            for key in kern:
                kern[key].append(k[key])
            tot.append(total)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if batch:
        runner.sync()
    else:
        runner.sync()
    replicas.barrier(ws)
    my_ms = replicas.max_over_ranks(float(sum(tot)), ws)
    value = replicas.whole_job_rate(N * args.steps, ws, my_ms * 1e-3) / 1e6
    if batch:
        runner.close()
    nbytes = n_fluid = n_liq = 0
    for s in sims:
        b_, f_, l_ = algorithmic_bytes(s.read(pslbm.F_TYPE)["type"], ns, fs, gs)
        nbytes, n_fluid, n_liq = nbytes + b_, n_fluid + f_, n_liq + l_
    for s in sims:
        s.close()
    del sims, runner
    bulk_ms = statistics.mean(kern["bulk"])
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = nbytes / (bulk_ms * 1e-3) / 1e9
    variant = f"{tshape[0]}x{tshape[1]} {STAGING_NAMES[staged]}"
    traffic = profile_traffic(args.workload, variant) if prec == pslbm.FP32 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": KERNEL_NAMES[staged], "variant": variant,
                "bytes_per_launch": nbytes, "kernel_ms": bulk_ms,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if "hbm_gbs" in peaks
                else "fallback 6.8 TB/s",
                "kernel_share": bulk_ms / statistics.mean(tot)}
    if prec == pslbm.FP64:
        # the FP64 path is bound by FP64 arithmetic, not by HBM
        alu = fp64_roofline(args.workload, variant, bulk_ms)
        if alu is not None:
            alu["kernel_share"] = roofline["kernel_share"]
            alu["hbm"] = {k: roofline[k] for k in ("achieved", "peak", "unit", "frac", "bytes_per_launch")}
            roofline = alu

    cfg = {"workload": WORKLOAD_NAMES[args.workload], "members": len(scenes), "nodes": N,
           "fluid_nodes": n_fluid, "liquid_nodes": n_liq, "precision": args.precision,
           "l2": ("flushed (256 MiB write) before every timed step" if flush is not None else
                  "not flushed: the state is far larger than the 129 MB L2"),
           "parallelism": f"{'instances sharded over' if batch else 'replicas on'} {ws} GPU(s), no data-path exchange",
           "tile": f"{tshape[0]}x{tshape[1]}", "staging": STAGING_NAMES[staged],
           "variant_choice": ("the library's autotuner (each open variant timed for 3 steps, in two passes, best pass kept)" if trials is None else
                              "each variant timed for 5 steps under the timed loop's conditions: " +
                              ", ".join(f"{k[0][0]}x{k[0][1]} {STAGING_NAMES[k[1]]} {v:.4f} ms"
                                        for k, v in sorted(trials.items())))}
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": my_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "fp32", "fp64": "f64", "fp32_f16": "fp32 (f16 solute storage)",
                      "fp32_bf16": "fp32 (bf16 solute storage)"}[args.precision],
            "data": "synthetic", "config": cfg, "roofline": roofline,
            "kernel_ms": {k: statistics.mean(v) for k, v in kern.items()},
            "gpu_launches": 3 * args.steps}
    if clk:
        line["clocks"] = clk

    if not args.skip_cpu:
        # end to end through the public API with host buffers: create every
        # member from its host arrays in pinned memory (host->device copy of
        # the scenes), then every step a step call and a read of that step's
        # result (the step count and status of every member) to the host, then
        # each member's budget (6 + ns doubles) read back after the last step
        keep, pscenes = [], []
        for sc in scenes:
            d = dict(sc)
            for k in ("mask", "rho1", "rho2", "conc", "vol"):
                d[k], t = pinned(sc[k])
                keep.append(t)
            pscenes.append(d)
        replicas.barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sims2 = make_sims(pscenes)
        if batch:
            r2 = pslbm.Batch(sims2, tile_x=tshape[0], tile_y=tshape[1])
            r2.set_staging(staged)
        else:
            r2 = sims2[0]
            r2.set_tile_shape(*tshape[:2])
            r2.set_staging(staged)
        mon_bytes = 0
        for _ in range(args.steps):
            r2.step(1)
            r2.monitor()
            mon_bytes += 16 * len(sims2) if batch else 64
        if batch:
            r2.close()
        # every member's budget into one device buffer (no allocation per
        # member), then one copy to the host
        nb = 6 + ns
        bud = torch.empty((len(sims2), nb), dtype=torch.float64, device="cuda")
        for i, s in enumerate(sims2):
            s.budget_device_noalloc(bud[i].data_ptr())
        with torch.cuda.stream(stream):
            budgets = bud.cpu()
        out_bytes = budgets.numel() * 8
        el = time.perf_counter() - t0
        for s in sims2:
            s.close()
        del keep, pscenes
        h2d = sum(sc["mask"].nbytes + sc["rho1"].nbytes + sc["rho2"].nbytes + sc["conc"].nbytes for sc in scenes)
        e2e_val = replicas.whole_job_rate(N * args.steps, ws, replicas.max_over_ranks(el, ws)) / 1e6
        line["e2e"] = {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                       "d2h_bytes_per_step": (mon_bytes + out_bytes) / args.steps,
                       "note": ("members created from host arrays in pinned memory inside the timed region; each "
                                "step's monitor (step count and status of every member) read to the host; every "
                                "member's budget read after the last step")}
        if rank == 0:
            line["cpu_baseline"] = cpu_baseline(args.workload)
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
