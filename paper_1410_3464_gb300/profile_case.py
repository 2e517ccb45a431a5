"""A fixed small case of the bulk kernel to run under ncu, and the summary of
what ncu measured on it.

    python -m paper_1410_3464_gb300.profile_case run [--warm 2] [--steps 3] [--only SHAPE:STAGING]
        porous discs 1024x512 (seed 1), FP32, three transported species: the
        bulk-kernel variants (tile 16x16 and 32x8, each with plain loads, TMA
        2-stage and TMA D2Q9-box staging; tiles 16x32 and 32x16, two nodes per
        thread, with plain loads and D2Q9-box staging) in that order, each for
        --warm then --steps single steps.  The working set (about 150 MB) is larger than
        the 129 MB L2, so DRAM counters mean something, and small enough for a
        multi-pass ncu capture.
    python -m paper_1410_3464_gb300.profile_case run --batch 32 [--warm 2] [--steps 3] [--only SHAPE:STAGING]
        the same for a batch of 32 members of the 256-member benchmark trace
        (every 8th request: sides 128-1024, about 6 M nodes, 1.8 GB of device
        state): small enough for a multi-pass ncu capture, large enough that
        DRAM counters mean something.  Its DRAM bytes per launch scale to the
        256-member batch by the ratio of the algorithmic bytes.
    python -m paper_1410_3464_gb300.profile_case summarize LAUNCHES.csv OUT.json [--batch 32]
        reads the ncu --csv --print-units base launch list of the run above
        (kernels matching k_bulk, metrics dram__bytes_read.sum,
        dram__bytes_write.sum, gpu__time_duration.sum) and writes, per variant,
        the mean DRAM bytes and duration of the launches after the warm-up,
        keyed by the hash of the device sources they were built from; for a
        batch also the traffic scaled to the full 256-member batch.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import statistics
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPES = ((16, 16), (32, 8), (16, 32), (32, 16))     # the last two: two nodes per thread, no staging 1
STAGINGS = (0, 1, 2)
STAGING_NAMES = {0: "plain loads", 1: "tma 2-stage", 2: "tma d2q9-box"}
WORKLOAD = "porous discs 1024x512 (seed 1), FP32, 3 species"


def kernel_source_hash(precision="fp32"):
    """Hash of the device sources the bulk kernels of a precision are compiled from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1410_3464_gb300", "csrc")
    units = {"fp32": ("kernels_f32.cu", "kernels_f32_n2.cu"), "fp64": ("kernels_f64.cu", "kernels_f64_n2.cu")}[precision]
    for f in ("device.cuh", "tma.cuh", "bulk.cuh", "kernels_impl.cuh") + units:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def variant_name(shape, staging):
    return f"{shape[0]}x{shape[1]} {STAGING_NAMES[staging]}"


def variants(only=None):
    out = [(s, g) for s in SHAPES for g in STAGINGS if g != 1 or s[0] * s[1] == 256]
    if only:
        sh, g = only.split(":")
        tx, ty = (int(v) for v in sh.split("x"))
        out = [((tx, ty), int(g))]
    return out


def batch_members(count):
    """Every (256 / count)-th request of the 256-member benchmark trace (seed 4)."""
    from . import inputs
    reqs = inputs.request_stream(256, seed=4, size_range=(128, 1024), budget_range=(1000, 10000),
                                 rate_range=(1e-6, 1e-1), porosity_range=(0.4, 0.8), stop_fraction=0.0)
    return reqs[::max(1, 256 // count)][:count], reqs


def algorithmic_bytes(types, ns):
    """FP32 bulk-kernel bytes of one step (fluid x 144 + liquid x 40 ns + 2 per node)."""
    return int((types <= 1).sum()) * 144 + int((types == 0).sum()) * 40 * ns + 2 * types.size


def run_batch(args):
    from . import inputs, pslbm
    members, _ = batch_members(args.batch)
    scenes = [inputs.request_scene(r) for r in members]
    sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                             precision=pslbm.FP32) for sc in scenes]
    for shape, g in variants(args.only):
        b = pslbm.Batch(sims, tile_x=shape[0], tile_y=shape[1])
        if g and not b.staging()[1]:
            raise SystemExit("TMA staging unavailable for this batch")
        b.set_staging(g)
        for _ in range(args.warm + args.steps):
            b.step(1)
        b.sync()
        b.close()
        print(f"{variant_name(shape, g)}: {args.warm} + {args.steps} bulk launches", flush=True)
    alg = sum(algorithmic_bytes(s.read(pslbm.F_TYPE)["type"], s.ns) for s in sims)
    print(json.dumps({"algorithmic_bytes_per_launch": alg, "members": len(sims),
                      "nodes": sum(s.nx * s.ny for s in sims)}), flush=True)
    for s in sims:
        s.close()
    return 0


def run(args):
    if args.batch:
        return run_batch(args)
    from . import inputs, pslbm
    sc = inputs.porous_discs(nx=1024, ny=512, seed=1)
    prec = pslbm.FP64 if args.fp64 else pslbm.FP32
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=prec) as sim:
        if not args.fp64 and not sim.staging()[1]:
            raise SystemExit("TMA staging unavailable on this device")
        vs = [v for v in variants(args.only) if not (args.fp64 and v[1] != 0)]
        for shape, g in vs:
            sim.set_staging(-1)
            sim.set_tile_shape(*shape)
            sim.set_staging(g)
            for _ in range(args.warm + args.steps):
                sim.step(1)
            sim.sync()
            print(f"{variant_name(shape, g)}: {args.warm} + {args.steps} bulk launches", flush=True)
    return 0


_SCALE = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9,
          "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1.0,
          "ns": 1e-9, "us": 1e-6, "ms": 1e-3, "s": 1.0}


def read_launches(path):
    """{launch id: (kernel name, {metric: value in bytes or seconds})} of an ncu csv."""
    rows = {}
    with open(path, newline="") as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if "Metric Name" not in r or r.get("ID") in (None, ""):
            continue
        lid = int(r["ID"])
        name, metrics = rows.setdefault(lid, (r["Kernel Name"], {}))
        v = float(r["Metric Value"].replace(",", ""))
        metrics[r["Metric Name"]] = v * _SCALE.get(r.get("Metric Unit", "").strip().lower(), 1.0)
    return rows


def summarize(args):
    rows = read_launches(args.csv)
    bulk = [rows[k] for k in sorted(rows) if "k_bulk" in rows[k][0]]
    vs = [v for v in variants(args.only) if not (args.fp64 and v[1] != 0)]
    if args.fp64:
        return summarize_fp64(args, bulk, vs)
    per = args.warm + args.steps
    if len(bulk) != per * len(vs):
        raise SystemExit(f"expected {per * len(vs)} bulk launches, found {len(bulk)}")
    out = {"kernel": ("k_bulk (plain loads) / k_bulk_tma (TMA-staged), FP32 storage, 3 species, " +
                      ("batch" if args.batch else "single simulation")),
           "workload": (f"{args.batch} members of the 256-member benchmark batch (every {256 // args.batch}th "
                        "request), FP32, 3 species" if args.batch else WORKLOAD),
           "source_hash": kernel_source_hash(),
           "traffic_per_launch": {}, "dram_bytes_read": {}, "dram_bytes_write": {}, "ncu_duration_us": {},
           "note": ("ncu replays each launch with caches flushed; dram bytes are per launch, means over the "
                    f"{args.steps} launches after {args.warm} warm-up launches of each variant; writes still "
                    "resident in L2 at kernel end are not counted"),
           "command": args.command}
    for i, (shape, g) in enumerate(vs):
        launches = bulk[i * per + args.warm:(i + 1) * per]
        want_tma = g != 0
        for name, _ in launches:
            if ("k_bulk_tma" in name) != want_tma:
                raise SystemExit(f"launch {name!r} does not match variant {variant_name(shape, g)}")
        rd = statistics.mean(m["dram__bytes_read.sum"] for _, m in launches)
        wr = statistics.mean(m["dram__bytes_write.sum"] for _, m in launches)
        du = statistics.mean(m["gpu__time_duration.sum"] for _, m in launches)
        key = variant_name(shape, g)
        out["traffic_per_launch"][key] = int(round(rd + wr))
        out["dram_bytes_read"][key] = int(round(rd))
        out["dram_bytes_write"][key] = int(round(wr))
        out["ncu_duration_us"][key] = round(du * 1e6, 2)
    if args.batch:
        # scale the small batch's DRAM bytes to the full 256-member batch by the
        # ratio of the algorithmic bytes (the kernel's traffic per node does not
        # depend on which members are in the batch)
        alg_small, alg_full = args.alg_small, args.alg_full
        out["algorithmic_bytes_small"] = alg_small
        out["algorithmic_bytes_full"] = alg_full
        out["traffic_measured_small"] = dict(out["traffic_per_launch"])
        out["traffic_per_launch"] = {k: int(round(v * alg_full / alg_small))
                                     for k, v in out["traffic_measured_small"].items()}
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out["traffic_per_launch"]))
    return 0


def summarize_fp64(args, bulk, vs):
    """FP64 operations per launch of the FP64 bulk kernel (plain loads): 2 per
    DFMA, 1 per DADD and DMUL, counted by ncu over the executed thread
    instructions, and the FP64 pipe's active share."""
    per = args.warm + args.steps
    if len(bulk) != per * len(vs):
        raise SystemExit(f"expected {per * len(vs)} bulk launches, found {len(bulk)}")
    out = {"kernel": "k_bulk<double> (plain loads), FP64, 3 species, single simulation",
           "workload": "porous discs 1024x512 (seed 1), FP64, 3 species", "source_hash": kernel_source_hash("fp64"),
           "fp64_flops_per_launch": {}, "fp64_pipe_active_pct": {}, "ncu_duration_us": {},
           "note": ("FP64 operations counted by ncu over executed thread instructions (DFMA as 2, DADD and DMUL as "
                    f"1), means over the {args.steps} launches after {args.warm} warm-up launches"),
           "command": args.command}
    for i, (shape, g) in enumerate(vs):
        launches = bulk[i * per + args.warm:(i + 1) * per]
        fl = statistics.mean(2 * m["sm__sass_thread_inst_executed_op_dfma_pred_on.sum"] +
                             m["sm__sass_thread_inst_executed_op_dadd_pred_on.sum"] +
                             m["sm__sass_thread_inst_executed_op_dmul_pred_on.sum"] for _, m in launches)
        key = variant_name(shape, g)
        out["fp64_flops_per_launch"][key] = int(round(fl))
        out["fp64_pipe_active_pct"][key] = round(statistics.mean(
            m["sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active"] for _, m in launches), 2)
        out["ncu_duration_us"][key] = round(statistics.mean(m["gpu__time_duration.sum"] for _, m in launches) * 1e6, 2)
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out["fp64_flops_per_launch"]))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    for name in ("run", "summarize"):
        p = sub.add_parser(name)
        p.add_argument("--warm", type=int, default=2)
        p.add_argument("--steps", type=int, default=3)
        p.add_argument("--only", default=None, help="one variant, e.g. 32x8:1")
        p.add_argument("--batch", type=int, default=0, help="members of the benchmark batch (0: one lattice)")
        p.add_argument("--fp64", action="store_true", help="the FP64 path (plain-load variants only)")
        if name == "summarize":
            p.add_argument("--alg-small", type=int, default=0, help="algorithmic bytes per launch of the run")
            p.add_argument("--alg-full", type=int, default=0, help="algorithmic bytes per launch of the full batch")
            p.add_argument("csv")
            p.add_argument("out")
            p.add_argument("--command", default="", help="the ncu command line that made the csv")
    args = ap.parse_args(argv)
    return run(args) if args.cmd == "run" else summarize(args)


if __name__ == "__main__":
    sys.exit(main())
