"""A fixed small case of the bulk kernel to run under ncu, and the summary of
what ncu measured on it.

    python -m paper_1410_3464_gb300.profile_case run [--warm 2] [--steps 3] [--only SHAPE:STAGING]
        porous discs 1024x512 (seed 1), FP32, three transported species: the
        bulk-kernel variants (tile 16x16 and 32x8, each with plain loads, TMA
        2-stage and TMA 1-stage staging) in that order, each for --warm then
        --steps single steps.  The working set (about 150 MB) is larger than
        the 129 MB L2, so DRAM counters mean something, and small enough for a
        multi-pass ncu capture.
    python -m paper_1410_3464_gb300.profile_case summarize LAUNCHES.csv OUT.json
        reads the ncu --csv --print-units base launch list of the run above
        (kernels matching k_bulk, metrics dram__bytes_read.sum,
        dram__bytes_write.sum, gpu__time_duration.sum) and writes, per variant,
        the mean DRAM bytes and duration of the launches after the warm-up,
        keyed by the hash of the device sources they were built from.
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
SHAPES = ((16, 16), (32, 8))
STAGINGS = (0, 1, 2)
STAGING_NAMES = {0: "plain loads", 1: "tma 2-stage", 2: "tma 1-stage"}
WORKLOAD = "porous discs 1024x512 (seed 1), FP32, 3 species"


def kernel_source_hash():
    """Hash of the device sources the FP32 bulk kernels are compiled from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1410_3464_gb300", "csrc")
    for f in ("device.cuh", "tma.cuh", "bulk.cuh", "kernels_impl.cuh", "kernels_f32.cu"):
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def variant_name(shape, staging):
    return f"{shape[0]}x{shape[1]} {STAGING_NAMES[staging]}"


def variants(only=None):
    out = [(s, g) for s in SHAPES for g in STAGINGS]
    if only:
        sh, g = only.split(":")
        tx, ty = (int(v) for v in sh.split("x"))
        out = [((tx, ty), int(g))]
    return out


def run(args):
    from . import inputs, pslbm
    sc = inputs.porous_discs(nx=1024, ny=512, seed=1)
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP32) as sim:
        if not sim.staging()[1]:
            raise SystemExit("TMA staging unavailable on this device")
        for shape, g in variants(args.only):
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
    vs = variants(args.only)
    per = args.warm + args.steps
    if len(bulk) != per * len(vs):
        raise SystemExit(f"expected {per * len(vs)} bulk launches, found {len(bulk)}")
    out = {"kernel": "k_bulk (plain loads) / k_bulk_tma (TMA-staged), FP32 storage, 3 species, single simulation",
           "workload": WORKLOAD, "source_hash": kernel_source_hash(),
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
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out["traffic_per_launch"]))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    for name in ("run", "summarize"):
        p = sub.add_parser(name)
        p.add_argument("--warm", type=int, default=2)
        p.add_argument("--steps", type=int, default=3)
        p.add_argument("--only", default=None, help="one variant, e.g. 32x8:1")
        if name == "summarize":
            p.add_argument("csv")
            p.add_argument("out")
            p.add_argument("--command", default="", help="the ncu command line that made the csv")
    args = ap.parse_args(argv)
    return run(args) if args.cmd == "run" else summarize(args)


if __name__ == "__main__":
    sys.exit(main())
