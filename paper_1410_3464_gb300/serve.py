"""Serving harness: drives the library's continuous-batching server with a
seeded Poisson request stream in real time and reports completion latencies
(p50, p99) and aggregate MLUPS, next to running every request alone, first in
first out, on the plain single-instance FP64 path over the same arrival trace.

    python -m paper_1410_3464_gb300.serve --requests 48 --max-side 512 --max-budget 2000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, pslbm


def run_server(trace, precision=pslbm.FP32, hbm_budget=150 * 10**9, chunk_steps=200, max_active=1024):
    """Replay `trace` against a Server in real time.  Returns per-request
    records (latency, steps) and the aggregate node-update rate."""
    scenes = [inputs.request_scene(r) for r in trace]      # prepared before the clock starts
    srv = pslbm.Server(precision=precision, hbm_budget_bytes=hbm_budget, chunk_steps=chunk_steps,
                       max_active=max_active)
    t0 = time.perf_counter()
    pending = list(range(len(trace)))
    ids = {}
    done = {}
    updates = 0
    while len(done) < len(trace):
        now = time.perf_counter() - t0
        while pending and trace[pending[0]]["arrival"] <= now:
            i = pending.pop(0)
            sc = scenes[i]
            ids[i] = srv.submit(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                                step_budget=trace[i]["step_budget"], stop_dv=trace[i]["stop_dv"])
        active = [i for i in ids if i not in done]
        if not active:
            if pending:
                time.sleep(max(0.0, trace[pending[0]]["arrival"] - (time.perf_counter() - t0)))
            continue
        srv.advance()
        now = time.perf_counter() - t0
        for i in active:
            st, n, b = srv.poll(ids[i])
            if st in (pslbm.REQ_DONE, pslbm.REQ_FAILED):
                done[i] = dict(latency=now - trace[i]["arrival"], steps=n, state=st)
                updates += trace[i]["nx"] * trace[i]["ny"] * n
                srv.release(ids[i])
    wall = time.perf_counter() - t0
    srv.close()
    return done, updates / (wall - trace[0]["arrival"]) / 1e6, wall


def run_alone_fifo(trace, precision=pslbm.FP64, chunk_steps=200):
    """Every request alone, in arrival order, on the single-instance path;
    latency = finish - arrival with a single server (queueing included)."""
    clock = 0.0
    out = {}
    updates = 0
    busy = 0.0
    for i, r in enumerate(trace):
        sc = inputs.request_scene(r)
        start = max(clock, r["arrival"])
        t0 = time.perf_counter()
        failed = False
        with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                              precision=precision) as sim:
            b = sim.read(pslbm.F_BUDGET)["budget"]
            ns = sim.ns
            v0 = b[3 + ns] + b[4 + ns]
            done = 0
            while done < r["step_budget"]:
                n = min(chunk_steps, r["step_budget"] - done)
                sim.step(n)
                done += n
                try:
                    b = sim.read(pslbm.F_BUDGET)["budget"]
                except pslbm.PslbmError:
                    failed = True
                    break
                v = b[3 + ns] + b[4 + ns]
                if r["stop_dv"] > 0 and v0 > 0 and abs(v - v0) >= r["stop_dv"] * v0:
                    break
        el = time.perf_counter() - t0
        busy += el
        clock = start + el
        out[i] = dict(latency=clock - r["arrival"], steps=done, failed=failed)
        updates += r["nx"] * r["ny"] * done
    return out, updates / busy / 1e6, clock


def percentile(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else float("nan")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--min-side", type=int, default=128)
    ap.add_argument("--max-side", type=int, default=512)
    ap.add_argument("--min-budget", type=int, default=200)
    ap.add_argument("--max-budget", type=int, default=2000)
    ap.add_argument("--mean-interarrival", type=float, default=0.02)
    ap.add_argument("--chunk", type=int, default=100)
    ap.add_argument("--hbm-budget-gb", type=float, default=150.0)
    ap.add_argument("--skip-baseline", action="store_true")
    a = ap.parse_args()
    trace = inputs.request_stream(a.requests, seed=a.seed, size_range=(a.min_side, a.max_side),
                                  budget_range=(a.min_budget, a.max_budget), mean_interarrival=a.mean_interarrival)
    done, mlups, wall = run_server(trace, hbm_budget=int(a.hbm_budget_gb * 1e9), chunk_steps=a.chunk)
    lat = [d["latency"] for d in done.values()]
    rep = {"workload": f"{a.requests} Poisson requests (seed {a.seed}), sides log-uniform {a.min_side}-{a.max_side}, "
                       f"budgets log-uniform {a.min_budget}-{a.max_budget} steps, half stopping at 5% solid-volume "
                       f"change, mean inter-arrival {a.mean_interarrival} s",
           "served_fp32": {"aggregate_mlups": mlups, "p50_latency_s": percentile(lat, 50),
                           "p99_latency_s": percentile(lat, 99), "wall_s": wall,
                           "failed": sum(1 for d in done.values() if d["state"] != pslbm.REQ_DONE)}}
    if not a.skip_baseline:
        base, bm, bwall = run_alone_fifo(trace, chunk_steps=a.chunk)
        bl = [d["latency"] for d in base.values()]
        rep["alone_fifo_fp64"] = {"aggregate_mlups": bm, "p50_latency_s": percentile(bl, 50),
                                  "p99_latency_s": percentile(bl, 99), "wall_s": bwall,
                                  "failed": sum(1 for d in base.values() if d["failed"])}
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
