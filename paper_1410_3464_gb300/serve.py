"""Serving harness: drives the library's continuous-batching server with a
seeded Poisson request stream in real time and reports completion latencies
(p50, p99) and aggregate MLUPS, next to running every request alone, first in
first out, on the plain single-instance FP64 path over the same arrival trace,
and, per request, the error of the served (FP32) final state against the
alone (FP64) one: max |a - b| / max |b| per field over the nodes where the
field is defined in both.

    python -m paper_1410_3464_gb300.serve --requests 48 --max-side 512 --max-budget 2000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, pslbm


def run_server(trace, precision=pslbm.FP32, hbm_budget=150 * 10**9, chunk_steps=200, max_active=1024,
               keep_fields=False):
    """Replay `trace` against a Server in real time.  Returns per-request
    records (latency, steps, and with keep_fields the final fields, fetched
    after the clock stops) and the aggregate node-update rate."""
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
                                step_budget=trace[i]["step_budget"], stop_dv=trace[i]["stop_dv"],
                                keep_fields=keep_fields)
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
    wall = time.perf_counter() - t0
    for i in done:
        if keep_fields and done[i]["state"] == pslbm.REQ_DONE:
            done[i]["fields"] = srv.fetch(ids[i])
        srv.release(ids[i])
    srv.close()
    return done, updates / (wall - trace[0]["arrival"]) / 1e6, wall


def field_errors(got, ref):
    """max |a - b| / max |b| per field over the nodes where it is defined in both
    runs (fluid for rho_1, rho_2, u; liquid for each concentration), and the
    number of nodes whose type differs."""
    fluid = (got["type"] <= 1) & (ref["type"] <= 1)
    liquid = (got["type"] == 0) & (ref["type"] == 0)
    out = {}
    for k in ("rho1", "rho2", "ux", "uy"):
        a, b = got[k][fluid], ref[k][fluid]
        den = float(np.abs(b).max()) if b.size else 0.0
        out[k] = float(np.abs(a - b).max() / den) if den > 0 else 0.0
    cerr = 0.0
    for k in range(ref["conc"].shape[0]):
        a, b = got["conc"][k][liquid], ref["conc"][k][liquid]
        den = float(np.abs(b).max()) if b.size else 0.0
        if den > 0:
            cerr = max(cerr, float(np.abs(a - b).max() / den))
    out["conc"] = cerr
    out["type_diff"] = int((got["type"] != ref["type"]).sum())
    return out


def run_alone_fifo(trace, precision=pslbm.FP64, chunk_steps=200, served=None):
    """Every request alone, in arrival order, on the single-instance path;
    latency = finish - arrival with a single server (queueing included).  With
    `served` (run_server records with fields) each request's final state is
    compared with the served one when both took the same number of steps."""
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
            ref = sim.read() if (served and not failed and "fields" in served.get(i, {})) else None
        el = time.perf_counter() - t0
        busy += el
        clock = start + el
        out[i] = dict(latency=clock - r["arrival"], steps=done, failed=failed)
        if ref is not None:
            got = served[i]["fields"]
            if served[i]["steps"] == done:
                out[i]["error"] = field_errors(got, ref)
            else:
                out[i]["error"] = {"steps_differ": [served[i]["steps"], done]}
            served[i].pop("fields")
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
    done, mlups, wall = run_server(trace, hbm_budget=int(a.hbm_budget_gb * 1e9), chunk_steps=a.chunk,
                                   keep_fields=not a.skip_baseline)
    lat = [d["latency"] for d in done.values()]
    rep = {"workload": f"{a.requests} Poisson requests (seed {a.seed}), sides log-uniform {a.min_side}-{a.max_side}, "
                       f"budgets log-uniform {a.min_budget}-{a.max_budget} steps, half stopping at 5% solid-volume "
                       f"change, mean inter-arrival {a.mean_interarrival} s",
           "served_fp32": {"aggregate_mlups": mlups, "p50_latency_s": percentile(lat, 50),
                           "p99_latency_s": percentile(lat, 99), "wall_s": wall,
                           "failed": sum(1 for d in done.values() if d["state"] != pslbm.REQ_DONE)}}
    if not a.skip_baseline:
        base, bm, bwall = run_alone_fifo(trace, chunk_steps=a.chunk, served=done)
        bl = [d["latency"] for d in base.values()]
        rep["alone_fifo_fp64"] = {"aggregate_mlups": bm, "p50_latency_s": percentile(bl, 50),
                                  "p99_latency_s": percentile(bl, 99), "wall_s": bwall,
                                  "failed": sum(1 for d in base.values() if d["failed"])}
        errs = {i: d["error"] for i, d in base.items() if "error" in d and "steps_differ" not in d["error"]}
        rep["served_fp32_vs_alone_fp64"] = {
            "requests_compared": len(errs),
            "requests_with_other_step_counts": sum(1 for d in base.values() if "steps_differ" in d.get("error", {})),
            "max_over_requests": {k: max(e[k] for e in errs.values()) for k in ("rho1", "rho2", "ux", "uy", "conc")}
            if errs else {},
            "median_over_requests": {k: float(np.median([e[k] for e in errs.values()]))
                                     for k in ("rho1", "rho2", "ux", "uy", "conc")} if errs else {},
            "requests_within_1e-4_on_rho1_u": sum(1 for e in errs.values()
                                                  if max(e["rho1"], e["ux"], e["uy"]) <= 1e-4),
            "per_request": {str(i): e for i, e in sorted(errs.items())}}
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
