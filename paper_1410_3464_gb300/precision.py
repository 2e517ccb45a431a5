"""Per-field error of the reduced-precision paths against the FP64 GPU path.

Runs one scene in FP64 and in the requested reduced precisions side by side,
and at each checkpoint reports, per field, the relative error
max |a - b| / max |b| over the nodes where the field is defined (fluid nodes for
densities and velocities, liquid nodes for concentrations), the number of
nodes whose type differs, and the budget drift.  The FP64 path itself matches
the CPU oracle within 1e-12 (tested), so it stands in for the exact solution
at sizes and step counts the oracle cannot reach.

    python -m paper_1410_3464_gb300.precision --scene porous --nx 512 --ny 256 \
        --steps 100,1000,10000 --precisions fp32,fp32_f16,fp32_bf16
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import inputs, pslbm

PRECISIONS = {"fp32": pslbm.FP32, "fp32_f16": pslbm.FP32_SOLUTE_F16, "fp32_bf16": pslbm.FP32_SOLUTE_BF16}


def rel(a, b, where):
    a, b = a[where], b[where]
    if b.size == 0:
        return 0.0
    den = float(np.abs(b).max())
    num = float(np.abs(a - b).max())
    return num / den if den > 0 else num


def rel_rms(a, b, where):
    a, b = a[where], b[where]
    if b.size == 0:
        return 0.0
    den = float(np.sqrt(np.mean(b * b)))
    num = float(np.sqrt(np.mean((a - b) ** 2)))
    return num / den if den > 0 else num


def field_errors(got, ref):
    fluid = ref["type"] <= 1
    liquid = ref["type"] == 0
    both_f = fluid & (got["type"] <= 1)
    both_l = liquid & (got["type"] == 0)
    out = {k: rel(got[k], ref[k], both_f) for k in ("rho1", "rho2", "ux", "uy")}
    out["rms"] = {k: rel_rms(got[k], ref[k], both_f) for k in ("rho1", "rho2", "ux", "uy")}
    for k in range(ref["conc"].shape[0]):
        out["rms"][f"conc{k}"] = rel_rms(got["conc"][k], ref["conc"][k], both_l)
    # share of fluid nodes whose rho_1 error exceeds 1e-4 of the field's maximum
    e1 = np.abs(got["rho1"] - ref["rho1"])[both_f]
    out["rho1_nodes_above_1e-4"] = float((e1 > 1e-4 * np.abs(ref["rho1"][both_f]).max()).mean()) if e1.size else 0.0
    for k in range(ref["conc"].shape[0]):
        out[f"conc{k}"] = rel(got["conc"][k], ref["conc"][k], both_l)
    out["vol_d"] = rel(got["vol"][0], ref["vol"][0], np.ones_like(fluid))
    out["type_diff_nodes"] = int((got["type"] != ref["type"]).sum())
    out["solid_diff_nodes"] = int(((got["type"] >= 2) & (got["type"] <= 3) ^
                                   (ref["type"] >= 2) & (ref["type"] <= 3)).sum())
    return out


def scene(args):
    if args.scene == "bubble":
        sc = inputs.bubble_grain(nx=args.nx, ny=args.ny, grain=(args.nx // 2, args.ny // 2, args.ny * 3 // 16),
                                 bubble=(args.nx * 3 // 16, args.ny // 2, args.ny * 5 // 32))
    else:
        kw = {} if args.k1 is None else {"k1": args.k1}
        sc = inputs.porous_discs(nx=args.nx, ny=args.ny, seed=args.seed, bubbles=args.bubbles,
                                 gas_yield=not args.no_gas_yield, **kw)
    p = dict(sc["params"])
    if args.rho_ref is not None:
        p["rho_ref"] = tuple(float(v) for v in args.rho_ref.split(","))
    if args.conc_ref is not None:
        c = [float(v) for v in args.conc_ref.split(",")]
        p["conc_ref"] = tuple(c + [0.0] * (len(p["conc_ref"]) - len(c)))
    sc["params"] = p
    return sc


def perturbed(sc, eps, seed=12345):
    """The same scene with rho_1 scaled by (1 + eps * u), u uniform in [-1, 1]
    (seeded) at fluid nodes: the FP64 path run from it shows how fast the flow
    itself amplifies a perturbation of relative size eps."""
    rng = np.random.default_rng(seed)
    r1 = sc["rho1"] * (1.0 + eps * rng.uniform(-1.0, 1.0, sc["rho1"].shape))
    return inputs.Scene(mask=sc["mask"], rho1=r1, rho2=sc["rho2"], conc=sc["conc"], vol=sc["vol"],
                        params=sc["params"])


def study(args):
    sc = scene(args)
    checkpoints = sorted(int(s) for s in args.steps.split(","))
    precs = [p for p in args.precisions.split(",") if p]
    sims = {"fp64": pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                                     precision=pslbm.FP64)}
    for p in precs:
        sims[p] = pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                                   precision=PRECISIONS[p])
    if args.perturb > 0:
        tw = perturbed(sc, args.perturb)
        sims["fp64_perturbed"] = pslbm.Simulation(tw["mask"], tw["params"], tw["rho1"], tw["rho2"], tw["conc"],
                                                  tw["vol"], precision=pslbm.FP64)
        precs = precs + ["fp64_perturbed"]
    rows = []
    done = 0
    failed = {}
    t0 = time.time()
    for c in checkpoints:
        for name, s in list(sims.items()):
            try:
                s.step(c - done)
                s.sync()
            except pslbm.PslbmError as e:      # a run that diverged is reported and dropped
                failed[name] = f"between steps {done} and {c}: {e}"
                s.close()
                del sims[name]
        done = c
        row = {"step": c, "failed": dict(failed)}
        if "fp64" not in sims:
            rows.append(row)
            break
        ref = sims["fp64"].read()
        for p in precs:
            if p not in sims:
                continue
            got = sims[p].read()
            row[p] = field_errors(got, ref)
            row[p]["budget_rel"] = [float(abs(g - r) / max(abs(r), 1e-300))
                                    for g, r in zip(got["budget"][:-1], ref["budget"][:-1])]
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
        if args.save_fields and c in args.save_at:
            np.savez_compressed(f"{args.save_fields}_{c}.npz", **{f"{p}_{k}": v for p in ["fp64"] + precs if p in sims
                                for k, v in sims[p].read().items()})
    for s in sims.values():
        s.close()
    return {"scene": args.scene, "nx": args.nx, "ny": args.ny, "seed": args.seed,
            "rho_ref": list(sc["params"]["rho_ref"]), "conc_ref": list(sc["params"]["conc_ref"]),
            "perturb": args.perturb, "failed": failed, "wall_s": time.time() - t0, "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--scene", choices=["bubble", "porous"], default="porous")
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--steps", default="100,1000,10000")
    ap.add_argument("--precisions", default="fp32,fp32_f16,fp32_bf16")
    ap.add_argument("--save-fields", default=None, help="path prefix: save all fields at each checkpoint")
    ap.add_argument("--save-at", default="", help="checkpoints to save fields at (default: all)")
    ap.add_argument("--bubbles", type=int, default=None, help="gas bubbles seeded in the porous scene")
    ap.add_argument("--k1", type=float, default=None, help="rate of R1 in the porous scene (default 1e-5)")
    ap.add_argument("--no-gas-yield", action="store_true",
                    help="porous scene without R1's gas product (stable on long lattices)")
    ap.add_argument("--rho-ref", default=None, help="population shift per fluid component, e.g. 0,0")
    ap.add_argument("--conc-ref", default=None, help="solute population shift per species, e.g. 0,0,0")
    ap.add_argument("--perturb", type=float, default=0.0,
                    help="also run FP64 from rho_1 perturbed by this relative size (flow sensitivity)")
    args = ap.parse_args(argv)
    args.save_at = {int(v) for v in args.save_at.split(",") if v} or {int(v) for v in args.steps.split(",")}
    print(json.dumps(study(args)))


if __name__ == "__main__":
    main()
