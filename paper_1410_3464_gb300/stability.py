"""How long variants of the porous workload stay inside the Eq. 13 domain.

    python -m paper_1410_3464_gb300.stability [--nx 4096] [--ny 2048] [--steps 50000]
        [--every 2500] [--precision fp32] [VARIANT ...]

Each variant of the porous scene (seed 4 unless it says otherwise) runs on the
GPU path in chunks of --every steps; after every chunk the monitor reports the
largest rho_1 over fluid nodes, and a device status (a density outside the
Eq. 13 domain, a non-finite density) ends the run.  One JSON line: per
variant, whether it reached --steps, the chunk in which it failed, and the
largest rho_1 after each chunk.  Variants (all others as the bench's porous
scene):
  base                 seeded bubbles (pore area / 2000), all reactions
  half_bubbles         half as many bubbles
  quarter_bubbles      a quarter as many
  small_bubbles        bubble radii U[3, 6] instead of U[4, 10]
  overpressure_1.005   inlet at 1.005 times the liquid density instead of 1.01
  half_small_op1005    the last three together (half the bubbles)
  no_bubbles           a single bubble
  k1_zero              no R1 (no gas source; with all solutes at 0, no chemistry)
  half_bubbles_k1_zero
  no_gas_yield         R1 without its gas product
  no_gas_k4_zero       ... and without R4
  no_gas_k4_1e-5       ... and R4 at 1e-5
"""
from __future__ import annotations

import argparse
import json
import time

from . import inputs, pslbm

VARIANTS = {
    "base": dict(),
    "half_bubbles": dict(bubbles="half"),
    "quarter_bubbles": dict(bubbles="quarter"),
    "small_bubbles": dict(bubble_r=(3.0, 6.0)),
    "overpressure_1.005": dict(overpressure=1.005),
    "half_small_op1005": dict(bubbles="half", bubble_r=(3.0, 6.0), overpressure=1.005),
    "no_bubbles": dict(bubbles=1),
    "k1_zero": dict(k1=0.0),
    "half_bubbles_k1_zero": dict(bubbles="half", k1=0.0),
    "no_gas_yield": dict(gas_yield=False),
    "no_gas_k4_zero": dict(gas_yield=False, k4=0.0),
    "no_gas_k4_1e-5": dict(gas_yield=False, k4=1e-5),
}
PRECISIONS = {"fp32": pslbm.FP32, "fp64": pslbm.FP64}


def scene(name, nx, ny, seed):
    kw = dict(VARIANTS[name])
    if kw.get("bubbles") in ("half", "quarter"):
        pore = int((inputs.porous_discs(nx=nx, ny=ny, seed=seed, bubbles=1)["mask"] <= 1).sum())
        kw["bubbles"] = max(1, pore // (4000 if kw["bubbles"] == "half" else 8000))
    return inputs.porous_discs(nx=nx, ny=ny, seed=seed, **kw)


def run(name, nx, ny, seed, steps, every, precision):
    sc = scene(name, nx, ny, seed)
    t0 = time.time()
    done, fail, max_rho1 = 0, None, []
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as s:
        while done < steps:
            n = min(every, steps - done)
            s.step(n)
            done += n
            try:
                _, m, _ = s.monitor()
                max_rho1.append(round(m, 4))
            except pslbm.PslbmError as e:
                fail = f"between {done - n} and {done}: {e}"
                break
    return dict(survived=fail is None, fail=fail, steps=done, max_rho1=max_rho1, wall_s=round(time.time() - t0, 1))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("variants", nargs="*", default=None)
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--steps", type=int, default=50000)
    ap.add_argument("--every", type=int, default=2500)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp32")
    args = ap.parse_args(argv)
    names = args.variants or list(VARIANTS)
    for n in names:
        if n not in VARIANTS:
            raise SystemExit(f"unknown variant {n}; choose from {', '.join(VARIANTS)}")
    out = {}
    for n in names:
        out[n] = run(n, args.nx, args.ny, args.seed, args.steps, args.every, PRECISIONS[args.precision])
    print(json.dumps(dict(workload=f"porous discs {args.nx}x{args.ny} (seed {args.seed}), {args.precision}",
                          checked_every=args.every, steps=args.steps, variants=out)), flush=True)


if __name__ == "__main__":
    main()
