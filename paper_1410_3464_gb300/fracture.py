"""Permeability against porosity of a dissolving fracture (App. C, Eq. A3), on
the GPU path.

    python -m paper_1410_3464_gb300.fracture --steps 200000 --every 10000

inputs.fracture() (L = 100, H = 90, initial aperture 30, pressure-driven
single-phase flow, R2 dissolving the fracture walls) runs on the FP64 path.
At every checkpoint:
  * the porosity of the medium is eps = 1 - sum(V_D) / (L (H - 2)), from the
    VOP volumes of the blocks (the wall rows are not part of the medium);
  * the permeability at the fixed reservoir pressures is proportional to the
    volumetric flow rate Q = sum over the column x = L / 2 of u_x (the
    velocity of Eq. 19), so k / k0 = Q / Q0.
Eq. A3 says k / k0 = (eps / eps0)^3 for a fracture that widens uniformly; the
exponent is fitted by least squares on log(k / k0) against log(eps / eps0).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, pslbm


def porosity(vol_d, L, H):
    """1 - solid volume of the medium (columns 1..L, rows 1..H-2) / its area."""
    return 1.0 - float(vol_d[1:H - 1, 1:L + 1].sum()) / float(L * (H - 2))


def flow_rate(ux, L):
    """Volumetric flow rate through the mid column."""
    return float(ux[:, L // 2 + 1].sum())


def run(steps=200000, every=10000, L=100, H=90, h0=30, k2=1e-4, settle=20000):
    sc = inputs.fracture(L=L, H=H, h0=h0, k2=k2)
    rows = []
    t0 = time.time()
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP64) as s:
        done = 0
        while done < steps:
            n = settle if done == 0 else every
            s.step(n)
            done += n
            f = s.read(pslbm.F_UX | pslbm.F_VOL | pslbm.F_TYPE)
            rows.append(dict(step=done, eps=porosity(f["vol_d"], L, H), Q=flow_rate(f["ux"], L),
                             fluid_rows_mid=int((f["type"][:, L // 2 + 1] == 0).sum())))
    e0, q0 = rows[0]["eps"], rows[0]["Q"]
    for r in rows:
        r["eps_ratio"] = r["eps"] / e0
        r["k_ratio"] = r["Q"] / q0
    x = np.log([r["eps_ratio"] for r in rows])
    y = np.log([r["k_ratio"] for r in rows])
    exponent = float(np.polyfit(x, y, 1)[0]) if x.max() - x.min() > 1e-6 else float("nan")
    return dict(workload=f"fracture {L}x{H}, aperture {h0}, k2 {k2}, FP64", exponent=exponent,
                seconds=time.time() - t0, rows=rows)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--steps", type=int, default=200000)
    ap.add_argument("--every", type=int, default=10000)
    ap.add_argument("--k2", type=float, default=1e-4)
    args = ap.parse_args(argv)
    print(json.dumps(run(args.steps, args.every, k2=args.k2)), flush=True)


if __name__ == "__main__":
    main()
