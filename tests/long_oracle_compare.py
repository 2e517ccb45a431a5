"""Compare saved GPU fields with the oracle on a long run (not a pytest file).

    python -m paper_1410_3464_gb300.precision --scene porous --nx 512 --ny 256 --seed 4 \
        --no-gas-yield --steps 2000 --precisions fp32 --save-fields f512       # on the GPU
    python tests/long_oracle_compare.py f512_2000.npz --nx 512 --ny 256 --seed 4 \
        --no-gas-yield --steps 2000                                           # here

runs the CPU oracle on the same seeded scene for the same number of steps (about
17 minutes for this one) and prints, per saved precision, the relative error
per field (max |a - b| / max |b| over the nodes where the field is defined in
both) and the number of nodes whose type differs.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import lbm  # noqa: E402
from paper_1410_3464_gb300 import inputs  # noqa: E402


def rel(a, b, where):
    a, b = a[where], b[where]
    den = float(np.abs(b).max()) if b.size else 0.0
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max() if a.size else 0.0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("fields")
    ap.add_argument("--nx", type=int, required=True)
    ap.add_argument("--ny", type=int, required=True)
    ap.add_argument("--seed", type=int, required=True)
    ap.add_argument("--steps", type=int, required=True)
    ap.add_argument("--no-gas-yield", action="store_true")
    a = ap.parse_args()
    sc = inputs.porous_discs(nx=a.nx, ny=a.ny, seed=a.seed, gas_yield=not a.no_gas_yield)
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    L.run(a.steps)
    o = L.fields()
    g = np.load(a.fields)
    out = {}
    for prec in sorted(k[:-len("_type")] for k in g.files if k.endswith("_type")):
        t = g[f"{prec}_type"]
        fl = (o["type"] <= 1) & (t <= 1)
        lq = (o["type"] == 0) & (t == 0)
        e = {k: rel(g[f"{prec}_{k}"], o[k], fl) for k in ("rho1", "rho2", "ux", "uy")}
        for k in range(o["conc"].shape[0]):
            e[f"conc{k}"] = rel(g[f"{prec}_conc"][k], o["conc"][k], lq)
        e["vol_d_abs"] = float(np.abs(g[f"{prec}_vol_d"] - o["vol_d"]).max())
        e["type_diff_nodes"] = int((t != o["type"]).sum())
        out[prec] = e
    print(json.dumps({"scene": f"porous {a.nx}x{a.ny} seed {a.seed}" + (" without R1's gas" if a.no_gas_yield else ""),
                      "steps": a.steps, "vs_oracle": out}))


if __name__ == "__main__":
    main()
