"""Static contact angle of a droplet on a flat wall (App. A2), on the GPU path.

    python -m paper_1410_3464_gb300.contact_angle --w -0.4 -0.2 0 0.1 0.14 --steps 30000
    python -m paper_1410_3464_gb300.contact_angle --w 0 --w2 -0.5 -1 -2 --steps 30000
        (the interaction on the gas component instead: w_1w = w, w_2w = each --w2)

Each run steps inputs.droplet(w=...) (201x201, rescaled C-S EOS at 0.65 T_c,
walls at the top and bottom rows, periodic sides) on the FP64 path and
measures the angle on the final density field:
  * the interface is the contour rho_1 = (rho_l + rho_g) / 2 of the bulk
    densities found in the field; on every row from `skip` rows above the
    wall face up to the droplet's top, its left and right crossings are found
    by linear interpolation between nodes;
  * a circle is fitted to those points by algebraic least squares
    (x^2 + y^2 = a x + b y + c);
  * theta = 90 deg + asin((y_c - y_w) / R), measured through the liquid,
    with y_w = 0.5 the wall face of the halfway bounce-back.
A centre below the wall face gives theta < 90 deg (wetting), above it
theta > 90 deg.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, pslbm


def interface_points(rho1, level, row_lo, row_hi, xc):
    """(x, y) crossings of rho1 = level left and right of column xc on rows
    row_lo .. row_hi (inclusive) whose row at xc is liquid."""
    xs, ys = [], []
    for y in range(row_lo, row_hi + 1):
        r = rho1[y]
        if r[xc] <= level:
            break
        i = xc
        while i > 0 and r[i - 1] > level:
            i -= 1
        if i == 0:
            continue
        xs.append(i - 1 + (level - r[i - 1]) / (r[i] - r[i - 1]))
        ys.append(float(y))
        j = xc
        while j < len(r) - 1 and r[j + 1] > level:
            j += 1
        if j == len(r) - 1:
            continue
        xs.append(j + (r[j] - level) / (r[j] - r[j + 1]))
        ys.append(float(y))
    return np.array(xs), np.array(ys)


def fit_circle(x, y):
    """Centre and radius of the least-squares circle x^2 + y^2 = a x + b y + c."""
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    a, b, c = np.linalg.lstsq(A, x * x + y * y, rcond=None)[0]
    xc, yc = a / 2.0, b / 2.0
    return xc, yc, math.sqrt(c + xc * xc + yc * yc)


def contact_angle(rho1, wall_y=0.5, skip=4):
    """Angle (degrees, through the liquid) of the droplet resting on the wall
    whose face is at y = wall_y (rows above it), with the fitted circle."""
    fluid = rho1[1:-1]
    rl, rg = float(fluid.max()), float(fluid[fluid > 0].min())
    level = 0.5 * (rl + rg)
    row0 = int(math.ceil(wall_y + skip))
    # the middle column of the droplet's liquid run on the first measured row
    liq = np.flatnonzero(rho1[row0] > level)
    xc = int(liq[len(liq) // 2]) if len(liq) else rho1.shape[1] // 2
    px, py = interface_points(rho1, level, row0, rho1.shape[0] - 2, xc)
    cx, cy, R = fit_circle(px, py)
    s = max(-1.0, min(1.0, (cy - wall_y) / R))
    return dict(theta_deg=90.0 + math.degrees(math.asin(s)), centre=(cx, cy), radius=R, points=int(len(px)),
                rho_l=rl, rho_g=rg, level=level)


def run(w, steps=30000, radius=50.0, nx=201, ny=201, precision=None, w2=0.0):
    sc = inputs.droplet(nx=nx, ny=ny, radius=radius, w=w, w2=w2)
    prec = pslbm.FP64 if precision is None else precision
    t0 = time.time()
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], None, None, precision=prec) as s:
        s.step(steps)
        s.sync()
        rho1 = s.read(pslbm.F_RHO1)["rho1"]
    out = contact_angle(rho1)
    out.update(w=w, w2=w2, steps=steps, seconds=time.time() - t0, initial_radius=radius)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--w", type=float, nargs="+", default=[-0.4, -0.2, 0.0, 0.1, 0.14])
    ap.add_argument("--steps", type=int, default=30000)
    ap.add_argument("--radius", type=float, default=50.0)
    ap.add_argument("--w2", type=float, nargs="+", default=[0.0],
                    help="interaction on the gas component (every pair of --w and --w2 is run)")
    args = ap.parse_args(argv)
    rows = []
    for w in args.w:
        for w2 in args.w2:
            try:
                rows.append(run(w, args.steps, args.radius, w2=w2))
            except pslbm.PslbmError as e:       # a run that left the EOS domain or diverged
                rows.append(dict(w=w, w2=w2, steps=args.steps, failed=str(e)))
    print(json.dumps(dict(workload="droplet on a flat wall, 201x201, rescaled C-S EOS at 0.65 Tc, FP64",
                          runs=rows)), flush=True)


if __name__ == "__main__":
    main()
