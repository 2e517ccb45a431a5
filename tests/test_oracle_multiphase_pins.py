"""Multiphase pins of the CPU oracle: coexistence densities and Laplace's law.

Both are fixed by thermodynamics and mechanics rather than by the oracle:

  * a flat liquid-vapour interface relaxes to bulk densities set by the
    Carnahan-Starling EOS of Eq. 12 (equal pressure on both sides, Eq. A1);
    the liquid density sits within a fraction of a per cent of the Maxwell
    equal-area value and the vapour density between the Shan-Chen mechanical
    stability value and the Maxwell value (Section 3.1 prints 0.3589 / 0.0067
    for these constants: its vapour lies in the same bracket);
  * the pressure jump across a static droplet grows linearly in 1/R (App. A1,
    Laplace's law), with no offset.

The interaction weights of Eqs. 11 and 13 decide both: the literal reading
w(1)=1/3, w(2)=1/12 together with the factor 6/G of Eq. 13 would make the
model's pressure c_s^2 rho + 3 (p_CS - c_s^2 rho), a different EOS whose bulk
densities miss these values by far.
"""
import math
import warnings

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq

from oracle import lbm
from paper_1410_3464_gb300 import inputs

A, B, R = 1.0, 4.0, 1.0
T = 0.7 * 0.0943294
G11 = -1.0


def p_cs(rho):
    """Eq. 12, typed out here independently of the oracle."""
    eta = B * rho / 4.0
    return rho * R * T * (1 + eta + eta ** 2 - eta ** 3) / (1 - eta) ** 3 - A * rho ** 2


def inv_psi(rho):
    """1/psi with psi^2 = 6/G (p - rho/3) (Eq. 13)."""
    return 1.0 / math.sqrt(6.0 / G11 * (p_cs(rho) - rho / 3.0))


def coexistence(weight):
    """Bulk densities (liquid, vapour) with equal pressure and zero weighted
    area int_{rg}^{rl} (p0 - p) dW = 0.  W = 1/rho is Maxwell's construction,
    W = 1/psi the Shan-Chen mechanical stability condition."""
    dp = lambda r, h=1e-7: (p_cs(r + h) - p_cs(r - h)) / (2 * h)
    s_lo = brentq(dp, 0.005, 0.12)          # spinodal points bracket the loop
    s_hi = brentq(dp, 0.12, 0.3)
    p_min = p_cs(s_hi)

    def vapour_at(rl):                      # p(rg) = p(rl) on the vapour branch
        return brentq(lambda r: p_cs(r) - p_cs(rl), 1e-9, s_lo)

    def area(rl):
        rg = vapour_at(rl)
        p0 = p_cs(rl)
        with warnings.catch_warnings():       # the integrand's end points are stiff
            warnings.simplefilter("ignore")
            return quad(lambda r: (p0 - p_cs(r)) * weight(r), rg, rl, limit=400, epsabs=1e-14)[0]

    # liquid densities whose pressure lies between the loop's minimum and maximum
    lo = brentq(lambda r: p_cs(r) - max(p_min, 1e-12), s_hi, 0.49)
    hi = brentq(lambda r: p_cs(r) - p_cs(s_lo), s_hi, 0.49)
    rl = brentq(area, lo + 1e-9, hi - 1e-9, xtol=1e-14)
    return rl, vapour_at(rl)


def w_maxwell(r):
    return -1.0 / r ** 2          # d(1/rho)/drho


def w_sc(r, h=1e-7):
    return (inv_psi(r + h) - inv_psi(r - h)) / (2 * h)


def test_flat_interface_coexistence():
    """A periodic 1x128 strip with a liquid slab, started at the Maxwell
    densities, relaxes to bulk densities with the liquid within 0.5 % of both
    the Maxwell and the Shan-Chen mechanical value and the vapour strictly
    between them (averaged over steps 2000-3000, which covers several periods
    of the slab's slowly damped breathing mode); the liquid also matches the
    paper's printed 0.3589 within 1 %."""
    rl_m, rg_m = coexistence(w_maxwell)
    rl_s, rg_s = coexistence(w_sc)
    assert abs(rl_m - 0.35813) < 1e-4 and abs(rg_m - 0.009294) < 1e-5
    assert rg_s < rg_m
    ny = 128
    p = lbm.default_params(1, ny)
    p.update(G12=0.0, G21=0.0, eos_T=T)
    y = np.arange(ny)
    prof = 0.5 * (np.tanh((y - ny / 4) / 3.0) - np.tanh((y - 3 * ny / 4) / 3.0))
    rho1 = (rg_m + (rl_m - rg_m) * prof)[:, None]
    rho2 = np.full((ny, 1), 1e-6)
    mask = np.where(rho1 > 0.5 * rl_m, lbm.LIQUID, lbm.GAS).astype(np.uint8)
    L = lbm.Lattice(mask, p, rho1, rho2)
    L.run(2000)
    acc = np.zeros(ny)
    for _ in range(1000):
        L.step()
        acc += L._density(0)[:, 0]
    r = acc / 1000
    rl, rg = r[ny // 2], r[0]
    assert abs(r[ny // 2 - 8:ny // 2 + 9] - rl).max() < 1e-3 * rl     # flat bulk
    assert abs(rl - rl_m) < 0.005 * rl_m
    assert abs(rl - rl_s) < 0.005 * rl_s
    assert rg_s < rg < rg_m
    assert abs(rl - 0.3589) < 0.01 * 0.3589
    assert abs(p_cs(rl) - p_cs(rg)) < 0.05 * abs(p_cs(rg))          # mechanical balance


@pytest.mark.slow
def test_laplace_law_static_droplet():
    """Static liquid droplets of radius 8, 10, 12 in a periodic 44x44 vapour
    box (1500 steps each): dp = p_CS(rho_in) - p_CS(rho_out) is linear in 1/R
    with R^2 > 0.999 and an intercept below 5 % of the largest jump; the
    droplet radius comes from the mass, not from the initial guess."""
    rl_m, rg_m = coexistence(w_maxwell)
    n = 44
    pts = []
    for R0 in (8.0, 10.0, 12.0):
        p = lbm.default_params(n, n)
        p.update(G12=0.0, G21=0.0, eos_T=T)
        y, x = np.mgrid[0:n, 0:n]
        d = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2)
        prof = 0.5 * (1 - np.tanh((d - R0) / 2.0))
        rho1 = rg_m + (rl_m - rg_m) * prof
        mask = np.where(rho1 > 0.5 * rl_m, lbm.LIQUID, lbm.GAS).astype(np.uint8)
        L = lbm.Lattice(mask, p, rho1, np.full((n, n), 1e-6))
        L.run(1500)
        r = L.fields()["rho1"]
        rin, rout = r[n // 2, n // 2], r[0, 0]
        radius = math.sqrt((r.sum() - rout * n * n) / (math.pi * (rin - rout)))
        pts.append((1.0 / radius, p_cs(rin) - p_cs(rout)))
    a = np.array(pts)
    M = np.vstack([a[:, 0], np.ones(len(a))]).T
    (slope, icpt), *_ = np.linalg.lstsq(M, a[:, 1], rcond=None)
    pred = M @ np.array([slope, icpt])
    r2 = 1 - ((a[:, 1] - pred) ** 2).sum() / ((a[:, 1] - a[:, 1].mean()) ** 2).sum()
    assert slope > 0                         # positive surface tension
    assert r2 > 0.999
    assert abs(icpt) < 0.05 * a[:, 1].max()


def test_wall_without_interaction_rests_at_ninety_degrees():
    """App. A2 and Section 5: a wall without solid-fluid interaction (w = 0)
    holds a droplet at 90 degrees.  Oracle, 41x31, droplet r = 10 on the bottom
    wall, 1500 steps (the angle is settled by then: 3000 steps give the same to
    0.1 degree); the circle fit of the rho_1 midpoint contour gives 86.8 degrees
    at this small radius (the 201x201 GPU runs give 89.4-89.7).  A reading in
    which every solid neighbour takes the centre node's own value gives about
    64 degrees."""
    from paper_1410_3464_gb300 import contact_angle as ca
    sc = inputs.droplet(nx=41, ny=31, radius=10.0, w=0.0)
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], None, None)
    L.run(1500)
    r1 = L.moments()[0]
    out = ca.contact_angle(np.where(L._fluid(L.type), r1, 0.0), skip=3)
    assert abs(out["theta_deg"] - 90.0) < 5.0, out
