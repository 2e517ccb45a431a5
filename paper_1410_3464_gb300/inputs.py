"""Seeded synthetic inputs: node-type masks, initial densities, concentrations,
solid volumes and parameter sets for the reactive two-phase LBM workloads.

This module only builds inputs (numbers and masks).  It contains none of the
method's arithmetic and imports neither the CUDA binding nor the CPU oracle, so
both sides of a parity test can consume the same arrays.

Node types: 0 liquid, 1 gas, 2 solid D(s), 3 solid F(s), 4 inert wall,
5 inlet reservoir, 6 outlet reservoir.

Workloads (sizes and structure of the paper's scene, Section 5: a mineral grain
immersed in liquid with a gas phase, walls with 90 degree contact angle, tau = 1,
D2Q5 transport with rest fraction J_0):

  * bubble_grain(): 128x64 channel, one D(s) grain r=12 at (64,32), one gas
    bubble r=10 at (24,32), species A (1.0) and B (0.0), A->B at k1=1e-3, B
    consumed at the grain surface at k2=1e-3 (first-order dissolution).
  * porous_discs(): seeded overlapping D(s) discs (radii U[8,24], porosity 0.6)
    in an x-channel between an inlet reservoir column (liquid at 1 % over the
    coexistence density) and an outlet reservoir column, with seeded gas slugs
    (bubbles) in the pore space; species B, E, F transported, A derived from the
    liquid density; R1 (k1=1e-5, gas-producing), R3 (k3=1e-1), R2 on D(s)
    (k2=1e-3), R4 on D(s)/F(s) (k4=1e-3).
  * beaker(): the paper's Section 5 scene (100x160, D(s) cylinder, free top
    outlet), stand-in rates.
  * droplet(): App. A2's static contact angle (201x201, a droplet on the
    bottom wall, solid-fluid interaction w).
  * fracture(): App. C's dissolving fracture (100x90, aperture 30 between two
    D(s) blocks, pressure-driven single-phase flow, R2 at the walls).
"""
from __future__ import annotations

import math

import numpy as np

LIQUID, GAS, SOLID_D, SOLID_F, WALL, INLET, OUTLET = range(7)
MAX_SPECIES = 4
IDX_ABSENT = -1
IDX_DERIVED = -2

# Carnahan-Starling constants.  "Original" a=1, b=4, R=1 (critical temperature
# 0.0943294 found numerically from dp/drho = d2p/drho2 = 0); "rescaled" set of
# Section 3.1 (T_c = 0.999954).
CS_ORIGINAL = dict(eos_a=1.0, eos_b=4.0, eos_R=1.0, Tc=0.0943294)
CS_RESCALED = dict(eos_a=0.09926, eos_b=0.18727, eos_R=0.2, Tc=0.999954)
# Coexistence densities (Maxwell equal-area construction) used only as initial
# values: original EOS at 0.7 Tc, rescaled EOS at 0.7 Tc.
COEX_ORIGINAL_07 = (0.35813, 0.009294)
COEX_RESCALED_07 = (7.6495, 0.19852)


def base_params(nx, ny):
    """Parameter dictionary with every feature off and the paper's fluid
    constants (G11=-1, G12=G21=0.001, a0=0.005, rho10=-0.008/ln a0, rho20=0.003,
    tau=1)."""
    return dict(
        nx=int(nx), ny=int(ny), periodic_x=1, periodic_y=1,
        tau=(1.0, 1.0), G11=-1.0, G12=0.001, G21=0.001,
        a0=0.005, rho10=-0.008 / math.log(0.005), rho20=0.003,
        w_adh=(0.0, 0.0), eos_a=1.0, eos_b=4.0, eos_R=1.0, eos_T=0.7 * CS_ORIGINAL["Tc"],
        body_force=(0.0, 0.0), rho_ref=(1.0, 1.0), rho_ref_gas=(0.0, 0.0), r1_surface_factor=1.0,
        inlet_axis=0, outlet_axis=0,
        n_species=0, idx_A=IDX_ABSENT, idx_B=IDX_ABSENT, idx_E=IDX_ABSENT, idx_F=IDX_ABSENT,
        J0=(0.0,) * MAX_SPECIES, tau_g=(1.0,) * MAX_SPECIES, conc_ref=(0.0,) * MAX_SPECIES,
        k1=0.0, inv_Keq=0.0, k3=0.0, k2=0.0, k4=0.0, C_F_sat=0.0,
        gas_yield=0.0, inv_M_C=0.0, c_total_per_rho1=0.0,
        Vbar_D=1.0, Vbar_F=1.0, V_split=2.0, seed=0,
        rho_in_liq=(0.0, 0.0), rho_in_gas=(0.0, 0.0), rho_out=(0.0, 0.0), rho_out_gas=(0.0, 0.0),
        inlet_period_liq=1, inlet_period_gas=0, inlet_ramp=0, conc_in=(0.0,) * MAX_SPECIES,
        conc_scale=(0.0,) * MAX_SPECIES,
    )


def _pad(vals, fill=0.0):
    vals = list(vals)
    return tuple(vals + [fill] * (MAX_SPECIES - len(vals)))


class Scene(dict):
    """mask [ny,nx] u8, rho1, rho2 [ny,nx] f64, conc [ns,ny,nx] f64 (or None),
    vol [2,ny,nx] f64 (or None), params dict."""


def bubble_grain(nx=128, ny=64, grain=(64, 32, 12), bubble=(24, 32, 10),
                 rho2_gas=0.002, rho2_liq=2e-5):
    """Plain-method scene: x-periodic channel, wall rows y=0 and y=ny-1, one
    D(s) grain, one gas bubble, liquid elsewhere at the coexistence densities of
    the original C-S EOS at 0.7 T_c; species A=1.0, B=0.0."""
    y, x = np.mgrid[0:ny, 0:nx]
    mask = np.full((ny, nx), LIQUID, dtype=np.uint8)
    gx, gy, gr = grain
    bx, by, br = bubble
    in_bubble = (x - bx) ** 2 + (y - by) ** 2 <= br * br
    mask[in_bubble] = GAS
    mask[(x - gx) ** 2 + (y - gy) ** 2 <= gr * gr] = SOLID_D
    mask[0, :] = WALL
    mask[ny - 1, :] = WALL
    rl, rg = COEX_ORIGINAL_07
    rho1 = np.where(mask == GAS, rg, rl).astype(np.float64)
    rho2 = np.where(mask == GAS, rho2_gas, rho2_liq).astype(np.float64)
    p = base_params(nx, ny)
    p.update(periodic_x=1, periodic_y=0, rho_ref=(rl, rho2_liq), rho_ref_gas=(rg, rho2_gas),
             n_species=2, idx_A=0, idx_B=1,
             J0=_pad([1.0 / 3.0, 1.0 / 3.0]), tau_g=_pad([0.8, 0.8], 1.0),
             conc_ref=_pad([1.0, 0.0]),
             k1=1e-3, k2=1e-3, Vbar_D=1.0, seed=1)
    conc = np.zeros((2, ny, nx))
    conc[0] = 1.0
    return Scene(mask=mask, rho1=rho1, rho2=rho2, conc=conc, vol=None, params=p)


def _splitmix64_stream(seed):
    """Seeded uniform stream in [0, 1) from the SplitMix64 generator."""
    mask64 = (1 << 64) - 1
    state = seed & mask64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & mask64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask64
        z ^= z >> 31
        yield (z >> 11) * (1.0 / (1 << 53))


def _liquid_spans_x(open_):
    """True if a 4-connected path of open nodes joins column 0 to the last column."""
    from scipy import ndimage
    lab, _ = ndimage.label(open_, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    left = set(np.unique(lab[:, 0])) - {0}
    right = set(np.unique(lab[:, -1])) - {0}
    return bool(left & right)


def discs_mask(nx, ny, seed, rmin=8.0, rmax=24.0, porosity=0.6, buffer=16, walls=True):
    """Overlapping D(s) discs with centres uniform over the domain minus
    `buffer` columns at each end, radii uniform in [rmin, rmax], added until the
    solid fraction of the interior reaches 1 - porosity.  Reseeds (seed+1, ...)
    until an open 4-connected path spans x.  Rows 0 and ny-1 are walls when
    `walls` is set."""
    y, x = np.mgrid[0:ny, 0:nx]
    for attempt in range(64):
        rng = _splitmix64_stream(seed + attempt)
        solid = np.zeros((ny, nx), dtype=bool)
        lo, hi = buffer, nx - buffer
        target = 1.0 - porosity
        interior = (x >= lo) & (x < hi)
        area = interior.sum()
        count = 0                      # solid nodes of the interior, kept incrementally
        while count < target * area:
            cx = lo + next(rng) * (hi - lo)
            cy = next(rng) * ny
            r = rmin + next(rng) * (rmax - rmin)
            x0, x1 = max(int(cx - r) - 1, lo), min(int(cx + r) + 2, hi)
            y0, y1 = max(int(cy - r) - 1, 0), min(int(cy + r) + 2, ny)
            sub = (x[y0:y1, x0:x1] - cx) ** 2 + (y[y0:y1, x0:x1] - cy) ** 2 <= r * r
            count += int((sub & ~solid[y0:y1, x0:x1]).sum())
            solid[y0:y1, x0:x1] |= sub
        mask = np.where(solid, SOLID_D, LIQUID).astype(np.uint8)
        if walls:
            mask[0, :] = WALL
            mask[ny - 1, :] = WALL
        if _liquid_spans_x(mask == LIQUID):
            return mask
    raise RuntimeError("no spanning pore space found")


def porous_discs(nx=1024, ny=512, seed=1, porosity=0.6, rmin=8.0, rmax=24.0,
                 k1=1e-5, k3=1e-1, k2=1e-3, k4=1e-3, rho2_gas=0.002, rho2_liq=2e-5,
                 bubbles=None, bubble_r=(4.0, 10.0), slug=None, overpressure=1.01, gas_mass=0.1, gas_yield=True):
    """Porous-medium scene: pressure-driven flow in x through seeded overlapping
    D(s) discs, with gas slugs in the pore space carried by the flow.

    The inlet reservoir column holds liquid at `overpressure` times the liquid
    coexistence density, the outlet column holds the coexistence density.  Gas
    slugs are seeded bubbles (count ~ pore area / 2000 nodes unless given,
    radii uniform in `bubble_r`) with a smooth tanh density profile of width 2.
    `slug=(P_l, P_g)` instead makes the inlet alternate liquid and gas states
    (sharp switch; used only for short runs).  Original C-S EOS at 0.7 T_c;
    species B, E, F transported and A derived from the liquid density.
    gas_yield=False keeps R1's chemistry (A -> B) but drops its gas product
    C(g) from the fluid (Eq. 27 sources zero): on long lattices the gas R1
    makes accumulates along the flow path until the liquid leaves the Eq. 13
    domain."""
    mask = discs_mask(nx, ny, seed, rmin, rmax, porosity)
    mask[1:ny - 1, 0] = INLET
    mask[1:ny - 1, nx - 1] = OUTLET
    rl, rg = COEX_ORIGINAL_07
    # mass units of Eq. 25b: C_A = 1 in liquid at rho_l, so M_A = rho_l; the gas
    # C(g) of R1 is light, M_C = 0.1 M_A (Eq. 27: S_2 = -S_1 = 0.5 R1 M_C)
    m_gas = gas_mass * rl
    y, x = np.mgrid[0:ny, 0:nx]
    pore = mask == LIQUID
    rng = _splitmix64_stream(seed * 7919 + 17)
    if bubbles is None:
        bubbles = max(1, int(pore.sum() // 2000))
    bubbles = int(bubbles)
    prof = np.zeros((ny, nx))          # 1 inside gas, 0 in liquid
    for _ in range(bubbles):
        for _try in range(100):
            cx = 16 + next(rng) * (nx - 32)
            cy = next(rng) * ny
            if pore[int(cy), int(cx)]:
                break
        r = bubble_r[0] + next(rng) * (bubble_r[1] - bubble_r[0])
        # the tanh profile is below 3e-9 beyond r + 20: evaluate it in a window
        h = int(r) + 21
        x0, x1 = max(int(cx) - h, 0), min(int(cx) + h + 1, nx)
        y0, y1 = max(int(cy) - h, 0), min(int(cy) + h + 1, ny)
        d = np.sqrt((x[y0:y1, x0:x1] - cx) ** 2 + (y[y0:y1, x0:x1] - cy) ** 2)
        prof[y0:y1, x0:x1] = np.maximum(prof[y0:y1, x0:x1], 0.5 * (1.0 - np.tanh((d - r) / 2.0)))
    prof = np.where(pore, prof, 0.0)
    mask[pore & (prof > 0.5)] = GAS
    fluid = (mask == LIQUID) | (mask == GAS)
    rho1 = np.where(fluid, rl + (rg - rl) * prof, 0.0)
    rho2 = np.where(fluid, rho2_liq + (rho2_gas - rho2_liq) * prof, 0.0)
    p = base_params(nx, ny)
    p.update(periodic_x=0, periodic_y=0, rho_ref=(rl, rho2_liq), rho_ref_gas=(rg, rho2_gas),
             n_species=3, idx_A=IDX_DERIVED, idx_B=0, idx_E=1, idx_F=2,
             J0=_pad([1.0 / 3.0] * 3), tau_g=_pad([0.8] * 3, 1.0), conc_ref=_pad([0.0] * 3),
             k1=k1, k3=k3, k2=k2, k4=k4, C_F_sat=0.0,
             gas_yield=0.5 * m_gas if gas_yield else 0.0, inv_M_C=1.0 / m_gas, c_total_per_rho1=1.0 / rl,
             Vbar_D=1.0, Vbar_F=1.0, V_split=2.0, seed=seed,
             rho_in_liq=(overpressure * rl, rho2_liq), rho_in_gas=(rg, rho2_gas),
             rho_out=(rl, rho2_liq), rho_out_gas=(rg, rho2_gas), conc_in=_pad([0.0] * 3),
             # 16-bit solute storage only: B, E, F reach about 0.2, 0.03 and 0.04
             # by 10,000 steps on the 1024x512 lattice; these scales put those
             # maxima near 1000, far from FP16's ceiling (65504), and keep values
             # down to a few 1e-9 in its normal range
             conc_scale=_pad([2.0 ** 12, 2.0 ** 15, 2.0 ** 14]))
    if slug is not None:
        p.update(inlet_period_liq=int(slug[0]), inlet_period_gas=int(slug[1]))
    conc = np.zeros((3, ny, nx))
    return Scene(mask=mask, rho1=rho1, rho2=rho2, conc=conc, vol=None, params=p)


def beaker(nx=100, ny=160, grain=(50, 50, 15), level=100, k1=1e-5, r1_surface=1000.0, k3=1e-1, k2=1e-3,
           k4=1e-7, gas_mass=0.001):
    """The paper's beaker scene (Section 5): a D(s) cylinder of radius 15 at
    (50, 50) in a 100x160 domain with walls left, right and at the bottom and a
    free outlet at the top; liquid below y = level (rho_1 = 8.31, rho_2 = 1e-4)
    and gas above (rho_1 = 0.05, rho_2 = 0.05); rescaled C-S EOS at 0.65 T_c;
    tau = 1; every solute with J0 = 0.9 and tau_g = 0.65 (D = 4.5e-8 m^2/s at
    1 mm and the fluid's time step); the liquid holds only A (C_A = 1).  A, B,
    E, F are all transported; R1 runs r1_surface times faster at the D(s)
    surface (Section 2).  The paper's Table 1 (rate constants) is missing: the
    rates are stand-ins, with k2, k4 below (1 - J0)/2.  At this EOS's liquid
    density (8.17, Eq. 13 domain limit 9.86) a liquid node that turns into F(s)
    hands its mass to two or three neighbours and pushes them out of the EOS
    domain, so k4 is slow (the paper's Fig. 9 also runs R4 at 1/10000 of its
    rate), and the gas C(g) is light (M_C = 0.001 rho_l).  With all four
    reactions on the scene runs 20,000 steps: the D(s) surface dissolves until
    a shell of precipitated F(s) covers it (from about 2,500 steps on)."""
    y, x = np.mgrid[0:ny, 0:nx]
    gas = y >= level
    mask = np.where(gas, GAS, LIQUID).astype(np.uint8)
    gx, gy, gr = grain
    mask[(x - gx) ** 2 + (y - gy) ** 2 <= gr * gr] = SOLID_D
    mask[:, 0] = WALL
    mask[:, nx - 1] = WALL
    mask[0, :] = WALL
    mask[ny - 1, 1:nx - 1] = OUTLET
    # the initial interface is a tanh profile of width 2 (a sharp step launches
    # compression waves that leave the EOS domain of Eq. 13)
    liq = 0.5 * (1.0 - np.tanh((y - level + 0.5) / 2.0))
    rho1 = 0.05 + (8.31 - 0.05) * liq
    rho2 = 0.05 + (1e-4 - 0.05) * liq
    fluid = (mask == LIQUID) | (mask == GAS)
    rho1 = np.where(fluid, rho1, 0.0)
    rho2 = np.where(fluid, rho2, 0.0)
    rl, rg = 8.17, 0.0537                 # Section 5.1: steady bulk densities
    m_gas = gas_mass * rl
    p = base_params(nx, ny)
    p.update(periodic_x=0, periodic_y=0, eos_a=CS_RESCALED["eos_a"], eos_b=CS_RESCALED["eos_b"],
             eos_R=CS_RESCALED["eos_R"], eos_T=0.65 * CS_RESCALED["Tc"],
             rho_ref=(rl, 1e-4), rho_ref_gas=(rg, 0.05),
             n_species=4, idx_A=0, idx_B=1, idx_E=2, idx_F=3,
             J0=_pad([0.9] * 4), tau_g=_pad([0.65] * 4, 1.0), conc_ref=_pad([0.0] * 4),
             k1=k1, r1_surface_factor=r1_surface, k3=k3, k2=k2, k4=k4, C_F_sat=0.0,
             gas_yield=0.5 * m_gas, inv_M_C=1.0 / m_gas,
             Vbar_D=1.0, Vbar_F=1.0, V_split=2.0, seed=7,
             rho_out=(rl, 1e-4), rho_out_gas=(rg, 0.05), outlet_axis=1)
    conc = np.zeros((4, ny, nx))
    conc[0][mask == LIQUID] = 1.0
    return Scene(mask=mask, rho1=rho1, rho2=rho2, conc=conc, vol=None, params=p)


def droplet(nx=201, ny=201, radius=50.0, w=0.0, width=2.0, w2=0.0):
    """Static contact angle (App. A2): a semicircular liquid droplet of the
    given radius centred on the bottom wall of an nx x ny domain with walls at
    the top and bottom rows and periodic sides; rescaled C-S EOS at 0.65 T_c
    (liquid 8.17 / gas 0.0537, density ratio about 150); tau = 1; no species.
    The wall faces sit halfway between the wall rows and the first fluid rows
    (y = 0.5 and y = ny - 1.5).  The solid-fluid interaction of Eq. 16 is
    w_1w = w on the liquid component and w_2w = w2 on the gas component."""
    y, x = np.mgrid[0:ny, 0:nx]
    xc, yw = (nx - 1) / 2.0, 0.5
    r = np.hypot(x - xc, y - yw)
    liq = 0.5 * (1.0 - np.tanh((r - radius) / width))
    mask = np.where(liq > 0.5, LIQUID, GAS).astype(np.uint8)
    mask[0, :] = WALL
    mask[ny - 1, :] = WALL
    rl, rg = 8.17, 0.0537
    rho1 = rg + (rl - rg) * liq
    rho2 = 0.05 + (1e-4 - 0.05) * liq
    fluid = mask <= GAS
    rho1 = np.where(fluid, rho1, 0.0)
    rho2 = np.where(fluid, rho2, 0.0)
    p = base_params(nx, ny)
    p.update(periodic_x=1, periodic_y=0, eos_a=CS_RESCALED["eos_a"], eos_b=CS_RESCALED["eos_b"],
             eos_R=CS_RESCALED["eos_R"], eos_T=0.65 * CS_RESCALED["Tc"], w_adh=(float(w), float(w2)),
             rho_ref=(rl, 1e-4), rho_ref_gas=(rg, 0.05))
    return Scene(mask=mask, rho1=rho1, rho2=rho2, conc=None, vol=None, params=p)


def fracture(L=100, H=90, h0=30, k2=1e-4, overpressure=1.001, conc_in=1.0, rho2_liq=2e-5):
    """Fracture dissolution (App. C): an aperture-h0 fracture between two D(s)
    blocks in an L x H medium.  Walls on the top and bottom rows (no slip); a
    fixed-density inlet reservoir column before the medium (liquid at
    `overpressure` times the coexistence density) and an outlet column after
    it at the coexistence density, so the flow is pressure driven; one phase
    (liquid everywhere), original C-S EOS at 0.7 T_c, tau = 1.  The only species
    B enters at conc_in and dissolves the fracture walls by R2 (first order,
    C_sat = 0; J0 = 1/3, tau_g = 0.8).  The blocks' faces toward the reservoirs
    touch no liquid, so, as in the paper, they do not react; a small k2 keeps
    the dissolution uniform along the fracture."""
    nx, ny = L + 2, H
    y, x = np.mgrid[0:ny, 0:nx]
    lo = (H - h0) // 2
    mask = np.full((ny, nx), LIQUID, np.uint8)
    mask[(y < lo) | (y >= lo + h0)] = SOLID_D
    mask[0, :] = WALL
    mask[ny - 1, :] = WALL
    mask[1:ny - 1, 0] = INLET
    mask[1:ny - 1, nx - 1] = OUTLET
    rl = COEX_ORIGINAL_07[0]
    fluid = mask == LIQUID
    rho1 = np.where(fluid, rl, 0.0)
    rho2 = np.where(fluid, rho2_liq, 0.0)
    p = base_params(nx, ny)
    p.update(periodic_x=0, periodic_y=0, rho_ref=(rl, rho2_liq),
             n_species=1, idx_A=IDX_ABSENT, idx_B=0, idx_E=IDX_ABSENT, idx_F=IDX_ABSENT,
             J0=_pad([1.0 / 3.0]), tau_g=_pad([0.8], 1.0), conc_ref=_pad([0.0]),
             k2=k2, Vbar_D=1.0, Vbar_F=1.0, V_split=2.0, seed=11,
             rho_in_liq=(overpressure * rl, rho2_liq), rho_in_gas=(overpressure * rl, rho2_liq),
             rho_out=(rl, rho2_liq), rho_out_gas=(rl, rho2_liq), conc_in=_pad([conc_in]))
    conc = np.zeros((1, ny, nx))
    return Scene(mask=mask, rho1=rho1, rho2=rho2, conc=conc, vol=None, params=p)


def _log_uniform(u, lo, hi):
    return math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


def request_stream(n, seed=5, size_range=(128, 2048), budget_range=(1000, 50000), rate_range=(1e-6, 1e-1),
                   porosity_range=(0.4, 0.8), stop_fraction=0.05, mean_interarrival=1.0, multiple=16):
    """Seeded stream of simulation requests: Poisson arrivals (exponential
    inter-arrival times with the given mean, in seconds), lattice sides
    log-uniform in `size_range` (rounded to a multiple of `multiple`), porosity
    uniform, each of k1, k3, k2, k4 log-uniform in `rate_range` (k2, k4 capped
    below (1 - J0)/2 = 1/3), step budget log-uniform (integer), half of the
    requests also stopping once the total solid volume changed by
    `stop_fraction`.  Returns a list of dicts (arrival, nx, ny, seed, porosity,
    rates, step_budget, stop_dv)."""
    rng = _splitmix64_stream(seed * 1000003 + 11)
    t = 0.0
    out = []
    for i in range(n):
        t += -mean_interarrival * math.log(max(1e-300, 1.0 - next(rng)))
        nx = int(round(_log_uniform(next(rng), *size_range) / multiple)) * multiple
        ny = int(round(_log_uniform(next(rng), *size_range) / multiple)) * multiple
        nx, ny = max(nx, 64), max(ny, 64)
        por = porosity_range[0] + next(rng) * (porosity_range[1] - porosity_range[0])
        k1, k3, k2, k4 = (_log_uniform(next(rng), *rate_range) for _ in range(4))
        k2, k4 = min(k2, 0.33), min(k4, 0.33)
        budget = int(_log_uniform(next(rng), *budget_range))
        stop = stop_fraction if next(rng) < 0.5 else 0.0
        out.append(dict(arrival=t, nx=nx, ny=ny, seed=seed * 100000 + i, porosity=por,
                        rates=(k1, k3, k2, k4), step_budget=budget, stop_dv=stop))
    return out


def request_scene(req):
    """The porous-medium scene of one request of request_stream().  R1 turns
    liquid mass into gas (Eq. 27); its rate is capped at 1e-4 so that the
    liquid does not vaporise within the step budget.  The inlet overpressure
    scales with the channel length so the driving gradient is the same for
    every size."""
    k1, k3, k2, k4 = req["rates"]
    k1 = min(k1, 1e-4)
    rmax = max(4.0, min(24.0, min(req["nx"], req["ny"]) / 6.0))
    # same inlet pressure gradient as the 1024-node-long channel at 1 % overpressure
    over = 1.0 + 0.01 * req["nx"] / 1024.0
    return porous_discs(nx=req["nx"], ny=req["ny"], seed=req["seed"], porosity=req["porosity"],
                        rmin=min(8.0, rmax / 2), rmax=rmax, k1=k1, k3=k3, k2=k2, k4=k4, overpressure=over)
