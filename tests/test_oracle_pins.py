"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints, a closed form, an exact invariant, or brute force on a tiny case.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import lbm

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def uniform_mask(nx, ny, t=lbm.LIQUID):
    return np.full((ny, nx), t, dtype=np.uint8)


def flow_off(p):
    """No pseudo-potential interactions: two ideal components (G = 0)."""
    p.update(G11=0.0, G12=0.0, G21=0.0)
    return p


# ---------------------------------------------------------------- lattice

def test_d2q9_isotropy():
    """Eqs. 7-8: weights sum to 1, first moment 0, second moment c_s^2 I,
    opposite directions are opposite vectors."""
    w = np.array(lbm.W9)
    ex, ey = np.array(lbm.EX9), np.array(lbm.EY9)
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs((w * ex).sum()) < 1e-15 and abs((w * ey).sum()) < 1e-15
    assert abs((w * ex * ex).sum() - 1 / 3) < 1e-15
    assert abs((w * ey * ey).sum() - 1 / 3) < 1e-15
    assert abs((w * ex * ey).sum()) < 1e-15
    for a in range(9):
        o = lbm.OPP9[a]
        assert ex[o] == -ex[a] and ey[o] == -ey[a]
    # Eq. 7 literally: axis directions at angles (a-1) pi/2, diagonals rotated by pi/4
    for a in range(1, 5):
        ang = (a - 1) * math.pi / 2
        assert (ex[a], ey[a]) == (round(math.cos(ang)), round(math.sin(ang)))
    for a in range(5, 9):
        ang = (a - 5) * math.pi / 2 + math.pi / 4
        assert (ex[a], ey[a]) == (round(math.sqrt(2) * math.cos(ang)), round(math.sqrt(2) * math.sin(ang)))


def test_feq_moments():
    """Eq. 8: sum f_eq = rho, sum f_eq e = rho u, sum f_eq e e = rho/3 I + rho u u."""
    rng = np.random.default_rng(0)
    rho, ux, uy = rng.uniform(0.1, 2, 50), rng.uniform(-0.1, 0.1, 50), rng.uniform(-0.1, 0.1, 50)
    f = np.array([lbm.feq9(a, rho, ux, uy) for a in range(9)])
    ex, ey = np.array(lbm.EX9)[:, None], np.array(lbm.EY9)[:, None]
    np.testing.assert_allclose(f.sum(0), rho, rtol=1e-14)
    np.testing.assert_allclose((f * ex).sum(0), rho * ux, atol=1e-15)
    np.testing.assert_allclose((f * ey).sum(0), rho * uy, atol=1e-15)
    np.testing.assert_allclose((f * ex * ex).sum(0), rho / 3 + rho * ux * ux, rtol=1e-13)
    np.testing.assert_allclose((f * ex * ey).sum(0), rho * ux * uy, atol=1e-15)


def test_geq5_moments():
    """Eqs. 21-22: sum g_eq = C, sum g_eq e = C u (for any rest fraction)."""
    for J0 in (0.0, 1 / 3, 0.9):
        C, ux, uy = 0.7, 0.03, -0.02
        g = [lbm.geq5(a, C, J0, ux, uy) for a in range(5)]
        assert abs(sum(g) - C) < 1e-15
        assert abs(sum(g[a] * lbm.EX5[a] for a in range(5)) - C * ux) < 1e-15
        assert abs(sum(g[a] * lbm.EY5[a] for a in range(5)) - C * uy) < 1e-15
        # second moment fixes the diffusivity: sum g e_x^2 = C (1 - J0)/2
        assert abs(sum(g[a] * lbm.EX5[a] ** 2 for a in range(5)) - C * (1 - J0) / 2) < 1e-15


# ---------------------------------------------------------------- EOS

def test_cs_critical_point_matches_paper():
    """Eq. 12 with a=1, b=4, R=1: dp/drho = d2p/drho2 = 0 at the critical
    point, which the paper prints as T_c = 0.094, rho_c = 0.13044."""
    gv = GOLDEN["cs_critical_original"]
    from scipy.optimize import fsolve

    def dp(r, T, h=1e-6):
        return (lbm.cs_pressure(r + h, 1, 4, 1, T) - lbm.cs_pressure(r - h, 1, 4, 1, T)) / (2 * h)

    def d2p(r, T, h=1e-4):
        return (lbm.cs_pressure(r + h, 1, 4, 1, T) - 2 * lbm.cs_pressure(r, 1, 4, 1, T)
                + lbm.cs_pressure(r - h, 1, 4, 1, T)) / h ** 2

    rc, Tc = fsolve(lambda v: [dp(v[0], v[1]), d2p(v[0], v[1]) * 1e-2], [0.13, 0.094], xtol=1e-12)
    assert abs(Tc - gv["Tc"]) < 5e-4           # paper prints 3 digits
    assert abs(rc - gv["rho_c"]) < 5e-4


def test_psi_consistent_with_pressure_A1():
    """Eq. 13 (psi from the EOS) and Eq. A1 (single-component pressure
    p = c_s^2 rho + c_s^2 G psi^2 / 2) must give back Eq. 12."""
    rho = np.linspace(0.001, 0.3, 200)      # inside the Eq. 13 domain at these T
    for T in (0.6 * 0.0943294, 0.7 * 0.0943294, 0.9 * 0.0943294):
        psi = lbm.psi1_of_rho(rho, 1, 4, 1, T, -1.0)
        p_a1 = rho / 3 + 0.5 / 3 * (-1.0) * psi ** 2
        np.testing.assert_allclose(p_a1, lbm.cs_pressure(rho, 1, 4, 1, T), rtol=1e-12, atol=1e-15)


def test_phi_constants_sign_change():
    """Eq. 15b with rho_10 = -0.008/ln(a_0): phi_2 vanishes at rho_1 = 0.008
    (natural log), as the paper's choice intends; Eq. 15a: phi_1(0) = 0."""
    gv = GOLDEN["interaction_constants"]
    p = lbm.default_params(4, 4)
    assert abs(lbm.phi2_of_rho1(gv["phi2_zero_rho1"], p["a0"], p["rho10"])) < 1e-15
    assert lbm.phi1_of_rho2(0.0, p["rho20"]) == 0.0
    assert p["a0"] == gv["a0"] and p["rho20"] == gv["rho20"] and p["G12"] == gv["G12"]


# ---------------------------------------------------------------- forces

def _lattice_with_density(rho1, rho2, p, mask=None):
    ny, nx = rho1.shape
    m = uniform_mask(nx, ny) if mask is None else mask
    return lbm.Lattice(m, p, rho1, rho2)


def test_cohesion_force_on_linear_psi():
    """Eq. 11 with the interaction weights: for a psi field linear in x and y
    the stencil sum is exactly c_s^2 grad psi, so F_11 = -G psi c_s^2 grad psi."""
    nx, ny = 12, 10
    p = lbm.default_params(nx, ny)
    p.update(periodic_x=0, periodic_y=0, G12=0.0, G21=0.0)
    T = p["eos_T"]
    # choose psi = 0.02 + 0.003 x + 0.002 y, invert Eq. 13 for rho on the gas branch
    from scipy.optimize import brentq
    yy, xx = np.mgrid[0:ny, 0:nx]
    psi_t = 0.02 + 0.003 * xx + 0.002 * yy
    rho1 = np.zeros((ny, nx))
    for i in range(ny):
        for j in range(nx):
            rho1[i, j] = brentq(lambda r: lbm.psi1_of_rho(r, 1, 4, 1, T, -1.0) - psi_t[i, j], 1e-9, 0.05)
    L = _lattice_with_density(rho1, np.full((ny, nx), 1e-3), p)
    r1, r2, j1, j2 = L.moments()
    F1x, F1y, _, _ = L._forces(L.type, r1, r2, 0 * r1, 0 * r1)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    np.testing.assert_allclose(F1x[inner], (1.0 * psi_t * (1 / 3) * 0.003)[inner], rtol=1e-9)
    np.testing.assert_allclose(F1y[inner], (1.0 * psi_t * (1 / 3) * 0.002)[inner], rtol=1e-9)


def test_intercomponent_force_on_quadratic_phi():
    """Eq. 14a: for phi_2 = c x^2 the stencil sum is exactly 2 c x / 3 (odd
    moments of the weights vanish), so F_12,x = -G12 phi_1 (2 c x / 3)."""
    nx, ny = 16, 6
    p = lbm.default_params(nx, ny)
    p.update(periodic_y=1, periodic_x=0, G11=0.0, G21=0.0, G12=0.5)
    xx = np.mgrid[0:ny, 0:nx][1].astype(float)
    # phi_2 = a0 - exp(-rho1/rho10) = c x^2 + phi0  -> rho1 = -rho10 ln(a0 - c x^2 - phi0)
    c, phi0 = 1e-5, -0.5
    rho1 = -p["rho10"] * np.log(p["a0"] - (c * xx ** 2 + phi0))
    rho2 = np.full((ny, nx), 0.002)
    L = _lattice_with_density(rho1, rho2, p)
    r1, r2, _, _ = L.moments()
    F1x, F1y, _, _ = L._forces(L.type, r1, r2, 0 * r1, 0 * r1)
    phi1 = lbm.phi1_of_rho2(r2, p["rho20"])
    inner = (slice(None), slice(1, nx - 1))
    np.testing.assert_allclose(F1x[inner], (-0.5 * phi1 * 2 * c * xx / 3)[inner], rtol=1e-7, atol=1e-16)
    np.testing.assert_allclose(F1y, 0.0, atol=1e-16)


def test_adhesion_force_sign_and_magnitude():
    """Eq. 16: next to a flat wall below, sum_a w s(x+e) e = (0, -(1/9 + 2/36)),
    so F_1w = w psi_1 (1/9 + 2/36) in +y: w > 0 repels (non-wetting, App. A2
    w = 0.14 -> 97 deg), w < 0 attracts; one row up the sum is zero."""
    nx, ny = 8, 6
    p = lbm.default_params(nx, ny)
    p.update(periodic_x=1, periodic_y=0, G12=0.0, G21=0.0, w_adh=(0.14, 0.0))
    m = uniform_mask(nx, ny)
    m[0, :] = lbm.WALL
    rho1 = np.full((ny, nx), 0.3)
    L = _lattice_with_density(rho1, np.full((ny, nx), 1e-3), p, m)
    r1, r2, _, _ = L.moments()
    F1x, F1y, _, _ = L._forces(L.type, r1, r2, 0 * r1, 0 * r1)
    psi = lbm.psi1_of_rho(r1[1, 0], 1, 4, 1, p["eos_T"], -1.0)
    # mirror-image wall: the cohesion sum of a uniform field is zero even beside the wall
    assert abs(F1y[1, 0] - 0.14 * psi * (1 / 9 + 2 / 36)) < 1e-15
    assert abs(F1y[2, 0]) < 1e-15
    assert np.all(np.abs(F1x) < 1e-15)


def test_gas_component_adhesion_sign_and_magnitude():
    """Eq. 16 for the gas component (psi_2 := rho_2): next to a flat wall below,
    F_2w = -w_2w rho_2 (0, -(1/9 + 2/36)), so w_2w < 0 pulls the gas toward the
    wall (the non-wetting calibration) with magnitude |w_2w| rho_2 / 6; the
    liquid component feels nothing from it, rows between the walls feel no
    wall, and the top row (a wall beyond the non-periodic edge) is pulled up."""
    nx, ny = 8, 6
    p = lbm.default_params(nx, ny)
    p.update(periodic_x=1, periodic_y=0, G12=0.0, G21=0.0, w_adh=(0.0, -4.0))
    m = uniform_mask(nx, ny)
    m[0, :] = lbm.WALL
    rho2 = np.full((ny, nx), 0.05)
    L = _lattice_with_density(np.full((ny, nx), 0.3), rho2, p, m)
    r1, r2, _, _ = L.moments()
    F1x, F1y, F2x, F2y = L._forces(L.type, r1, r2, 0 * r1, 0 * r1)
    assert abs(F2y[1, 0] - (-4.0 * 0.05 / 6.0)) < 1e-15
    assert np.all(np.abs(F2y[2:ny - 1]) < 1e-15)
    assert abs(F2y[ny - 1, 0] - 4.0 * 0.05 / 6.0) < 1e-15
    assert np.all(np.abs(F2x) < 1e-15)
    assert np.all(np.abs(F1y) < 1e-15) and np.all(np.abs(F1x) < 1e-15)


def test_flat_wall_is_a_mirror_for_the_cohesion_sums():
    """Walls are 90-degree walls (App. A2, Section 5): in the Eq. 11 and 14 sums
    a solid neighbour takes its mirror image across a flat wall, so next to a
    flat wall a field that varies along the wall but not across it feels no
    wall-normal cohesion force, exactly as far from the wall.  (Taking the
    centre node's own value for the diagonal wall neighbours would leave
    w(2) (psi(x+1, 2) + psi(x-1, 2) - 2 psi(x, 1)) in the normal sum.)"""
    nx, ny = 16, 8
    p = lbm.default_params(nx, ny)
    p.update(periodic_x=1, periodic_y=0, G12=0.0, G21=0.0, w_adh=(0.0, 0.0))
    m = uniform_mask(nx, ny)
    m[0, :] = lbm.WALL
    m[ny - 1, :] = lbm.WALL
    x = np.arange(nx)
    # a density varying along x only (periodic), inside the EOS domain
    rho1 = np.tile(0.30 + 0.04 * np.sin(2 * np.pi * x / nx), (ny, 1))
    L = _lattice_with_density(rho1, np.full((ny, nx), 1e-3), p, m)
    r1, r2, _, _ = L.moments()
    F1x, F1y, _, _ = L._forces(L.type, r1, r2, 0 * r1, 0 * r1)
    assert np.all(np.abs(F1y[1:ny - 1]) < 1e-15)
    # the force along the wall is the bulk one on every fluid row
    np.testing.assert_allclose(F1x[1], F1x[ny // 2], rtol=0, atol=1e-15)
    assert np.abs(F1x[ny // 2]).max() > 1e-4


# ---------------------------------------------------------------- flow

def test_closed_domain_mass_conservation():
    """Eq. 6 with halfway bounce-back: a closed two-phase domain with an
    obstacle conserves each component's mass to rounding over many steps."""
    from paper_1410_3464_gb300 import inputs
    sc = inputs.bubble_grain(nx=48, ny=32, grain=(30, 16, 5), bubble=(12, 16, 5))
    p = dict(sc["params"])
    p.update(k1=0.0, k2=0.0)
    L = lbm.Lattice(sc["mask"], p, sc["rho1"], sc["rho2"], sc["conc"], None)
    b0 = L.budget()
    L.run(150)
    b1 = L.budget()
    assert abs(b1[1] - b0[1]) < 1e-12 * b0[1]
    assert abs(b1[2] - b0[2]) < 1e-12 * b0[2]


def _poiseuille_error(H, tau=1.0, g=1e-6):
    nx, ny = 4, H + 2
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=1, periodic_y=0, tau=(tau, tau), body_force=(g, 0.0))
    m = uniform_mask(nx, ny)
    m[0, :] = lbm.WALL
    m[-1, :] = lbm.WALL
    rho1 = np.full((ny, nx), 1.0)
    rho2 = np.full((ny, nx), 0.01)
    L = lbm.Lattice(m, p, rho1, rho2)
    nu = (tau - 0.5) / 3
    steps = int(1.6 * H * H / nu)     # ~16 e-folds of the slowest mode H^2/(pi^2 nu)
    L.run(steps)
    u = L.fields()["ux"][1:-1, 0]
    y = np.arange(1, ny - 1)
    exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    return np.abs(u - exact).max() / exact.max()


@pytest.mark.slow
def test_poiseuille_profile_second_order():
    """Body-force channel flow between halfway bounce-back walls: the profile
    is the parabola u = g/(2 nu) (y - y0)(y1 - y), nu = (tau - 1/2)/3 (Eq. 10),
    with walls half a link outside the last fluid rows; the error falls as H^-2."""
    e8 = _poiseuille_error(8)
    e16 = _poiseuille_error(16)
    assert e16 < 5e-3
    assert 3.0 < e8 / e16 < 5.0


# ---------------------------------------------------------------- transport

def _pulse_lattice(nx, ny, J0, tau_g, u=(0.0, 0.0)):
    p = flow_off(lbm.default_params(nx, ny))
    p.update(n_species=1, idx_A=0, J0=(J0, 0, 0, 0), tau_g=(tau_g, 1, 1, 1))
    rho1 = np.full((ny, nx), 1.0)
    rho2 = np.full((ny, nx), 0.01)
    conc = np.zeros((1, ny, nx))
    conc[0, ny // 2, nx // 2] = 1.0
    L = lbm.Lattice(uniform_mask(nx, ny), p, rho1, rho2, conc)
    theta_off = -1.0
    L.theta = theta_off          # every node liquid
    if u != (0.0, 0.0):
        for s, r in ((0, rho1), (1, rho2)):
            for a in range(9):
                L.f[s, a] = lbm.feq9(a, r, np.full_like(r, u[0]), np.full_like(r, u[1]))
    return L


def _moments(C):
    ny, nx = C.shape
    y, x = np.mgrid[0:ny, 0:nx]
    m = C.sum()
    cx, cy = (C * x).sum() / m, (C * y).sum() / m
    vx = (C * (x - cx) ** 2).sum() / m
    return m, cx, cy, vx


def _run_pulse(L, n):
    for _ in range(n):
        L.step()
        L.theta = -1.0
    return L.fields()["conc"][0]


def test_diffusion_variance_growth_eq24():
    """Eqs. 20-24 at u = 0: the variance of a pulse grows by exactly 2D per
    step per axis once the initial transient has decayed, D = (1 - J0)(tau - 1/2)/2."""
    for J0, tau in ((1 / 3, 0.8), (0.0, 1.0), (0.2, 1.3)):
        # 25 steps: the transient decays as (1 - 1/tau)^n; the support (25 nodes)
        # stays inside the 64-node periodic box
        L = _pulse_lattice(64, 64, J0, tau)
        C1 = _run_pulse(L, 25)
        C2 = _run_pulse(L, 1)
        D = 0.5 * (1 - J0) * (tau - 0.5)
        m1, _, _, v1 = _moments(C1)
        m2, _, _, v2 = _moments(C2)
        assert abs(m2 - 1.0) < 1e-13
        assert abs((v2 - v1) - 2 * D) < 1e-10


def test_unit_mapping_matches_paper():
    """Section 5: dx = 1e-3 m, nu = 1e-6 m^2/s at tau = 1 and J0 = 0.9,
    tau_g = 0.65 give D = 4.5e-8 m^2/s.  The diffusivity is measured from the
    oracle's pulse spreading, not from Eq. 24."""
    gv = GOLDEN["unit_mapping"]
    L = _pulse_lattice(96, 96, gv["J0"], gv["tau_g"])
    C1 = _run_pulse(L, 40)
    C2 = _run_pulse(L, 1)
    D_lat = 0.5 * (_moments(C2)[3] - _moments(C1)[3])
    nu_lat = (gv["tau_fluid"] - 0.5) / 3
    dt = nu_lat * gv["dx"] ** 2 / gv["nu_phys"]
    assert abs(D_lat * gv["dx"] ** 2 / dt - gv["D_phys"]) < 1e-6 * gv["D_phys"]


def test_advection_centre_moves_with_fluid():
    """Eq. 21 with u from Eq. 19: in a uniform flow the centre of mass of a
    solute pulse moves exactly u per step."""
    u = (0.05, -0.02)
    L = _pulse_lattice(96, 96, 1 / 3, 0.8, u)
    # the pulse starts at rest equilibrium; its first moment relaxes to C u as
    # (1 - 1/tau)^n, so measure after 20 steps ((-0.25)^20 ~ 1e-12)
    C0 = _run_pulse(L, 20)
    _, x0, y0, _ = _moments(C0)
    C = _run_pulse(L, 30)
    _, x1, y1, _ = _moments(C)
    assert abs((x1 - x0) - 30 * u[0]) < 1e-11
    assert abs((y1 - y0) - 30 * u[1]) < 1e-11


# ---------------------------------------------------------------- reactions

def _uniform_reactor(ns, conc, **kw):
    nx, ny = 6, 5
    p = flow_off(lbm.default_params(nx, ny))
    p.update(n_species=ns, J0=(1 / 3,) * 4, tau_g=(0.8,) * 4)
    p.update(kw)
    rho1 = np.full((ny, nx), 1.0)
    rho2 = np.full((ny, nx), 0.2)
    c = np.zeros((ns, ny, nx))
    for k in range(ns):
        c[k] = conc[k]
    L = lbm.Lattice(uniform_mask(nx, ny), p, rho1, rho2, c)
    L.theta = -1.0
    return L


def test_first_order_decay_closed_form():
    """Eq. 5a (irreversible), Eq. 28 and Eq. 27: a uniform liquid with A -> B
    at rate k1 has C_A(n) = C0 (1 - k1)^n exactly, C_A + C_B = C0, and the
    liquid component loses gas_yield * (C0 - C_A(n)) per node to the gas one."""
    k1, y = 0.01, 0.5
    L = _uniform_reactor(2, (1.0, 0.0), idx_A=0, idx_B=1, k1=k1, gas_yield=y)
    r10, r20 = L.moments()[0][0, 0], L.moments()[1][0, 0]
    crossed = None
    for n in range(1, 121):
        L.step()
        L.theta = -1.0
        fl = L.fields()
        CA, CB = fl["conc"][0], fl["conc"][1]
        exact = (1 - k1) ** n
        np.testing.assert_allclose(CA, exact, rtol=1e-12)
        np.testing.assert_allclose(CA + CB, 1.0, rtol=1e-12)
        np.testing.assert_allclose(fl["rho1"], r10 - y * (1 - exact), rtol=1e-12)
        np.testing.assert_allclose(fl["rho2"], r20 + y * (1 - exact), rtol=1e-12)
        if crossed is None and CB[0, 0] >= CA[0, 0]:
            crossed = CA[0, 0]
    # Section 5.3: A and B cross at half the initial concentration
    frac = GOLDEN["ab_symmetry"]["crossing_fraction"]
    assert abs(crossed - frac) < k1


def test_r1_surface_enhancement_total_production():
    """Section 2: A decomposes in the bulk and 1000 times faster at the surface
    of D(s).  With one inert D(s) node (k2 = 0) in a uniform periodic liquid of
    C_A = 1, C_B = 0, one step produces, in total, exactly
    k1 (N_liquid + (f - 1) N_surface) of B, N_surface being the liquid nodes
    that share an axis link with the D(s) node (counted here directly: 4), since
    the D2Q5 rest fractions sum to one and streaming and bounce-back conserve
    mass."""
    nx, ny, k1 = 9, 8, 1e-4
    for f in (1.0, 1000.0):
        p = flow_off(lbm.default_params(nx, ny))
        p.update(n_species=2, idx_A=0, idx_B=1, J0=(1 / 3,) * 4, tau_g=(0.8,) * 4, k1=k1,
                 r1_surface_factor=f)
        mask = uniform_mask(nx, ny)
        mask[4, 3] = lbm.SOLID_D
        liquid = mask == lbm.LIQUID
        surface = sum(int(liquid[(4 + dy) % ny, (3 + dx) % nx]) for dx, dy in ((1, 0), (0, 1), (-1, 0), (0, -1)))
        assert surface == 4
        c = np.zeros((2, ny, nx))
        c[0][liquid] = 1.0
        L = lbm.Lattice(mask, p, np.full((ny, nx), 1.0), np.full((ny, nx), 0.2), c)
        L.theta = -1.0
        L.step()
        total_b = L.fields()["conc"][1][liquid].sum()
        assert abs(total_b - k1 * (liquid.sum() + (f - 1.0) * surface)) < 1e-15 * liquid.sum()


def test_reversible_r1_equilibrium_is_stationary():
    """Eq. 5a: with C_A = C_B sqrt(C_C)/K_eq the net rate vanishes."""
    inv_keq, rho2 = 3.0, 0.2
    CB = 0.4
    CA = inv_keq * CB * math.sqrt(rho2 * 2.0)
    L = _uniform_reactor(2, (CA, CB), idx_A=0, idx_B=1, k1=0.05, inv_Keq=inv_keq, inv_M_C=2.0, gas_yield=0.5)
    L.run(5)
    fl = L.fields()
    np.testing.assert_allclose(fl["conc"][0], CA, rtol=1e-13)
    np.testing.assert_allclose(fl["conc"][1], CB, rtol=1e-13)
    # a perturbation relaxes toward it: more A than equilibrium -> A decreases
    L2 = _uniform_reactor(2, (CA * 1.1, CB), idx_A=0, idx_B=1, k1=0.05, inv_Keq=inv_keq, inv_M_C=2.0)
    L2.step()
    assert L2.fields()["conc"][0][0, 0] < CA * 1.1


def test_r3_invariants():
    """Eq. 5c and Eq. 28: B + E -> F conserves C_B - C_E, C_B + C_F and
    C_E + C_F; one step from (0.5, 0.3, 0) at k3 = 0.1 removes 0.015 of B."""
    L = _uniform_reactor(3, (0.5, 0.3, 0.0), idx_B=0, idx_E=1, idx_F=2, k3=0.1)
    L.step()
    L.theta = -1.0
    c = L.fields()["conc"]
    np.testing.assert_allclose(c[0], 0.485, rtol=1e-13)
    np.testing.assert_allclose(c[1], 0.285, rtol=1e-13)
    np.testing.assert_allclose(c[2], 0.015, rtol=1e-13)
    for _ in range(50):
        L.step()
        L.theta = -1.0
    c = L.fields()["conc"]
    np.testing.assert_allclose(c[0] - c[1], 0.2, rtol=1e-12)
    np.testing.assert_allclose(c[0] + c[2], 0.5, rtol=1e-12)
    np.testing.assert_allclose(c[1] + c[2], 0.3, rtol=1e-12)


def test_derived_species_a():
    """Section 4.1: the last aqueous species is the total liquid concentration
    minus the transported ones.  With C_A derived from rho_1 and only R1 on,
    d C_B = k1 C_A per step, which the closed form of one step fixes."""
    k1, c_tot = 0.02, 2.0
    L = _uniform_reactor(1, (0.5,), idx_A=lbm.IDX_DERIVED, idx_B=0, k1=k1, c_total_per_rho1=c_tot)
    L.step()
    c = L.fields()["conc"][0]
    np.testing.assert_allclose(c, 0.5 + k1 * (c_tot * 1.0 - 0.5), rtol=1e-13)


# ---------------------------------------------------------------- reactive wall

def _robin_channel(L_rows, k, J0, tau_g, C0, steps):
    """x-periodic strip: row 0 mineral D(s), rows 1..L liquid, row L+1 inlet
    reservoir holding C0; species B consumed at the mineral by R2."""
    nx, ny = 3, L_rows + 2
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=1, periodic_y=0, n_species=2, idx_B=0, idx_E=1,
             J0=(J0, J0, 0, 0), tau_g=(tau_g, tau_g, 1, 1), k2=k, Vbar_D=1e-9,
             rho_in_liq=(1.0, 0.01), rho_out=(1.0, 0.01), conc_in=(C0, 0.0, 0, 0))
    m = uniform_mask(nx, ny)
    m[0, :] = lbm.SOLID_D
    m[-1, :] = lbm.INLET
    rho1 = np.full((ny, nx), 1.0)
    rho2 = np.full((ny, nx), 0.01)
    conc = np.zeros((2, ny, nx))
    conc[0, 1:-1] = C0
    L = lbm.Lattice(m, p, rho1, rho2, conc)
    for _ in range(steps):
        L.step()
        L.theta = 0.5
    return L


def test_reactive_wall_robin_closed_form():
    """Eqs. 29-31 with the halfway link rule: the steady 1D solution between a
    reactive wall (consumption k C_w) and a reservoir at C0 is linear with slope
    b = C0 / (L + tau_g - 1/2 + D/k) and link flux q = D b.  The flux of the
    product E leaving through the reservoir side equals q, so its slope is -q/D."""
    for (Lr, k, J0, tau_g) in ((8, 0.05, 0.0, 1.0), (6, 0.02, 1 / 3, 0.8)):
        C0 = 1.0
        D = 0.5 * (1 - J0) * (tau_g - 0.5)
        # ~22 e-folds of the slowest diffusive mode 4 L^2 / (pi^2 D)
        L = _robin_channel(Lr, k, J0, tau_g, C0, int(9 * Lr * Lr / D))
        b = C0 / (Lr + tau_g - 0.5 + D / k)
        C = L.fields()["conc"]
        y = np.arange(1, Lr + 1)
        Cw = D * b / k
        np.testing.assert_allclose(C[0][1:-1, 0], Cw + b * (y - 0.5), rtol=1e-9)
        q = L.last_qB[4][1, 0]          # link from row 1 toward the mineral below
        assert abs(q - D * b) < 1e-10
        slopeE = np.diff(C[1][1:-1, 0])
        np.testing.assert_allclose(slopeE, -q / D, rtol=1e-8)


def test_vop_bookkeeping_conserves_b():
    """Eqs. 32-33 with the link rule: in a closed box with no homogeneous
    reactions, sum C_B - sum V_D / Vbar_D is invariant (R2, B + D(s) -> E:
    every unit of B taken at the wall dissolves one molar volume of D(s))."""
    nx, ny = 10, 9
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=0, periodic_y=0, n_species=1, idx_B=0, J0=(1 / 3, 0, 0, 0),
             tau_g=(0.8, 1, 1, 1), k2=0.05, Vbar_D=0.3, V_split=1e30)
    m = uniform_mask(nx, ny)
    m[3:6, 3:6] = lbm.SOLID_D
    m[0, :] = m[-1, :] = lbm.WALL
    m[:, 0] = m[:, -1] = lbm.WALL
    rho1 = np.ones((ny, nx))
    rho2 = np.full((ny, nx), 0.01)
    conc = np.zeros((1, ny, nx))
    conc[0][m == lbm.LIQUID] = 0.8
    vol = np.zeros((2, ny, nx))
    vol[0][m == lbm.SOLID_D] = 50.0
    L = lbm.Lattice(m, p, rho1, rho2, conc, vol)
    inv0 = L.budget()[3] - L.V[0].sum() / p["Vbar_D"]
    for _ in range(200):
        L.step()
        L.theta = 0.5
    inv1 = L.budget()[3] - L.V[0].sum() / p["Vbar_D"]
    assert L.budget()[3] < 0.5 * 0.8 * (m == lbm.LIQUID).sum()
    assert abs(inv1 - inv0) < 1e-12 * abs(inv0)


# ---------------------------------------------------------------- status changes

def test_splitmix64_reference_vector():
    """The counter-based generator behind the VOP overflow choice is SplitMix64;
    its first outputs from state 1234567 are published."""
    want = [int(v) for v in GOLDEN["splitmix64_seed_1234567"]["outputs"]]
    s = 1234567
    got = []
    for _ in range(5):
        got.append(lbm.splitmix64(s))
        s = (s + 0x9E3779B97F4A7C15) & lbm.MASK64
    assert got == want


def test_dissolution_flip_and_fill():
    """A mineral node whose volume is used up turns liquid (Step 4-5); it is
    refilled at rest with the mean density of its surviving fluid neighbours
    and the mean concentration of its surviving liquid neighbours (brute force
    on the post-streaming neighbour values)."""
    nx, ny = 7, 7
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=1, periodic_y=1, n_species=1, idx_B=0, J0=(1 / 3, 0, 0, 0),
             tau_g=(0.8, 1, 1, 1), k2=0.05, Vbar_D=1.0)
    m = uniform_mask(nx, ny)
    m[3, 3] = lbm.SOLID_D
    rng = np.random.default_rng(3)
    rho1 = rng.uniform(0.9, 1.1, (ny, nx))
    rho2 = rng.uniform(0.01, 0.02, (ny, nx))
    conc = rng.uniform(0.5, 1.0, (1, ny, nx))
    vol = np.zeros((2, ny, nx))
    vol[0, 3, 3] = 1e-6
    L = lbm.Lattice(m, p, rho1, rho2, conc, vol)
    L.theta = 0.5
    # brute force: run the same step with the node kept solid (huge volume) to get
    # the post-streaming neighbour values
    p_ref = dict(p, V_split=1e30)
    L_ref = lbm.Lattice(m, p_ref, rho1, rho2, conc, np.where(vol > 0, 1e9, 0.0))
    L_ref.theta = 0.5
    L.step()
    L_ref.step()
    assert L.type[3, 3] == lbm.LIQUID and L_ref.type[3, 3] == lbm.SOLID_D
    fr = L_ref.fields()
    nbrs = [(3, 4), (4, 3), (3, 2), (2, 3)]
    r1 = np.mean([fr["rho1"][q] for q in nbrs])
    c = np.mean([fr["conc"][0][q] for q in nbrs])
    fl = L.fields()
    assert abs(fl["rho1"][3, 3] - r1) < 1e-13
    assert abs(fl["conc"][0][3, 3] - c) < 1e-13
    for a in range(9):
        assert abs(L.f[0, a, 3, 3] - lbm.W9[a] * r1) < 1e-15
    assert L.V[0, 3, 3] == 0.0


def test_dissolution_fill_closed_form():
    """The S->L fill (Section 4.5, R9) and the reactive link rule (R7) by hand.
    A uniform liquid at rest (no interactions, so it stays at rest and a
    bounce-back returns what it receives) surrounds one D(s) node of tiny V_D.
    In one step each of its four axis neighbours keeps all its populations but
    the one that meets the mineral, which comes back as g_out (1 - kappa) /
    (1 + kappa) (C_sat = 0, kappa = k2 / (2 J_a)); the node dissolves and is
    refilled at rest with the neighbours' densities and the mean of their
    concentrations: C0 (1 - J_a (1 - (1 - kappa) / (1 + kappa)) / J ), J = 1."""
    nx, ny = 7, 7
    p = flow_off(lbm.default_params(nx, ny))
    J0, k2, C0, r1, r2 = 1 / 3, 0.05, 0.7, 1.0, 0.015
    p.update(periodic_x=1, periodic_y=1, n_species=1, idx_B=0, J0=(J0, 0, 0, 0), tau_g=(0.8, 1, 1, 1),
             k2=k2, Vbar_D=1.0)
    m = uniform_mask(nx, ny)
    m[3, 3] = lbm.SOLID_D
    vol = np.zeros((2, ny, nx))
    vol[0, 3, 3] = 1e-6
    L = lbm.Lattice(m, p, np.full((ny, nx), r1), np.full((ny, nx), r2), np.full((1, ny, nx), C0), vol)
    L.theta = 0.5
    L.step()
    Ja = (1 - J0) / 4
    kappa = k2 / (2 * Ja)
    c_nbr = C0 - Ja * C0 + Ja * C0 * (1 - kappa) / (1 + kappa)
    fl = L.fields()
    assert L.type[3, 3] == lbm.LIQUID
    for q in [(3, 4), (4, 3), (3, 2), (2, 3)]:
        assert abs(fl["conc"][0][q] - c_nbr) < 1e-15
    for q in [(2, 2), (2, 4), (4, 2), (4, 4), (0, 0)]:
        assert abs(fl["conc"][0][q] - C0) < 1e-15
    assert abs(fl["conc"][0][3, 3] - c_nbr) < 1e-15
    assert abs(fl["rho1"][3, 3] - r1) < 1e-15 and abs(fl["rho2"][3, 3] - r2) < 1e-15
    assert abs(fl["ux"][3, 3]) < 1e-15 and abs(fl["uy"][3, 3]) < 1e-15
    for a in range(9):
        assert abs(L.f[0, a, 3, 3] - lbm.W9[a] * r1) < 1e-15
        assert abs(L.f[1, a, 3, 3] - lbm.W9[a] * r2) < 1e-15
    assert L.V[0, 3, 3] == 0.0


def test_overflow_flip_conserves_volume_and_mass():
    """Precipitation overflow (VOP): a node whose volume reaches V_split keeps
    1 and puts the excess into the liquid neighbour picked by SplitMix64; the
    vanished liquid's mass goes to its surviving neighbours, so the fluid mass
    is unchanged and sum V_F + Vbar_F * (F taken at the wall) is invariant."""
    nx, ny = 8, 8
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=1, periodic_y=1, n_species=1, idx_F=0, J0=(1 / 3, 0, 0, 0),
             tau_g=(0.8, 1, 1, 1), k4=0.1, Vbar_F=2.0, V_split=2.0, seed=77)
    m = uniform_mask(nx, ny)
    m[4, 4] = lbm.SOLID_F
    rho1 = np.full((ny, nx), 1.0)
    rho2 = np.full((ny, nx), 0.01)
    conc = np.zeros((1, ny, nx))
    conc[0][m == lbm.LIQUID] = 1.0
    vol = np.zeros((2, ny, nx))
    vol[1, 4, 4] = 1.999
    L = lbm.Lattice(m, p, rho1, rho2, conc, vol)
    L.theta = 0.5
    m0 = L.budget()
    L.step()
    assert (L.type == lbm.SOLID_F).sum() == 2
    nliq = [(4, 5), (5, 4), (4, 3), (3, 4)]       # E, N, W, S of (4, 4)
    r = lbm.splitmix64(lbm.overflow_key(77, 0, 4 * nx + 4))
    tgt = nliq[r % 4]
    assert L.type[tgt] == lbm.SOLID_F
    qsum = sum(L.last_qF[lbm.OPP5[b]][nliq[b - 1]] for b in range(1, 5))
    total = 1.999 + 2.0 * qsum
    assert abs(L.V[1, 4, 4] - 1.0) < 1e-15
    assert abs(L.V[1][tgt] - (total - 1.0)) < 1e-15
    m1 = L.budget()
    assert abs(m1[1] - m0[1]) < 1e-12 * m0[1]
    assert abs(m1[2] - m0[2]) < 1e-12 * m0[2]


def test_liquid_to_gas_amendment_conserves_solute():
    """Section 4.5, Step 2: a liquid node whose density falls below the
    threshold becomes gas and hands its solute to its liquid neighbours, so the
    total solute is unchanged; the gas node holds none."""
    nx, ny = 9, 9
    p = flow_off(lbm.default_params(nx, ny))
    p.update(n_species=1, idx_A=0, J0=(1 / 3, 0, 0, 0), tau_g=(0.8, 1, 1, 1))
    m = uniform_mask(nx, ny)
    rho1 = np.full((ny, nx), 1.0)
    rho1[4, 4] = 0.2
    rho2 = np.full((ny, nx), 0.01)
    conc = np.full((1, ny, nx), 0.5)
    conc[0, 4, 4] = 3.0
    L = lbm.Lattice(m, p, rho1, rho2, conc)
    L.theta = 0.5
    c0 = L.budget()[3]
    L.step()
    assert L.type[4, 4] == lbm.GAS
    assert abs(L.budget()[3] - c0) < 1e-13 * c0
    assert np.all(L.g[:, :, 4, 4] == 0.0)
