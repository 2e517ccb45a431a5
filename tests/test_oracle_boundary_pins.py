"""Pins of the oracle's reservoir boundaries and of the gas-to-liquid amendment.

The reservoirs (an inlet column whose state alternates liquid and gas slugs
with linear ramps, and an outlet column that follows the phase arriving from
upstream) are the open boundaries of the pressure-driven porous workload; the
paper's own scene has only a free top outlet (Section 5), so their definition
is this library's and is stated once more here by hand.  The appearing-node
rule is the amendment of Section 4.5 (Step 2) for a gas node that turns
liquid.  Every expected value below is computed by hand from that definition
(a piecewise-linear weight, a choice between two given states, the Eq. 8
equilibrium at a given density and velocity, a mean of given neighbour
concentrations), not by the oracle.
"""
import numpy as np
import pytest

from oracle import lbm


def flow_off(p):
    """Two ideal components (G = 0): no pseudo-potential forces."""
    p.update(G11=0.0, G12=0.0, G21=0.0)
    return p


def moving_lattice(m, p, rho1, rho2, u, conc=None):
    """A lattice whose fluid populations start at the Eq. 8 equilibrium of a
    uniform velocity u (the oracle's own initial state is at rest)."""
    L = lbm.Lattice(m, p, rho1, rho2, conc)
    fluid = (m == lbm.LIQUID) | (m == lbm.GAS)
    ux = np.full(m.shape, u[0])
    uy = np.full(m.shape, u[1])
    for a in range(9):
        L.f[0, a] = np.where(fluid, lbm.feq9(a, rho1, ux, uy), 0.0)
        L.f[1, a] = np.where(fluid, lbm.feq9(a, rho2, ux, uy), 0.0)
    return L


# Weight of the gas state at the inlet over one period of a 5-step liquid slug
# and a 3-step gas slug with a 2-step ramp: the last two steps of each slug
# blend linearly toward the next state in thirds (1/3, 2/3 into gas; 2/3, 1/3
# back to liquid); with no ramp the switch is sharp.
SLUG_5_3_RAMP_2 = [0.0, 0.0, 0.0, 1 / 3, 2 / 3, 1.0, 2 / 3, 1 / 3]
SLUG_5_3_SHARP = [0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0]


@pytest.mark.parametrize("ramp,expected", [(2, SLUG_5_3_RAMP_2), (0, SLUG_5_3_SHARP)])
def test_inlet_slug_weight_over_two_periods(ramp, expected):
    nx, ny = 6, 3
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=0, periodic_y=1, inlet_period_liq=5, inlet_period_gas=3, inlet_ramp=ramp,
             rho_in_liq=(1.0, 0.0), rho_in_gas=(0.0, 1.0))
    m = np.full((ny, nx), lbm.LIQUID, np.uint8)
    m[:, 0] = lbm.INLET
    rho1 = np.where(m == lbm.LIQUID, 1.0, 0.0)
    rho2 = np.where(m == lbm.LIQUID, 0.01, 0.0)
    L = lbm.Lattice(m, p, rho1, rho2)
    zero = np.zeros((ny, nx))
    for t in range(16):
        r1, r2, _, _ = L._reservoir_state(L.type, rho1, rho2, zero, zero, t, 0.5)
        wg = expected[t % 8]
        np.testing.assert_allclose(r1[:, 0], 1.0 - wg, rtol=0, atol=1e-15, err_msg=f"t={t}")
        np.testing.assert_allclose(r2[:, 0], wg, rtol=0, atol=1e-15, err_msg=f"t={t}")
        assert np.all(r1[:, 1:] == 0.0) and np.all(r2[:, 1:] == 0.0)


@pytest.mark.parametrize("axis", [0, 1])
def test_outlet_follows_the_phase_of_the_node_upstream(axis):
    """Outlet along x (column nx-1 drains x-1) and along y (row ny-1 drains
    y-1): liquid state where the upstream node is marked liquid, gas state
    where it is marked gas."""
    n = 6
    p = flow_off(lbm.default_params(n, n))
    p.update(periodic_x=1 if axis == 1 else 0, periodic_y=1 if axis == 0 else 0, outlet_axis=axis,
             rho_out=(0.9, 0.01), rho_out_gas=(0.05, 0.3))
    m = np.full((n, n), lbm.LIQUID, np.uint8)
    rho1 = np.full((n, n), 1.0)
    rho2 = np.full((n, n), 0.01)
    gas_lanes = (0, 3, 4)                 # lanes whose upstream node is gas
    for k in range(n):
        if axis == 0:
            m[k, n - 1] = lbm.OUTLET
            if k in gas_lanes:
                m[k, n - 2] = lbm.GAS
                rho1[k, n - 2] = 0.1      # below the threshold 0.5
            # the node two upstream is of the other phase: it must not matter
            rho1[k, n - 3] = 1.0 if k in gas_lanes else 0.1
        else:
            m[n - 1, k] = lbm.OUTLET
            if k in gas_lanes:
                m[n - 2, k] = lbm.GAS
                rho1[n - 2, k] = 0.1
            rho1[n - 3, k] = 1.0 if k in gas_lanes else 0.1
    rho1 = np.where(m == lbm.OUTLET, 0.0, rho1)
    rho2 = np.where(m == lbm.OUTLET, 0.0, rho2)
    L = lbm.Lattice(m, p, rho1, rho2)
    zero = np.zeros((n, n))
    r1, r2, _, _ = L._reservoir_state(L.type, rho1, rho2, zero, zero, 0, 0.5)
    for k in range(n):
        at = (k, n - 1) if axis == 0 else (n - 1, k)
        want = (0.05, 0.3) if k in gas_lanes else (0.9, 0.01)
        assert r1[at] == want[0] and r2[at] == want[1], (k, r1[at], r2[at])


def test_reservoirs_push_the_equilibrium_of_their_state_at_the_neighbour_velocity():
    """One step of a channel flowing at u = (0.04, 0.02) between an inlet column
    (rho = 1.05, 0.02; species at 0.7) and an outlet column (liquid state
    0.95, 0.015): the populations that enter the first and last fluid columns
    from the reservoirs are Eq. 8 at the reservoir density and the velocity of
    that fluid column, w_a rho (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u^2), and the
    inlet's solute populations are Eq. 21, C_in (J_a + e.u / 2)."""
    nx, ny = 6, 3
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=0, periodic_y=1, rho_in_liq=(1.05, 0.02), rho_out=(0.95, 0.015),
             rho_out_gas=(0.05, 0.3), n_species=1, idx_A=0, J0=(1 / 3, 0, 0, 0), tau_g=(1.0, 1, 1, 1),
             conc_in=(0.7, 0, 0, 0))
    m = np.full((ny, nx), lbm.LIQUID, np.uint8)
    m[:, 0] = lbm.INLET
    m[:, nx - 1] = lbm.OUTLET
    fluid = m == lbm.LIQUID
    rho1 = np.where(fluid, 1.0, 0.0)
    rho2 = np.where(fluid, 0.01, 0.0)
    conc = np.zeros((1, ny, nx))
    L = moving_lattice(m, p, rho1, rho2, (0.04, 0.02), conc)
    L.theta = 0.5
    L.step()
    # 1 + 3 e.u + 4.5 (e.u)^2 - 1.5 |u|^2 with |u|^2 = 0.002, by hand
    into_first = {1: 1.1242, 5: 1.1932, 8: 1.0588}     # e.u = 0.04, 0.06, 0.02
    into_last = {3: 0.8842, 6: 0.9388, 7: 0.8332}      # e.u = -0.04, -0.02, -0.06
    for y in range(ny):
        for a, fac in into_first.items():
            assert abs(L.f[0, a, y, 1] - lbm.W9[a] * 1.05 * fac) < 1e-15
            assert abs(L.f[1, a, y, 1] - lbm.W9[a] * 0.02 * fac) < 1e-16
        for a, fac in into_last.items():
            assert abs(L.f[0, a, y, nx - 2] - lbm.W9[a] * 0.95 * fac) < 1e-15
            assert abs(L.f[1, a, y, nx - 2] - lbm.W9[a] * 0.015 * fac) < 1e-16
        # the inlet's solute: C_in (1/6 + 0.04 / 2) into the first column along +x
        assert abs(L.g[0, 1, y, 1] - 0.7 * (1 / 6 + 0.02)) < 1e-15


def test_outlet_concentration_is_the_upstream_value_the_step_starts_from():
    """The outlet column's solute state is the concentration of the liquid node
    upstream of it as the step begins, before that node takes a share of a
    vanishing neighbour's solute (Step 2): here the upstream node holds 0.5 and
    receives 3.0 / 3 from its west neighbour, which turns gas; the population
    the outlet sends back into it (at rest, tau_g = 1) is J_a 0.5 = 0.5 / 6."""
    nx, ny = 6, 3
    p = flow_off(lbm.default_params(nx, ny))
    p.update(periodic_x=0, periodic_y=1, rho_out=(1.0, 0.01), rho_out_gas=(0.05, 0.3),
             n_species=1, idx_A=0, J0=(1 / 3, 0, 0, 0), tau_g=(1.0, 1, 1, 1))
    m = np.full((ny, nx), lbm.LIQUID, np.uint8)
    m[:, nx - 1] = lbm.OUTLET
    fluid = m == lbm.LIQUID
    rho1 = np.where(fluid, 1.0, 0.0)
    rho1[1, nx - 3] = 0.2                  # vanishes: liquid -> gas
    rho2 = np.where(fluid, 0.01, 0.0)
    conc = np.where(fluid, 0.5, 0.0)[None].copy()
    conc[0, 1, nx - 3] = 3.0
    L = lbm.Lattice(m, p, rho1, rho2, conc)
    L.theta = 0.5
    L.step()
    assert L.type[1, nx - 3] == lbm.GAS
    assert abs(L.g[0, 3, 1, nx - 2] - 0.5 / 6.0) < 1e-15
    # the upstream node itself did receive its share (three liquid receivers:
    # north, south and east of the vanishing node)
    c_up = L.g[0, :, 1, nx - 2].sum()
    assert c_up > 0.5 + 0.5 / 6.0


def test_gas_node_turning_liquid_takes_the_mean_of_its_surviving_liquid_neighbours():
    """Section 4.5, Step 2, appearing node: a gas node marked liquid takes, at
    equilibrium, the mean concentration of its neighbours that were liquid and
    stay liquid; a neighbour that is itself appearing, or gas, does not count.
    Centre (2, 2): east 0.3 and north 0.6 survive, west (2, 1) appears too,
    south (1, 2) stays gas, so its value is 0.45.  The west node's surviving
    neighbours all hold 0.5, so it takes 0.5.  After one step at rest with
    tau_g = 1 the centre holds J_0 0.45 plus J_a times what streams in: 0.3
    from the east, 0.6 from the north, 0.5 from the west and its own 0.45
    bounced back at the gas node south of it."""
    n = 5
    p = flow_off(lbm.default_params(n, n))
    p.update(n_species=1, idx_A=0, J0=(1 / 3, 0, 0, 0), tau_g=(1.0, 1, 1, 1))
    m = np.full((n, n), lbm.LIQUID, np.uint8)
    m[2, 2] = lbm.GAS        # appears (rho_1 above the threshold)
    m[2, 1] = lbm.GAS        # appears too
    m[1, 2] = lbm.GAS        # stays gas
    rho1 = np.full((n, n), 1.0)
    rho1[1, 2] = 0.1
    rho2 = np.full((n, n), 0.01)
    conc = np.full((1, n, n), 0.5)
    conc[0, 2, 3] = 0.3      # east of the centre
    conc[0, 3, 2] = 0.6      # north of the centre
    L = lbm.Lattice(m, p, rho1, rho2, conc)
    L.theta = 0.5
    c0 = L.budget()[3]
    L.step()
    assert L.type[2, 2] == lbm.LIQUID and L.type[2, 1] == lbm.LIQUID and L.type[1, 2] == lbm.GAS
    want = (1 / 3) * 0.45 + (1 / 6) * (0.3 + 0.6 + 0.5 + 0.45)
    assert abs(L.g[0, :, 2, 2].sum() - want) < 1e-15
    # the appearing nodes created solute: 0.45 + 0.5 more than before
    assert abs(L.budget()[3] - (c0 + 0.45 + 0.5)) < 1e-13
