"""Plain FP64 CPU oracle of the pore-scale two-phase multi-mixture lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This module is the correctness reference for the CUDA
library.  Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does.  It shares no code with the
CUDA path.

It follows Chen, Kang, Tang, Robinson, He, Tao, "Pore-scale simulation of
multicomponent multiphase reactive transport with dissolution and precipitation"
(arXiv 1410.3464):

  * Section 3.1, Eqs. 6-19: two-component pseudo-potential (Shan-Chen) D2Q9 LBM
    with a Carnahan-Starling liquid component and an ideal gas component;
  * Section 3.2, Eqs. 20-24: D2Q5 mass-transport LBM for each aqueous solute;
  * Section 4, Eqs. 25-28: two-phase multi-mixture model (solutes only in the
    liquid phase, liquid-gas interface no-flux, last aqueous species derived);
  * Section 4.3-4.6, Eqs. 29-35: heterogeneous reactions at liquid-solid links
    and the volume-of-pixel (VOP) solid update with node status changes;
  * Section 4.7: the numerical procedure (Steps 1-5).

Everything is whole-array numpy in float64 (one array per intermediate, explicit
loops over lattice directions, Python loops over the few interface nodes that
change status).  Where the paper is silent or garbled this module implements the
readings listed in the design notes (force weights w(1)=1/9, w(2)=1/36; the
reactive link rule; the VOP overflow rule; the status-change amendments; the
lagged half-maximum liquid threshold).  Each function names the equation it
follows.

Array layout: 2D fields are [ny, nx] indexed [y, x]; populations are
f[component][direction][y, x] and g[species][direction][y, x].
"""
from __future__ import annotations

import numpy as np

# Node types (Fig. 2: liquid, gas, solid D(s), solid F(s); plus inert walls and
# fixed-state reservoir nodes for inflow/outflow boundaries).
LIQUID, GAS, SOLID_D, SOLID_F, WALL, INLET, OUTLET = range(7)

# Eq. 7: D2Q9 velocity set, alpha = 0 rest, 1-4 axis, 5-8 diagonal.
EX9 = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY9 = (0, 0, 1, 0, -1, 1, 1, -1, -1)
OPP9 = (0, 3, 4, 1, 2, 7, 8, 5, 6)
# Eq. 8 weights.
W9 = (4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
      1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0)
# Interaction weights w(|e|^2) of Eqs. 11, 14, 16.  Reading: w(1)=1/9, w(2)=1/36,
# so that sum_a w e_x^2 = c_s^2 = 1/3, which is the normalisation Eq. 13 (factor
# 6/G) and Eq. A1 (factor c_s^2/2) both assume.
WF = (0.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
      1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0)
# Section 3.2: D2Q5 is the D2Q9 set without the diagonals.
EX5 = EX9[:5]
EY5 = EY9[:5]
OPP5 = (0, 3, 4, 1, 2)

CS2 = 1.0 / 3.0  # lattice sound speed squared (c = 1)

MASK64 = (1 << 64) - 1


def splitmix64(state: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea, Flood 2014) whose
    state before the call is `state`: the state advances by the golden-ratio
    increment and the output is the mixed new state."""
    z = (state + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def overflow_key(seed: int, step: int, node: int) -> int:
    """Counter for the VOP overflow choice: seed xor (step << 40) xor node."""
    return (int(seed) ^ ((int(step) << 40) & MASK64) ^ int(node)) & MASK64


# ---------------------------------------------------------------- equations

def cs_pressure(rho, a, b, R, T):
    """Eq. 12: Carnahan-Starling equation of state p(rho)."""
    eta = b * rho / 4.0
    return rho * R * T * (1.0 + eta + eta * eta - eta * eta * eta) / (1.0 - eta) ** 3 - a * rho * rho


def psi1_argument(rho, a, b, R, T, G11):
    """The quantity under the square root of Eq. 13: 6/G11 (p(rho) - c_s^2 rho)."""
    return 6.0 / G11 * (cs_pressure(rho, a, b, R, T) - CS2 * rho)


def psi1_of_rho(rho, a, b, R, T, G11):
    """Eq. 13: effective mass of the liquid component from the C-S EOS."""
    arg = psi1_argument(rho, a, b, R, T, G11)
    if np.any(arg < 0):
        raise EOSDomainError("Eq. 13 square-root argument is negative")
    return np.sqrt(arg)


def phi1_of_rho2(rho2, rho20):
    """Eq. 15a: phi_1 = 1 - exp(-rho_2 / rho_20)."""
    return 1.0 - np.exp(-rho2 / rho20)


def phi2_of_rho1(rho1, a0, rho10):
    """Eq. 15b: phi_2 = a_0 - exp(-rho_1 / rho_10)."""
    return a0 - np.exp(-rho1 / rho10)


def feq9(a, rho, ux, uy):
    """Eq. 8: D2Q9 equilibrium of direction a (c = 1)."""
    eu = EX9[a] * ux + EY9[a] * uy
    uu = ux * ux + uy * uy
    return W9[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu)


def j5(a, J0):
    """Eq. 22: D2Q5 rest fraction J_0 and J_{1..4} = (1 - J_0)/4."""
    return J0 if a == 0 else (1.0 - J0) / 4.0


def geq5(a, C, J0, ux, uy):
    """Eq. 21: D2Q5 equilibrium g^eq = C (J_a + e_a.u / 2)."""
    return C * (j5(a, J0) + 0.5 * (EX5[a] * ux + EY5[a] * uy))


class EOSDomainError(ValueError):
    pass


class NonFiniteError(ValueError):
    pass


# ---------------------------------------------------------------- parameters

MAX_SPECIES = 4
IDX_ABSENT = -1
IDX_DERIVED = -2


def default_params(nx, ny):
    """Parameter set with the paper's fluid constants (Section 3.1: G11 = -1,
    a0 = 0.005, rho10 = -0.008/ln(a0), rho20 = 0.003, G12 = G21 = 0.001,
    tau = 1) and everything else switched off."""
    return dict(
        nx=nx, ny=ny, periodic_x=1, periodic_y=1,
        tau=(1.0, 1.0), G11=-1.0, G12=0.001, G21=0.001,
        a0=0.005, rho10=-0.008 / np.log(0.005), rho20=0.003,
        w_adh=(0.0, 0.0), eos_a=1.0, eos_b=4.0, eos_R=1.0, eos_T=0.7 * 0.09432936,
        body_force=(0.0, 0.0), rho_ref=(1.0, 1.0),
        n_species=0, idx_A=IDX_ABSENT, idx_B=IDX_ABSENT, idx_E=IDX_ABSENT, idx_F=IDX_ABSENT,
        J0=(0.0,) * MAX_SPECIES, tau_g=(1.0,) * MAX_SPECIES, conc_ref=(0.0,) * MAX_SPECIES,
        k1=0.0, inv_Keq=0.0, k3=0.0, k2=0.0, k4=0.0, C_F_sat=0.0,
        gas_yield=0.0, inv_M_C=0.0, c_total_per_rho1=0.0,
        Vbar_D=1.0, Vbar_F=1.0, V_split=2.0, seed=0,
        rho_in_liq=(0.0, 0.0), rho_in_gas=(0.0, 0.0), rho_out=(0.0, 0.0), rho_out_gas=(0.0, 0.0),
        inlet_period_liq=1, inlet_period_gas=0, inlet_ramp=0, conc_in=(0.0,) * MAX_SPECIES,
        r1_surface_factor=1.0, inlet_axis=0, outlet_axis=0,
    )


# ---------------------------------------------------------------- the lattice

class Lattice:
    """State of one simulation: populations f (2 components x 9), g (species x 5),
    node types, solid volumes V_D, V_F, the liquid threshold and the step count.
    """

    def __init__(self, mask, params, rho1=None, rho2=None, conc=None, vol=None):
        p = dict(params)
        self.p = p
        self.nx, self.ny = int(p["nx"]), int(p["ny"])
        self.px, self.py = bool(p["periodic_x"]), bool(p["periodic_y"])
        self.ns = int(p["n_species"])
        mask = np.asarray(mask, dtype=np.uint8).reshape(self.ny, self.nx)
        self.type = mask.copy()
        fluid = self._fluid(self.type)
        liquid = self.type == LIQUID
        shape = (self.ny, self.nx)
        r1 = np.zeros(shape) if rho1 is None else np.asarray(rho1, dtype=np.float64).reshape(shape)
        r2 = np.zeros(shape) if rho2 is None else np.asarray(rho2, dtype=np.float64).reshape(shape)
        r1 = np.where(fluid, r1, 0.0)
        r2 = np.where(fluid, r2, 0.0)
        zero = np.zeros(shape)
        # Initial state: equilibrium at rest (Eq. 8, Eq. 21).
        self.f = np.zeros((2, 9) + shape)
        for a in range(9):
            self.f[0, a] = np.where(fluid, feq9(a, r1, zero, zero), 0.0)
            self.f[1, a] = np.where(fluid, feq9(a, r2, zero, zero), 0.0)
        self.g = np.zeros((self.ns, 5) + shape)
        if conc is not None:
            c = np.asarray(conc, dtype=np.float64).reshape((self.ns,) + shape)
            for k in range(self.ns):
                for a in range(5):
                    self.g[k, a] = np.where(liquid, j5(a, p["J0"][k]) * c[k], 0.0)
        self.V = np.zeros((2,) + shape)
        if vol is None:
            self.V[0] = np.where(self.type == SOLID_D, 1.0, 0.0)
            self.V[1] = np.where(self.type == SOLID_F, 1.0, 0.0)
        else:
            self.V[:] = np.asarray(vol, dtype=np.float64).reshape((2,) + shape)
        self.t = 0
        rho1_now, _ = self._density(0), None
        self.theta = 0.5 * self._fluid_max(rho1_now, fluid)

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _fluid(typ):
        return (typ == LIQUID) | (typ == GAS)

    @staticmethod
    def _reservoir(typ):
        return (typ == INLET) | (typ == OUTLET)

    @staticmethod
    def _mineral(typ):
        return (typ == SOLID_D) | (typ == SOLID_F)

    @staticmethod
    def _fluid_max(rho1, fluid):
        return float(rho1[fluid].max()) if np.any(fluid) else 0.0

    def nb(self, a, dx, dy, fill):
        """Field value at (x + dx, y + dy): periodic wrap where the axis is
        periodic, `fill` outside the domain otherwise."""
        ny, nx = a.shape
        xs = np.arange(nx) + dx
        ys = np.arange(ny) + dy
        if self.px:
            xs = xs % nx
        if self.py:
            ys = ys % ny
        vx = (xs >= 0) & (xs < nx)
        vy = (ys >= 0) & (ys < ny)
        out = np.full_like(a, fill)
        out[np.ix_(vy, vx)] = a[np.ix_(ys[vy], xs[vx])]
        return out

    def nb_coord(self, y, x, dx, dy):
        """Coordinates of the neighbour (x + dx, y + dy) or None outside."""
        xx, yy = x + dx, y + dy
        if self.px:
            xx %= self.nx
        if self.py:
            yy %= self.ny
        if 0 <= xx < self.nx and 0 <= yy < self.ny:
            return yy, xx
        return None

    def _density(self, comp):
        """Eq. 9a: rho_sigma = sum_a f_sigma,a (summed in direction order)."""
        f = self.f[comp]
        r = f[0].copy()
        for a in range(1, 9):
            r = r + f[a]
        return r

    def _momentum(self, comp):
        """Eq. 9b: rho_sigma u_sigma = sum_a f_sigma,a e_a."""
        f = self.f[comp]
        jx = np.zeros_like(f[0])
        jy = np.zeros_like(f[0])
        for a in range(1, 9):
            if EX9[a]:
                jx = jx + EX9[a] * f[a]
            if EY9[a]:
                jy = jy + EY9[a] * f[a]
        return jx, jy

    def _conc(self, g):
        """Eq. 23: C_k = sum_a g_k,a (direction order)."""
        c = g[0].copy()
        for a in range(1, 5):
            c = c + g[a]
        return c

    def _axes(self):
        """Offsets of the node downstream of an inlet and upstream of an outlet:
        along x (axis 0: x + 1, x - 1) or along y (axis 1: y + 1, y - 1)."""
        ia, oa = int(self.p.get("inlet_axis", 0)), int(self.p.get("outlet_axis", 0))
        return ((1, 0) if ia == 0 else (0, 1)), ((-1, 0) if oa == 0 else (0, -1))

    def _reservoir_state(self, typ, rho1, rho2, jx, jy, t, theta):
        """Reservoir nodes hold a fixed equilibrium state that they push into
        their fluid neighbours: an inlet whose densities alternate between a
        liquid and a gas state (gas slugs), and an outlet at fixed density.  The
        velocity is that of the node next to it (downstream of an inlet,
        upstream of an outlet) when that node is fluid, else zero."""
        p = self.p
        inlet, outlet = typ == INLET, typ == OUTLET
        pl, pg = int(p["inlet_period_liq"]), int(p["inlet_period_gas"])
        ramp = int(p.get("inlet_ramp", 0))
        wg = 0.0                    # weight of the gas state: slugs with linear ramps
        if pg > 0:
            ph = t % (pl + pg)
            if ph < pl:
                wg = (ph - (pl - ramp) + 1) / (ramp + 1) if (ramp > 0 and ph >= pl - ramp) else 0.0
            else:
                wg = 1.0 - (ph - (pl + pg - ramp) + 1) / (ramp + 1) if (ramp > 0 and ph >= pl + pg - ramp) else 1.0
        rin = [(1.0 - wg) * p["rho_in_liq"][s] + wg * p["rho_in_gas"][s] for s in range(2)]
        fluid = self._fluid(typ)
        (idx, idy), (odx, ody) = self._axes()
        # outlet: liquid or gas state by the marking of the node upstream
        up_liq = self.nb(fluid & (rho1 > theta), odx, ody, False)
        ro = [np.where(up_liq, p["rho_out"][s], p["rho_out_gas"][s]) for s in range(2)]
        r1 = np.where(inlet, rin[0], np.where(outlet, ro[0], 0.0))
        r2 = np.where(inlet, rin[1], np.where(outlet, ro[1], 0.0))
        rho = rho1 + rho2
        with np.errstate(invalid="ignore", divide="ignore"):
            ux = np.where(fluid, (jx) / np.where(fluid, rho, 1.0), 0.0)
            uy = np.where(fluid, (jy) / np.where(fluid, rho, 1.0), 0.0)
        # neighbour used for the velocity
        ux_res = np.where(inlet, self.nb(ux, idx, idy, 0.0), np.where(outlet, self.nb(ux, odx, ody, 0.0), 0.0))
        uy_res = np.where(inlet, self.nb(uy, idx, idy, 0.0), np.where(outlet, self.nb(uy, odx, ody, 0.0), 0.0))
        return r1, r2, ux_res, uy_res

    # -- observables -------------------------------------------------------
    def moments(self):
        return self._density(0), self._density(1), self._momentum(0), self._momentum(1)

    def _forces(self, typ, rho1, rho2, r1res, r2res):
        """Eqs. 11-16: F_1 = F_11 + F_12 + F_1w + rho_1 g, F_2 = F_21 + F_2w + rho_2 g.
        In the cohesion (Eq. 11) and inter-component (Eq. 14) sums a solid
        neighbour takes the value of its mirror image across the wall (a
        symmetry wall), so that with w = 0 the wall is neither wetting nor
        non-wetting (90 degrees, as App. A2 and Section 5 state):
          * an axis neighbour's mirror image is the centre node itself;
          * a diagonal neighbour (x + ex, y + ey) on a flat wall is mirrored
            onto the live one of (x + ex, y) and (x, y + ey) when exactly one
            of them is live; otherwise (a corner) it takes the centre's value.
        Wetting is set only by the adhesion term of Eq. 16, whose wall density
        s is 1 at solid nodes (and outside a non-periodic edge) and 0 at fluid
        and reservoir nodes."""
        p = self.p
        fluid = self._fluid(typ)
        res = self._reservoir(typ)
        live = fluid | res
        r1 = np.where(fluid, rho1, np.where(res, r1res, 0.0))
        r2 = np.where(fluid, rho2, np.where(res, r2res, 0.0))
        if p["G11"] != 0.0:
            arg = np.where(live, psi1_argument(r1, p["eos_a"], p["eos_b"], p["eos_R"], p["eos_T"], p["G11"]), 0.0)
            if np.any(arg[live] < 0):
                raise EOSDomainError("Eq. 13 square-root argument is negative")
            psi1 = np.sqrt(np.where(live, arg, 0.0))
        else:
            psi1 = np.zeros_like(r1)
        phi1 = np.where(live, phi1_of_rho2(r2, p["rho20"]), 0.0)
        phi2 = np.where(live, phi2_of_rho1(r1, p["a0"], p["rho10"]), 0.0)
        s = np.where(live, 0.0, 1.0)

        def wsum(field):
            # sum_a w(|e_a|^2) field(x + e_a) e_a, a = 1..8, a solid neighbour
            # replaced by its mirror image as above
            sx = np.zeros_like(field)
            sy = np.zeros_like(field)
            for a in range(1, 9):
                ex, ey = EX9[a], EY9[a]
                v = self.nb(field, ex, ey, 0.0)
                if ex != 0 and ey != 0:
                    live_h = self.nb(live, ex, 0, False)
                    live_v = self.nb(live, 0, ey, False)
                    image = np.where(live_h & ~live_v, self.nb(field, ex, 0, 0.0),
                                     np.where(live_v & ~live_h, self.nb(field, 0, ey, 0.0), field))
                else:
                    image = field
                v = np.where(self.nb(live, ex, ey, False), v, image)
                sx = sx + WF[a] * v * ex
                sy = sy + WF[a] * v * ey
            return sx, sy

        spx, spy = wsum(psi1)
        s21x, s21y = wsum(phi2)   # neighbours' phi_2, for F_12
        s12x, s12y = wsum(phi1)   # neighbours' phi_1, for F_21
        sfull = self.nb(s, 0, 0, 1.0)
        ssx = np.zeros_like(s)
        ssy = np.zeros_like(s)
        for a in range(1, 9):
            v = self.nb(sfull, EX9[a], EY9[a], 1.0)
            ssx = ssx + WF[a] * v * EX9[a]
            ssy = ssy + WF[a] * v * EY9[a]
        gx, gy = p["body_force"]
        G11, G12, G21 = p["G11"], p["G12"], p["G21"]
        w1, w2 = p["w_adh"]
        # Eq. 11 (sigma = 1), Eq. 14a, Eq. 16 (psi_2 := rho_2 for the ideal gas)
        F1x = -G11 * psi1 * spx - G12 * phi1 * s21x - w1 * psi1 * ssx + rho1 * gx
        F1y = -G11 * psi1 * spy - G12 * phi1 * s21y - w1 * psi1 * ssy + rho1 * gy
        # Eq. 14b, Eq. 16
        F2x = -G21 * phi2 * s12x - w2 * rho2 * ssx + rho2 * gx
        F2y = -G21 * phi2 * s12y - w2 * rho2 * ssy + rho2 * gy
        z = np.zeros_like(rho1)
        return (np.where(fluid, F1x, z), np.where(fluid, F1y, z),
                np.where(fluid, F2x, z), np.where(fluid, F2y, z))

    def _velocities(self, rho1, rho2, j1, j2, F):
        """Eqs. 17-19: common velocity u', forced equilibrium velocities, and the
        physical velocity u_r."""
        t1, t2 = self.p["tau"]
        F1x, F1y, F2x, F2y = F
        den = rho1 / t1 + rho2 / t2
        upx = (j1[0] / t1 + j2[0] / t2) / den
        upy = (j1[1] / t1 + j2[1] / t2) / den
        # a component with no mass at a node carries no forced velocity shift
        z1 = rho1 == 0.0
        z2 = rho2 == 0.0
        r1s = np.where(z1, 1.0, rho1)
        r2s = np.where(z2, 1.0, rho2)
        u1x = upx + np.where(z1, 0.0, t1 * F1x / r1s)
        u1y = upy + np.where(z1, 0.0, t1 * F1y / r1s)
        u2x = upx + np.where(z2, 0.0, t2 * F2x / r2s)
        u2y = upy + np.where(z2, 0.0, t2 * F2y / r2s)
        rho = rho1 + rho2
        urx = (j1[0] + j2[0] + 0.5 * (F1x + F2x)) / rho
        ury = (j1[1] + j2[1] + 0.5 * (F1y + F2y)) / rho
        return (u1x, u1y), (u2x, u2y), (urx, ury)

    def fields(self):
        """Observable fields of the current state: rho_1, rho_2 and u_r (Eq. 19)
        at fluid nodes (0 elsewhere), concentrations at liquid nodes, node
        types and solid volumes."""
        typ = self.type
        fluid = self._fluid(typ)
        rho1, rho2, j1, j2 = self.moments()
        r1res, r2res, _, _ = self._reservoir_state(typ, rho1, rho2, j1[0] + j2[0], j1[1] + j2[1], self.t, self.theta)
        F = self._forces(typ, rho1, rho2, r1res, r2res)
        with np.errstate(invalid="ignore", divide="ignore"):
            _, _, ur = self._velocities(np.where(fluid, rho1, 1.0), np.where(fluid, rho2, 1.0), j1, j2, F)
        out = dict(
            rho1=np.where(fluid, rho1, 0.0), rho2=np.where(fluid, rho2, 0.0),
            ux=np.where(fluid, ur[0], 0.0), uy=np.where(fluid, ur[1], 0.0),
            type=typ.copy(), vol_d=self.V[0].copy(), vol_f=self.V[1].copy(),
        )
        liquid = typ == LIQUID
        out["conc"] = np.stack([np.where(liquid, self._conc(self.g[k]), 0.0) for k in range(self.ns)]) \
            if self.ns else np.zeros((0, self.ny, self.nx))
        return out

    def budget(self):
        """[max rho_1, sum rho_1, sum rho_2 (fluid nodes), sum C_k (liquid nodes),
        sum V_D, sum V_F]."""
        typ = self.type
        fluid = self._fluid(typ)
        rho1, rho2 = self._density(0), self._density(1)
        out = [self._fluid_max(rho1, fluid), float(rho1[fluid].sum()), float(rho2[fluid].sum())]
        liquid = typ == LIQUID
        for k in range(self.ns):
            out.append(float(self._conc(self.g[k])[liquid].sum()))
        out += [float(self.V[0].sum()), float(self.V[1].sum())]
        return np.array(out)

    # -- one time step -----------------------------------------------------
    def step(self):
        """One time step, in the order of Section 4.7 with the cut between time
        steps placed after the streaming of Step 1 (so marking and solute
        transport use the moments of the populations the step starts from):

          1. moments (Eq. 9) and liquid/gas marking against the lagged
             half-maximum threshold (Section 4.5);
          2. concentration amendment at nodes whose marking changed (Step 2);
          3. pseudo-potentials, forces and velocities (Eqs. 11-19);
          4. homogeneous reaction sources (Eqs. 5a, 5c, 27, 28);
          5. fluid collision and streaming with halfway bounce-back (Eq. 6, Step 1);
          6. solute collision and streaming, liquid only, with no-flux and
             reactive links (Eqs. 20-24, 26, 29-31, Step 3);
          7. VOP volume update and status changes (Eqs. 32-35, Step 4);
          8. amendment of flipped nodes (Step 5);
          9. next threshold = half the maximum liquid-component density.
        """
        p = self.p
        t = self.t
        typ = self.type
        ny, nx, ns = self.ny, self.nx, self.ns
        fluid = self._fluid(typ)
        res = self._reservoir(typ)
        mineral = self._mineral(typ)
        inlet, outlet = typ == INLET, typ == OUTLET

        # 1. moments (Eq. 9)
        rho1, rho2 = self._density(0), self._density(1)
        j1, j2 = self._momentum(0), self._momentum(1)
        if not (np.all(np.isfinite(rho1[fluid])) and np.all(np.isfinite(rho2[fluid]))):
            raise NonFiniteError("non-finite density")
        theta = self.theta
        new_max = self._fluid_max(rho1, fluid)
        r1res, r2res, uxres, uyres = self._reservoir_state(typ, rho1, rho2, j1[0] + j2[0], j1[1] + j2[1], t, theta)
        # marking (Section 4.5): liquid iff rho_1 > theta
        liq_new = fluid & (rho1 > theta)
        res_liq = res & (r1res > theta)
        old_liq = fluid & (typ == LIQUID)

        # 2. concentration amendment at marking changes
        C = np.stack([self._conc(self.g[k]) for k in range(ns)]) if ns else np.zeros((0, ny, nx))
        C_pre = C.copy()
        g = self.g.copy()
        if ns:
            vanish = np.argwhere(old_liq & ~liq_new)
            appear = fluid & ~old_liq & liq_new
            surviving = old_liq & liq_new
            dC = np.zeros_like(C)
            for (y, x) in vanish:
                recv = []
                for a in range(1, 5):
                    q = self.nb_coord(y, x, EX5[a], EY5[a])
                    if q is not None and liq_new[q]:
                        recv.append(q)
                if recv:
                    for q in recv:
                        dC[:, q[0], q[1]] += C[:, y, x] / len(recv)
            base = np.zeros_like(C)
            for (y, x) in np.argwhere(appear):
                src = []
                for a in range(1, 5):
                    q = self.nb_coord(y, x, EX5[a], EY5[a])
                    if q is not None and surviving[q]:
                        src.append(q)
                if src:
                    acc = np.zeros(ns)
                    for q in src:
                        acc = acc + C[:, q[0], q[1]]
                    base[:, y, x] = acc / len(src)
            for k in range(ns):
                J0 = p["J0"][k]
                for a in range(5):
                    ja = j5(a, J0)
                    g[k, a] = np.where(appear, ja * (base[k] + dC[k]),
                                       np.where(surviving, g[k, a] + ja * dC[k], g[k, a]))
            C = np.stack([self._conc(g[k]) for k in range(ns)])

        # 3. forces and velocities
        F = self._forces(typ, rho1, rho2, r1res, r2res)
        with np.errstate(invalid="ignore", divide="ignore"):
            safe1 = np.where(fluid, rho1, 1.0)
            safe2 = np.where(fluid, rho2, 1.0)
            u1, u2, ur = self._velocities(safe1, safe2, j1, j2, F)

        # 4. homogeneous reactions at liquid nodes (Eqs. 5a, 5c, 27, 28)
        S = np.zeros((ns, ny, nx))
        S1 = np.zeros((ny, nx))
        S2 = np.zeros((ny, nx))
        iA, iB, iE, iF = p["idx_A"], p["idx_B"], p["idx_E"], p["idx_F"]
        zero = np.zeros((ny, nx))
        if ns:
            CB = C[iB] if iB >= 0 else zero
            CE = C[iE] if iE >= 0 else zero
            if iA >= 0:
                CA = C[iA]
            elif iA == IDX_DERIVED:
                tot = zero.copy()
                for k in range(ns):
                    tot = tot + C[k]
                CA = np.maximum(0.0, p["c_total_per_rho1"] * rho1 - tot)
            else:
                CA = zero
            CC = rho2 * p["inv_M_C"]
            # Section 2: A decomposes in the bulk and, faster by a factor, at the
            # surface of D(s): liquid nodes sharing an axis link with a D(s) node
            fac = float(p.get("r1_surface_factor", 1.0)) or 1.0
            touch_d = np.zeros((ny, nx), dtype=bool)
            for b in range(1, 5):
                touch_d |= self.nb(typ, EX5[b], EY5[b], WALL) == SOLID_D
            k1 = np.where(touch_d, p["k1"] * fac, p["k1"])
            R1 = k1 * (CA - p["inv_Keq"] * CB * np.sqrt(np.maximum(CC, 0.0)))
            R3 = p["k3"] * CB * CE
            R1 = np.where(liq_new, R1, 0.0)
            R3 = np.where(liq_new, R3, 0.0)
            if iA >= 0:
                S[iA] = S[iA] - R1
            if iB >= 0:
                S[iB] = S[iB] + R1 - R3
            if iE >= 0:
                S[iE] = S[iE] - R3
            if iF >= 0:
                S[iF] = S[iF] + R3
            S1 = -p["gas_yield"] * R1
            S2 = p["gas_yield"] * R1

        # 5. fluid collision (Eq. 6 with Eq. 8 at u_eq) and streaming
        rhos = (rho1, rho2)
        us = (u1, u2)
        Ss = (S1, S2)
        fnew = self.f.copy()
        src_typ = {}
        for a in range(9):
            src_typ[a] = self.nb(typ, -EX9[a], -EY9[a], WALL)
        for s_ in range(2):
            tau = p["tau"][s_]
            fstar = np.empty_like(self.f[s_])
            for a in range(9):
                fe = feq9(a, rhos[s_], us[s_][0], us[s_][1])
                fstar[a] = self.f[s_, a] - (self.f[s_, a] - fe) / tau + W9[a] * Ss[s_]
            rres = (r1res, r2res)[s_]
            for a in range(9):
                st = src_typ[a]
                from_fluid = self._fluid(st)
                from_res = self._reservoir(st)
                pulled = self.nb(fstar[a], -EX9[a], -EY9[a], 0.0)
                fres = feq9(a, rres, uxres, uyres)
                pulled_res = self.nb(fres, -EX9[a], -EY9[a], 0.0)
                val = np.where(from_fluid, pulled, np.where(from_res, pulled_res, fstar[OPP9[a]]))
                fnew[s_, a] = np.where(fluid, val, self.f[s_, a])

        # 6. solute collision (Eqs. 20-22, u = u_r) and streaming, liquid nodes only
        gnew = np.zeros_like(self.g)
        qB = np.zeros((5, ny, nx))   # link flux of B from node x toward mineral x + e_d
        qF = np.zeros((5, ny, nx))
        if ns:
            gstar = np.zeros_like(g)
            for k in range(ns):
                J0, tg = p["J0"][k], p["tau_g"][k]
                for a in range(5):
                    ge = C[k] * (j5(a, J0) + 0.5 * (EX5[a] * ur[0] + EY5[a] * ur[1]))
                    gstar[k, a] = g[k, a] - (g[k, a] - ge) / tg + j5(a, J0) * S[k]
            # reservoir equilibrium pushed into liquid neighbours
            Cres = np.zeros((ns, ny, nx))
            for k in range(ns):
                cin = p["conc_in"][k]
                # outlet: concentration of the node upstream at the start of
                # the step when it is liquid, else 0
                cl = np.where(liq_new, C_pre[k], 0.0)
                (_, _), (odx, ody) = self._axes()
                Cres[k] = np.where(inlet, cin, np.where(outlet, self.nb(cl, odx, ody, 0.0), 0.0))
            k2, k4, Csat = p["k2"], p["k4"], p["C_F_sat"]
            for a in range(5):
                st = src_typ[a]
                src_liq = self.nb(liq_new, -EX5[a], -EY5[a], False)
                src_resl = self.nb(res_liq, -EX5[a], -EY5[a], False)
                d = OPP5[a]   # direction from x toward the source node
                for k in range(ns):
                    if a == 0:
                        gnew[k, 0] = np.where(liq_new, gstar[k, 0], 0.0)
                        continue
                    pulled = self.nb(gstar[k, a], -EX5[a], -EY5[a], 0.0)
                    gres = geq5(a, Cres[k], p["J0"][k], uxres, uyres)
                    pulled_res = self.nb(gres, -EX5[a], -EY5[a], 0.0)
                    out = gstar[k, d]
                    val = np.where(src_liq, pulled, np.where(src_resl, pulled_res, out))
                    gnew[k, a] = np.where(liq_new, val, 0.0)
            # reactive links (Eqs. 29-31): x liquid, source node a mineral
            for a in range(1, 5):
                st = src_typ[a]
                d = OPP5[a]
                onD = liq_new & (st == SOLID_D)
                onM = liq_new & ((st == SOLID_D) | (st == SOLID_F))
                if iB >= 0 and k2 != 0.0:
                    Jw = (1.0 - p["J0"][iB]) / 4.0
                    kap = k2 / (2.0 * Jw)
                    out = gstar[iB, d]
                    # back = out (1 - kap) / (1 + kap); the flux out - back
                    # written without the cancellation of two near values
                    q = out * (2.0 * kap / (1.0 + kap))
                    back = out - q
                    gnew[iB, a] = np.where(onD, back, gnew[iB, a])
                    qB[d] = np.where(onD, q, 0.0)
                    if iE >= 0:
                        gnew[iE, a] = np.where(onD, gstar[iE, d] + q, gnew[iE, a])
                if iF >= 0 and k4 != 0.0:
                    Jw = (1.0 - p["J0"][iF]) / 4.0
                    kap = k4 / (2.0 * Jw)
                    out = gstar[iF, d]
                    # back = (out (1 - kap) + k4 C_sat) / (1 + kap), flux as above
                    q = out * (2.0 * kap / (1.0 + kap)) - k4 * Csat / (1.0 + kap)
                    back = out - q
                    gnew[iF, a] = np.where(onM, back, gnew[iF, a])
                    qF[d] = np.where(onM, q, 0.0)

        # 7. VOP volume update (Eqs. 33, 35) and status decisions
        V = self.V.copy()
        newtyp = typ.copy()
        newtyp[fluid] = np.where(liq_new[fluid], LIQUID, GAS)
        dissolve = []
        choice = {}
        touch = np.zeros((ny, nx), dtype=bool)
        for b in range(1, 5):
            touch |= self.nb(liq_new, EX5[b], EY5[b], False)
        for (y, x) in np.argwhere(mineral & touch):
            sB = 0.0
            sF = 0.0
            nliq = []
            for b in range(1, 5):          # gather in E, N, W, S order
                q = self.nb_coord(y, x, EX5[b], EY5[b])
                if q is None or not liq_new[q]:
                    continue
                nliq.append(q)
                link = OPP5[b]           # direction from the neighbour toward (y, x)
                sB = sB + qB[link][q]
                sF = sF + qF[link][q]
            if not nliq:
                continue
            if typ[y, x] == SOLID_D:
                V[0, y, x] = V[0, y, x] - p["Vbar_D"] * sB
            V[1, y, x] = V[1, y, x] + p["Vbar_F"] * sF
            if V[0, y, x] < 0.0:
                V[0, y, x] = 0.0
            total = V[0, y, x] + V[1, y, x]
            if total <= 0.0:
                dissolve.append((y, x))
                V[0, y, x] = 0.0
                V[1, y, x] = 0.0
                continue
            newtyp[y, x] = SOLID_D if V[0, y, x] > 0.0 else SOLID_F
            if total >= p["V_split"]:
                excess = total - 1.0
                V[1, y, x] = V[1, y, x] - excess
                r = splitmix64(overflow_key(int(p["seed"]), t, y * nx + x))
                choice[(y, x)] = (tuple(int(v) for v in nliq[r % len(nliq)]), excess)
        # apply status changes: dissolved nodes become liquid; chosen liquid
        # neighbours become F(s) holding the excess of every mineral that chose
        # them (summed in E, N, W, S order)
        vanish_mask = np.zeros((ny, nx), dtype=bool)
        new_mask = np.zeros((ny, nx), dtype=bool)
        for (y, x) in dissolve:
            newtyp[y, x] = LIQUID
            new_mask[y, x] = True
        for tgt in sorted({c[0] for c in choice.values()}):
            y, x = tgt
            acc = 0.0
            for b in range(1, 5):
                q = self.nb_coord(y, x, EX5[b], EY5[b])
                if q is None:
                    continue
                c = choice.get((int(q[0]), int(q[1])))
                if c is not None and c[0] == tgt:
                    acc = acc + c[1]
            newtyp[y, x] = SOLID_F
            vanish_mask[y, x] = True
            V[0, y, x] = 0.0
            V[1, y, x] = acc

        # 8. amendment of flipped nodes (Step 5)
        surviving = fluid & ~vanish_mask
        surv_liq = surviving & liq_new
        rn1 = fnew[0, 0].copy()
        rn2 = fnew[1, 0].copy()
        for a in range(1, 9):
            rn1 = rn1 + fnew[0, a]
            rn2 = rn2 + fnew[1, a]
        Cn = np.stack([self._conc(gnew[k]) for k in range(ns)]) if ns else np.zeros((0, ny, nx))
        f_out = fnew.copy()
        g_out = gnew.copy()
        for (y, x) in np.argwhere(new_mask):
            sr = [0.0, 0.0]
            nf = 0
            sc = np.zeros(ns)
            nl = 0
            for b in range(1, 5):
                q = self.nb_coord(y, x, EX5[b], EY5[b])
                if q is None:
                    continue
                if surviving[q]:
                    sr[0] = sr[0] + rn1[q]
                    sr[1] = sr[1] + rn2[q]
                    nf += 1
                if surv_liq[q]:
                    sc = sc + Cn[:, q[0], q[1]]
                    nl += 1
            r_new = (sr[0] / nf, sr[1] / nf) if nf else tuple(p["rho_ref"])
            c_new = sc / nl if nl else np.zeros(ns)
            for a in range(9):
                f_out[0, a, y, x] = feq9(a, r_new[0], 0.0, 0.0)
                f_out[1, a, y, x] = feq9(a, r_new[1], 0.0, 0.0)
            for k in range(ns):
                for a in range(5):
                    g_out[k, a, y, x] = j5(a, p["J0"][k]) * c_new[k]
        # receivers gather the mass of vanishing neighbours (E, N, W, S order)
        near = np.zeros((ny, nx), dtype=bool)
        for b in range(1, 5):
            near |= self.nb(vanish_mask, EX5[b], EY5[b], False)
        for (y, x) in np.argwhere(surviving & near):
            add = [0.0, 0.0]
            addc = np.zeros(ns)
            hit = False
            for b in range(1, 5):
                v = self.nb_coord(y, x, EX5[b], EY5[b])
                if v is None or not vanish_mask[v]:
                    continue
                nf = 0
                nl = 0
                for c in range(1, 5):
                    w = self.nb_coord(v[0], v[1], EX5[c], EY5[c])
                    if w is None:
                        continue
                    nf += int(surviving[w])
                    nl += int(surv_liq[w])
                add[0] = add[0] + rn1[v] / nf
                add[1] = add[1] + rn2[v] / nf
                hit = True
                if surv_liq[y, x] and nl:
                    addc = addc + Cn[:, v[0], v[1]] / nl
            if not hit:
                continue
            for a in range(9):
                f_out[0, a, y, x] = f_out[0, a, y, x] + W9[a] * add[0]
                f_out[1, a, y, x] = f_out[1, a, y, x] + W9[a] * add[1]
            if surv_liq[y, x]:
                for k in range(ns):
                    for a in range(5):
                        g_out[k, a, y, x] = g_out[k, a, y, x] + j5(a, p["J0"][k]) * addc[k]
        for (y, x) in np.argwhere(vanish_mask):
            g_out[:, :, y, x] = 0.0

        # 9. commit
        self.f = f_out
        self.g = g_out
        self.V = V
        self.type = newtyp
        self.theta = 0.5 * new_max
        self.t = t + 1
        self.last_qB = qB
        self.last_qF = qF

    def run(self, n):
        for _ in range(n):
            self.step()
        return self
