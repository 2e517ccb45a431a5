"""GPU FP64 path vs the CPU oracle, element by element, through the C ABI.

Tolerance: 1e-12 relative per field (max |gpu - oracle| / max |oracle| over the
nodes where the field is defined) after the stated number of steps; node types
bit-exact.  Both sides evaluate the same formulas in FP64 and differ only in
rounding order (fused multiply-add, summation grouping), ~1e-16 per operation.
"""
import numpy as np
import pytest

from oracle import lbm
from paper_1410_3464_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def pslbm():
    from paper_1410_3464_gb300 import build, pslbm as m
    build.build()
    return m


def rel(a, b, where=None):
    if where is not None:
        a, b = a[where], b[where]
    den = np.abs(b).max() if b.size else 0.0
    if den == 0.0:
        return float(np.abs(a).max()) if a.size else 0.0
    return float(np.abs(a - b).max() / den)


def run_both(pslbm, sc, steps, precision=0):
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as sim:
        sim.step(steps)
        got = sim.read()
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    L.run(steps)
    ref = L.fields()
    ref["budget"] = L.budget()
    return got, ref, L


def compare(got, ref, tol=TOL, what=""):
    np.testing.assert_array_equal(got["type"], ref["type"], err_msg=f"{what} node types")
    fluid = ref["type"] <= 1
    liquid = ref["type"] == 0
    for name in ("rho1", "rho2", "ux", "uy"):
        e = rel(got[name], ref[name], fluid)
        assert e <= tol, f"{what} {name}: {e:.3e}"
    for k in range(ref["conc"].shape[0]):
        e = rel(got["conc"][k], ref["conc"][k], liquid)
        assert e <= tol, f"{what} conc[{k}]: {e:.3e}"
    e = rel(got["vol_d"], ref["vol_d"])
    assert e <= tol, f"{what} V_D: {e:.3e}"
    e = rel(got["vol_f"], ref["vol_f"])
    assert e <= tol, f"{what} V_F: {e:.3e}"
    b = got["budget"]
    rb = ref["budget"]
    np.testing.assert_allclose(b[:-1], rb, rtol=1e-11, atol=1e-300, err_msg=f"{what} budget")


def test_bubble_grain_128x64_100_steps(pslbm):
    """The plain-method scene (128x64, bubble + grain, 2 species, FP64) after 100 steps."""
    sc = inputs.bubble_grain()
    got, ref, L = run_both(pslbm, sc, 100)
    compare(got, ref, what="bubble_grain")
    assert got["budget"][-1] == 100


def test_marking_changes_happen(pslbm):
    """The bubble scene relaxes its sharp interface: nodes change between
    liquid and gas in the first steps, so the Step-2 amendment is exercised."""
    sc = inputs.bubble_grain(nx=64, ny=40, grain=(44, 20, 6), bubble=(16, 20, 7))
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], None)
    changed = 0
    for _ in range(30):
        t0 = L.type.copy()
        L.step()
        changed += int(((t0 <= 1) & (L.type <= 1) & (t0 != L.type)).sum())
    assert changed > 0
    got, ref, _ = run_both(pslbm, sc, 30)
    compare(got, ref, what="marking")


def test_dissolution_flips(pslbm):
    """Grain whose surface nodes hold little volume: several nodes dissolve and
    are refilled (Steps 4-5)."""
    sc = inputs.bubble_grain(nx=64, ny=40, grain=(32, 20, 7), bubble=(10, 20, 4))
    p = dict(sc["params"])
    p.update(k2=0.05, Vbar_D=1.0)
    sc["params"] = p
    conc = sc["conc"].copy()
    conc[1][sc["mask"] == 0] = 0.8            # B present from the start
    sc["conc"] = conc
    vol = np.zeros((2,) + sc["mask"].shape)
    vol[0][sc["mask"] == 2] = 1.0
    rng = np.random.default_rng(11)
    surf = (sc["mask"] == 2) & ((np.roll(sc["mask"], 1, 0) == 0) | (np.roll(sc["mask"], -1, 0) == 0) |
                                 (np.roll(sc["mask"], 1, 1) == 0) | (np.roll(sc["mask"], -1, 1) == 0))
    vol[0][surf] = rng.uniform(0.005, 0.4, surf.sum())
    sc["vol"] = vol
    got, ref, L = run_both(pslbm, sc, 60)
    assert (ref["type"] == 2).sum() < (sc["mask"] == 2).sum(), "no node dissolved"
    compare(got, ref, what="dissolution")


def test_precipitation_overflow(pslbm):
    """F(s) nodes near the overflow threshold with F in solution: overflow into
    liquid neighbours picked by SplitMix64, and redistribution of the vanished
    liquid's mass (Steps 4-5)."""
    nx, ny = 48, 32
    p = inputs.base_params(nx, ny)
    p.update(G11=0.0, G12=0.0, G21=0.0, periodic_x=1, periodic_y=1, rho_ref=(1.0, 0.01),
             n_species=2, idx_B=0, idx_F=1, J0=(1 / 3, 1 / 3, 0, 0), tau_g=(0.8, 0.8, 1, 1),
             k4=0.02, k2=0.02, Vbar_F=0.2, V_split=2.0, seed=1234)
    mask = np.zeros((ny, nx), np.uint8)
    rng = np.random.default_rng(5)
    pts = rng.integers(0, [ny, nx], size=(25, 2))
    vol = np.zeros((2, ny, nx))
    for y, x in pts:
        mask[y, x] = 3
        vol[1, y, x] = rng.uniform(1.975, 1.999)
    mask[10:14, 20:24] = 2
    vol[0][mask == 2] = 1.0
    rho1 = np.where(mask <= 1, 1.0 + 0.01 * rng.standard_normal((ny, nx)), 0.0)
    rho2 = np.where(mask <= 1, 0.01, 0.0)
    conc = np.zeros((2, ny, nx))
    conc[0][mask == 0] = 0.5
    conc[1][mask == 0] = rng.uniform(0.5, 1.0, (mask == 0).sum())
    sc = dict(mask=mask, rho1=rho1, rho2=rho2, conc=conc, vol=vol, params=p)
    got, ref, L = run_both(pslbm, sc, 40)
    assert (ref["type"] == 3).sum() > 25, "no overflow happened"
    compare(got, ref, what="overflow")


def test_porous_inlet_outlet_small(pslbm):
    """Porous-medium workload at 160x96 with inlet slugs (liquid 20 / gas 10
    steps), outlet, 3 species, derived A, R1-R4, for 45 steps."""
    sc = inputs.porous_discs(nx=160, ny=96, seed=7, slug=(20, 10))
    got, ref, _ = run_both(pslbm, sc, 45)
    compare(got, ref, what="porous")


@pytest.mark.parametrize("nx,ny,px,py", [(37, 13, 1, 1), (5, 3, 1, 1), (70, 9, 0, 1), (33, 17, 0, 0)])
def test_ragged_and_tiny_lattices(pslbm, nx, ny, px, py):
    """Sizes that are not multiples of the 32x8 tile (and smaller than it),
    periodic or walled."""
    rng = np.random.default_rng(nx * 100 + ny)
    p = inputs.base_params(nx, ny)
    p.update(periodic_x=px, periodic_y=py, rho_ref=(0.3, 1e-3), n_species=2, idx_A=0, idx_B=1,
             J0=(1 / 3, 0.2, 0, 0), tau_g=(0.8, 1.1, 1, 1), k1=0.01, k2=0.02, gas_yield=0.5, inv_M_C=1.0)
    mask = np.where(rng.random((ny, nx)) < 0.12, 2, 0).astype(np.uint8)
    rl, rg = inputs.COEX_ORIGINAL_07
    rho1 = np.where(mask == 0, rl * (1 + 0.01 * rng.standard_normal((ny, nx))), 0.0)
    gas = rng.random((ny, nx)) < 0.1
    mask[(mask == 0) & gas] = 1
    rho1[mask == 1] = rg
    rho2 = np.where(mask == 1, 0.002, 2e-5) * (mask <= 1)
    conc = np.stack([np.where(mask == 0, 1.0, 0.0), np.where(mask == 0, 0.2, 0.0)])
    sc = dict(mask=mask, rho1=rho1, rho2=rho2, conc=conc, vol=None, params=p)
    got, ref, _ = run_both(pslbm, sc, 25)
    compare(got, ref, what=f"{nx}x{ny}")


@pytest.mark.parametrize("ns", [0, 1, 4])
def test_species_counts(pslbm, ns):
    """Kernel instantiations for 0, 1 and 4 transported species."""
    sc = inputs.bubble_grain(nx=48, ny=24, grain=(30, 12, 4), bubble=(10, 12, 4))
    p = dict(sc["params"])
    p.update(n_species=ns, idx_A=0 if ns else -1, idx_B=1 if ns > 1 else -1, idx_E=2 if ns > 2 else -1,
             idx_F=3 if ns > 3 else -1, J0=(1 / 3, 0.1, 0.5, 0.25), tau_g=(0.8, 0.9, 1.2, 0.7),
             k1=2e-3, k3=0.05, k4=0.01 if ns > 3 else 0.0, k2=0.02 if ns > 1 else 0.0)
    sc["params"] = p
    conc = np.zeros((ns,) + sc["mask"].shape)
    for k in range(ns):
        conc[k][sc["mask"] == 0] = 1.0 / (k + 1)
    sc["conc"] = conc if ns else None
    got, ref, _ = run_both(pslbm, sc, 30)
    compare(got, ref, what=f"ns={ns}")


def test_adhesion_and_body_force(pslbm):
    """Non-zero fluid-solid interaction (Eq. 16) and a body force."""
    sc = inputs.bubble_grain(nx=64, ny=32, grain=(40, 16, 6), bubble=(14, 16, 5))
    p = dict(sc["params"])
    p.update(w_adh=(-0.02, 0.01), body_force=(1e-6, -2e-6))
    sc["params"] = p
    got, ref, _ = run_both(pslbm, sc, 40)
    compare(got, ref, what="adhesion")


def test_porous_full_size_1024x512(pslbm):
    """The porous-medium workload at its full 1024x512 size on the FP64 path,
    for 6 steps (the oracle's cost bounds the step count; the GPU path is the
    same at every step)."""
    sc = inputs.porous_discs()
    got, ref, _ = run_both(pslbm, sc, 6)
    compare(got, ref, what="porous 1024x512")


@pytest.mark.parametrize("shape", [(32, 8), (16, 16)])
def test_porous_full_size_benchmark_configuration(pslbm, shape):
    """The benchmark's own launch configuration -- FP32 with phase-shifted
    storage, the TMA-staged bulk kernel with two stages, the single-simulation
    parameter block -- on the full 1024x512 workload against the FP64 oracle
    after 6 steps: FP32 tolerance 1e-5 relative (about a hundred FP32 roundings
    of the largest values), node types bit-exact."""
    sc = inputs.porous_discs()
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP32) as sim:
        sim.set_tile_shape(*shape)
        sim.set_staging(1)
        sim.step(6)
        assert sim.staging() == (1, True)
        got = sim.read()
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    L.run(6)
    ref = L.fields()
    np.testing.assert_array_equal(got["type"], ref["type"])
    fluid, liquid = ref["type"] <= 1, ref["type"] == 0
    for name in ("rho1", "rho2", "ux", "uy"):
        e = rel(got[name], ref[name], fluid)
        assert e <= 1e-5, f"{name}: {e:.3e}"
    for k in range(ref["conc"].shape[0]):
        e = rel(got["conc"][k], ref["conc"][k], liquid)
        assert e <= 1e-5, f"conc[{k}]: {e:.3e}"


def test_r1_surface_enhancement(pslbm):
    """Section 2: R1 runs 1000 times faster at liquid nodes sharing a link with
    D(s); the plain scene with the enhancement on, 100 steps."""
    sc = inputs.bubble_grain()
    p = dict(sc["params"])
    p.update(k1=1e-5, r1_surface_factor=1000.0)
    sc["params"] = p
    got, ref, _ = run_both(pslbm, sc, 100)
    compare(got, ref, what="R1 surface enhancement")


@pytest.mark.parametrize("k1,surface", [(2e-3, 1.0), (2e-5, 100.0)])
def test_reversible_r1(pslbm, k1, surface):
    """Eq. 5a with the back reaction: R1 = k1 (C_A - C_B sqrt(C_C) / K_eq), with
    C_C = rho_2 / M_C taken from the gas component, on the plain scene (the
    bubble supplies C(g); R1 also turns liquid mass into gas, Eq. 27), without
    and with the Section 2 surface enhancement (100 times faster at the grain:
    2e-3 there); 100 steps, FP64 path against the oracle at 1e-12.  B starts at 0.3, so the back reaction is active from the
    first step, and at the bubble, where C_C is large, R1 runs backwards."""
    sc = inputs.bubble_grain()
    p = dict(sc["params"])
    p.update(k1=k1, inv_Keq=40.0, inv_M_C=1.0 / (0.1 * 0.35813), gas_yield=0.05 * 0.35813,
             r1_surface_factor=surface, k2=0.0)
    sc["params"] = p
    sc["conc"] = sc["conc"].copy()
    sc["conc"][1] = 0.3
    got, ref, L = run_both(pslbm, sc, 100)
    compare(got, ref, what=f"reversible R1 (surface x{surface:g})")
    # the back reaction is not negligible here: somewhere in the liquid the
    # oracle's back rate is at least half the forward rate
    liquid = ref["type"] == 0
    CC = np.maximum(ref["rho2"] * p["inv_M_C"], 0.0)
    back = ref["conc"][1] * np.sqrt(CC) * p["inv_Keq"]
    assert np.max(back[liquid] / ref["conc"][0][liquid]) > 0.5


def test_beaker_scene_free_top_outlet(pslbm):
    """The paper's beaker (Section 5): D(s) cylinder r = 15 at (50, 50) in
    100x160, walls left, right and bottom, a free outlet on the top row (outlet
    along y), rescaled C-S EOS at 0.65 T_c, four transported species, R1 with the
    surface enhancement, R2-R4; 120 steps."""
    sc = inputs.beaker()
    got, ref, _ = run_both(pslbm, sc, 120)
    compare(got, ref, what="beaker")


@pytest.mark.parametrize("w", [-0.2, 0.0])
def test_droplet_contact_line(pslbm, w):
    """A droplet on a flat wall (App. A2 scene, 48x32, r = 10, rescaled C-S EOS):
    the mirror-image wall in the cohesion sums and the Eq. 16 adhesion at the
    contact line, 150 steps on the FP64 path against the oracle."""
    sc = inputs.droplet(nx=48, ny=32, radius=10.0, w=w)
    got, ref, _ = run_both(pslbm, sc, 150)
    compare(got, ref, what=f"droplet w={w}")


def test_beaker_runs_with_all_reactions(pslbm):
    """The beaker with R1 (surface enhanced) to R4 on, 5000 steps on the FP64
    and FP32 paths: no error, and the dissolving D(s) surface is passivated by
    a shell of precipitated F(s) (R2 acts only on D(s) links; a D(s) node whose
    V_D is gone but holds some V_F turns into F(s) rather than liquid), as in
    the oracle, which shows the same shell (84 F(s) nodes, V_D = 625) from
    2,500 steps on."""
    for prec in (pslbm.FP64, pslbm.FP32):
        sc = inputs.beaker()
        with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                              precision=prec) as s:
            s.step(5000)
            f = s.read()
        nF = int((f["type"] == 3).sum())
        assert nF > 40, nF
        assert 600.0 < f["vol"][0].sum() < 700.0
        assert np.isfinite(f["rho1"]).all()


def test_plain_scene_full_length_2000_steps(pslbm):
    """The plain-method scene for its full 2000 steps on the FP64 path.  The
    two sides differ only in rounding order (about 1e-16 per operation); the
    flow does not amplify perturbations measurably (an FP64 run started from a
    1e-7 perturbation stays within 1e-7), so after 2000 steps the difference
    stays within 1e-10 relative per field."""
    sc = inputs.bubble_grain()
    got, ref, L = run_both(pslbm, sc, 2000)
    compare(got, ref, tol=1e-10, what="bubble_grain 2000 steps")
    assert got["budget"][-1] == 2000


def test_batch_equals_alone(pslbm):
    """Two simulations of different sizes stepped as one batch give bit-identical
    fields to the same simulations stepped alone."""
    a = inputs.porous_discs(nx=72, ny=48, seed=5, slug=(8, 4))
    b = inputs.porous_discs(nx=96, ny=40, seed=3, slug=(10, 5))
    alone = []
    for sc in (a, b):
        with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"]) as s:
            s.step(25)
            alone.append(s.read())
    sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
            for sc in (a, b)]
    bt = pslbm.Batch(sims)
    bt.step(25)
    bt.sync()
    bt.close()
    for s, ref in zip(sims, alone):
        got = s.read()
        for k in ("rho1", "rho2", "ux", "uy", "conc", "type", "vol"):
            assert np.array_equal(got[k], ref[k]), k
        s.close()


def test_step_counts_and_graph_replay(pslbm):
    """Steps split over several calls (graph replays of different lengths)
    give the same state as one call."""
    sc = inputs.bubble_grain(nx=64, ny=32, grain=(40, 16, 6), bubble=(14, 16, 5))
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"]) as s1:
        s1.step(71)
        r1 = s1.read()
        assert s1.steps() == 71
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"]) as s2:
        for n in (1, 5, 32, 0, 33):
            s2.step(n)
        r2 = s2.read()
    for k in ("rho1", "ux", "conc", "type", "vol"):
        assert np.array_equal(r1[k], r2[k]), k


def test_tile_shapes_and_autotune_agree(pslbm):
    """The step kernels exist for 16x16 and 32x8 tiles (one node per thread)
    and 16x32 and 32x16 tiles (two nodes per thread); a run pinned to any
    shape and an autotuned run (which times the four twice on its first 32
    steps: rows of 600 bytes leave no staged variant) give bit-identical fields, and
    the autotuned handle reports its choice."""
    sc = inputs.porous_discs(nx=150, ny=90, seed=21, slug=(12, 6))
    res = []
    for shape in ((16, 16), (32, 8), (16, 32), (32, 16), (0, 0)):
        with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"]) as s:
            s.set_tile_shape(*shape)
            s.step(40)
            tx, ty, tuned = s.tile_shape()
            assert tuned
            if shape != (0, 0):
                assert (tx, ty) == shape
            else:
                assert (tx, ty) in ((16, 16), (32, 8), (16, 32), (32, 16))
            res.append(s.read())
    for r in res[1:]:
        for k in ("rho1", "rho2", "ux", "uy", "conc", "type", "vol"):
            assert np.array_equal(r[k], res[0][k]), k
