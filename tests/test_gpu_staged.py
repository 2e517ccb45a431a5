"""TMA-staged bulk kernels against the plain-load kernel and the oracle.

The staged kernels (two stages and one stage) run the plain kernel's per-node arithmetic on populations
that the TMA unit copied into shared memory, so every field must be
bit-identical between the two, for both tile shapes, every species count, the
16-bit solute storages, periodic wrap (ring nodes across the edge come from
global memory), ragged edges (zero-filled box elements outside the lattice),
lattices narrower than the box, and batches.  The FP32 path (either kernel)
also matches the FP64 oracle within FP32 tolerance after 100 steps.
"""
import numpy as np
import pytest

from oracle import lbm
from paper_1410_3464_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho1", "rho2", "ux", "uy", "conc", "type", "vol", "budget")
STAGED = (1, 2)          # TMA-staged with two stages; with one stage


@pytest.fixture(scope="module")
def pslbm():
    from paper_1410_3464_gb300 import build, pslbm as m
    build.build()
    return m


def run(pslbm, sc, steps, precision, staging, shape=(16, 16)):
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as s:
        s.set_tile_shape(*shape)
        s.set_staging(staging)
        s.step(steps)
        used, avail = s.staging()
        assert used == staging and avail
        return s.read()


def assert_same(a, b, what):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k], equal_nan=True), f"{what}: {k}"


def periodic_bubble(nx, ny, seed=3):
    """Liquid with a gas bubble, periodic in x and y, species A -> B; the
    bubble sits across the corner so that the wrap carries the interface."""
    sc = inputs.bubble_grain(nx=nx, ny=ny, grain=(nx // 2, ny // 2, min(nx, ny) // 6),
                             bubble=(2, 2, min(nx, ny) // 5))
    p = dict(sc["params"])
    p.update(periodic_x=1, periodic_y=1)
    mask = sc["mask"].copy()
    mask[0, :] = lbm.LIQUID
    mask[-1, :] = lbm.LIQUID
    y, x = np.mgrid[0:ny, 0:nx]
    d2 = np.minimum(x, nx - x) ** 2 + np.minimum(y, ny - y) ** 2
    gas = d2 <= (min(nx, ny) // 5) ** 2
    mask[gas] = lbm.GAS
    mask[~gas & (mask == lbm.GAS)] = lbm.LIQUID
    rl, rg = inputs.COEX_ORIGINAL_07
    rho1 = np.where(mask == lbm.GAS, rg, rl).astype(np.float64)
    rho2 = np.where(mask == lbm.GAS, 0.002, 2e-5)
    return inputs.Scene(mask=mask, rho1=rho1, rho2=rho2, conc=sc["conc"], vol=None, params=p)


@pytest.mark.parametrize("shape", [(16, 16), (32, 8)])
@pytest.mark.parametrize("nx,ny", [(96, 64), (100, 50), (40, 24)])
def test_staged_equals_plain_porous(pslbm, shape, nx, ny):
    sc = inputs.porous_discs(nx=nx, ny=ny, seed=61, rmin=3, rmax=8)
    a = run(pslbm, sc, 40, pslbm.FP32, 0, shape)
    for staging in STAGED:
        b = run(pslbm, sc, 40, pslbm.FP32, staging, shape)
        assert_same(a, b, f"porous {nx}x{ny} {shape} staging {staging}")


@pytest.mark.parametrize("shape", [(16, 16), (32, 8)])
@pytest.mark.parametrize("nx,ny", [(128, 64), (36, 20), (8, 40)])
def test_staged_equals_plain_periodic_wrap(pslbm, shape, nx, ny):
    sc = periodic_bubble(nx, ny)
    a = run(pslbm, sc, 60, pslbm.FP32, 0, shape)
    if nx >= 64:                     # small bubbles dissolve within the run
        assert (a["type"] == lbm.GAS).any()
    for staging in STAGED:
        b = run(pslbm, sc, 60, pslbm.FP32, staging, shape)
        assert_same(a, b, f"periodic {nx}x{ny} {shape} staging {staging}")


@pytest.mark.parametrize("shape", [(16, 16), (32, 8)])
def test_staged_equals_plain_beaker(pslbm, shape):
    """Outlet along y, four species, R1 surface enhancement, partial tiles
    (100 = 6 x 16 + 4)."""
    sc = inputs.beaker()
    a = run(pslbm, sc, 60, pslbm.FP32, 0, shape)
    for staging in STAGED:
        b = run(pslbm, sc, 60, pslbm.FP32, staging, shape)
        assert_same(a, b, f"beaker {shape} staging {staging}")


@pytest.mark.parametrize("ns", [0, 1, 2, 4])
def test_staged_equals_plain_species_counts(pslbm, ns):
    sc = inputs.porous_discs(nx=64, ny=48, seed=71)
    p = dict(sc["params"])
    conc = sc["conc"]
    if ns < 3:
        p.update(n_species=ns, idx_A=lbm.IDX_DERIVED if ns else lbm.IDX_ABSENT, idx_B=0 if ns >= 1 else -1,
                 idx_E=1 if ns >= 2 else -1, idx_F=-1)
        conc = conc[:ns] if ns else None
    elif ns == 4:
        p.update(n_species=4, idx_A=3)
        conc = np.concatenate([conc, np.full((1,) + conc.shape[1:], 0.5)])
    sc = inputs.Scene(mask=sc["mask"], rho1=sc["rho1"], rho2=sc["rho2"], conc=conc, vol=None, params=p)
    a = run(pslbm, sc, 30, pslbm.FP32, 0)
    for staging in STAGED:
        b = run(pslbm, sc, 30, pslbm.FP32, staging)
        assert_same(a, b, f"ns={ns} staging {staging}")


@pytest.mark.parametrize("prec", ["FP32_SOLUTE_F16", "FP32_SOLUTE_BF16"])
@pytest.mark.parametrize("shape", [(16, 16), (32, 8)])
def test_staged_equals_plain_16bit_solutes(pslbm, prec, shape):
    sc = inputs.porous_discs(nx=120, ny=72, seed=81)
    a = run(pslbm, sc, 30, getattr(pslbm, prec), 0, shape)
    for staging in STAGED:
        b = run(pslbm, sc, 30, getattr(pslbm, prec), staging, shape)
        assert_same(a, b, f"{prec} staging {staging}")


def test_staged_batch_equals_alone(pslbm):
    scs = [inputs.porous_discs(nx=64 + 32 * i, ny=48 + 16 * i, seed=90 + i) for i in range(3)]
    refs = [run(pslbm, sc, 25, pslbm.FP32, 0) for sc in scs]
    sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                             precision=pslbm.FP32) for sc in scs]
    b = pslbm.Batch(sims)
    b.set_staging(2)
    b.step(25)
    b.sync()
    assert b.staging() == (2, True)
    b.close()
    for s, ref in zip(sims, refs):
        assert_same(s.read(), ref, "batch")
        s.close()


def test_staging_availability(pslbm):
    ok = inputs.porous_discs(nx=64, ny=48, seed=5)
    odd = inputs.porous_discs(nx=66, ny=48, seed=5)          # rows of 264 B: not a multiple of 16
    with pslbm.Simulation(ok["mask"], ok["params"], ok["rho1"], ok["rho2"], ok["conc"], precision=pslbm.FP32) as s:
        assert s.staging()[1]
    with pslbm.Simulation(odd["mask"], odd["params"], odd["rho1"], odd["rho2"], odd["conc"],
                          precision=pslbm.FP32) as s:
        assert not s.staging()[1]
        with pytest.raises(pslbm.PslbmError):
            s.set_staging(1)
        s.set_staging(0)
    with pslbm.Simulation(ok["mask"], ok["params"], ok["rho1"], ok["rho2"], ok["conc"], precision=pslbm.FP64) as s:
        assert s.staging() == (False, False)
    # 16-bit solutes need rows of 8 nodes
    p = inputs.porous_discs(nx=68, ny=48, seed=5)
    with pslbm.Simulation(p["mask"], p["params"], p["rho1"], p["rho2"], p["conc"],
                          precision=pslbm.FP32_SOLUTE_F16) as s:
        assert not s.staging()[1]


def test_autotune_over_variants_agrees(pslbm):
    """An autotuned run (ten variants, each timed twice, on its first 80
    steps) equals a run pinned to the plain 16x16 kernel."""
    sc = inputs.porous_discs(nx=128, ny=96, seed=7)
    ref = run(pslbm, sc, 100, pslbm.FP32, 0)
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP32) as s:
        s.step(100)
        assert s.tile_shape()[2]
        got = s.read()
    assert_same(got, ref, "autotuned")


@pytest.mark.parametrize("staging", [0, 1, 2])
def test_fp32_matches_oracle_100_steps(pslbm, staging):
    """FP32 compute with shifted FP32 storage vs the FP64 oracle on the plain
    scene (128x64, 100 steps): 1e-4 relative per field, node types equal."""
    sc = inputs.bubble_grain()
    got = run(pslbm, sc, 100, pslbm.FP32, staging)
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    L.run(100)
    ref = L.fields()
    np.testing.assert_array_equal(got["type"], ref["type"])
    fluid, liquid = ref["type"] <= 1, ref["type"] == 0
    for name in ("rho1", "rho2", "ux", "uy"):
        a, b = got[name][fluid], ref[name][fluid]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max(), name
    for k in range(ref["conc"].shape[0]):
        a, b = got["conc"][k][liquid], ref["conc"][k][liquid]
        assert np.abs(a - b).max() <= 1e-4 * max(np.abs(b).max(), 1e-30), k
