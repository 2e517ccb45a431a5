"""Bulk kernels with two nodes per thread (tiles 16x32 and 32x16).

A thread of these kernels computes the nodes (tx, ty) and (tx, ty + 256 / TX)
of its tile with the per-node arithmetic of the one-node kernels, so every
field must be bit-identical to the one-node plain kernel: FP64 and the FP32
storages, every species count, periodic wrap, ragged and tiny lattices,
reservoirs along x and y, batches; with plain loads and with the staged D2Q9
box (staging 2; the box has no x halo, so the side ring columns come from
global memory).  The FP64 two-node kernel also matches the oracle at 1e-12,
and the FP32 one on the full 1024x512 workload within FP32 tolerance.
"""
import numpy as np
import pytest

from oracle import lbm
from paper_1410_3464_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho1", "rho2", "ux", "uy", "conc", "type", "vol", "budget")
TWO = ((32, 16), (16, 32))


@pytest.fixture(scope="module")
def pslbm():
    from paper_1410_3464_gb300 import build, pslbm as m
    build.build()
    return m


def run(pslbm, sc, steps, precision, shape, staging=0):
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as s:
        s.set_tile_shape(*shape)
        s.set_staging(staging)
        s.step(steps)
        tx, ty, tuned = s.tile_shape()
        assert (tx, ty) == tuple(shape) and tuned
        return s.read()


def assert_same(a, b, what):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k], equal_nan=True), f"{what}: {k}"


def rel(a, b, where):
    a, b = a[where], b[where]
    den = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max() if a.size else 0.0)


@pytest.mark.parametrize("staging", [0, 2])
@pytest.mark.parametrize("shape", TWO)
@pytest.mark.parametrize("nx,ny", [(96, 64), (100, 50), (40, 24), (20, 12)])
def test_two_nodes_equal_one_node_porous(pslbm, shape, staging, nx, ny):
    """Porous scenes with inlet and outlet columns; 100 x 50 and 20 x 12 leave
    partial tiles in both directions (20 x 12 is smaller than one tile)."""
    sc = inputs.porous_discs(nx=nx, ny=ny, seed=61, rmin=3, rmax=8)
    ref = run(pslbm, sc, 40, pslbm.FP32, (32, 8))
    got = run(pslbm, sc, 40, pslbm.FP32, shape, staging)
    assert_same(got, ref, f"porous {nx}x{ny} {shape} staging {staging}")


@pytest.mark.parametrize("staging", [0, 2])
@pytest.mark.parametrize("shape", TWO)
@pytest.mark.parametrize("nx,ny", [(128, 64), (36, 20), (8, 40)])
def test_two_nodes_equal_one_node_periodic(pslbm, shape, staging, nx, ny):
    """Periodic in x and y with a gas bubble across the corner: ring nodes and
    pushes wrap around both edges, and partial tiles stand for wrapped nodes."""
    from test_gpu_staged import periodic_bubble
    sc = periodic_bubble(nx, ny)
    ref = run(pslbm, sc, 60, pslbm.FP32, (16, 16))
    got = run(pslbm, sc, 60, pslbm.FP32, shape, staging)
    assert_same(got, ref, f"periodic {nx}x{ny} {shape} staging {staging}")


@pytest.mark.parametrize("shape", TWO)
def test_two_nodes_staged_beaker(pslbm, shape):
    """Outlet along y, four species, R1 surface enhancement, partial tiles
    (100 = 6 x 16 + 4): staged two-node kernel equal to the one-node plain one."""
    sc = inputs.beaker()
    ref = run(pslbm, sc, 60, pslbm.FP32, (16, 16))
    got = run(pslbm, sc, 60, pslbm.FP32, shape, 2)
    assert_same(got, ref, f"beaker {shape}")


@pytest.mark.parametrize("shape", TWO)
def test_two_nodes_fp64_matches_oracle_beaker(pslbm, shape):
    """The beaker (outlet along y, four species, R1 surface enhancement,
    partial tiles) in FP64 against the oracle after 120 steps, 1e-12."""
    sc = inputs.beaker()
    got = run(pslbm, sc, 120, pslbm.FP64, shape)
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    L.run(120)
    ref = L.fields()
    np.testing.assert_array_equal(got["type"], ref["type"])
    fluid, liquid = ref["type"] <= 1, ref["type"] == 0
    for name in ("rho1", "rho2", "ux", "uy"):
        assert rel(got[name], ref[name], fluid) <= 1e-12, name
    for k in range(ref["conc"].shape[0]):
        assert rel(got["conc"][k], ref["conc"][k], liquid) <= 1e-12, k
    assert rel(got["vol_d"], ref["vol_d"], np.ones_like(ref["vol_d"], bool)) <= 1e-12


def test_two_nodes_fp64_equals_one_node_marking_changes(pslbm):
    """The plain scene with marking changes and dissolution flips in FP64:
    two-node and one-node kernels bit-identical."""
    sc = inputs.bubble_grain()
    p = dict(sc["params"])
    p.update(k2=5e-2)
    sc = inputs.Scene(**dict(sc, params=p))
    ref = run(pslbm, sc, 300, pslbm.FP64, (16, 16))
    got = run(pslbm, sc, 300, pslbm.FP64, (16, 32))
    assert_same(got, ref, "bubble_grain fp64")


@pytest.mark.parametrize("ns", [0, 1, 2, 4])
def test_two_nodes_species_counts(pslbm, ns):
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
    ref = run(pslbm, sc, 30, pslbm.FP32, (32, 8))
    for staging in (0, 2):
        got = run(pslbm, sc, 30, pslbm.FP32, (32, 16), staging)
        assert_same(got, ref, f"ns={ns} staging {staging}")


@pytest.mark.parametrize("prec", ["FP32_SOLUTE_F16", "FP32_SOLUTE_BF16"])
def test_two_nodes_16bit_solutes(pslbm, prec):
    sc = inputs.porous_discs(nx=120, ny=72, seed=81)
    ref = run(pslbm, sc, 30, getattr(pslbm, prec), (32, 8))
    for staging in (0, 2):
        got = run(pslbm, sc, 30, getattr(pslbm, prec), (32, 16), staging)
        assert_same(got, ref, f"{prec} staging {staging}")


@pytest.mark.parametrize("staging", [0, 2])
def test_two_nodes_batch_equals_alone(pslbm, staging):
    """A batch on 32x16 tiles: members of different sizes, one frozen early by
    its step limit, equal to each member run alone on 32x8 tiles."""
    scs = [inputs.porous_discs(nx=64 + 32 * i, ny=48 + 16 * i, seed=90 + i) for i in range(3)]
    refs = [run(pslbm, sc, 25, pslbm.FP32, (32, 8)) for sc in scs[:2]]
    refs.append(run(pslbm, scs[2], 10, pslbm.FP32, (32, 8)))
    sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                             precision=pslbm.FP32) for sc in scs]
    sims[2].set_step_limit(10)
    b = pslbm.Batch(sims, 32, 16)
    b.set_staging(staging)
    b.step(25)
    b.sync()
    assert b.tile_shape()[:2] == (32, 16) and b.staging() == (staging, True)
    b.close()
    for s, ref in zip(sims, refs):
        assert_same(s.read(), ref, "batch")
        s.close()


@pytest.mark.parametrize("staging", [0, 2])
def test_two_nodes_full_size_benchmark_workload(pslbm, staging):
    """The 1024x512 porous workload in FP32 on 32x16 tiles against the FP64
    oracle after 6 steps: 1e-5 relative, node types bit-exact."""
    sc = inputs.porous_discs()
    got = run(pslbm, sc, 6, pslbm.FP32, (32, 16), staging)
    L = lbm.Lattice(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"])
    L.run(6)
    ref = L.fields()
    np.testing.assert_array_equal(got["type"], ref["type"])
    fluid, liquid = ref["type"] <= 1, ref["type"] == 0
    for name in ("rho1", "rho2", "ux", "uy"):
        assert rel(got[name], ref[name], fluid) <= 1e-5, name
    for k in range(ref["conc"].shape[0]):
        assert rel(got["conc"][k], ref["conc"][k], liquid) <= 1e-5, k


def test_two_node_shapes_stage_the_d2q9_box_only(pslbm):
    """The two-node shapes have staging 2 (the D2Q9 box) but not staging 1
    (the D2Q9 and D2Q5 boxes would not fit two blocks per SM): fixing staging
    1 on a two-node shape (in either order) is rejected and leaves the handle
    as it was; the autotuner's choice is one of the six variants of one node
    per thread or the four of two nodes per thread, and equals the pinned
    runs."""
    sc = inputs.porous_discs(nx=128, ny=96, seed=7)
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP32) as s:
        assert s.staging()[1]
        s.set_tile_shape(32, 16)
        with pytest.raises(pslbm.PslbmError):
            s.set_staging(1)
        s.set_staging(2)
        s.set_tile_shape(32, 8)
        s.set_staging(1)
        with pytest.raises(pslbm.PslbmError):
            s.set_tile_shape(16, 32)
        assert s.tile_shape()[:2] == (32, 8)
        with pytest.raises(pslbm.PslbmError):
            s.set_tile_shape(64, 4)
    ref = run(pslbm, sc, 100, pslbm.FP32, (32, 16))
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP32) as s:
        s.step(100)
        tx, ty, tuned = s.tile_shape()
        assert tuned and (tx, ty) in ((16, 16), (32, 8), (16, 32), (32, 16))
        staged, _ = s.staging()
        assert not (staged == 1 and tx * ty == 512)
        got = s.read()
    assert_same(got, ref, "autotuned")
