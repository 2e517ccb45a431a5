"""The create path: one device allocation per simulation, the inputs staged in
the second population buffer, the solid volumes and the first threshold
derived on the device.

- volumes derived from the node types equal the same volumes passed in;
- the first threshold equals half the initial maximum of rho_1 over fluid
  nodes, read back through the monitor;
- a handle's device bytes stay within the estimate the server admits by;
- handles created and destroyed in a loop (the arena freed each time) give
  the same results as the first.
"""
import numpy as np
import pytest

from oracle import lbm
from paper_1410_3464_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho1", "rho2", "ux", "uy", "conc", "type", "vol", "budget")


@pytest.fixture(scope="module")
def pslbm():
    from paper_1410_3464_gb300 import build, pslbm as m
    build.build()
    return m


def sim(pslbm, sc, vol, precision):
    return pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], vol,
                            precision=precision)


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_volumes_from_types_equal_given_volumes(pslbm, prec):
    """A porous scene with D(s) grains and an F(s) patch: V from the mask on the
    device (vol = NULL) and the same V passed in give identical runs."""
    sc = inputs.porous_discs(nx=96, ny=64, seed=11, rmin=3, rmax=8)
    mask = sc["mask"].copy()
    solid = np.argwhere(mask == lbm.SOLID_D)
    for (y, x) in solid[::7]:
        mask[y, x] = lbm.SOLID_F
    sc = inputs.Scene(**dict(sc, mask=mask))
    vol = np.zeros((2,) + mask.shape)
    vol[0][mask == lbm.SOLID_D] = 1.0
    vol[1][mask == lbm.SOLID_F] = 1.0
    p = getattr(pslbm, prec)
    with sim(pslbm, sc, None, p) as a, sim(pslbm, sc, vol, p) as b:
        assert np.array_equal(a.read(pslbm.F_VOL)["vol"], vol)
        a.step(40)
        b.step(40)
        ra, rb = a.read(), b.read()
    for k in FIELDS:
        assert np.array_equal(ra[k], rb[k], equal_nan=True), k


def test_first_threshold_is_half_the_initial_maximum(pslbm):
    sc = inputs.bubble_grain()
    fluid = sc["mask"] <= 1
    with sim(pslbm, sc, None, pslbm.FP64) as s:
        n, m, st = s.monitor()
        assert n == 0 and st == 0
        assert m == float(sc["rho1"][fluid].max())


def test_device_bytes_within_the_estimate(pslbm):
    for nx, ny, seed in ((96, 64, 1), (100, 50, 2), (20, 12, 3)):
        sc = inputs.porous_discs(nx=nx, ny=ny, seed=seed, rmin=3, rmax=8)
        for prec in (pslbm.FP64, pslbm.FP32, pslbm.FP32_SOLUTE_F16):
            est = pslbm.estimate_device_bytes(sc["params"], prec)
            with sim(pslbm, sc, None, prec) as s:
                s.step(5)
                used = s.device_bytes()
            assert used <= est, (nx, ny, prec, used, est)


def test_repeated_create_destroy_same_results(pslbm):
    sc = inputs.porous_discs(nx=64, ny=48, seed=5)
    ref = None
    for _ in range(12):
        with sim(pslbm, sc, None, pslbm.FP32) as s:
            s.step(20)
            r = s.read()
        if ref is None:
            ref = r
        for k in FIELDS:
            assert np.array_equal(r[k], ref[k], equal_nan=True), k
