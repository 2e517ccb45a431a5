"""The per-step monitor (pslbm_monitor): step count, the maximum rho_1 the last
step found (Section 4.5: half of it is the next liquid threshold) and status.

The bulk kernel takes the maximum over the state a step starts from, so after
k + 1 steps the monitor reports the maximum of the state after k steps, which
the budget read-out gives independently (same FP32 sums, exact maximum)."""
import numpy as np
import pytest

from paper_1410_3464_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pslbm():
    from paper_1410_3464_gb300 import build, pslbm as m
    build.build()
    return m


@pytest.mark.parametrize("precision", [0, 1])
def test_monitor_reports_last_step_maximum(pslbm, precision):
    sc = inputs.porous_discs(nx=96, ny=64, seed=13)
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as s:
        n0, m0, st0 = s.monitor()
        assert n0 == 0 and st0 == 0
        assert m0 == s.read(pslbm.F_BUDGET)["budget"][0]      # the initial maximum
        for k in (1, 7, 40):
            before = s.read(pslbm.F_BUDGET)["budget"][0]
            s.step(1)
            n, m, st = s.monitor()
            assert st == 0
            assert n == s.steps()
            assert m == before, (k, m, before)
            s.step(k)


def test_monitor_reports_a_nonfinite_state(pslbm):
    sc = inputs.porous_discs(nx=64, ny=48, seed=14)
    rho1 = sc["rho1"].copy()
    y, x = np.argwhere(sc["mask"] == 0)[5]
    rho1[y, x] = np.nan
    with pslbm.Simulation(sc["mask"], sc["params"], rho1, sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP32) as s:
        s.step(2)
        with pytest.raises(pslbm.PslbmError):
            s.monitor()
