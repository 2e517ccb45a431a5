"""The allocation-free budget entry point (pslbm_budget_device_noalloc).

Some callers cannot allocate device memory at the moment they want the budget:
a host that hands the library a fixed memory pool and forbids later
allocation, or a real-time loop where an allocation could stall.  They call
this entry point, which keeps its partial sums in a file-scope device array;
it must give the same numbers as pslbm_read_fields(PSLBM_F_BUDGET), bit for bit,
on every storage precision.  This file is collected last so that a failure here
comes after every other test.
"""
import numpy as np
import pytest

from paper_1410_3464_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pslbm():
    from paper_1410_3464_gb300 import build, pslbm as m
    build.build()
    return m


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_noalloc_budget_matches_read_fields(pslbm, precision):
    import torch
    sc = inputs.porous_discs(nx=200, ny=120, seed=9, slug=(10, 5))
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as sim:
        sim.step(15)
        n = 6 + sim.ns
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        for call in range(2):                       # two calls in a row
            ref = sim.read(pslbm.F_BUDGET)["budget"]
            sim.budget_device_noalloc(out.data_ptr())
            sim.sync()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), f"call {call}"
            # same reduction grid and order as read_fields: the same bits
            assert np.array_equal(got, ref), f"call {call}: {got} != {ref}"
            sim.step(3)


def test_noalloc_rejects_null_output(pslbm):
    sc = inputs.porous_discs(nx=64, ny=32, seed=2, slug=(10, 5))
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"]) as sim:
        with pytest.raises(pslbm.PslbmError) as e:
            sim.budget_device_noalloc(None)
        assert e.value.status == -1
