"""Fracture dissolution (App. C, Eq. A3) on the GPU path: a 30-wide fracture
in a 100x90 medium widens as R2 dissolves its walls under pressure-driven
flow; the permeability (the flow rate at the fixed reservoir pressures)
against the porosity from the VOP volumes follows a power law of exponent 3."""
import pytest

pytestmark = pytest.mark.gpu


def test_permeability_porosity_cubic_law():
    from paper_1410_3464_gb300 import fracture
    out = fracture.run(steps=120000, every=20000)
    rows = out["rows"]
    assert rows[-1]["eps_ratio"] > 1.35          # the fracture has widened by a third at least
    assert all(b["eps"] > a["eps"] for a, b in zip(rows, rows[1:]))
    assert abs(out["exponent"] - 3.0) < 0.2, out["exponent"]
