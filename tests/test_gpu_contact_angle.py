"""Static contact angle (App. A2) on the GPU path, 201x201, FP64.

The walls are symmetry (mirror-image) walls in the cohesion sums, so with no
solid-fluid interaction (w = 0) the droplet must rest at 90 degrees, as the
paper states for w = 0 and for the beaker walls (Section 5); an attractive
interaction (w < 0) makes the wall wetting, the angle falling nearly linearly
with w (the paper: w = -0.4 gives 74.2 degrees with its own constants)."""
import pytest

pytestmark = pytest.mark.gpu


def test_contact_angle_ninety_degrees_without_interaction():
    from paper_1410_3464_gb300 import contact_angle as ca
    out = ca.run(0.0, steps=30000)
    assert abs(out["theta_deg"] - 90.0) < 2.0, out


def test_contact_angle_falls_with_attractive_interaction():
    from paper_1410_3464_gb300 import contact_angle as ca
    th = [ca.run(w, steps=30000)["theta_deg"] for w in (-0.3, -0.15, 0.0)]
    assert th[0] < th[1] < th[2]
    assert 65.0 < th[0] < 85.0
    # nearly linear: the midpoint within 2 degrees of the chord
    assert abs(th[1] - 0.5 * (th[0] + th[2])) < 2.0
