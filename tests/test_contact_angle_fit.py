"""The contact-angle measurement (App. A2) recovers the angle of a known
circular cap: synthetic tanh droplets whose circle centre lies on, below and
above the wall face give 90 degrees, 90 - asin(15/60) and 90 + asin(10/45)."""
import math

import numpy as np
import pytest

from paper_1410_3464_gb300 import contact_angle as ca


@pytest.mark.parametrize("yc_off,R", [(0.0, 50.0), (-15.0, 60.0), (10.0, 45.0)])
def test_circle_fit_recovers_cap_angle(yc_off, R):
    ny = nx = 201
    y, x = np.mgrid[0:ny, 0:nx]
    r = np.hypot(x - 100.0, y - (0.5 + yc_off))
    rho = 0.0537 + (8.17 - 0.0537) * 0.5 * (1.0 - np.tanh((r - R) / 2.0))
    rho[0, :] = 0.0
    rho[-1, :] = 0.0
    out = ca.contact_angle(rho)
    assert abs(out["theta_deg"] - (90.0 + math.degrees(math.asin(yc_off / R)))) < 0.05
    assert abs(out["radius"] - R) < 0.05
