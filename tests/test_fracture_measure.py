"""The fracture measurement (App. C): the porosity of the undissolved medium
is the aperture over the medium's height, h0 / (H - 2) (the two wall rows are
not medium), and the flow rate sums the mid column."""
import numpy as np

from paper_1410_3464_gb300 import fracture, inputs


def test_initial_porosity_is_aperture_over_height():
    L, H, h0 = 100, 90, 30
    sc = inputs.fracture(L=L, H=H, h0=h0)
    vol_d = (sc["mask"] == inputs.SOLID_D).astype(float)
    assert abs(fracture.porosity(vol_d, L, H) - h0 / (H - 2)) < 1e-15


def test_flow_rate_sums_the_mid_column():
    L, H = 100, 90
    ux = np.zeros((H, L + 2))
    y = np.arange(H)
    ux[:, L // 2 + 1] = np.where((y >= 30) & (y < 60), (y - 29.5) * (59.5 - y), 0.0)
    assert abs(fracture.flow_rate(ux, L) - ux[:, L // 2 + 1].sum()) < 1e-12
