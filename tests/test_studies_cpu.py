"""The convergence study's model definitions (Sec. V: production HHLB(6;7) x HLB(6;7) at
delta = 1, 10 and HHLB(10;16) x HLB(6;7) at delta = 0.1, S = 16; reference
HHLB(10;50) x HLB(6;7), S = 48; A = 0.98, u_w = sqrt(2)) and its extrapolation, on the CPU."""
import math

import numpy as np
import pytest

from paper_1810_07803_gb300 import lbc, studies


@pytest.mark.parametrize("delta,orders", [(0.1, (10, 16)), (1.0, (6, 7)), (10.0, (6, 7))])
def test_models_of_the_paper(delta, orders):
    p = studies.production(delta, 0.66, 2.0 / 3.0)
    r = studies.reference(delta, 0.66, 2.0 / 3.0)
    assert (p["Nexp_x"], p["Qx"], p["Nexp_y"], p["Qy"]) == (*orders, 6, 7)
    assert (r["Nexp_x"], r["Qx"], r["Nexp_y"], r["Qy"]) == (10, 50, 6, 7)
    assert studies.S_of(p) == 16 and studies.S_of(r) == 48
    for m in (p, r):
        assert m["stretch_A"] == 0.98 and m["u_right"] == -m["u_left"] == math.sqrt(2.0)
        assert m["half_channel"] == 1 and m["local_dt"] == 1 and m["precision"] == "fp64"
        lbc.make_params(m)   # a valid lbc_params


def test_full_channel_and_compensated_variants():
    p = studies.production(1.0, 0.66, 2.0 / 3.0, half=False, precision="fp32", compensated=True)
    assert p["Nx"] == 32 and studies.S_of(p) == 16 and p["half_channel"] == 0 and p["compensated"] == 1
    assert studies.production(1.0, 0.66, 2.0 / 3.0, compensated=True)["compensated"] == 0   # FP64: no remainder


def test_aitken_is_exact_on_a_geometric_sequence():
    limit, c, q = 0.37, 0.2, 0.6
    x = [limit + c * q ** k for k in range(3)]
    assert studies.aitken(*x) == pytest.approx(limit, rel=1e-14)
    assert studies.aitken(1.0, 1.0, 1.0) == 1.0          # no change: the last value
    assert studies.aitken(1.0, 2.0, 4.0) == 4.0          # diverging: the last value


def test_pi_number_is_minus_half_the_shear_stress():
    m = np.zeros((10, 5))
    m[lbc.MOMENT_NAMES.index("P_xy")] = -0.4
    pi, spread = studies.pi_number(m)
    assert pi == pytest.approx(0.2) and spread == 0.0
