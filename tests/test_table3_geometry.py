"""Pin of the Table 3 analytical spreading lengths (App. D) by plane
geometry (no lattice code): the construction of ``table3_geometry`` -- a
straight 1|2 interface normal to the wall, 120-degree junctions for equal
tensions, the prescribed wall angles and equal drop areas -- reproduces
every printed analytical length of Table 3 to the printed three decimals,
and its symmetric case agrees with the closed forms (L1 = L3 = 1.5 r and
the root of a quadratic for L2)."""
import json
import math
import os

import pytest

import table3_geometry as T

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table3_spreading_lengths.json")


def test_phase1_quadrature():
    """Area of the phase-1 region (half disc of radius r centred at (-a, 0),
    cut at x = 0) by quadrature equals pi r^2 / 3 + sqrt(3) r^2 / 8."""
    r, a, _ = T.phase1()
    n = 200000
    hx = (r + a) / n
    area = sum(math.sqrt(max(r * r - ((-(a + r) + (k + 0.5) * hx) + a) ** 2, 0.0)) * hx for k in range(n))
    assert abs(area - math.pi / 2) < 1e-6


@pytest.mark.parametrize("k", [0, 1, 2])
def test_table3_analytical_lengths(k):
    with open(GOLD) as fh:
        g = json.load(fh)
    L = T.spreading_lengths(g["theta34_deg"][k])
    for i, name in enumerate(("analytical_L1", "analytical_L2", "analytical_L3")):
        assert abs(L[i] - g[name][k]) <= 6e-4, (name, L[i], g[name][k])


def test_symmetric_case_closed_form():
    L1, L2, L3 = T.spreading_lengths(90.0)
    r, _, _ = T.phase1()
    assert abs(L1 - 1.5 * r) < 1e-12
    assert abs(L3 - L1) < 1e-6
    assert abs(L2 - T.symmetric_L2()) < 1e-6


def test_contact_points_skip_rounding_sign_changes():
    """The GPU test's contact-point reader: a sign change of C_a - C_b
    counts only where C_a + C_b > 1/2, so the rounding-level sign changes
    inside a third phase (both fields ~0) are not taken for an interface,
    and the real crossing is located to within interpolation error."""
    import numpy as np
    from test_gpu_table3 import contact_points
    x = np.arange(200, dtype=np.float64)
    ca = 0.5 * (1.0 - np.tanh((x - 120.3) / 4.0))          # phase a on the left
    cb = 0.5 * (1.0 + np.tanh((x - 120.3) / 4.0))          # phase b on the right
    third = (x < 60)                                         # a third phase on the far left
    ca[third] = 1e-9 * np.sin(x[third])                      # rounding-level values of both
    cb[third] = 1e-9 * np.cos(x[third])
    p = contact_points(ca, cb)
    assert len(p) == 1 and abs(p[0] - 120.3) < 0.05, p
    d = ca - cb
    naive = [i for i in range(len(d) - 1) if (d[i] >= 0) != (d[i + 1] >= 0)]
    assert len(naive) > 1                                    # what the first-sign-change reader saw
