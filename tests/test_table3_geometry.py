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
