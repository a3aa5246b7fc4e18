"""Pin of the Table 2 golden values by plane geometry (no lattice code).

A semicircular compound drop of radius R split at its axis into two
quarter discs (phases 1 and 2) under equal surface tensions and
theta_13 = theta_23 = 90 deg settles, by symmetry, with a vertical 1-2
interface, 120-degree angles at the triple junction, and 1-3 and 2-3 arcs
that meet the wall at 90 deg: each arc is centred on the wall, at distance
a from the axis, with radius r = 2a (its tangent at the junction rises 30
deg from the horizontal).  Phase 1 then fills the half disc of radius r
less the circular segment beyond the axis, pi r^2 / 3 + sqrt(3) r^2 / 8,
which must equal pi R^2 / 4; its footprint is L1 = a + r = 1.5 r.
"""
import json
import math
import os

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table2_spreading_lengths.json")


def symmetric_length():
    r = math.sqrt((math.pi / 4.0) / (math.pi / 3.0 + math.sqrt(3.0) / 8.0))
    return 1.5 * r


def test_segment_area_formula():
    """The area of the half disc of radius r centred at (-r/2, 0) to the
    left of the axis, by numerical quadrature."""
    r, n = 1.0, 200000
    a = r / 2.0
    h = (r + a) / n
    area = 0.0
    for k in range(n):
        x = -(a + r) + (k + 0.5) * h
        area += math.sqrt(max(r * r - (x + a) ** 2, 0.0)) * h
    assert abs(area - (math.pi / 3.0 + math.sqrt(3.0) / 8.0)) < 1e-6


def test_table2_symmetric_case():
    with open(GOLD) as fh:
        g = json.load(fh)
    i = g["theta13_deg"].index(90.0)
    L = symmetric_length()
    assert abs(L - g["analytical_L1"][i]) < 5e-4
    assert abs(L - g["analytical_L2"][i]) < 5e-4
