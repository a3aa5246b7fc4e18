"""bench.py's algorithmic byte counts (the roofline numerators), counted
here plane by plane from the state layout the kernels move, so that a
change to either side shows:

* 2D step: per node the 9N populations read and written, psi, the N-1
  angle planes when the angle is a per-node field, and the 2N+3 lagged
  planes (a, psi C_i u for i < N, T_xx, T_yy, T_xy, psi m.u) read and
  written -- 392 B at N = 4 with the angle field in FP32 (the imbibition
  workload);
* 3D step: 7(N-1) D3Q7 and 15 D3Q15 populations and the 3N+7 lagged planes
  (a_xy, a_yz, a_zx, psi C_i u, six T components, psi m.u) read and
  written, and psi -- 364 B at N = 3 in FP32 (the sphere workload); the
  fused kernel moves exactly that, the three-kernel update kernel adds the
  N-1 volume fractions and N chemical potentials it reads (384 B).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _lagged_2d(N):
    return 1 + 2 * (N - 1) + 3 + 1          # a, psi C_i u (x, y), T (3), psi m.u


def _lagged_3d(N):
    return 3 + 3 * (N - 1) + 6 + 1          # a (3), psi C_i u (x, y, z), T (6), psi m.u


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("tf", [False, True])
def test_2d_step_floats(N, tf):
    want = 2 * 9 * N + 1 + ((N - 1) if tf else 0) + 2 * _lagged_2d(N)
    assert bench.step_floats_per_node(N, tf) == want


def test_2d_headline_bytes():
    assert 4 * bench.step_floats_per_node(4, True) == 392


@pytest.mark.parametrize("N", [2, 3, 4])
def test_3d_step_bytes(N):
    want = 2 * (7 * (N - 1) + 15) + 2 * _lagged_3d(N) + 1
    assert bench.step_bytes_per_node_3d(N, False, 1) == want
    assert bench.step_bytes_per_node_3d(N, True, 1) == want + (N - 1)
    k = bench.kernel_bytes_per_node_3d(N, False, 1)
    assert k["fused_step"] == want
    assert k["update"] == want + (N - 1) + N


def test_3d_headline_bytes():
    assert bench.step_bytes_per_node_3d(3, False, 4) == 364
    assert bench.kernel_bytes_per_node_3d(3, False, 4)["update"] == 384
