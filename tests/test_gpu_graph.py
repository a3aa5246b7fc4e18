"""The fused 2D step replayed as a CUDA graph (two steps per replay, captured
on first use) against the same step launched kernel by kernel: with
profiling on, ddcc_step takes the plain launches, so two handles of the
same problem, one profiled and one not, must agree bit for bit after any
sequence of step calls -- including calls of fewer than four steps (plain),
odd counts and calls that start on the second ping-pong copy.  FP32 and
FP64, periodic and walled, with a per-node angle field."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10314_gb300 import build as B
    B.build()
    import paper_2311_10314_gb300 as D
    return D


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("periodic_y", [1, 0])
def test_graph_replay_matches_plain_launches(D, precision, periodic_y):
    from paper_2311_10314_gb300 import _lib
    pb = W.random_problem(70, 45, 3, seed=21, periodic_y=periodic_y, theta_field=True, width=5.0)
    sims = [D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision)
            for _ in range(2)]
    _lib.ddcc_profile(sims[0].h, True)          # plain launches
    for n in (1, 5, 2, 9, 4, 3, 12):
        for s in sims:
            s.step(n)
        _lib.ddcc_kernel_times(sims[0].h)        # keep the event record short
    assert sims[0].steps == sims[1].steps == 36
    a, b = sims[0].fields(), sims[1].fields()
    for k in ("C", "ux", "uy", "P", "mu"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(sims[0].mass(), sims[1].mass())
    for s in sims:
        s.close()
