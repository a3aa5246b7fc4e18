"""The fused 2D step replayed as a CUDA graph (two steps per replay, captured
on first use) against the same step launched kernel by kernel: with
profiling on, ddcc_step takes the plain launches, so two handles of the
same problem, one profiled and one not, must agree bit for bit after any
sequence of step calls -- including calls of fewer than four steps (plain),
odd counts and calls that start on the second ping-pong copy.  FP32 and
FP64, periodic and walled, with a per-node angle field.  And the read-out
fields kept between reads of one state are formed anew after a step (2D
and 3D)."""
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


def test_read_after_step_sees_the_new_state(D):
    """The read-out fields are formed once per state: reading, stepping and
    reading again gives the new state's fields (as a handle that was only
    read at the end), in 2D and in 3D (where C and mu are kept)."""
    pb = W.random_problem(64, 40, 3, seed=8, periodic_y=1, theta_field=True, width=5.0)
    a = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=D.DDCC_FP64)
    b = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=D.DDCC_FP64)
    a.step(3)
    first = a.fields()
    a.step(6)
    b.step(9)
    fa, fb = a.fields(), b.fields()
    assert not np.array_equal(first["C"], fa["C"])
    for k in ("C", "ux", "uy", "P", "mu"):
        assert np.array_equal(fa[k], fb[k]), k
    a.close()
    b.close()
    p3 = W.random_problem_3d(20, 12, 10, 3, seed=4, theta_field=True)
    a = D.Sim3D(p3.params, p3.psi, p3.C0, p3.cos_theta, p3.cos_theta_field, precision=D.DDCC_FP64)
    b = D.Sim3D(p3.params, p3.psi, p3.C0, p3.cos_theta, p3.cos_theta_field, precision=D.DDCC_FP64)
    a.step(2)
    first = a.fields()
    a.step(3)
    b.step(5)
    fa, fb = a.fields(), b.fields()
    assert not np.array_equal(first["C"], fa["C"])
    for k in ("C", "ux", "uy", "uz", "P", "mu"):
        assert np.array_equal(fa[k], fb[k]), k
    a.close()
    b.close()
