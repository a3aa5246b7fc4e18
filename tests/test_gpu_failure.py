"""Failure detection without a GPU fault: a bounded wait whose completion
never comes runs out, the kernel returns, the host reads DDCC_ERR_TIMEOUT,
and the CUDA context stays usable (a simulation steps and matches the
oracle afterwards)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10314_gb300 import build as B
    B.build()
    import paper_2311_10314_gb300 as D
    return D


def test_bounded_wait_runs_out_and_context_survives(ddcc):
    from paper_2311_10314_gb300 import _lib
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert _lib.ddcc_selftest_bounded_wait(stream, flag.data_ptr(), True) == _lib.DDCC_OK
    for _ in range(2):
        assert _lib.ddcc_selftest_bounded_wait(stream, flag.data_ptr(), False) == _lib.DDCC_ERR_TIMEOUT
        assert int(flag.item()) == 1
    assert _lib.ddcc_selftest_bounded_wait(stream, flag.data_ptr(), True) == _lib.DDCC_OK
    pb = W.random_problem(40, 27, 3, seed=2, periodic_y=0, theta_field=True, width=6.0)
    o = Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field)
    o.step(20)
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=ddcc.DDCC_FP64)
    sim.step(20)
    got = sim.fields()
    sim.close()
    fl = pb.psi >= 0.01
    assert np.abs(o.macroscopic()["C"].numpy() - got["C"])[:, fl].max() <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_population_reported(ddcc, precision):
    """A state with NaN populations, loaded from host memory through
    ddcc_load_state, makes ddcc_mass return DDCC_ERR_NONFINITE; the context
    stays usable and the clean state still gives finite masses."""
    from paper_2311_10314_gb300 import _lib
    pb = W.random_problem(40, 27, 3, seed=2, periodic_y=0, theta_field=True, width=6.0)
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision)
    sim.step(3)
    clean = sim.save_state().cpu()
    m_clean = sim.mass()
    bad = clean.clone()
    N = pb.params["nphase"]
    planes = 9 * N + 2 * N + 3
    plane_bytes = (bad.numel() - 256) // planes
    es = 8 if precision == 0 else 4
    view = bad[256:256 + plane_bytes].view(torch.float64 if es == 8 else torch.float32)
    view[:] = float("nan")                 # the rest population of phase 1
    sim.load_state(bad)
    with pytest.raises(_lib.DdccError) as ei:
        sim.mass()
    assert ei.value.status == _lib.DDCC_ERR_NONFINITE
    sim.load_state(clean)
    assert np.array_equal(sim.mass(), m_clean)
    sim.close()


@pytest.mark.parametrize("bad", [0.0, -1e-3, 1.0 + 1e-12, float("nan")])
@pytest.mark.parametrize("where", [0, 4097, -1])
def test_create_rejects_psi_outside_unit_interval(ddcc, bad, where):
    """psi must lie in (0, 1] at every node: one bad value anywhere (first
    node, inside a later block of the scan, last node) gives
    DDCC_ERR_PARAM from create, and the same field without it is
    accepted."""
    from paper_2311_10314_gb300 import _lib
    pb = W.random_problem(96, 64, 2, seed=3, periodic_y=1, width=4.0)
    psi = pb.psi.copy()
    psi.reshape(-1)[where] = bad
    with pytest.raises(_lib.DdccError) as ei:
        ddcc.Sim(pb.params, psi, pb.C0, pb.cos_theta, precision=ddcc.DDCC_FP32)
    assert ei.value.status == _lib.DDCC_ERR_PARAM
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, precision=ddcc.DDCC_FP32)
    sim.close()
