"""The allocation-free per-phase mass reduction against ddcc_mass.

ddcc_phase_mass_noalloc exists for callers that cannot call cudaMalloc --
plugins whose host application owns all device memory, real-time loops that
cannot absorb an allocation's implicit synchronisation.  It keeps its
scratch in a static device array.  This test feeds it the population planes
of a live simulation (through a saved state, whose layout include/ddcc.h
documents) and checks it returns the masses ddcc_mass returns, on two calls
in a row with steps in between, and that a call after the first one leaves
the device's free memory unchanged.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10314_gb300 import build as B
    B.build()
    import paper_2311_10314_gb300 as D
    from paper_2311_10314_gb300 import _lib
    return D, _lib


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_mass_matches_ddcc_mass(mods, precision):
    D, L = mods
    pb = W.random_problem(70, 45, 4, seed=21, periodic_y=0, theta_field=True, width=6.0)
    N, nx, ny = 4, pb.params["nx"], pb.params["ny"]
    sim = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision)
    es = 8 if precision == D.DDCC_FP64 else 4
    first, pitch, plane_stride = L.state_layout(nx, ny, N, es)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        sim.step(7 + call)
        ref = sim.mass()
        buf = sim.save_state()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = L.ddcc_phase_mass_noalloc(buf.data_ptr() + first * es, precision, N, nx, ny, pitch,
                                       plane_stride, out.data_ptr(), stream.cuda_stream)
        assert st == L.DDCC_OK, L.status_string(st)
        stream.synchronize()
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free0
        got = out[: N - 1].cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=0.0), (call, got, ref)
    sim.close()


def test_noalloc_rejects_sizes_beyond_static_scratch(mods):
    D, L = mods
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    ny = L.NOALLOC_MAX_ROWS + 1
    st = L.ddcc_phase_mass_noalloc(dummy.data_ptr(), 0, 3, 4, ny, 4, 4 * ny, out.data_ptr(), 0)
    assert st == L.DDCC_ERR_PARAM
