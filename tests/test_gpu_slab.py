"""The y-slab decomposition on the GPU: several slabs of one grid held on
one GPU (``slab.LocalSlabs``) and one rank exchanging with itself
(``SlabRun`` with a one-rank ``TorchExchange``) step the same state as one
``Sim`` of the whole grid.  The kernels do the same arithmetic node by node
whatever the slab's height, so every own row of every population and
lagged plane matches bit for bit, FP64 and FP32, and the FP64 masses of the
own rows, summed, match the whole grid's.  This covers ``ddcc_get_rows`` /
``ddcc_set_rows`` and the halo bookkeeping; the exchange between GPUs
(NCCL) is not run here (one GPU)."""
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


def _whole_rows(D, sim, y0, n):
    from paper_2311_10314_gb300 import _lib
    N = sim.N
    dt = torch.float64 if sim.precision == D.DDCC_FP64 else torch.float32
    buf = torch.empty((9 * N + 2 * N + 3, n, sim.nx), dtype=dt, device="cuda")
    _lib.ddcc_get_rows(sim.h, y0, n, buf.data_ptr())
    return buf.cpu().numpy()


@pytest.mark.parametrize("world,precision", [(2, 0), (3, 0), (3, 1)])
def test_local_slabs_match_whole_grid(D, world, precision):
    from paper_2311_10314_gb300 import slab
    pb = W.random_problem(96, 45, 3, seed=9, theta_field=True, width=6.0, body_force=(1e-5, 0.0))
    whole = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision)
    ls = slab.LocalSlabs(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, world, precision, D.Sim)
    steps = 40
    whole.step(steps)
    ls.step(steps)
    ny = pb.params["ny"]
    for r, st in enumerate(ls.steppers):
        y0, y1 = slab.slab_rows(ny, world, r)
        got = st.get_rows(slab.HALO, y1 - y0).cpu().numpy()
        assert np.array_equal(got, _whole_rows(D, whole, y0, y1 - y0)), r
    assert np.allclose(ls.mass(), whole.mass(), rtol=1e-12 if precision == 0 else 1e-6, atol=0)
    ls.close()
    whole.close()


def test_one_rank_exchanges_with_itself(D):
    from paper_2311_10314_gb300 import slab
    pb = W.config4_imbibition(nx=256, ny=256)
    whole = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=D.DDCC_FP32)
    st = slab.GpuSlab(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, 0, 256, D.DDCC_FP32, D.Sim)
    run = slab.SlabRun(st, 256, slab.TorchExchange(0, 1))
    whole.step(25)
    run.step(25)
    assert np.array_equal(run.own_rows().cpu().numpy(), _whole_rows(D, whole, 0, 256))
    assert np.allclose(run.mass(), whole.mass(), rtol=1e-6, atol=0)
    st.close()
    whole.close()
