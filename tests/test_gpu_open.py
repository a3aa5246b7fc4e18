"""GPU path with open x ends (inflow at x = 0, outflow at x = nx - 1,
DDCC_FLAG_OPEN_X + ddcc_set_inflow) against the FP64 oracle's reading of
Sec. 4.5's parabolic inflow/outflow.

Bars: FP64 1e-10 in C (psi >= 0.01), rho and u after 150 steps, through the
fused tile kernel (wide grids) and the plain-load fallback (narrow ones);
FP32 1e-4 in C on psi >= 0.5; the Sec. 4.5 wavy channel with its inflow runs
1500 steps finite.
"""
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


def _open_problem(nx, ny, N, seed, py):
    rng = np.random.default_rng(seed)
    pb = W.random_problem(nx, ny, N, seed=seed, periodic_x=0, periodic_y=py, theta_field=True, width=6.0)
    y = np.arange(ny) + 0.5
    u_in = 0.02 * 4.0 * y * (ny - y) / ny ** 2 + 0.003 * rng.standard_normal(ny)
    C_in = rng.uniform(0.0, 0.9 / (N - 1), size=(N - 1, ny))
    return pb, (u_in, C_in)


@pytest.mark.parametrize("nx,ny,N,py", [(48, 30, 2, 0), (57, 33, 3, 1), (44, 36, 4, 0), (21, 17, 3, 0)])
def test_open_ends_fp64_parity(ddcc, nx, ny, N, py):
    pb, ox = _open_problem(nx, ny, N, seed=nx + N, py=py)
    o = Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, open_x=ox)
    o.step(150)
    ref = {k: v.numpy() for k, v in o.macroscopic().items()}
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=ddcc.DDCC_FP64,
                   open_x=ox)
    sim.step(150)
    got = sim.fields()
    sim.close()
    fl = pb.psi >= 0.01
    assert np.abs(ref["C"] - got["C"])[:, fl].max() <= 1e-10
    assert np.abs(ref["rho"] - got["rho"])[fl].max() <= 1e-10
    assert max(np.abs(ref["ux"] - got["ux"]).max(), np.abs(ref["uy"] - got["uy"]).max()) <= 1e-10


def test_open_ends_fp32_against_oracle(ddcc):
    pb, ox = _open_problem(57, 33, 3, seed=60, py=0)
    o = Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, open_x=ox)
    o.step(150)
    ref = o.macroscopic()["C"].numpy()
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=ddcc.DDCC_FP32,
                   open_x=ox)
    sim.step(150)
    got = sim.fields()["C"]
    sim.close()
    assert np.abs(ref - got)[:, pb.psi >= 0.5].max() <= 1e-4


def test_open_ends_rejected_where_unsupported(ddcc):
    pb, ox = _open_problem(48, 30, 2, seed=1, py=0)
    prm = dict(pb.params, periodic_x=1)
    with pytest.raises(ddcc.DdccError):
        ddcc.Sim(prm, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, open_x=ox)
    with pytest.raises(ddcc.DdccError):
        ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, open_x=ox, path="sweep")


@pytest.mark.parametrize("precision", [0, 1])
def test_wavy_channel_with_inflow(ddcc, precision):
    pb = W.config6_wavy_channel()
    prm = dict(pb.params, periodic_x=0, body_force=[0.0, 0.0])
    sim = ddcc.Sim(prm, None, pb.C0, walls=pb.extra["walls"], open_x=pb.extra["open_x"],
                   precision=precision)
    sim.step(1500)
    C = sim.read(ddcc.FIELD_C)
    ux = sim.read(ddcc.FIELD_UX)
    sim.close()
    assert np.isfinite(C).all() and np.isfinite(ux).all()
    gap = pb.psi >= 0.5
    assert ux[gap].mean() > 0.0
