"""GPU path for a solid of several parts (Sec. 4.5): psi = prod_k psi_k and
the wetting term sum_k cos(theta^k_jq) |grad psi_k|, created through
ddcc_create_walls, against the FP64 oracle's direct form of the paper's
expression.

Bars: FP64 1e-10 in C (psi >= 0.01), u, rho after 150 steps; FP32 1e-4 in C
on psi >= 0.5; the Sec. 4.5 wavy channel runs 2000 steps with mass conserved
(1e-13 FP64, 1e-6 FP32).
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


def _channel(nx, ny, N, seed, uniform=False):
    rng = np.random.default_rng(seed)
    x, y = np.meshgrid(np.arange(nx) + 0.0, np.arange(ny) + 0.0)
    xi = W.SOLID_XI
    psi1 = W.psi_from_distance(y - 7.3 - 2.0 * np.sin(2 * np.pi * x / nx), xi=xi)
    psi2 = W.psi_from_distance(ny - 7.4 + 1.5 * np.cos(2 * np.pi * x / nx) - y, xi=xi)
    C0 = np.zeros((N - 1, ny, nx))
    C0[0] = W.drop_profile(np.hypot(x - 0.35 * nx, y - 9.0), 6.0, 4.0)
    if N > 2:
        C0[1] = W.drop_profile(np.hypot(x - 0.68 * nx, y - ny + 10.0), 5.0, 4.0) * (1 - C0[0])
    prm = W.base_params(nx, ny, N, periodic_x=1, periodic_y=0, sigma=0.01, width=4.0, xi=xi,
                        tau=0.8, eta=0.5)
    if uniform:
        cos1 = rng.uniform(-0.7, 0.7, size=N - 1)
        cos2 = rng.uniform(-0.7, 0.7, size=N - 1)
    else:
        cos1 = rng.uniform(-0.7, 0.7, size=(N - 1, ny, nx))
        cos2 = rng.uniform(-0.7, 0.7, size=(N - 1, ny, nx))
    return prm, [(psi1, cos1), (psi2, cos2)], C0


def _ref(prm, walls, C0, steps):
    o = Oracle(prm, None, C0, None, walls=walls)
    o.step(steps)
    m = o.macroscopic()
    return {k: v.numpy() for k, v in m.items()}, o.psi.numpy()


@pytest.mark.parametrize("nx,ny,N,uniform", [(48, 36, 2, False), (61, 40, 3, False), (50, 38, 3, True),
                                             (45, 41, 4, False)])
def test_walls_fp64_parity(ddcc, nx, ny, N, uniform):
    prm, walls, C0 = _channel(nx, ny, N, seed=nx + N, uniform=uniform)
    ref, psi = _ref(prm, walls, C0, 150)
    sim = ddcc.Sim(prm, None, C0, walls=walls, precision=ddcc.DDCC_FP64)
    assert np.array_equal(sim.read(ddcc.FIELD_PSI), psi)
    sim.step(150)
    got = sim.fields()
    sim.close()
    fl = psi >= 0.01
    assert np.abs(ref["C"] - got["C"])[:, fl].max() <= 1e-10
    assert np.abs(ref["rho"] - got["rho"])[fl].max() <= 1e-10
    assert max(np.abs(ref["ux"] - got["ux"]).max(), np.abs(ref["uy"] - got["uy"]).max()) <= 1e-10


def test_walls_fp32_against_oracle(ddcc):
    prm, walls, C0 = _channel(61, 40, 3, seed=3)
    ref, psi = _ref(prm, walls, C0, 150)
    sim = ddcc.Sim(prm, None, C0, walls=walls, precision=ddcc.DDCC_FP32)
    sim.step(150)
    got = sim.fields()
    sim.close()
    assert np.abs(ref["C"] - got["C"])[:, psi >= 0.5].max() <= 1e-4


def test_flat_second_wall_matches_single_solid(ddcc):
    prm, walls, C0 = _channel(48, 36, 3, seed=9)
    psi1, cos1 = walls[0]
    out = []
    for kw in (dict(walls=[(psi1, cos1), (np.ones_like(psi1), walls[1][1])]),
               dict(psi=psi1, cos_theta_field=cos1)):
        psi = kw.pop("psi", None)
        sim = ddcc.Sim(prm, psi, C0, precision=ddcc.DDCC_FP64, **kw)
        sim.step(100)
        out.append(sim.fields())
        sim.close()
    for k in ("C", "ux", "uy", "P"):
        assert np.abs(out[0][k] - out[1][k]).max() <= 1e-12, k


@pytest.mark.parametrize("precision", [0, 1])
def test_wavy_channel_runs_and_conserves(ddcc, precision):
    pb = W.config6_wavy_channel()
    sim = ddcc.Sim(pb.params, None, pb.C0, walls=pb.extra["walls"], precision=precision)
    m0 = sim.mass()
    sim.step(2000)
    m1 = sim.mass()
    C = sim.read(ddcc.FIELD_C)
    ux = sim.read(ddcc.FIELD_UX)
    sim.close()
    assert np.isfinite(C).all() and np.isfinite(ux).all()
    assert (np.abs(m1 - m0) / np.abs(m0)).max() <= (1e-13 if precision == 0 else 1e-6)
    assert ux[pb.psi >= 0.5].mean() > 0.0     # the body force drives the channel flow
