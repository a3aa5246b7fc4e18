"""Edge and degenerate cases of the GPU path through the C ABI.

* the smallest grids the ABI accepts (3 x 3 and 5 x 4), periodic and
  walled, N = 2..4, FP64 against the oracle element by element (1e-10):
  ghost frames wider than the domain, the plain-load fallback kernels;
* a grid one column narrower / wider than the TMA boxes need (pitch 32 vs
  64), so both the fallback and the fused tile kernel see ragged tiles;
* a fluid at rest with no second phase and psi = 1 stays exactly at rest;
* a single phase filling the whole fluid (C = 1) stays put to round-off.
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


def _small_problem(nx, ny, N, px, py, seed):
    rng = np.random.default_rng(seed)
    psi = rng.uniform(0.2, 1.0, size=(ny, nx))
    C0 = rng.uniform(0.0, 0.9 / (N - 1), size=(N - 1, ny, nx))
    cf = rng.uniform(-0.7, 0.7, size=(N - 1, ny, nx))
    prm = W.base_params(nx, ny, N, periodic_x=px, periodic_y=py, sigma=0.01, width=3.0,
                        tau=0.8, eta=0.5)
    return prm, psi, C0, cf


@pytest.mark.parametrize("nx,ny,N,px,py", [(3, 3, 2, 1, 1), (3, 3, 3, 0, 0), (5, 4, 4, 1, 0),
                                           (4, 5, 3, 0, 1)])
def test_smallest_grids_match_oracle(ddcc, nx, ny, N, px, py):
    prm, psi, C0, cf = _small_problem(nx, ny, N, px, py, seed=nx * 10 + ny + N)
    o = Oracle(prm, psi, C0, None, cf)
    o.step(40)
    ref = o.macroscopic()
    sim = ddcc.Sim(prm, psi, C0, cos_theta_field=cf, precision=ddcc.DDCC_FP64)
    sim.step(40)
    got = sim.fields()
    sim.close()
    assert np.abs(ref["C"].numpy() - got["C"]).max() <= 1e-10
    assert max(np.abs(ref["ux"].numpy() - got["ux"]).max(), np.abs(ref["uy"].numpy() - got["uy"]).max()) <= 1e-10


@pytest.mark.parametrize("nx", [23, 24, 25, 32, 33])
def test_box_width_boundary_matches_oracle(ddcc, nx):
    """pitch = round_up(nx + 8, 32): 32 for nx <= 24 (plain-load tile
    fallback), 64 above (fused TMA tile kernel with a ragged last tile)."""
    pb = W.random_problem(nx, 19, 3, seed=nx, periodic_y=0, theta_field=True, width=6.0)
    o = Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field)
    o.step(60)
    ref = o.macroscopic()
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=ddcc.DDCC_FP64)
    sim.step(60)
    got = sim.fields()
    sim.close()
    fl = pb.psi >= 0.01
    assert np.abs(ref["C"].numpy() - got["C"])[:, fl].max() <= 1e-10
    assert np.abs(ref["ux"].numpy() - got["ux"]).max() <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_fluid_at_rest_stays_at_rest(ddcc, precision):
    nx, ny = 48, 40
    prm = W.base_params(nx, ny, 2, sigma=0.01, width=4.0, tau=0.8)
    psi = np.ones((ny, nx))
    C0 = np.zeros((1, ny, nx))
    sim = ddcc.Sim(prm, psi, C0, cos_theta=np.array([0.3]), precision=precision)
    sim.step(200)
    f = sim.fields()
    sim.close()
    for k in ("ux", "uy", "P"):
        assert np.abs(f[k]).max() == 0.0, k
    assert np.abs(f["C"][0]).max() == 0.0


@pytest.mark.parametrize("precision", [0, 1])
def test_single_phase_filling_the_fluid_stays(ddcc, precision):
    nx, ny = 48, 40
    pb = W.random_problem(nx, ny, 2, seed=3, periodic_y=0, theta_field=False, width=4.0)
    C0 = np.ones((1, ny, nx))
    sim = ddcc.Sim(pb.params, pb.psi, C0, pb.cos_theta, precision=precision)
    m0 = sim.mass()
    sim.step(300)
    f = sim.fields()
    m1 = sim.mass()
    sim.close()
    tol = 1e-12 if precision == 0 else 1e-5
    assert np.abs(f["C"][0] - 1.0)[pb.psi >= 0.01].max() <= tol
    assert max(np.abs(f["ux"]).max(), np.abs(f["uy"]).max()) <= tol
    assert np.abs(m1 - m0).max() / m0.max() <= (1e-14 if precision == 0 else 1e-6)


@pytest.mark.parametrize("N,seed,periodic_y", [(2, 1, 1), (2, 4, 0), (3, 2, 0), (3, 6, 1), (4, 3, 1),
                                               (4, 20, 0)])
def test_random_small_inputs_50_steps(ddcc, N, seed, periodic_y):
    """The brute-force cases of the two oracle transcriptions (every input
    random node by node: psi, fractions, angles, rho, nu, sigma, d0, eta,
    every relaxation rate, a body force): FP64 GPU against the oracle after
    50 steps, populations and lagged fields through the saved state."""
    pb = W.random_small(N, seed, periodic_y=periodic_y)
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field,
                   precision=ddcc.DDCC_FP64)
    sim.step(50)
    got = sim.fields()
    mass = sim.mass()
    sim.close()
    o = Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field)
    o.step(50)
    ref = o.macroscopic()
    for k in ("C", "rho", "ux", "uy", "P", "mu"):
        r = ref[k].numpy()
        err = np.abs(r - got[k]).max()
        assert err <= 1e-10 * max(1.0, np.abs(r).max()), (k, err)
    assert np.allclose(mass, o.mass().numpy(), rtol=1e-13, atol=0)
