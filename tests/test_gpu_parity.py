"""GPU parity: the sm_103a path through the C ABI against the FP64 oracle.

Bars (element by element on the same seeded inputs):
  FP64: max |dC_i| <= 1e-10 on nodes with psi >= 0.01, max psi |dC_i| <=
        1e-10 everywhere, max |d rho| <= 1e-10 (psi >= 0.01), max |du| <=
        1e-10 everywhere, after the stated number of steps.
  FP32: max |dC_i| <= 1e-4 on nodes with psi >= 0.5 (stated FP32 error).
Cases span several 32 x 8 tiles with ragged tails, periodic and walled axes,
N = 2, 3, 4, uniform and per-node contact angles, d0 != 1/3 and a body force.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import Oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32_C = 1e-4


@pytest.fixture(scope="module")
def ddcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10314_gb300 import build as B
    B.build()
    import paper_2311_10314_gb300 as D
    return D


def _oracle_fields(pb, steps):
    o = Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field)
    o.step(steps)
    m = o.macroscopic()
    out = {k: v.numpy() for k, v in m.items()}
    out["mass"] = o.mass().numpy()
    return out


def _gpu_fields(D, pb, steps, precision, path="tile"):
    sim = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision,
                path=path)
    sim.step(steps)
    out = sim.fields()
    out["mass"] = sim.mass()
    sim.close()
    return out


def _errors(pb, ref, got):
    psi = pb.psi
    fl = psi >= 0.01
    dC = np.abs(ref["C"] - got["C"])
    return dict(
        C=float(dC[:, fl].max()),
        C_psi=float((psi[None] * dC).max()),
        rho=float(np.abs(ref["rho"] - got["rho"])[fl].max()),
        u=float(max(np.abs(ref["ux"] - got["ux"]).max(), np.abs(ref["uy"] - got["uy"]).max())),
        psiP=float((psi * np.abs(ref["P"] - got["P"])).max()),
        mass=float((np.abs(ref["mass"] - got["mass"]) / np.abs(ref["mass"])).max()),
    )


CASES = [
    # (nx, ny, N, seed, periodic_y, theta_field, width, steps)
    (37, 23, 2, 3, 1, False, 4.0, 200),
    (33, 29, 2, 9, 0, True, 4.0, 200),
    (48, 40, 3, 5, 0, True, 6.0, 200),
    (61, 37, 3, 7, 1, False, 6.0, 200),
    (50, 44, 4, 6, 1, True, 6.0, 150),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d_N%d_s%d" % c[:4])
def test_fp64_parity_random(ddcc, case):
    nx, ny, N, seed, py, tf, width, steps = case
    pb = W.random_problem(nx, ny, N, seed=seed, periodic_y=py, theta_field=tf, width=width)
    ref = _oracle_fields(pb, steps)
    got = _gpu_fields(ddcc, pb, steps, ddcc.DDCC_FP64)
    e = _errors(pb, ref, got)
    assert e["C"] <= TOL64 and e["C_psi"] <= TOL64, e
    assert e["rho"] <= TOL64 and e["u"] <= TOL64, e
    assert e["mass"] <= 1e-13, e


def test_fp64_parity_walled_box_d0_body_force(ddcc):
    """Both axes walled, d0 = 0.4 (s21 != s22), a body force, N = 3."""
    pb = W.random_problem(45, 38, 3, seed=11, periodic_x=0, periodic_y=0, theta_field=True,
                          width=6.0, d0=0.4, body_force=(2e-5, -1e-5))
    ref = _oracle_fields(pb, 150)
    got = _gpu_fields(ddcc, pb, 150, ddcc.DDCC_FP64)
    e = _errors(pb, ref, got)
    assert e["C"] <= TOL64 and e["C_psi"] <= TOL64 and e["rho"] <= TOL64 and e["u"] <= TOL64, e


def test_fp64_initial_state(ddcc):
    pb = W.random_problem(40, 27, 4, seed=2, periodic_y=0, theta_field=True, width=6.0)
    ref = _oracle_fields(pb, 0)
    got = _gpu_fields(ddcc, pb, 0, ddcc.DDCC_FP64)
    e = _errors(pb, ref, got)
    assert max(e["C"], e["rho"], e["u"], e["psiP"]) <= 1e-13, e
    assert np.abs(ref["mu"] - got["mu"])[:, pb.psi >= 0.01].max() <= 1e-12


@pytest.fixture(scope="module")
def droplet_ref():
    pb = W.config1_droplet_wall()
    return pb, _oracle_fields(pb, 1000)


@pytest.mark.parametrize("path", ["tile", "sweep"])
def test_fp64_parity_droplet_wall_1000_steps(ddcc, droplet_ref, path):
    """The 64 x 64 semicircular droplet on a psi-embedded wall, 1000 steps:
    the stated FP64 bar (1e-10 in C, rho and u), through both step paths."""
    pb, ref = droplet_ref
    got = _gpu_fields(ddcc, pb, 1000, ddcc.DDCC_FP64, path=path)
    e = _errors(pb, ref, got)
    assert e["C"] <= TOL64 and e["C_psi"] <= TOL64 and e["rho"] <= TOL64 and e["u"] <= TOL64, e


def test_fp64_parity_lens(ddcc):
    pb = W.config2_lens(nx=96, ny=96)
    ref = _oracle_fields(pb, 300)
    got = _gpu_fields(ddcc, pb, 300, ddcc.DDCC_FP64)
    e = _errors(pb, ref, got)
    assert e["C"] <= TOL64 and e["C_psi"] <= TOL64 and e["rho"] <= TOL64 and e["u"] <= TOL64, e


@pytest.mark.parametrize("path", ["tile", "sweep"])
def test_fp32_against_oracle_droplet_wall(ddcc, droplet_ref, path):
    pb, ref = droplet_ref
    got = _gpu_fields(ddcc, pb, 1000, ddcc.DDCC_FP32, path=path)
    bulk = pb.psi >= 0.5
    err = np.abs(ref["C"] - got["C"])[:, bulk].max()
    assert err <= TOL32_C, err
    assert np.abs(ref["ux"] - got["ux"]).max() <= 1e-5


def test_fp32_against_oracle_random_n4(ddcc):
    pb = W.random_problem(50, 44, 4, seed=6, periodic_y=1, theta_field=True, width=6.0)
    ref = _oracle_fields(pb, 150)
    got = _gpu_fields(ddcc, pb, 150, ddcc.DDCC_FP32)
    bulk = pb.psi >= 0.5
    err = np.abs(ref["C"] - got["C"])[:, bulk].max()
    assert err <= TOL32_C, err


@pytest.mark.parametrize("precision", [0, 1])
def test_mass_conserved_on_gpu(ddcc, precision):
    pb = W.random_problem(70, 45, 3, seed=4, periodic_y=0, theta_field=True, width=6.0)
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision)
    m0 = sim.mass()
    sim.step(500)
    m1 = sim.mass()
    drift = np.abs(m1 - m0) / np.abs(m0)
    assert drift.max() <= (1e-13 if precision == 0 else 1e-6), drift
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_save_load_resumes_bit_exact(ddcc, precision):
    pb = W.random_problem(41, 35, 3, seed=8, periodic_y=0, theta_field=False, width=6.0)
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, precision=precision)
    sim.step(20)
    buf = sim.save_state()
    host = buf.cpu()
    sim.step(30)
    a = sim.fields()
    sim.load_state(buf)
    assert sim.steps == 20
    sim.step(30)
    b = sim.fields()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    sim.load_state(host)
    sim.step(30)
    c = sim.fields()
    for k in a:
        assert np.array_equal(a[k], c[k]), k
    sim.close()


def test_full_size_imbibition_fp32_properties(ddcc):
    """The 4096^2, N = 4 porous-imbibition workload in the launch
    configuration the benchmark times: finite, sum_i C_i = 1, and the FP64
    mass reduction conserved to FP32 round-off."""
    pb = W.config4_imbibition()
    sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field,
                   precision=ddcc.DDCC_FP32)
    m0 = sim.mass()
    sim.step(20)
    m1 = sim.mass()
    assert (np.abs(m1 - m0) / m0).max() <= 1e-6
    C = np.stack([sim.read(ddcc._lib.FIELD_C + i) for i in range(3)])
    assert np.isfinite(C).all()
    sim.close()


SWEEP_CASES = [
    # (nx, ny, N, seed, periodic_x, periodic_y, theta_field, width, precision)
    (70, 45, 3, 4, 1, 0, True, 6.0, 0),
    (96, 40, 4, 13, 1, 1, True, 6.0, 0),
    (67, 53, 2, 14, 0, 0, False, 4.0, 0),
    (130, 37, 3, 15, 0, 1, True, 6.0, 0),
    (70, 45, 3, 4, 1, 0, True, 6.0, 1),
    (150, 66, 4, 16, 1, 1, True, 6.0, 1),
]


@pytest.mark.parametrize("case", SWEEP_CASES, ids=lambda c: "%dx%d_N%d_p%d%d_fp%d" % (
    c[0], c[1], c[2], c[4], c[5], 64 if c[8] == 0 else 32))
def test_sweep_matches_tile_kernel(ddcc, case):
    """The TMA row-sweep step and the tile step compute the same update
    (FP64: to round-off; FP32: to FP32 round-off) over 60 steps, on
    periodic and walled axes, with uniform and per-node angles."""
    nx, ny, N, seed, px, py, tf, width, prec = case
    pb = W.random_problem(nx, ny, N, seed=seed, periodic_x=px, periodic_y=py, theta_field=tf,
                          width=width)
    out = []
    for path in ("sweep", "tile"):
        sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field,
                       precision=prec, path=path)
        assert sim.path == path
        sim.step(60)
        out.append(sim.fields())
        sim.close()
    tol = 1e-12 if prec == 0 else 2e-5
    for k in ("C", "ux", "uy", "rho"):
        err = np.abs(out[0][k] - out[1][k])
        if k in ("C", "rho"):
            err = err[..., pb.psi >= 0.01]
        assert err.max() <= tol, (k, err.max())


def test_benchmark_workload_paths(ddcc):
    pb = W.config4_imbibition(nx=512, ny=512)
    for prec in (0, 1):
        for path in ("tile", "sweep"):
            sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field,
                           precision=prec, path=path)
            assert sim.path == path
            sim.close()
