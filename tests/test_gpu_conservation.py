"""FP32 phase-mass conservation in steady flows (GPU).

A drop at rest is the hard case for FP32: the rest population carries nearly
all of psi C, so its update rounds at the ulp of psi C with the same error
every step.  The step recovers that rounding error exactly (TwoSum) and
moves it onto a moving population.  Without it the 64^2 wall drop lost
2.6e-6 of its phase mass in 3.3e4 steps (2D) and the 96^3 drop on a sphere
2.9e-4 in 6e4 steps (3D); with it both stay within 1e-8.
"""
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


def test_fp32_mass_of_a_drop_at_rest_2d(D):
    pb = W.config1_droplet_wall()
    sim = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, precision=D.DDCC_FP32)
    m0 = sim.mass()
    sim.step(50000)
    m1 = sim.mass()
    sim.close()
    assert (np.abs(m1 - m0) / m0).max() <= 1e-8


def test_fp32_mass_of_a_drop_at_rest_3d(D):
    pb = W.config9_drop_on_sphere(theta_deg=90.0, L=96, Rs=12.0, R0=24.0)
    sim = D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, precision=D.DDCC_FP32)
    m0 = sim.mass()
    sim.step(30000)
    m1 = sim.mass()
    sim.close()
    assert (np.abs(m1 - m0) / m0).max() <= 1e-8
