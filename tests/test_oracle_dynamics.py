"""Pins of the oracle's whole time step against what the paper fixes.

* Conservation: sum_x psi C_i = sum_x sum_p f^i_p is constant to round-off
  (Eqs. B.5b-c: the collision keeps sum_p f and sum_p F = 0; streaming and
  halfway bounce-back move populations without loss), on periodic and
  walled grids, N = 2..4, with uniform and per-node contact angles.
* Reduction consistency (Sec. 2.1, Table 1): an absent phase stays absent
  and the N-phase run equals the (N-1)-phase run.  Exact to round-off when
  the flow is frozen, and with flow when the absent phase is one of the
  evolved ones; approximate when it is the derived phase C_N.
* Shear-wave decay gives the viscosity of Eq. 16 for both the s21 rows
  (diagonal wave) and the s22 row (axis wave), at d0 = 1/3 and 0.4.
* Laplace law: the pressure jump of a static drop is sigma / R (2D).
* Wetting direction of Eq. 2.14: a drop prescribed 60 deg spreads on the
  wall, 90 deg holds its footprint, 120 deg retracts.
* Mobility of Eq. 17: a small mode around C = 1/2 grows at the linearised
  Cahn-Hilliard rate (m0 / 2) k^2 (2 beta - (3 eps sigma / 4) k^2) within 1%.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import ddcc_oracle as O


def _oracle(pb, **kw):
    return O.Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, **kw)


@pytest.mark.parametrize("nx,ny,N,seed,py,tf,width", [
    (33, 29, 2, 9, 0, True, 4.0),
    (23, 19, 2, 3, 1, False, 4.0),
    (48, 40, 3, 5, 0, True, 6.0),
    (50, 44, 4, 6, 1, True, 6.0),
])
def test_mass_conserved(nx, ny, N, seed, py, tf, width):
    pb = W.random_problem(nx, ny, N, seed=seed, periodic_y=py, theta_field=tf, width=width)
    o = _oracle(pb)
    m0 = o.mass()
    o.step(150)
    m1 = o.mass()
    assert torch.isfinite(o.f).all()
    assert ((m1 - m0).abs() / m0).max().item() < 1e-13
    # C_N is derived, so sum_i C_i = 1 exactly up to rounding
    C = o.macroscopic()["C"]
    assert (C.sum(0) - 1.0).abs().max().item() < 1e-12


def _reduction_pair(frozen, absent):
    p2 = W.config1_droplet_wall(nx=48, ny=40, R=10, wall=8)
    p3 = W.config1_droplet_wall(nx=48, ny=40, R=10, wall=8, nphase=3, absent_phase=absent)
    # the present ambient phase keeps the N = 2 density and viscosity
    p3.params["rho"] = [1.0, 1.0, 1.0]
    o2, o3 = _oracle(p2, frozen_flow=frozen), _oracle(p3, frozen_flow=frozen)
    o2.step(150)
    o3.step(150)
    return o2.macroscopic(), o3.macroscopic()


@pytest.mark.parametrize("absent", [2, 3])
def test_reduction_consistency_frozen_flow(absent):
    a2, a3 = _reduction_pair(True, absent)
    assert (a2["C"][0] - a3["C"][0]).abs().max().item() < 1e-12
    assert a3["C"][absent - 1].abs().max().item() < 1e-12


def test_reduction_consistency_evolved_phase_absent():
    """With flow: phase 2 (evolved) absent; the ternary run reproduces the
    binary run and C_2 stays zero to round-off."""
    a2, a3 = _reduction_pair(False, 2)
    assert (a2["C"][0] - a3["C"][0]).abs().max().item() < 1e-11
    assert (a2["ux"] - a3["ux"]).abs().max().item() < 1e-13
    assert a3["C"][1].abs().max().item() < 1e-13


def test_reduction_consistency_derived_phase_absent():
    """With flow and the derived phase C_3 absent, C_1 + C_2 = 1 holds only
    up to the weak compressibility of the flow LB (div(psi u) != 0 at the
    discrete level): small, and largest in the solid where psi is small."""
    a2, a3 = _reduction_pair(False, 3)
    p = W.config1_droplet_wall(nx=48, ny=40, R=10, wall=8).psi
    fluid = torch.as_tensor(p >= 0.5)
    assert a3["C"][2][fluid].abs().max().item() < 2e-3
    assert (a2["C"][0] - a3["C"][0])[fluid].abs().max().item() < 5e-3


def _shear_decay(d0, diag, L=32, steps=300, nu=0.1, U=1e-3):
    prm = W.base_params(L, L, 2, sigma=0.01, d0=d0)
    prm["nu"] = [nu, nu]
    o = O.Oracle(prm, np.ones((L, L)), np.ones((1, L, L)), np.array([0.0]))
    yy, xx = torch.meshgrid(torch.arange(L, dtype=O.DT), torch.arange(L, dtype=O.DT),
                            indexing="ij")
    k = 2 * math.pi / L
    if diag:
        ph, k2 = k * (xx + yy), 2 * k * k
        ux, uy = U * torch.sin(ph) / math.sqrt(2), -U * torch.sin(ph) / math.sqrt(2)
    else:
        ph, k2 = k * yy, k * k
        ux, uy = U * torch.sin(ph), torch.zeros_like(ph)
    zero = torch.zeros_like(ph)
    s = O.s_vector(o.psi, torch.ones_like(ph), (ux, uy), (zero, zero), o.w, o.cs2)
    o.g = O.g_equilibrium(zero, s, prm["rho0"], o.w, o.cs2)

    def amp():
        return (o.macroscopic()["ux"] * torch.sin(ph)).sum().item()
    a0 = amp()
    o.step(steps)
    return -math.log(amp() / a0) / (k2 * steps)


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4])
@pytest.mark.parametrize("diag", [False, True])
def test_shear_wave_viscosity_eq16(d0, diag):
    nu = _shear_decay(d0, diag)
    assert abs(nu / 0.1 - 1.0) < 0.01


def test_laplace_law():
    """Delta P = sigma / R for a static drop (psi = 1), time-averaged over
    the acoustic oscillation, within 5% (diffuse-interface corrections are
    O(W / R))."""
    L, R, sigma, Wd = 48, 12.0, 0.01, 4.0
    prm = W.base_params(L, L, 2, sigma=sigma, width=Wd)
    yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    r = np.sqrt((xx - L / 2) ** 2 + (yy - L / 2) ** 2)
    o = O.Oracle(prm, np.ones((L, L)), W.drop_profile(r, R, Wd)[None], np.array([0.0]))
    o.step(300)
    vals = []
    inside, outside = r < R - 2 * Wd, r > R + 2 * Wd
    for _ in range(140):
        o.step(5)
        P = o.P.numpy()
        vals.append(P[inside].mean() - P[outside].mean())
    ratio = float(np.mean(vals)) * R / sigma
    assert abs(ratio - 1.0) < 0.05


def test_wetting_direction():
    """Footprint on the first fluid rows after 500 steps: larger for 60 deg,
    unchanged for 90 deg, smaller for 120 deg (Eq. 2.14 sign, reading R11)."""
    out = {}
    for th in (60.0, 90.0, 120.0):
        pb = W.config1_droplet_wall(nx=64, ny=40, R=12, wall=8, theta_deg=th)
        o = _oracle(pb)
        row = 10
        L0 = o.macroscopic()["C"][0][row].sum().item()
        o.step(500)
        out[th] = o.macroscopic()["C"][0][row].sum().item() - L0
    assert out[60.0] > 1.0
    assert abs(out[90.0]) < 0.5
    assert out[120.0] < -1.0


def _ch_growth(prm, L=64, ny=4, steps=1200):
    """Growth rate of a small cos(2 pi x / L) perturbation of C = 1/2 with the
    flow frozen, against the linearised Cahn-Hilliard rate."""
    x = np.arange(L) + 0.0
    k = 2 * math.pi / L
    C0 = (0.5 + 1e-4 * np.cos(k * x))[None, None, :].repeat(ny, axis=1)
    o = O.Oracle(prm, np.ones((ny, L)), C0, np.array([0.0]), frozen_flow=True)

    def amp():
        return float((o.macroscopic()["C"][0].numpy()[0] - 0.5) @ np.cos(k * x))
    o.step(100)
    a0 = amp()
    o.step(steps)
    return math.log(amp() / a0) / steps, k


@pytest.mark.parametrize("width,tau", [(4.0, 0.8), (4.0, 1.0), (6.0, 0.8)])
def test_cahn_hilliard_growth_rate_eq17(width, tau):
    """N = 2, psi = 1, C = 1/2: the flux of phase 1 is M_11 grad mu_1 +
    M_12 grad mu_2 = 2 m0 C1 C2 grad mu_1 (mu_2 = -mu_1) and mu_1 =
    2 beta g'(C) - (3 eps sigma / 4) lap C, so a mode exp(i k x) grows at
    omega = (m0 / 2) k^2 (2 beta - (3 eps sigma / 4) k^2) with g''(1/2) = -1.
    With the stencil's own Laplacian eigenvalue in place of -k^2 the oracle
    matches within 1% for two mobilities (Eq. 17: m0 = (1/s1 - 1/2) eta cs2)
    and two widths (beta = 3 sigma / eps, reading R1)."""
    sigma = 0.01
    prm = W.base_params(64, 4, 2, sigma=sigma, width=width, tau=tau)
    om, k = _ch_growth(prm)
    w, cs2 = O.weights(prm["d0"]).numpy(), prm["d0"]
    lam = sum(2 * w[p] * (math.cos(k * cx) - 1) / cs2 for p, (cx, cy) in enumerate(O.C_VEL) if p)
    pred = (prm["m0"] / 2) * (-lam) * (2 * 3 * sigma / width + 0.75 * width * sigma * lam)
    assert abs(om / pred - 1.0) < 0.01, (om, pred)
