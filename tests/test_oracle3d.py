"""Pins of the three-dimensional oracle (D3Q7 phase / D3Q15 flow lattices)
against facts the paper or the mathematics fixes independently of how the
oracle computes them:

* the weights of Sec. 3 give the textbook D3Q15 set (2/9, 1/9, 1/72) at
  d0 = 1/3 and the textbook D3Q7 set (1/4, 1/8) at d0 = 1/4, and have the
  isotropic moments the Taylor analysis of App. B needs;
* the D3Q15 Hermite rows are orthogonal under those weights (closed-form
  norms); Lambda = H^-1 S H meets Eq. B.5a and has the spectrum S;
* the equilibria and sources meet the moment conditions of Eqs. B.5b-e;
* the rest component of Lambda_g^-1 G - G / 2 reproduces the 3D constants
  K = 1 - 2 d0 and H = K (3 - 7 d0)(s21 - 2) / 2 printed below Eq. 19;
* the stencils are exact on quadratics and have zero total flux;
* a flat tanh interface is stationary up to the stencils' truncation;
* the step conserves sum_x psi C_i to round-off, keeps an absent evolved
  phase absent (reduction consistency) and reproduces the N - 1 phase run;
* shear waves decay at the viscosity of Eq. 16 for the s22 rows (axis
  wave) and the s21 rows (diagonal wave);
* the whole step commutes with a cyclic permutation of the axes and with a
  mirror reflection (catches a wrong sign or index in one component);
* the wetting term of Eq. 2.14 acts in the right direction in 3D (a drop
  on a flat wall spreads at 60 deg and retracts at 120 deg);
* a small mode around C = 1/2 grows at the linearised Cahn-Hilliard rate
  set by the Eq. 17 mobility, beta and kappa (within 1%);
* the linearised bulk flow update with the Eq. 19 pressure: with equal
  rates (BGK) the checkerboard mode k = (pi, pi, pi) has the closed-form
  eigenvalues 1 - s and -1; with the rates of Sec. 4.4 (s0 = 1, s4 = 1.2)
  it grows; with the 3D workloads' s4 = 0.8 no Fourier mode grows.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import ddcc_oracle3d as O

D0S = [1.0 / 3.0, 0.25, 0.4]


def test_weights_textbook_values():
    assert torch.allclose(O.weights15(1.0 / 3.0),
                          torch.tensor([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8, dtype=O.DT), atol=1e-16)
    assert torch.allclose(O.weights7(0.25), torch.tensor([0.25] + [0.125] * 6, dtype=O.DT),
                          atol=1e-16)


@pytest.mark.parametrize("d0", D0S)
def test_weight_moments(d0):
    for w, vel in ((O.weights7(d0), O.C7), (O.weights15(d0), O.C15)):
        c = O.velocities(vel)
        assert abs(w.sum().item() - 1.0) < 1e-15
        M2 = torch.einsum("p,pa,pb->ab", w, c, c)
        assert torch.allclose(M2, d0 * torch.eye(3, dtype=O.DT), atol=1e-15)
        assert torch.allclose(torch.einsum("p,pa->a", w, c), torch.zeros(3, dtype=O.DT))
    w, c = O.weights15(d0), O.velocities(O.C15)
    # fourth moments of the flow lattice: the Delta + delta^(4) structure
    assert abs((w * c[:, 0] ** 4).sum().item() - d0) < 1e-15
    assert abs((w * c[:, 0] ** 2 * c[:, 2] ** 2).sum().item() - d0 * d0) < 1e-15


@pytest.mark.parametrize("d0", D0S)
def test_hermite15_rows_orthogonal(d0):
    H, w = O.hermite15(d0), O.weights15(d0)
    G = H @ torch.diag(w) @ H.T
    e = d0 * (1 - d0)
    w0 = 1 - 3 * d0 + 2 * d0 * d0
    norms = [1.0] + [d0] * 3 + [e] * 3 + [d0 * d0] * 3 + [d0 * e] * 3 + [d0 * d0, d0 * d0 * w0]
    assert torch.allclose(G, torch.diag(torch.tensor(norms, dtype=O.DT)), atol=1e-15)


def _rates(seed, n):
    g = torch.Generator().manual_seed(seed)
    return (0.5 + 1.4 * torch.rand(n, generator=g, dtype=O.DT)).tolist()


@pytest.mark.parametrize("d0", D0S)
def test_collision_B5a(d0):
    cs2 = d0
    s0, s1, s21, s22, s3, s4 = _rates(3, 6)
    for H, vel, s in ((O.hermite7(d0), O.C7, O.rates7(s0, s1, s21)),
                      (O.hermite15(d0), O.C15, O.rates15(s0, s1, s21, s22, s3, s4))):
        Lam = O.collision_matrix(H, s)
        c = O.velocities(vel)
        Q = len(vel)
        assert torch.allclose(Lam.sum(dim=0), torch.full((Q,), s0, dtype=O.DT), atol=1e-13)
        for a in range(3):
            assert torch.allclose((c[:, a:a + 1] * Lam).sum(dim=0), s1 * c[:, a], atol=1e-13)
            lhs = (c[:, a:a + 1] ** 2 * Lam).sum(dim=0)
            assert torch.allclose(lhs, s21 * (c[:, a] ** 2 - cs2) + cs2 * s0, atol=1e-13)
        if Q == 15:
            for a, b in O.PAIRS:
                lhs = ((c[:, a] * c[:, b])[:, None] * Lam).sum(dim=0)
                assert torch.allclose(lhs, s22 * c[:, a] * c[:, b], atol=1e-13)


@pytest.mark.parametrize("d0", D0S)
def test_collision_spectrum(d0):
    s = _rates(11, 15)
    r15 = O.rates15(s[0], s[1], s[2], s[3], s[4], s[5])
    for H, rr in ((O.hermite7(d0), O.rates7(s[0], s[1], s[2])), (O.hermite15(d0), r15)):
        ev = torch.linalg.eigvals(O.collision_matrix(H, rr))
        assert ev.imag.abs().max().item() < 1e-10
        assert torch.allclose(torch.sort(ev.real).values,
                              torch.sort(torch.tensor(rr, dtype=O.DT)).values, atol=1e-10)


def _rand(shape, seed, lo=-1.0, hi=1.0):
    g = torch.Generator().manual_seed(seed)
    return lo + (hi - lo) * torch.rand(shape, generator=g, dtype=O.DT)


def _mom(vel, idx, v):
    """sum_p prod_{a in idx} c_pa v_p."""
    c = O.velocities(vel)
    k = torch.ones(len(vel), dtype=O.DT)
    for a in idx:
        k = k * c[:, a]
    return torch.einsum("p,p...->...", k, v)


@pytest.mark.parametrize("d0", D0S)
def test_f_equilibrium_and_source_B5bc(d0):
    w, cs2 = O.weights7(d0), d0
    shp = (3, 4, 5)
    psiC, psimu = _rand(shp, 1, 0, 1), _rand(shp, 2)
    u = tuple(_rand(shp, 3 + a, -0.1, 0.1) for a in range(3))
    eta = 0.77
    feq = O.f_equilibrium(psiC, psimu, u, eta, w, cs2)
    assert torch.allclose(feq.sum(0), psiC, atol=1e-14)
    for a in range(3):
        assert torch.allclose(_mom(O.C7, [a], feq), psiC * u[a], atol=1e-14)
        for b in range(3):
            ref = cs2 * eta * psimu if a == b else torch.zeros(shp, dtype=O.DT)
            assert torch.allclose(_mom(O.C7, [a, b], feq), ref, atol=1e-14)
    V = tuple(_rand(shp, 9 + a) for a in range(3))
    F = O.f_source(V, w, cs2)
    assert F.sum(0).abs().max().item() < 1e-15
    for a in range(3):
        assert torch.allclose(_mom(O.C7, [a], F), V[a], atol=1e-15)


@pytest.mark.parametrize("d0", D0S)
def test_g_equilibrium_B5d(d0):
    w, cs2 = O.weights15(d0), d0
    shp = (2, 3, 4)
    psi, rho = _rand(shp, 11, 0.1, 1), _rand(shp, 12, 0.5, 2)
    u = tuple(_rand(shp, 13 + a, -0.1, 0.1) for a in range(3))
    mC = tuple(_rand(shp, 17 + a, -0.05, 0.05) for a in range(3))
    psiP, rho0 = _rand(shp, 21), 1.3
    geq = O.g_equilibrium(psiP, O.s_vector(psi, rho, u, mC, w, cs2), rho0, w, cs2)
    assert torch.allclose(geq.sum(0), torch.full(shp, rho0, dtype=O.DT), atol=1e-14)
    for a in range(3):
        assert torch.allclose(_mom(O.C15, [a], geq), psi * rho * u[a], atol=1e-14)
        for b in range(3):
            ref = psi * rho * u[a] * u[b] + 0.5 * (psi * mC[a] * u[b] + psi * u[a] * mC[b])
            if a == b:
                ref = ref + psiP
            assert torch.allclose(_mom(O.C15, [a, b], geq), ref, atol=1e-14)
            for g in range(3):
                ref = torch.zeros(shp, dtype=O.DT)
                for d in range(3):
                    delta = float(a == b) * float(g == d) + float(a == g) * float(b == d) \
                        + float(b == g) * float(a == d)
                    extra = (1.0 - 3.0 * cs2) if a == b == g == d else 0.0
                    ref = ref + psi * rho * (cs2 * delta + extra) * u[d]
                assert torch.allclose(_mom(O.C15, [a, b, g], geq), ref, atol=1e-14)


@pytest.mark.parametrize("d0", D0S)
def test_g_source_B5e(d0):
    w, cs2 = O.weights15(d0), d0
    shp = (2, 2, 3)
    a0 = _rand(shp, 31)
    F = tuple(_rand(shp, 32 + a) for a in range(3))
    M = [_rand(shp, 40 + k) for k in range(6)]
    G = O.g_source(a0, F, M, w, cs2)
    assert torch.allclose(G.sum(0), a0, atol=1e-14)
    full = {(0, 0): M[0], (1, 1): M[1], (2, 2): M[2]}
    for k, (a, b) in enumerate(O.PAIRS):
        full[(a, b)] = full[(b, a)] = M[3 + k]
    for a in range(3):
        assert torch.allclose(_mom(O.C15, [a], G), F[a], atol=1e-14)
        for b in range(3):
            ref = full[(a, b)] + (cs2 * a0 if a == b else 0.0)
            assert torch.allclose(_mom(O.C15, [a, b], G), ref, atol=1e-14)


@pytest.mark.parametrize("d0", D0S)
def test_pressure_constants_from_collision_matrix(d0):
    """App. C: the rest component of Lambda_g^-1 G - G / 2 for the force
    term G of Eq. 3.10 (with M^{2G} at d_t T = 0) is
    [K (1 - d0)(2 - s0) / (2 s0)] psi u . grad rho + (H / s21) u . grad(psi rho)
    with the 3D K and H printed below Eq. 19."""
    w, cs2 = O.weights15(d0), d0
    s0, s1, s21, s22, s3, s4 = _rates(5, 6)
    Lam = O.collision_matrix(O.hermite15(d0), O.rates15(s0, s1, s21, s22, s3, s4))
    shp = (5,)
    a0 = _rand(shp, 51)
    F = tuple(_rand(shp, 52 + a) for a in range(3))
    u = [_rand(shp, 55 + a, -0.1, 0.1) for a in range(3)]
    gpr = [_rand(shp, 58 + a) for a in range(3)]
    ugpr = u[0] * gpr[0] + u[1] * gpr[1] + u[2] * gpr[2]
    M = [2 * cs2 * u[a] * gpr[a] + (1 - 3 * cs2) * ugpr for a in range(3)]
    M += [cs2 * (u[a] * gpr[b] + gpr[a] * u[b]) for (a, b) in O.PAIRS]
    G = O.g_source(a0, F, M, w, cs2)
    rest = (torch.linalg.inv(Lam) @ G)[0] - 0.5 * G[0]
    K, Hc = O.pressure_constants(d0, s21)
    ref = K * (1 - d0) * (2 - s0) / (2 * s0) * a0 + Hc / s21 * ugpr
    assert torch.allclose(rest, ref, atol=1e-13)
    # K itself: minus the rest component of the dual of a diagonal
    # second-order row
    assert abs(-torch.linalg.inv(O.hermite15(d0))[0, 4].item() - K) < 1e-14


def _poly3(shape):
    z, y, x = torch.meshgrid(*(torch.arange(n, dtype=O.DT) for n in shape), indexing="ij")
    return x, y, z


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.25])
def test_stencils_exact_on_quadratics(d0):
    shape = (7, 8, 9)
    w, cs2 = O.weights15(d0), d0
    x, y, z = _poly3(shape)
    chi = 0.3 + 1.7 * x - 0.4 * y + 0.9 * z + 0.25 * x * x - 0.6 * x * y + 0.11 * y * y \
        + 0.2 * y * z - 0.35 * z * z + 0.15 * x * z
    g = O.grad(chi, w, cs2)
    ref = (1.7 + 0.5 * x - 0.6 * y + 0.15 * z, -0.4 - 0.6 * x + 0.22 * y + 0.2 * z,
           0.9 + 0.2 * y - 0.7 * z + 0.15 * x)
    inner = (slice(1, -1),) * 3
    for a in range(3):
        assert torch.allclose(g[a][inner], ref[a][inner], atol=1e-12)
    psi = 0.5 + 0.03 * x - 0.02 * y + 0.01 * z
    C = 0.1 * x * x + 0.07 * x * y - 0.05 * y * y + 0.2 * x + 0.04 * z * z - 0.03 * y * z
    out = O.div_psi_grad(psi, C, w, cs2)
    Cx, Cy, Cz = 0.2 * x + 0.07 * y + 0.2, 0.07 * x - 0.1 * y - 0.03 * z, 0.08 * z - 0.03 * y
    lap = 0.2 - 0.1 + 0.08
    ref = 0.03 * Cx - 0.02 * Cy + 0.01 * Cz + psi * lap
    assert torch.allclose(out[inner], ref[inner], atol=1e-12)


def test_div_psi_grad_zero_total_flux():
    g = torch.Generator().manual_seed(4)
    psi = 0.2 + 0.8 * torch.rand(6, 7, 5, generator=g, dtype=O.DT)
    C = torch.rand(6, 7, 5, generator=g, dtype=O.DT)
    assert abs(O.div_psi_grad(psi, C, O.weights15(1 / 3), 1 / 3).sum().item()) < 1e-13


def _flat_residual(width):
    nx, sigma = 256, 0.01
    x = torch.arange(nx, dtype=O.DT)
    c = 0.5 * (torch.tanh(2 * (x - nx / 4) / width) - torch.tanh(2 * (x - 3 * nx / 4) / width))
    C1 = c[None, None, :].repeat(2, 3, 1)
    psi = torch.ones_like(C1)
    prm = {"sigma": [[0, sigma], [sigma, 0]], "width": width}
    cp = O.pair_cosines([torch.full_like(psi, 0.3)], prm["sigma"])
    _, mu, _ = O.chemical_potentials([C1, 1 - C1], psi, cp, prm, O.weights15(1 / 3), 1 / 3)
    bulk_max = (2 * 3 * sigma / width * O.g_prime(C1).abs()).max().item()
    return mu[0].abs().max().item() / bulk_max


def test_flat_interface_stationary():
    """A tanh(2x / epsilon) profile is the equilibrium of Eq. 2.1 (with
    beta = 3 sigma / epsilon): mu ~ 0 up to second-order truncation."""
    r8, r16 = _flat_residual(8.0), _flat_residual(16.0)
    assert r8 < (4 / 8.0) ** 2 / 6 and r16 < (4 / 16.0) ** 2 / 6
    assert 3.0 < r8 / r16 < 5.0


def _oracle(pb, **kw):
    return O.Oracle3D(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, **kw)


@pytest.mark.parametrize("shape,N,seed,tf", [((9, 10, 11), 2, 1, True), ((8, 12, 10), 3, 2, False),
                                             ((10, 9, 12), 4, 3, True)])
def test_mass_conserved(shape, N, seed, tf):
    nz, ny, nx = shape
    pb = W.random_problem_3d(nx, ny, nz, N, seed=seed, theta_field=tf)
    o = _oracle(pb)
    m0 = o.mass()
    o.step(40)
    m1 = o.mass()
    assert torch.isfinite(o.f).all() and torch.isfinite(o.g).all()
    assert ((m1 - m0).abs() / m0).max().item() < 1e-13
    assert (o.macroscopic()["C"].sum(0) - 1.0).abs().max().item() < 1e-12


def test_reduction_evolved_phase_absent():
    """Three phases with phase 2 (evolved) absent reproduce the two-phase
    run with flow: phase 3 takes the role of the binary's phase 2 (same
    density, viscosity, sigma_13 = sigma_12, theta_13 = theta_12).  With
    sigma_12 = sigma_23 the absent phase's chemical potential vanishes
    identically, so its distributions stay exactly at rest."""
    nz, ny, nx = 10, 11, 12
    pb = W.random_problem_3d(nx, ny, nz, 2, seed=7)
    p2 = pb.params
    p3 = W.base_params_3d(nx, ny, nz, 3, width=p2["width"])
    s12 = p2["sigma"][0][1]
    p3["sigma"] = [[0.0, 0.011, s12], [0.011, 0.0, 0.011], [s12, 0.011, 0.0]]
    p3["rho"] = [p2["rho"][0], 0.7, p2["rho"][1]]
    p3["nu"] = [p2["nu"][0], 0.12, p2["nu"][1]]
    p3["eta"] = [p2["eta"][0], 0.9]
    p3["m0"] = p2["m0"]
    C3 = np.concatenate([pb.C0, np.zeros_like(pb.C0)])
    o2 = O.Oracle3D(p2, pb.psi, pb.C0, pb.cos_theta)
    o3 = O.Oracle3D(p3, pb.psi, C3, np.array([pb.cos_theta[0], -0.4]))
    o2.step(30)
    o3.step(30)
    a2, a3 = o2.macroscopic(), o3.macroscopic()
    assert (a2["C"][0] - a3["C"][0]).abs().max().item() < 1e-11
    assert a3["C"][1].abs().max().item() < 1e-13
    for k in ("ux", "uy", "uz"):
        assert (a2[k] - a3[k]).abs().max().item() < 1e-13


def _shear_decay(d0, mode, L=32, steps=300, nu=0.1, U=1e-3):
    shape = {"y": (1, L, 1), "z": (L, 1, 1), "xy": (1, L, L), "yz": (L, L, 1)}[mode]
    nz, ny, nx = shape
    prm = W.base_params_3d(nx, ny, nz, 2, d0=d0)
    prm["nu"] = [nu, nu]
    o = O.Oracle3D(prm, np.ones(shape), np.ones((1,) + shape), np.array([0.0]))
    x, y, z = _poly3(shape)
    k = 2 * math.pi / L
    zero = torch.zeros(shape, dtype=O.DT)
    if mode == "y":          # u_x(y): the s22 row xy
        ph, k2, u, comp, sgn = k * y, k * k, None, 0, 1.0
        u = (U * torch.sin(ph), zero, zero)
    elif mode == "z":        # u_y(z): the s22 row yz
        ph, k2, comp, sgn = k * z, k * k, 1, 1.0
        u = (zero, U * torch.sin(ph), zero)
    elif mode == "xy":       # diagonal wave: the s21 rows
        ph, k2, comp, sgn = k * (x + y), 2 * k * k, 0, 1.0
        u = (U * torch.sin(ph) / math.sqrt(2), -U * torch.sin(ph) / math.sqrt(2), zero)
    else:
        ph, k2, comp, sgn = k * (y + z), 2 * k * k, 1, 1.0
        u = (zero, U * torch.sin(ph) / math.sqrt(2), -U * torch.sin(ph) / math.sqrt(2))
    s = O.s_vector(o.psi, torch.ones(shape, dtype=O.DT), u, (zero, zero, zero), o.w15, o.cs2)
    o.g = O.g_equilibrium(zero, s, prm["rho0"], o.w15, o.cs2)
    key = ("ux", "uy", "uz")[comp]

    def amp():
        return sgn * (o.macroscopic()[key] * torch.sin(ph)).sum().item()
    a0 = amp()
    o.step(steps)
    return -math.log(amp() / a0) / (k2 * steps)


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.25])
@pytest.mark.parametrize("mode", ["y", "z", "xy", "yz"])
def test_shear_wave_viscosity_eq16(d0, mode):
    assert abs(_shear_decay(d0, mode) / 0.1 - 1.0) < 0.01


def _run(pb, steps):
    o = _oracle(pb)
    o.step(steps)
    return o.macroscopic()


def test_axis_permutation_symmetry():
    """(x, y, z) -> (y, z, x): the step commutes with the cyclic rotation of
    the axes; velocity components rotate with it."""
    nz, ny, nx = 7, 8, 9
    pb = W.random_problem_3d(nx, ny, nz, 3, seed=12, theta_field=True)
    a = _run(pb, 12)
    rot = lambda arr: np.ascontiguousarray(np.asarray(arr).transpose(
        tuple(range(np.ndim(arr) - 3)) + tuple(np.ndim(arr) - 3 + k for k in (1, 2, 0))))
    p2 = dict(pb.params)
    p2["nz"], p2["ny"], p2["nx"] = ny, nx, nz
    pr = W.Problem("rot", p2, rot(pb.psi), rot(pb.C0), pb.cos_theta, rot(pb.cos_theta_field))
    b = _run(pr, 12)
    assert (b["C"] - torch.as_tensor(rot(a["C"].numpy()))).abs().max().item() < 1e-12
    # new (x', y', z') = (z, x, y) in old axes
    for new, old in (("ux", "uz"), ("uy", "ux"), ("uz", "uy")):
        assert (b[new] - torch.as_tensor(rot(a[old].numpy()))).abs().max().item() < 1e-13
    assert (b["P"] - torch.as_tensor(rot(a["P"].numpy()))).abs().max().item() < 1e-13


def test_mirror_symmetry():
    """x -> -x (periodic): C and P mirror, u_x changes sign."""
    nz, ny, nx = 7, 8, 9
    pb = W.random_problem_3d(nx, ny, nz, 2, seed=13, theta_field=True)
    a = _run(pb, 12)
    flip = lambda arr: np.ascontiguousarray(np.roll(np.flip(np.asarray(arr), -1), 1, -1))
    pr = W.Problem("mir", pb.params, flip(pb.psi), flip(pb.C0), pb.cos_theta,
                   flip(pb.cos_theta_field))
    b = _run(pr, 12)
    assert (b["C"] - torch.as_tensor(flip(a["C"].numpy()))).abs().max().item() < 1e-12
    assert (b["ux"] + torch.as_tensor(flip(a["ux"].numpy()))).abs().max().item() < 1e-13
    for k in ("uy", "uz", "P"):
        assert (b[k] - torch.as_tensor(flip(a[k].numpy()))).abs().max().item() < 1e-13


def _bulk_update(d0, s, k):
    """Linearised flow update at rest (psi = rho = 1) for the Fourier mode
    k: g -> shift(k) (g - Lambda (g - g^eq(P(g), J(g)))), with P from the
    moving populations as in Eq. 19."""
    w, cs2 = O.weights15(d0).numpy(), d0
    c = O.velocities(O.C15).numpy()
    Lam = O.collision_matrix(O.hermite15(d0), s).numpy()
    E = np.zeros((15, 15))
    for j in range(15):
        g = np.zeros(15)
        g[j] = 1.0
        P = cs2 / (1 - w[0]) * g[1:].sum()
        geq = w * P / cs2 + w * (c @ (c.T @ g)) / cs2
        geq[0] = (w[0] - 1) * P / cs2
        E[:, j] = geq
    return np.exp(-1j * (c @ np.asarray(k)))[:, None] * (np.eye(15) - Lam @ (np.eye(15) - E))


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4])
def test_checkerboard_mode_bgk_closed_form(d0):
    s = 1.3
    ev = np.linalg.eigvals(_bulk_update(d0, [s] * 15, (math.pi,) * 3))
    # on the symmetric (rest, moving) pair: eigenvalues 1 - s and -1
    assert np.abs(np.abs(ev).max() - 1.0) < 1e-12
    assert np.min(np.abs(ev - (1 - s))) < 1e-12 and np.min(np.abs(ev + 1.0)) < 1e-12


def _rates_from_params(prm, nu=0.1):
    d0 = prm["d0"]
    s21, s22 = O.flow_shear_rates(nu, d0)
    sg = prm["s_g"]
    return O.rates15(sg[0], sg[1], s21, s22, sg[2], sg[3])


def test_checkerboard_mode_paper_rates_grow():
    prm = W.base_params_3d(8, 8, 8, 2, d0=0.4)
    prm["s_g"] = [1.0, 1.2, 1.2, 1.2]
    ev = np.linalg.eigvals(_bulk_update(0.4, _rates_from_params(prm), (math.pi,) * 3))
    assert np.abs(ev).max() > 1.3


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4])
def test_workload_rates_linearly_stable(d0):
    prm = W.base_params_3d(8, 8, 8, 2, d0=d0)
    s = _rates_from_params(prm)
    ks = np.linspace(0.0, math.pi, 7)
    worst = max(np.abs(np.linalg.eigvals(_bulk_update(d0, s, (a, b, c)))).max()
                for a in ks for b in ks for c in ks)
    assert worst <= 1.0 + 1e-12


def test_wetting_direction_3d():
    """Eq. 2.14's wetting term in 3D: a hemispherical drop on a flat wall
    (psi from the distance to the floor and ceiling planes) prescribed
    60 deg spreads its footprint on the first fluid layer, 120 deg shrinks
    it (theta measured inside the drop, as in 2D)."""
    nx, ny, nz = 28, 18, 28
    x, y, z = np.meshgrid(np.arange(nx) + 0.0, np.arange(ny) + 0.0, np.arange(nz) + 0.0, indexing="xy")
    x, y, z = (np.transpose(a, (2, 0, 1)) for a in (x, y, z))      # (nz, ny, nx)
    yw = 4.0
    psi = W.psi_from_distance(np.minimum(y - yw, ny - 1 - yw - y))
    r = np.sqrt((x - nx / 2 + 0.3) ** 2 + (y - yw) ** 2 + (z - nz / 2 + 0.2) ** 2)
    C0 = W.drop_profile(r, 8.0, 4.0)[None]
    prm = W.base_params_3d(nx, ny, nz, 2, sigma=0.01, width=4.0)
    layer = int(yw) + 1

    def footprint(theta):
        o = O.Oracle3D(prm, psi, C0, np.array([math.cos(math.radians(theta))]))
        a0 = (o.macroscopic()["C"][0].numpy()[:, layer, :] > 0.5).sum()
        o.step(300)
        return (o.macroscopic()["C"][0].numpy()[:, layer, :] > 0.5).sum() - a0
    spread60, spread120 = footprint(60.0), footprint(120.0)
    assert spread60 > 0 > spread120, (spread60, spread120)


@pytest.mark.parametrize("d0,tau", [(1.0 / 3.0, 0.8), (0.4, 1.0)])
def test_cahn_hilliard_growth_rate_eq17(d0, tau):
    """The linearised Cahn-Hilliard growth of a small cos(2 pi x / L)
    perturbation of C = 1/2 (N = 2, psi = 1, flow frozen) on the D3Q7 phase
    lattice: omega = (m0 / 2) k^2 (2 beta - (3 eps sigma / 4) k^2), with the
    D3Q15 stencil's Laplacian eigenvalue for -k^2, within 1% (Eq. 17, and
    at d0 = 0.4 where the D3Q7 rest weight is negative)."""
    L, sigma, width = 64, 0.01, 4.0
    prm = W.base_params_3d(L, 1, 1, 2, sigma=sigma, width=width, tau=tau, d0=d0)
    x = np.arange(L) + 0.0
    k = 2 * math.pi / L
    C0 = (0.5 + 1e-4 * np.cos(k * x))[None, None, None, :]
    o = O.Oracle3D(prm, np.ones((1, 1, L)), C0, np.array([0.0]), frozen_flow=True)

    def amp():
        return float((o.macroscopic()["C"][0].numpy()[0, 0] - 0.5) @ np.cos(k * x))
    o.step(100)
    a0 = amp()
    o.step(1200)
    om = math.log(amp() / a0) / 1200
    w = O.weights15(d0).numpy()
    lam = sum(2 * w[p] * (math.cos(k * c[0]) - 1) / d0 for p, c in enumerate(O.C15) if p)
    pred = (prm["m0"] / 2) * (-lam) * (2 * 3 * sigma / width + 0.75 * width * sigma * lam)
    assert abs(om / pred - 1.0) < 0.01, (om, pred)
