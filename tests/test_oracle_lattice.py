"""Pins of the oracle's lattice, collision matrix, equilibria and sources.

Each test checks an oracle function against a fact the paper or the
mathematics fixes independently of how the oracle computes it:
the D2Q9 weights of Sec. 3 (golden values at d0 = 1/3 and their moments),
the orthogonality of the Hermite rows under those weights, the moment
conditions of Eq. B.5a-e on random node states, and the eigenvalues of
Lambda = H^-1 S H.
"""
import json
import math
import os

import pytest
import torch

from oracle import ddcc_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
D0S = [1.0 / 3.0, 0.4, 0.5, 0.3]


def test_weights_golden_d0_third():
    with open(os.path.join(GOLD, "d2q9_weights.json")) as fh:
        gold = json.load(fh)
    w = O.weights(gold["d0"])
    assert torch.allclose(w, torch.tensor(gold["weights"], dtype=O.DT), atol=1e-15)


@pytest.mark.parametrize("d0", D0S)
def test_weight_moments(d0):
    """sum w = 1, sum w c c = d0 I (= cs2 I), sum w cx^2 cy^2 = cs2^2,
    sum w cx^4 = d0 c^2 (the Delta + delta^(4) structure of Eq. B.5d)."""
    w, c = O.weights(d0), O.velocities()
    assert abs(w.sum().item() - 1.0) < 1e-15
    M2 = torch.einsum("p,pa,pb->ab", w, c, c)
    assert torch.allclose(M2, d0 * torch.eye(2, dtype=O.DT), atol=1e-15)
    assert abs((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum().item() - d0 * d0) < 1e-15
    assert abs((w * c[:, 0] ** 4).sum().item() - d0) < 1e-15
    # odd moments vanish
    assert torch.allclose(torch.einsum("p,pa->a", w, c), torch.zeros(2, dtype=O.DT))
    assert abs((w * c[:, 0] ** 3).sum().item()) < 1e-16


@pytest.mark.parametrize("d0", D0S)
def test_hermite_rows_orthogonal(d0):
    """The Hermite rows are orthogonal under omega(d0) with the closed-form
    norms 1, d0, d0, d0(1-d0), d0(1-d0), d0^2, d0^2(1-d0) (x2), d0^2(1-d0)^2."""
    H, w = O.hermite_matrix(d0), O.weights(d0)
    G = H @ torch.diag(w) @ H.T
    e = d0 * (1 - d0)
    norms = torch.tensor([1, d0, d0, e, e, d0 * d0, d0 * e, d0 * e, e * e], dtype=O.DT)
    assert torch.allclose(G, torch.diag(norms), atol=1e-15)


def _rates(seed):
    g = torch.Generator().manual_seed(seed)
    return (0.5 + 1.4 * torch.rand(6, generator=g, dtype=O.DT)).tolist()


@pytest.mark.parametrize("d0", D0S)
def test_collision_B5a(d0):
    """Eq. B.5a: sum_p Lambda_pq = s0, sum_p c_p Lambda_pq = s1 c_q, and the
    second moment relaxes the Hermite rows cc - cs2 I with s21 (diagonal)
    and s22 (off-diagonal) on top of cs2 s0 I."""
    s0, s1, s21, s22, s3, s4 = _rates(7)
    Lam = O.collision_matrix(d0, O.relaxation_vector(s0, s1, s21, s22, s3, s4))
    c = O.velocities()
    cs2 = d0
    assert torch.allclose(Lam.sum(dim=0), torch.full((9,), s0, dtype=O.DT), atol=1e-13)
    for a in range(2):
        lhs = (c[:, a:a + 1] * Lam).sum(dim=0)
        assert torch.allclose(lhs, s1 * c[:, a], atol=1e-13)
    cx, cy = c[:, 0], c[:, 1]
    lhs_xx = (cx[:, None] ** 2 * Lam).sum(dim=0)
    assert torch.allclose(lhs_xx, s21 * (cx ** 2 - cs2) + cs2 * s0, atol=1e-13)
    lhs_xy = ((cx * cy)[:, None] * Lam).sum(dim=0)
    assert torch.allclose(lhs_xy, s22 * cx * cy, atol=1e-13)


@pytest.mark.parametrize("d0", D0S)
def test_collision_spectrum(d0):
    s = [0.9, 1.1, 1.1, 1.3, 1.3, 0.7, 1.6, 1.6, 1.9]
    Lam = O.collision_matrix(d0, s)
    ev = torch.linalg.eigvals(Lam)
    assert torch.allclose(ev.imag, torch.zeros(9, dtype=O.DT), atol=1e-10)
    assert torch.allclose(torch.sort(ev.real).values, torch.sort(torch.tensor(s, dtype=O.DT)).values,
                          atol=1e-10)


def _rand(shape, seed, lo=-1.0, hi=1.0):
    g = torch.Generator().manual_seed(seed)
    return lo + (hi - lo) * torch.rand(shape, generator=g, dtype=O.DT)


@pytest.mark.parametrize("d0", D0S)
def test_f_equilibrium_B5b(d0):
    """Eq. B.5b: sum f^eq = psi C, sum c f^eq = psi C u,
    sum c c f^eq = cs2 eta psi mu I."""
    w, c, cs2 = O.weights(d0), O.velocities(), d0
    shp = (5, 7)
    psiC, psimu = _rand(shp, 1, 0, 1), _rand(shp, 2)
    u = (_rand(shp, 3, -0.1, 0.1), _rand(shp, 4, -0.1, 0.1))
    eta = 0.83
    feq = O.f_equilibrium(psiC, psimu, u, eta, w, cs2)
    assert torch.allclose(feq.sum(0), psiC, atol=1e-14)
    for a in range(2):
        assert torch.allclose(torch.einsum("p,pyx->yx", c[:, a], feq), psiC * u[a], atol=1e-14)
    for a in range(2):
        for b in range(2):
            m = torch.einsum("p,pyx->yx", c[:, a] * c[:, b], feq)
            ref = cs2 * eta * psimu if a == b else torch.zeros_like(psimu)
            assert torch.allclose(m, ref, atol=1e-14)


@pytest.mark.parametrize("d0", D0S)
def test_f_source_B5c(d0):
    """Eq. B.5c: sum F = 0, sum c F = V."""
    w, c, cs2 = O.weights(d0), O.velocities(), d0
    V = (_rand((4, 6), 5), _rand((4, 6), 6))
    F = O.f_source(V, w, cs2)
    assert torch.allclose(F.sum(0), torch.zeros(4, 6, dtype=O.DT), atol=1e-15)
    for a in range(2):
        assert torch.allclose(torch.einsum("p,pyx->yx", c[:, a], F), V[a], atol=1e-15)


@pytest.mark.parametrize("d0", D0S)
def test_g_equilibrium_B5d(d0):
    """Eq. B.5d: sum g^eq = rho0, sum c g^eq = psi rho u,
    sum c c g^eq = psi rho u u + psi (m^C u + u m^C)/2 + psi P I,
    sum c c c g^eq = psi rho (cs2 Delta + delta^(4)) . u."""
    w, c, cs2 = O.weights(d0), O.velocities(), d0
    shp = (3, 5)
    psi, rho = _rand(shp, 11, 0.1, 1), _rand(shp, 12, 0.5, 2)
    u = (_rand(shp, 13, -0.1, 0.1), _rand(shp, 14, -0.1, 0.1))
    mC = (_rand(shp, 15, -0.05, 0.05), _rand(shp, 16, -0.05, 0.05))
    psiP = _rand(shp, 17)
    rho0 = 1.7
    s = O.s_vector(psi, rho, u, mC, w, cs2)
    geq = O.g_equilibrium(psiP, s, rho0, w, cs2)
    assert torch.allclose(geq.sum(0), torch.full(shp, rho0, dtype=O.DT), atol=1e-14)
    for a in range(2):
        assert torch.allclose(torch.einsum("p,pyx->yx", c[:, a], geq), psi * rho * u[a], atol=1e-14)
    for a in range(2):
        for b in range(2):
            m = torch.einsum("p,pyx->yx", c[:, a] * c[:, b], geq)
            ref = psi * rho * u[a] * u[b] + 0.5 * (psi * mC[a] * u[b] + psi * u[a] * mC[b])
            if a == b:
                ref = ref + psiP
            assert torch.allclose(m, ref, atol=1e-14)
    # third moment: Delta_abgd u_d cs2 + delta^(4) (c^2 - 3 cs2) for a=b=g
    for a in range(2):
        for b in range(2):
            for g in range(2):
                m = torch.einsum("p,pyx->yx", c[:, a] * c[:, b] * c[:, g], geq)
                ref = torch.zeros(shp, dtype=O.DT)
                for d in range(2):
                    delta = float(a == b) * float(g == d) + float(a == g) * float(b == d) \
                        + float(b == g) * float(a == d)
                    extra = (1.0 - 3.0 * cs2) if (a == b == g == d) else 0.0
                    ref = ref + psi * rho * (cs2 * delta + extra) * u[d]
                assert torch.allclose(m, ref, atol=1e-14)


@pytest.mark.parametrize("d0", D0S)
def test_g_source_B5e(d0):
    """Eq. B.5e: sum G = psi u . grad rho, sum c G = F,
    sum c c G = cs2 psi u . grad rho I + M^{2G}."""
    w, c, cs2 = O.weights(d0), O.velocities(), d0
    shp = (4, 4)
    a0 = _rand(shp, 21)
    F = (_rand(shp, 22), _rand(shp, 23))
    M = (_rand(shp, 24), _rand(shp, 25), _rand(shp, 26))
    G = O.g_source(a0, F, M, w, cs2)
    assert torch.allclose(G.sum(0), a0, atol=1e-14)
    for a in range(2):
        assert torch.allclose(torch.einsum("p,pyx->yx", c[:, a], G), F[a], atol=1e-14)
    Mt = [[M[0], M[2]], [M[2], M[1]]]
    for a in range(2):
        for b in range(2):
            m = torch.einsum("p,pyx->yx", c[:, a] * c[:, b], G)
            ref = Mt[a][b] + (cs2 * a0 if a == b else 0.0)
            assert torch.allclose(m, ref, atol=1e-14)


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4])
def test_rates_from_eq16_eq17(d0):
    """Eq. 16 and Eq. 17 inverted by the oracle give back nu and m0."""
    nu = torch.tensor([0.01, 0.1, 0.3], dtype=O.DT)
    s21, s22 = O.flow_shear_rates(nu, d0)
    assert torch.allclose((1 / s21 - 0.5) * (1 - d0) / 2, nu, atol=1e-15)
    assert torch.allclose((1 / s22 - 0.5) * d0, nu, atol=1e-15)
    prm = {"d0": d0, "m0": 0.07, "eta": [0.8, 1.3]}
    for s1, eta in zip(O.derived_rates(prm), prm["eta"]):
        assert math.isclose((1 / s1 - 0.5) * eta * d0, 0.07, rel_tol=1e-14)
