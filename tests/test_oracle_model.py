"""Pins of the oracle's stencils, chemical potential and mobility.

* Stencils (reading R7) are exact on polynomials of degree <= 2.
* With mirror ghosts the discrete div(psi grad C) has zero total (no flux
  through an outer wall) and so does it on a periodic grid.
* g'(C) agrees with a central difference of g(C) = C^2 (C - 1)^2.
* A flat tanh(2x/epsilon) interface is stationary: mu vanishes up to the
  stencil's truncation error only with beta_ij = 3 sigma_ij / epsilon
  (reading R1 of Eq. 2.1); the printed inverse form fails.
* For N = 2 the chemical potentials of Eq. 2.14 satisfy mu_1 = -mu_2 at
  every node, for any psi and contact angle: the bulk, gradient and wetting
  terms are each odd under exchanging the phases.
* The mobility of Eq. 2.5 has zero row and column sums.
* Eq. 2.9 returns the prescribed theta_iN for pairs with phase N and is
  antisymmetric in cosine.
"""
import math

import pytest
import torch

from oracle import ddcc_oracle as O


def _poly_fields(nx, ny):
    y, x = torch.meshgrid(torch.arange(ny, dtype=O.DT), torch.arange(nx, dtype=O.DT),
                          indexing="ij")
    return x, y


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4])
def test_gradient_exact_on_quadratics(d0):
    nx, ny = 12, 10
    grid = O.Grid(nx, ny, 0, 0)
    w, cs2 = O.weights(d0), d0
    x, y = _poly_fields(nx, ny)
    chi = 0.3 + 1.7 * x - 0.4 * y + 0.25 * x * x - 0.6 * x * y + 0.11 * y * y
    gx, gy = grid.grad(chi, w, cs2)
    ex = 1.7 + 0.5 * x - 0.6 * y
    ey = -0.4 - 0.6 * x + 0.22 * y
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    assert torch.allclose(gx[inner], ex[inner], atol=1e-12)
    assert torch.allclose(gy[inner], ey[inner], atol=1e-12)


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4])
def test_div_psi_grad_exact(d0):
    """div(psi grad C) = grad psi . grad C + psi lap C for psi linear and
    C quadratic."""
    nx, ny = 11, 9
    grid = O.Grid(nx, ny, 0, 0)
    w, cs2 = O.weights(d0), d0
    x, y = _poly_fields(nx, ny)
    psi = 0.5 + 0.03 * x - 0.02 * y
    C = 0.1 * x * x + 0.07 * x * y - 0.05 * y * y + 0.2 * x
    out = grid.div_psi_grad(psi, C, w, cs2)
    Cx = 0.2 * x + 0.07 * y + 0.2
    Cy = 0.07 * x - 0.1 * y
    ref = 0.03 * Cx - 0.02 * Cy + psi * (0.2 - 0.1)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    assert torch.allclose(out[inner], ref[inner], atol=1e-12)


@pytest.mark.parametrize("px,py", [(1, 1), (1, 0), (0, 0)])
def test_div_psi_grad_zero_total_flux(px, py):
    g = torch.Generator().manual_seed(3)
    nx, ny = 13, 9
    grid = O.Grid(nx, ny, px, py)
    w = O.weights(1 / 3)
    psi = 0.2 + 0.8 * torch.rand(ny, nx, generator=g, dtype=O.DT)
    C = torch.rand(ny, nx, generator=g, dtype=O.DT)
    tot = grid.div_psi_grad(psi, C, w, 1 / 3).sum().item()
    assert abs(tot) < 1e-13


def test_g_prime_matches_difference():
    C = torch.linspace(-0.2, 1.2, 57, dtype=O.DT)
    h = 1e-5
    fd = (O.g_poly(C + h) - O.g_poly(C - h)) / (2 * h)
    assert torch.allclose(O.g_prime(C), fd, atol=1e-9)
    # g has its minima at 0 and 1 (the two pure phases)
    assert abs(O.g_prime(torch.tensor(0.0)).item()) == 0.0
    assert abs(O.g_prime(torch.tensor(1.0)).item()) == 0.0


def _flat_interface(nx, width, sigma):
    """Two flat tanh(2 x / epsilon) interfaces on a periodic strip."""
    x = torch.arange(nx, dtype=O.DT)
    x1, x2 = nx / 4.0, 3.0 * nx / 4.0
    c = 0.5 * (torch.tanh(2 * (x - x1) / width) - torch.tanh(2 * (x - x2) / width))
    ny = 4
    C1 = c[None, :].repeat(ny, 1)
    return C1, ny


def _flat_residual(width):
    nx, sigma = 256, 0.01
    C1, ny = _flat_interface(nx, width, sigma)
    grid = O.Grid(nx, ny, 1, 1)
    w, cs2 = O.weights(1 / 3), 1 / 3
    psi = torch.ones(ny, nx, dtype=O.DT)
    s = sigma
    prm = {"sigma": [[0, s], [s, 0]], "width": width}
    cos_pairs = O.pair_cosines([torch.full_like(psi, 0.3)], prm["sigma"])
    psi_mu, mu, _ = O.chemical_potentials(grid, [C1, 1 - C1], psi, cos_pairs, prm, w, cs2)
    bulk_max = (2 * 3 * sigma / width * O.g_prime(C1).abs()).max().item()
    return mu[0].abs().max().item() / bulk_max


def test_flat_interface_stationary():
    """A tanh(2x/epsilon) profile is the equilibrium of Eq. 2.1: mu_1 ~ 0 up
    to the stencils' second-order truncation, which falls ~4x when epsilon
    doubles.  Bounds: (4/epsilon)^2 / 6 of the bulk term's largest value."""
    r8, r16 = _flat_residual(8.0), _flat_residual(16.0)
    assert r8 < (4 / 8.0) ** 2 / 6
    assert r16 < (4 / 16.0) ** 2 / 6
    assert 3.0 < r8 / r16 < 5.0


def test_flat_interface_rejects_printed_beta():
    """With the printed beta = 3 epsilon / sigma the same profile leaves a
    residual many times the bulk scale (reading R1)."""
    width, sigma, nx = 8.0, 0.01, 256
    C1, ny = _flat_interface(nx, width, sigma)
    grid = O.Grid(nx, ny, 1, 1)
    w, cs2 = O.weights(1 / 3), 1 / 3
    psi = torch.ones(ny, nx, dtype=O.DT)
    bulk_max = (2 * 3 * sigma / width * O.g_prime(C1).abs()).max().item()
    bulk_bad = 2 * (3 * width / sigma) * (O.g_prime(C1) - O.g_prime(torch.ones_like(C1)))
    lap = (3 * width / 4) * sigma * grid.div_psi_grad(psi, 1 - C1, w, cs2)
    assert (bulk_bad + lap).abs().max().item() > 100 * bulk_max


def test_two_phase_mu_antisymmetric():
    g = torch.Generator().manual_seed(5)
    nx, ny = 17, 12
    grid = O.Grid(nx, ny, 1, 0)
    w, cs2 = O.weights(0.4), 0.4
    psi = 1e-3 + torch.rand(ny, nx, generator=g, dtype=O.DT)
    C1 = torch.rand(ny, nx, generator=g, dtype=O.DT)
    ct = [torch.cos(math.pi * torch.rand(ny, nx, generator=g, dtype=O.DT))]
    prm = {"sigma": [[0, 0.013], [0.013, 0]], "width": 4.5}
    cos_pairs = O.pair_cosines(ct, prm["sigma"])
    psi_mu, mu, _ = O.chemical_potentials(grid, [C1, 1 - C1], psi, cos_pairs, prm, w, cs2)
    assert torch.allclose(psi_mu[0], -psi_mu[1], atol=1e-15)
    # and the wetting term is not trivially zero on this input
    cos0 = O.pair_cosines([torch.zeros_like(psi)], prm["sigma"])
    psi_mu0, _, _ = O.chemical_potentials(grid, [C1, 1 - C1], psi, cos0, prm, w, cs2)
    assert (psi_mu[0] - psi_mu0[0]).abs().max().item() > 1e-3


@pytest.mark.parametrize("N", [2, 3, 4])
def test_mobility_zero_sums(N):
    g = torch.Generator().manual_seed(N)
    C = [torch.rand(5, 6, generator=g, dtype=O.DT) for _ in range(N)]
    M = O.mobility(C, 0.07)
    for i in range(N):
        row = sum(M[i][j] for j in range(N))
        col = sum(M[j][i] for j in range(N))
        assert row.abs().max().item() < 1e-16
        assert col.abs().max().item() < 1e-16
        assert torch.allclose(M[i][i], 0.07 * C[i] * sum(C[j] for j in range(N) if j != i))


def test_pair_cosines_eq29():
    sigma = [[0, 0.015, 0.005, 0.02], [0.015, 0, 0.01, 0.03],
             [0.005, 0.01, 0, 0.012], [0.02, 0.03, 0.012, 0]]
    ct = [torch.tensor([0.3], dtype=O.DT), torch.tensor([-0.6], dtype=O.DT), torch.tensor([0.1], dtype=O.DT)]
    cp = O.pair_cosines(ct, sigma)
    N = 4
    for i in range(N - 1):
        assert math.isclose(cp[i][N - 1].item(), ct[i].item(), rel_tol=1e-14)
        assert math.isclose(cp[N - 1][i].item(), -ct[i].item(), rel_tol=1e-14)
    for i in range(N):
        for j in range(N):
            if i != j:
                assert math.isclose(cp[i][j].item(), -cp[j][i].item(), rel_tol=1e-14)
    # Eq. 2.9 written out for (1, 2)
    ref = (0.02 * 0.3 - 0.03 * -0.6) / 0.015
    assert math.isclose(cp[0][1].item(), ref, rel_tol=1e-14)
