"""FP64 CPU oracle of one DD-CCLB time step (test infrastructure).

This module is test infrastructure: only the tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  The CUDA path never
calls it and shares no code with it.

It is a plain, slow, literal transcription of the lattice Boltzmann method
of Sec. 3 for the diffuse-domain consistent and conservative (DD-CC)
equations of Sec. 2.3, on the D2Q9 lattice, in float64 torch CPU ops over
whole grids (torch also gives the autograd reference for gradients).  The
order of operations follows the paper: moments (Sec. 3, recovery of phi C_i),
chemical potential (Eq. 2.14), mobility (Eq. 2.5), the remainder S_i (Eq. 3.7),
mass-diffusion flux m^C (Sec. 2.2), force F and velocity (Sec. 3), pressure
(Eq. 19), equilibria and sources (Eqs. 3.5, 3.6, 3.8, 3.10), the collision
with Lambda = H^-1 S H (Sec. 3, H built from Hermite polynomials and
inverted numerically), and streaming (Eqs. 3.1, 3.2).

Notation: the paper's phi (solid characteristic function) is ``psi`` here,
C_i are the volume fractions, N the number of phases.  Phases 1..N-1 carry
distributions f^i; C_N = 1 - sum_{i<N} C_i.  Lattice units dx = dt = c = 1.

Readings taken where the paper is silent or ambiguous (each is also listed
with its justification in the design notes):
  R1  beta_ij = 3 sigma_ij / epsilon (the printed 3 epsilon / sigma_ij is
      inverted: only this form gives the tanh(2x/epsilon) profile and the
      surface tension sigma).
  R2  H rows (S order): 1, cx, cy, cx^2-cs2, cy^2-cs2, cx cy,
      (cx^2-cs2) cy, cx (cy^2-cs2), (cx^2-cs2)(cy^2-cs2); these are the
      Hermite polynomials orthogonal under the d0 weights and reproduce both
      viscosity relations of Eq. 16.
  R3  the alpha/alpha-bar sums of s_p and G count the off-diagonal pair once
      (the form that satisfies Eqs. B.5d and B.5e).
  R4  a = psi (m^C_x u_y - u_x m^C_y) / 2 enters F lagged by one step; the
      damping -(1-psi) u / eps0^3 is implicit in u; u and the Eq. 19
      pressure P are solved jointly per node (P grad psi in F makes u affine
      in P and Eq. 19 quadratic in P; the root that tends to the linear one
      as the quadratic term vanishes is taken).  The antisymmetric
      divergence -div(psi (m^C u - u m^C) / 2) contracts the first index,
      as the convective flux div(m u) of Eq. 2.13c does: (d_y a, -d_x a).
  R5  rho0 = params['rho0'] (it cancels in every moment difference).
  R6  the s_0 of Eq. 19 is the p = 0 value of s_p; m^{phi C} is m = rho u + m^C.
  R7  isotropic stencils with the lattice weights; time derivatives are
      backward differences with zero history.
  R8  psi is clamped below by psi_min by the input generator.
  R9  N-1 phases evolved, C_N = 1 - sum.
  R10 cos(theta_jq) from Eq. 2.9 for every pair, with sigma_NN = 0.
  R14 outer walls: halfway bounce-back for f and g; mirror ghost nodes
      for C, psi, mu and a.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64

# D2Q9 velocities, Sec. 3: p = 0 rest, 1-4 axis, 5-8 diagonal
C_VEL = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1),
         (1, 1), (-1, 1), (-1, -1), (1, -1))
OPPOSITE = (0, 3, 4, 1, 2, 7, 8, 5, 6)


# ----------------------------------------------------------------------------
# lattice, Sec. 3 (D2Q9 block)
# ----------------------------------------------------------------------------

def weights(d0: float) -> torch.Tensor:
    """D2Q9 weights omega_p(d0): (1-d0)^2, (d0-d0^2)/2, d0^2/4 (Sec. 3)."""
    w0 = 1.0 - 2.0 * d0 + d0 * d0
    w1 = (d0 - d0 * d0) / 2.0
    w2 = d0 * d0 / 4.0
    return torch.tensor([w0, w1, w1, w1, w1, w2, w2, w2, w2], dtype=DT)


def velocities() -> torch.Tensor:
    return torch.tensor(C_VEL, dtype=DT)


def hermite_matrix(d0: float) -> torch.Tensor:
    """H of Sec. 3 (reading R2): row a evaluated at every velocity c_p."""
    cs2 = d0
    rows = []
    for (cx, cy) in C_VEL:
        rows.append([1.0, cx, cy, cx * cx - cs2, cy * cy - cs2, cx * cy,
                     cx * cx * cy - cs2 * cy, cx * cy * cy - cs2 * cx,
                     cx * cx * cy * cy - cs2 * (cx * cx + cy * cy) + cs2 * cs2])
    return torch.tensor(rows, dtype=DT).T.contiguous()    # (9 moments, 9 p)


def relaxation_vector(s0, s1, s21, s22, s3, s4):
    """diag(S) = (s0, s1, s1, s21, s21, s22, s3, s3, s4), Sec. 3."""
    return [s0, s1, s1, s21, s21, s22, s3, s3, s4]


def collision_matrix(d0: float, s) -> torch.Tensor:
    """Lambda = H^-1 S H (Sec. 3); ``s`` is the 9 diagonal rates."""
    H = hermite_matrix(d0)
    return torch.linalg.inv(H) @ torch.diag(torch.tensor(s, dtype=DT)) @ H


# ----------------------------------------------------------------------------
# neighbour access, stencils (reading R7) and boundaries (reading R14)
# ----------------------------------------------------------------------------

class Grid:
    """Index maps for neighbour access on an nx x ny lattice."""

    def __init__(self, nx, ny, periodic_x, periodic_y):
        self.nx, self.ny = int(nx), int(ny)
        self.px, self.py = bool(periodic_x), bool(periodic_y)
        self._cache = {}

    @staticmethod
    def _axis(n, d, periodic):
        i = torch.arange(n) + d
        valid = (i >= 0) & (i < n)
        if periodic:
            return i % n, torch.ones(n, dtype=torch.bool)
        mirrored = torch.where(i < 0, -i - 1, torch.where(i >= n, 2 * n - i - 1, i))
        return mirrored, valid

    def maps(self, dx, dy):
        key = (dx, dy)
        if key not in self._cache:
            ix, vx = self._axis(self.nx, dx, self.px)
            iy, vy = self._axis(self.ny, dy, self.py)
            self._cache[key] = (ix, iy, vy[:, None] & vx[None, :])
        return self._cache[key]

    def nb(self, a, dx, dy):
        """a(x + dx, y + dy): periodic wrap, or the mirror ghost at a wall."""
        ix, iy, _ = self.maps(dx, dy)
        return a.index_select(-2, iy).index_select(-1, ix)

    def grad(self, chi, w, cs2):
        """Isotropic gradient sum_p w_p c_p chi(x + c_p) / cs2."""
        gx = torch.zeros_like(chi)
        gy = torch.zeros_like(chi)
        for p, (cx, cy) in enumerate(C_VEL):
            if p == 0:
                continue
            v = self.nb(chi, cx, cy) * w[p] / cs2
            gx = gx + cx * v
            gy = gy + cy * v
        return gx, gy

    def div_psi_grad(self, psi, C, w, cs2):
        """div(psi grad C) = sum_p 2 w_p psi_{x+c_p/2} (C(x+c_p) - C(x)) / cs2
        with psi_{x+c_p/2} = (psi(x) + psi(x+c_p)) / 2."""
        out = torch.zeros_like(C)
        for p, (cx, cy) in enumerate(C_VEL):
            if p == 0:
                continue
            psi_mid = 0.5 * (psi + self.nb(psi, cx, cy))
            out = out + 2.0 * w[p] * psi_mid * (self.nb(C, cx, cy) - C) / cs2
        return out

    def stream(self, post):
        """Pull streaming of post-collision populations (..., 9, ny, nx):
        new_p(x) = post_p(x - c_p), or post_{opp(p)}(x) where x - c_p lies
        beyond an outer wall (halfway bounce-back)."""
        out = []
        for p, (cx, cy) in enumerate(C_VEL):
            ix, iy, valid = self.maps(-cx, -cy)
            pulled = post[..., p, :, :].index_select(-2, iy).index_select(-1, ix)
            bounced = post[..., OPPOSITE[p], :, :]
            out.append(torch.where(valid, pulled, bounced))
        return torch.stack(out, dim=-3)


# ----------------------------------------------------------------------------
# model pieces, Sec. 2
# ----------------------------------------------------------------------------

def g_poly(C):
    """g(C) = C^2 (C - 1)^2 (Sec. 2.1)."""
    return C * C * (C - 1.0) ** 2


def g_prime(C):
    """g'(C) = 2 C (C - 1)^2 + 2 C^2 (C - 1)."""
    return 2.0 * C * (C - 1.0) ** 2 + 2.0 * C * C * (C - 1.0)


def beta_matrix(sigma, width):
    """beta_ij = 3 sigma_ij / epsilon (reading R1 of Eq. 2.1)."""
    N = len(sigma)
    return [[3.0 * sigma[i][j] / width for j in range(N)] for i in range(N)]


def pair_cosines(cos_iN, sigma):
    """cos(theta_jq) for all phase pairs from the N-1 angles theta_iN by
    Eq. 2.9 (reading R10); ``cos_iN`` is a list of N-1 tensors.  Returns a
    nested list [j][q] (None on the diagonal)."""
    N = len(sigma)
    cN = list(cos_iN) + [torch.zeros_like(cos_iN[0])]   # theta_NN term: sigma_NN = 0
    out = [[None] * N for _ in range(N)]
    for j in range(N):
        for q in range(N):
            if j != q:
                out[j][q] = (sigma[j][N - 1] * cN[j] - sigma[q][N - 1] * cN[q]) / sigma[j][q]
    return out


def chemical_potentials(grid, C, psi, cos_pairs, prm, w, cs2, walls=None):
    """psi mu_i for i = 1..N by Eq. 2.14 and mu_i = psi mu_i / psi.

    With ``walls`` -- a list of (cos_pairs_k, psi_k) for solids given by
    their own characteristic functions psi_k with psi = prod_k psi_k -- the
    wetting term is the Sec. 4.5 form sum_k cos(theta^k_jq) |grad psi_k|
    in place of cos(theta_jq) |grad psi| (``cos_pairs`` is then unused)."""
    N = len(C)
    sigma = prm["sigma"]
    eps = prm["width"]
    beta = beta_matrix(sigma, eps)
    L = [grid.div_psi_grad(psi, C[j], w, cs2) for j in range(N)]
    gpx, gpy = grid.grad(psi, w, cs2)
    if walls is None:
        terms = [(cos_pairs, torch.sqrt(gpx * gpx + gpy * gpy))]
    else:
        terms = []
        for cp_k, psi_k in walls:
            kx, ky = grid.grad(psi_k, w, cs2)
            terms.append((cp_k, torch.sqrt(kx * kx + ky * ky)))
    psi_mu = []
    for i in range(N):
        bulk = torch.zeros_like(psi)
        grad_term = torch.zeros_like(psi)
        wet = torch.zeros_like(psi)
        for j in range(N):
            bulk = bulk + 2.0 * beta[i][j] * psi * (g_prime(C[i]) - g_prime(C[i] + C[j]))
            grad_term = grad_term + 0.75 * eps * sigma[i][j] * L[j]
            for cp, abs_grad in terms:
                inner = torch.zeros_like(psi)
                for q in range(N):
                    if q != j:
                        inner = inner + cp[j][q] * C[j] * C[q]
                wet = wet + 3.0 * sigma[i][j] * inner * abs_grad
        psi_mu.append(bulk + grad_term + wet)
    mu = [pm / psi for pm in psi_mu]
    return psi_mu, mu, (gpx, gpy)


def mobility(C, m0):
    """M_ij = -m0 C_i C_j (i != j), M_ii = -sum_{j != i} M_ij (Eq. 2.5)."""
    N = len(C)
    M = [[None] * N for _ in range(N)]
    for i in range(N):
        for j in range(N):
            if i != j:
                M[i][j] = -m0 * C[i] * C[j]
    for i in range(N):
        acc = torch.zeros_like(C[0])
        for j in range(N):
            if j != i:
                acc = acc + M[i][j]
        M[i][i] = -acc
    return M


# ----------------------------------------------------------------------------
# equilibria and sources, Sec. 3
# ----------------------------------------------------------------------------

def f_equilibrium(psiC, psi_mu, u, eta, w, cs2):
    """f^{i,eq}_p of Eq. 3.5 for one phase -> (9, ny, nx)."""
    out = []
    for p, (cx, cy) in enumerate(C_VEL):
        if p == 0:
            out.append((w[0] - 1.0) * eta * psi_mu + psiC)
        else:
            cu = cx * psiC * u[0] + cy * psiC * u[1]
            out.append(w[p] * eta * psi_mu + w[p] * cu / cs2)
    return torch.stack(out)


def f_source(V, w, cs2):
    """F^i_p = w_p c_p . V / cs2 (Eq. 3.6) with
    V = d_t(psi C_i u) + cs2 eta_i (mu_i grad psi - S_i)."""
    out = []
    for p, (cx, cy) in enumerate(C_VEL):
        out.append(w[p] * (cx * V[0] + cy * V[1]) / cs2)
    return torch.stack(out)


def s_vector(psi, rho, u, mC, w, cs2, c2=1.0):
    """s_p of Sec. 3 (below Eq. 3.10), reading R3 for the xy term."""
    Axx = psi * rho * u[0] * u[0] + psi * mC[0] * u[0]
    Ayy = psi * rho * u[1] * u[1] + psi * mC[1] * u[1]
    Axy = psi * rho * u[0] * u[1] + 0.5 * (psi * mC[0] * u[1] + psi * u[0] * mC[1])
    out = []
    for p, (cx, cy) in enumerate(C_VEL):
        t1 = (cx * psi * rho * u[0] + cy * psi * rho * u[1]) / cs2
        t2 = (Axx * (cx * cx - cs2) + Ayy * (cy * cy - cs2)) / (c2 * cs2 - cs2 * cs2)
        t3 = Axy * cx * cy / (cs2 * cs2)
        out.append(w[p] * (t1 + t2 + t3))
    return torch.stack(out)


def g_equilibrium(psiP, s, rho0, w, cs2):
    """g^eq_p of Eq. 3.8."""
    out = []
    for p in range(9):
        if p == 0:
            out.append((w[0] - 1.0) * psiP / cs2 + rho0 + s[0])
        else:
            out.append(w[p] * psiP / cs2 + s[p])
    return torch.stack(out)


def g_source(psi_u_grad_rho, F, M2G, w, cs2, c2=1.0):
    """G_p of Eq. 3.10 with the second-order tensor M^{2G} (xx, yy, xy)."""
    Mxx, Myy, Mxy = M2G
    out = []
    for p, (cx, cy) in enumerate(C_VEL):
        t = psi_u_grad_rho + (cx * F[0] + cy * F[1]) / cs2
        t = t + (Mxx * (cx * cx - cs2) + Myy * (cy * cy - cs2)) / (c2 * cs2 - cs2 * cs2)
        t = t + Mxy * cx * cy / (cs2 * cs2)
        out.append(w[p] * t)
    return torch.stack(out)


def apply_collision(Lam, v):
    """(Lambda v)_p = sum_q Lambda_pq v_q for a (9, ny, nx) field; ``Lam``
    is (9, 9) or per node (ny, nx, 9, 9)."""
    if Lam.dim() == 2:
        return torch.einsum("pq,qyx->pyx", Lam, v)
    return torch.einsum("yxpq,qyx->pyx", Lam, v)


# ----------------------------------------------------------------------------
# the step
# ----------------------------------------------------------------------------

def derived_rates(prm):
    """Per-phase s_1^{f_i} from m0 = (1/s1 - 1/2) eta_i cs2 (Eq. 17)."""
    cs2 = prm["d0"]
    return [1.0 / (prm["m0"] / (eta * cs2) + 0.5) for eta in prm["eta"]]


def pressure_constants(d0: float, s21):
    """K = 1 - d0 and H = K (1 - 2 d0)(s21 - 2), the two-dimensional
    constants printed below Eq. 19."""
    K = 1.0 - d0
    return K, K * (1.0 - 2.0 * d0) * (s21 - 2.0)


def eq19_coefficients(d0: float, s0: float, s21):
    """The coefficients of Eq. 19's velocity terms: A of psi u . grad rho
    (1/2 + K (1 - d0)(2 - s0) / (2 s0)), K/2 of d_t(psi m . u) and H / s21
    of u . grad(psi rho), with the 2D K and H."""
    K, Hc = pressure_constants(d0, s21)
    A = 0.5 + K * (1.0 - d0) * (2.0 - s0) / (2.0 * s0)
    return A, K / 2.0, Hc / s21


def flow_shear_rates(nu, d0, c2=1.0):
    """s21, s22 from nu by Eq. 16."""
    cs2 = d0 * c2
    s21 = 1.0 / (2.0 * nu / (c2 - cs2) + 0.5)
    s22 = 1.0 / (nu / cs2 + 0.5)
    return s21, s22


class Oracle:
    """State and time stepping of the DD-CCLB method on one CPU.

    Fields: ``f`` (N-1, 9, ny, nx), ``g`` (9, ny, nx) with g_0 holding rho0,
    lagged ``P``, ``a``, ``psiCu`` (N-1, 2), ``T`` (3: xx, yy, xy) and
    ``psimu`` (psi m . u), all float64 on the CPU.
    """

    def __init__(self, params, psi, C0, cos_theta, cos_theta_field=None,
                 frozen_flow=False, walls=None, open_x=None):
        prm = dict(params)
        self.prm = prm
        self.N = int(prm["nphase"])
        self.nx, self.ny = int(prm["nx"]), int(prm["ny"])
        self.grid = Grid(self.nx, self.ny, prm["periodic_x"], prm["periodic_y"])
        self.d0 = float(prm["d0"])
        self.cs2 = self.d0
        self.w = weights(self.d0)
        self.frozen = bool(frozen_flow)
        # walls: list of (psi_k, cos_k) -- solids with their own
        # characteristic functions and angles theta^k_iN ((N-1,) uniform or
        # (N-1, ny, nx)); psi = prod_k psi_k (Sec. 4.5)
        self.walls = None
        if walls is not None:
            self.walls = []
            prod = None
            for psi_k, cos_k in walls:
                pk = torch.as_tensor(psi_k, dtype=DT)
                ck = torch.as_tensor(cos_k, dtype=DT)
                if ck.dim() == 1:
                    ck = ck[:, None, None].expand(-1, self.ny, self.nx)
                cp = pair_cosines([ck[i] for i in range(self.N - 1)], prm["sigma"])
                self.walls.append((cp, pk))
                prod = pk if prod is None else prod * pk
            psi = prod
        self.psi = torch.as_tensor(psi, dtype=DT)
        if self.walls is not None:
            self.cos_iN = [torch.zeros((self.ny, self.nx), dtype=DT) for _ in range(self.N - 1)]
        elif cos_theta_field is not None:
            ct = torch.as_tensor(cos_theta_field, dtype=DT)
            self.cos_iN = [ct[i] for i in range(self.N - 1)]
        else:
            self.cos_iN = [torch.full((self.ny, self.nx), float(cos_theta[i]), dtype=DT)
                           for i in range(self.N - 1)]
        sf = prm["s_f"]
        self.Lam_f = [collision_matrix(self.d0, relaxation_vector(
            sf[0], s1, sf[1], sf[2], sf[3], sf[4])) for s1 in derived_rates(prm)]
        self.H = hermite_matrix(self.d0)
        self.Hinv = torch.linalg.inv(self.H)
        # open_x: (u_in (ny,), C_in (N-1, ny)) -- inflow at x = 0 and outflow
        # at x = nx - 1 with the prescribed velocity profile (reading R22)
        self.open_x = None
        if open_x is not None:
            if prm["periodic_x"]:
                raise ValueError("open boundaries need a non-periodic x axis")
            self.open_x = (torch.as_tensor(open_x[0], dtype=DT), torch.as_tensor(open_x[1], dtype=DT))
        self.init_state(torch.as_tensor(C0, dtype=DT))

    # -- pieces -------------------------------------------------------------

    def volume_fractions(self, f):
        """phi C_i = sum_p f^i_p (Sec. 3), C_i = phi C_i / phi, C_N = 1 - sum."""
        psiC = [f[i].sum(dim=0) for i in range(self.N - 1)]
        C = [pc / self.psi for pc in psiC]
        CN = torch.ones_like(self.psi)
        for Ci in C:
            CN = CN - Ci
        return psiC, C + [CN]

    def init_state(self, C0):
        """Reading R13: f = f^eq(C0, mu(C0), u = 0), g = g^eq(P = 0, u = 0),
        lagged fields zero."""
        N = self.N
        C = [C0[i] for i in range(N - 1)]
        CN = torch.ones_like(self.psi)
        for Ci in C:
            CN = CN - Ci
        C = C + [CN]
        cos_pairs = pair_cosines(self.cos_iN, self.prm["sigma"])
        psi_mu, _, _ = chemical_potentials(self.grid, C, self.psi, cos_pairs,
                                           self.prm, self.w, self.cs2, self.walls)
        zero = torch.zeros_like(self.psi)
        self.f = torch.stack([
            f_equilibrium(self.psi * C[i], psi_mu[i], (zero, zero),
                          self.prm["eta"][i], self.w, self.cs2)
            for i in range(N - 1)])
        s0 = torch.zeros((9, self.ny, self.nx), dtype=DT)
        self.g = g_equilibrium(zero, s0, self.prm["rho0"], self.w, self.cs2)
        self.P = zero.clone()
        self.a = zero.clone()
        self.psiCu = torch.zeros((N - 1, 2, self.ny, self.nx), dtype=DT)
        self.T = torch.zeros((3, self.ny, self.nx), dtype=DT)
        self.psimu = zero.clone()
        self.steps = 0

    def fields(self):
        """Everything the step computes before collision (a1-a6, a10)."""
        prm, grid, w, cs2 = self.prm, self.grid, self.w, self.cs2
        N, psi = self.N, self.psi
        psiC, C = self.volume_fractions(self.f)
        rho = torch.zeros_like(psi)
        nu = torch.zeros_like(psi)
        for i in range(N):
            rho = rho + C[i] * prm["rho"][i]
            nu = nu + C[i] * prm["nu"][i]
        s21, s22 = flow_shear_rates(nu, self.d0)
        cos_pairs = pair_cosines(self.cos_iN, prm["sigma"])
        psi_mu, mu, grad_psi = chemical_potentials(grid, C, psi, cos_pairs,
                                                   prm, w, cs2, self.walls)
        gradC = [grid.grad(C[j], w, cs2) for j in range(N)]
        gradmu = [grid.grad(mu[j], w, cs2) for j in range(N)]
        M = mobility(C, prm["m0"])
        m0 = prm["m0"]
        S = []
        for i in range(N - 1):
            Sx = (psi * M[i][i] - psi * m0) / m0 * gradmu[i][0]
            Sy = (psi * M[i][i] - psi * m0) / m0 * gradmu[i][1]
            for j in range(N):
                if j != i:
                    Sx = Sx + psi * M[i][j] / m0 * gradmu[j][0]
                    Sy = Sy + psi * M[i][j] / m0 * gradmu[j][1]
            S.append((Sx, Sy))
        mCx = torch.zeros_like(psi)
        mCy = torch.zeros_like(psi)
        for i in range(N):
            for j in range(N):
                mCx = mCx - prm["rho"][i] * M[i][j] * gradmu[j][0]
                mCy = mCy - prm["rho"][i] * M[i][j] * gradmu[j][1]
        # force without the pressure-wall and damping terms; a is lagged
        Fx = torch.zeros_like(psi)
        Fy = torch.zeros_like(psi)
        for i in range(N):
            Fx = Fx + psi_mu[i] * gradC[i][0]
            Fy = Fy + psi_mu[i] * gradC[i][1]
        dax, day = grid.grad(self.a, w, cs2)
        Fx = Fx + day
        Fy = Fy - dax
        b = prm["body_force"]
        Fx = Fx + psi * rho * b[0]
        Fy = Fy + psi * rho * b[1]
        eps0 = prm["eps0"]
        damp = (1.0 - psi) / eps0 ** 3
        d0 = self.d0
        grad_rho = grid.grad(rho, w, cs2)
        grad_psirho = grid.grad(psi * rho, w, cs2)
        A, Kh, Hs = eq19_coefficients(d0, prm["s_g"][0], s21)
        cP = cs2 / (1.0 - w[0])
        sum_g = torch.zeros_like(psi)
        for p in range(1, 9):
            sum_g = sum_g + self.g[p]
        if self.frozen:
            ux = torch.zeros_like(psi)
            uy = torch.zeros_like(psi)
            P = self.P
        else:
            Jx = torch.zeros_like(psi)
            Jy = torch.zeros_like(psi)
            for p, (cx, cy) in enumerate(C_VEL):
                Jx = Jx + cx * self.g[p]
                Jy = Jy + cy * self.g[p]
            # Velocity (Sec. 3): psi rho u = J + F/2 with
            # F = F0 + P grad psi - (1 - psi) u / eps0^3, so u = u0 + P e.
            den = psi * rho + 0.5 * damp
            u0x = (Jx + 0.5 * Fx) / den
            u0y = (Jy + 0.5 * Fy) / den
            ex = 0.5 * grad_psi[0] / den
            ey = 0.5 * grad_psi[1] / den
            # Pressure, Eq. 19, with s_0 = -w0 psi m . u / (1 - cs2) and
            # psi m . u = psi rho |u|^2 + psi m^C . u:
            #   psi P = cP [G0 + beta . u + gamma |u|^2]
            bx = (A * psi * grad_rho[0] + (Kh - w[0] / (1.0 - cs2)) * psi * mCx
                  + Hs * grad_psirho[0])
            by = (A * psi * grad_rho[1] + (Kh - w[0] / (1.0 - cs2)) * psi * mCy
                  + Hs * grad_psirho[1])
            gam = (Kh - w[0] / (1.0 - cs2)) * psi * rho
            G0 = sum_g - Kh * self.psimu
            # joint solve of u = u0 + P e and Eq. 19 (reading R4):
            # qa P^2 + qb P + qc = 0, the root that tends to -qc/qb
            qa = cP * gam * (ex * ex + ey * ey)
            qb = cP * (bx * ex + by * ey + 2.0 * gam * (u0x * ex + u0y * ey)) - psi
            qc = cP * (G0 + bx * u0x + by * u0y + gam * (u0x * u0x + u0y * u0y))
            disc = torch.clamp(qb * qb - 4.0 * qa * qc, min=0.0)
            root = torch.sqrt(disc)
            P = -2.0 * qc / torch.where(qb < 0, qb - root, qb + root)
            ux = u0x + P * ex
            uy = u0y + P * ey
            Fx = Fx + P * grad_psi[0]
            Fy = Fy + P * grad_psi[1]
        Fx = Fx - damp * ux
        Fy = Fy - damp * uy
        u_grad_rho = ux * grad_rho[0] + uy * grad_rho[1]
        psimu = psi * (rho * (ux * ux + uy * uy) + mCx * ux + mCy * uy)
        psiP = psi * P
        return dict(psiC=psiC, C=C, rho=rho, nu=nu, s21=s21, s22=s22,
                    psi_mu=psi_mu, mu=mu, grad_psi=grad_psi, gradC=gradC,
                    gradmu=gradmu, M=M, S=S, mC=(mCx, mCy), F=(Fx, Fy),
                    u=(ux, uy), psiP=psiP, P=P,
                    u_grad_rho=u_grad_rho, grad_psirho=grad_psirho,
                    psimu=psimu)

    def step(self, n=1):
        for _ in range(int(n)):
            self._step()

    def _step(self):
        prm, w, cs2, N, psi = self.prm, self.w, self.cs2, self.N, self.psi
        fl = self.fields()
        ux, uy = fl["u"]
        # phase LB, Eqs. 3.1, 3.5-3.7
        f_post = []
        new_psiCu = []
        for i in range(N - 1):
            eta = prm["eta"][i]
            psiCu = (fl["psiC"][i] * ux, fl["psiC"][i] * uy)
            dt_x = psiCu[0] - self.psiCu[i, 0]
            dt_y = psiCu[1] - self.psiCu[i, 1]
            Vx = dt_x + cs2 * eta * (fl["mu"][i] * fl["grad_psi"][0] - fl["S"][i][0])
            Vy = dt_y + cs2 * eta * (fl["mu"][i] * fl["grad_psi"][1] - fl["S"][i][1])
            feq = f_equilibrium(fl["psiC"][i], fl["psi_mu"][i], (ux, uy), eta, w, cs2)
            Fi = f_source((Vx, Vy), w, cs2)
            Lam = self.Lam_f[i]
            fi = self.f[i]
            post = fi - apply_collision(Lam, fi - feq) + Fi - 0.5 * apply_collision(Lam, Fi)
            f_post.append(post)
            new_psiCu.append(torch.stack(psiCu))
        if self.frozen:
            g_post = self.g
            T = self.T
            a = self.a
        else:
            mCx, mCy = fl["mC"]
            rho = fl["rho"]
            s = s_vector(psi, rho, (ux, uy), (mCx, mCy), w, cs2)
            geq = g_equilibrium(fl["psiP"], s, prm["rho0"], w, cs2)
            T = torch.stack([psi * mCx * ux, psi * mCy * uy,
                             0.5 * (psi * mCx * uy + psi * ux * mCy)])
            dT = T - self.T
            gpr = fl["grad_psirho"]
            ugpr = ux * gpr[0] + uy * gpr[1]
            c2 = 1.0
            Mxx = dT[0] + cs2 * 2.0 * ux * gpr[0] + (c2 - 3.0 * cs2) * ugpr
            Myy = dT[1] + cs2 * 2.0 * uy * gpr[1] + (c2 - 3.0 * cs2) * ugpr
            Mxy = dT[2] + cs2 * (ux * gpr[1] + gpr[0] * uy)
            G = g_source(psi * fl["u_grad_rho"], fl["F"], (Mxx, Myy, Mxy), w, cs2)
            sg = prm["s_g"]
            rates = torch.stack([torch.full_like(psi, sg[0]), torch.full_like(psi, sg[1]),
                                 torch.full_like(psi, sg[1]), fl["s21"], fl["s21"],
                                 fl["s22"], torch.full_like(psi, sg[2]),
                                 torch.full_like(psi, sg[2]), torch.full_like(psi, sg[3])])
            # Lambda^g = H^-1 S(x) H applied node by node
            def lam_g(v):
                m = torch.einsum("ap,pyx->ayx", self.H, v)
                return torch.einsum("pa,ayx->pyx", self.Hinv, rates * m)
            g_post = self.g - lam_g(self.g - geq) + G - 0.5 * lam_g(G)
            a = 0.5 * psi * (mCx * uy - ux * mCy)
        self.f = self.grid.stream(torch.stack(f_post))
        if not self.frozen:
            self.g = self.grid.stream(g_post)
            self.P = fl["P"]       # diagnostics only; P is not lagged
            self.a = a
            self.T = T
            self.psimu = fl["psimu"]
        self.psiCu = torch.stack(new_psiCu)
        if self.open_x is not None:
            self.open_boundaries()
        self.steps += 1

    def open_boundaries(self):
        """Reading R22 of the inflow/outflow of Sec. 4.5: after streaming, the
        columns x = 0 (inlet) and x = nx - 1 (outlet) are reset to equilibrium
        (Eqs. 3.5, 3.8 with mu = 0 and m^C = 0) at the prescribed velocity
        (u_in(y), 0); C is C_in(y) at the inlet and copied from x = nx - 2 at
        the outlet; P is copied from the neighbouring column, taken from Eq. 19
        without its velocity terms, psi P = c_P (sum_{p>0} g_p - K/2 psi m.u);
        the lagged fields are those of that state."""
        prm, N, w, cs2 = self.prm, self.N, self.w, self.cs2
        u_in, C_in = self.open_x
        K, _ = pressure_constants(self.d0, 0.0)
        cP = cs2 / (1.0 - w[0])
        for xb, xn in ((0, 1), (self.nx - 1, self.nx - 2)):
            psib = self.psi[:, xb]
            psin = self.psi[:, xn]
            if xb == 0:
                Cb = [C_in[i] for i in range(N - 1)]
            else:
                Cb = [self.f[i, :, :, xn].sum(dim=0) / psin for i in range(N - 1)]
            CN = torch.ones_like(psib)
            for c in Cb:
                CN = CN - c
            rho = CN * prm["rho"][N - 1]
            for i in range(N - 1):
                rho = rho + Cb[i] * prm["rho"][i]
            sum_g = self.g[1:, :, xn].sum(dim=0)
            Pn = cP * (sum_g - K / 2.0 * self.psimu[:, xn]) / psin
            psiP = psib * Pn
            zero = torch.zeros_like(psib)
            u = (u_in, zero)
            for i in range(N - 1):
                self.f[i, :, :, xb] = f_equilibrium(psib * Cb[i], zero, u, prm["eta"][i], w, cs2)
            s_b = s_vector(psib, rho, u, (zero, zero), w, cs2)
            self.g[:, :, xb] = g_equilibrium(psiP, s_b, prm["rho0"], w, cs2)
            self.a[:, xb] = zero
            for i in range(N - 1):
                self.psiCu[i, 0, :, xb] = psib * Cb[i] * u_in
                self.psiCu[i, 1, :, xb] = zero
            self.T[:, :, xb] = 0.0
            self.psimu[:, xb] = psib * rho * u_in * u_in

    # -- diagnostics --------------------------------------------------------

    def mass(self):
        """Per-phase sum_x sum_p f^i_p (= sum_x psi C_i)."""
        return self.f.sum(dim=(1, 2, 3))

    def macroscopic(self):
        """C_1..C_N, rho, u_x, u_y, P and mu_1..mu_N of the current state,
        as the next step computes them."""
        fl = self.fields()
        return dict(C=torch.stack(fl["C"]), rho=fl["rho"], ux=fl["u"][0],
                    uy=fl["u"][1], P=fl["P"], mu=torch.stack(fl["mu"]))
