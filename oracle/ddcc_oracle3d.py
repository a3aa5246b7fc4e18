"""FP64 CPU oracle of one three-dimensional DD-CCLB time step (test
infrastructure).

This module is test infrastructure: only the tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  The CUDA path never
calls it and shares no code with it.

It transcribes the lattice Boltzmann method of Sec. 3 for the DD-CC
equations of Sec. 2.3 in three dimensions: the phase distributions f^i on
the D3Q7 lattice and the flow distributions g on the D3Q15 lattice, with
the weights and relaxation orders printed in Sec. 3 and the 3D constants
K = 1 - 2 d0 and H = K (3 - 7 d0)(s21 - 2) / 2 of the pressure (Eq. 19).
Every other formula -- the chemical potential (Eq. 2.14), the mobility
(Eq. 2.5), the remainder S_i (Eq. 3.7), the mass-diffusion flux m^C, the
force F, the velocity, the equilibria and sources (Eqs. 3.5, 3.6, 3.8,
3.10) and M^{2G} -- is the dimension-free form of Sec. 3, written out with
three components.  Fields are float64 torch tensors shaped (nz, ny, nx).

Readings taken in addition to those of the two-dimensional oracle:
  R23 Hermite rows (S order).  D3Q7: 1, cx, cy, cz, cx^2 - cs2, cy^2 - cs2,
      cz^2 - cs2.  D3Q15: 1; cx, cy, cz; c_a^2 - cs2 (a = x, y, z);
      cx cy, cy cz, cz cx; cx (cy^2 - cs2), cy (cz^2 - cs2), cz (cx^2 - cs2),
      cx cy cz; cx^2 cy^2 cz^2 - cs2 |c|^2 + 2 cs2^2.  The D3Q15 rows are
      orthogonal under the weights omega_p(d0) (the last is the one
      direction left orthogonal to the others), which makes the rest
      component of Lambda^-1 give exactly the K and H of Eq. 19.  Parity
      unpinned for the third-order rows: they enter only through s3, and
      no test fixes them beyond orthogonality and the spectrum of Lambda.
  R24 isotropic stencils with the D3Q15 weights, as R7 does with D2Q9.
  R25 the antisymmetric tensor A = psi (m^C u - u m^C) / 2 has three
      components a_xy, a_yz, a_zx, lagged one step as in R4; the force
      takes -div A contracted on the first index (as R4).
  R26 the joint per-node solve of u and P of R4 in three components.
  R27 the box is periodic along every axis; solids enter through psi only.
"""
from __future__ import annotations

import torch

DT = torch.float64

# D3Q7 (phase) and D3Q15 (flow) velocities, Sec. 3
C7 = ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
C15 = ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
       (1, 1, 1), (-1, 1, 1), (1, -1, 1), (-1, -1, 1),
       (1, 1, -1), (-1, 1, -1), (1, -1, -1), (-1, -1, -1))


# ----------------------------------------------------------------------------
# lattices, Sec. 3 (D3Q7 and D3Q15 blocks)
# ----------------------------------------------------------------------------

def weights7(d0: float) -> torch.Tensor:
    """D3Q7 weights: 1 - 3 d0 at rest, d0 / 2 on the six axes."""
    return torch.tensor([1.0 - 3.0 * d0] + [d0 / 2.0] * 6, dtype=DT)


def weights15(d0: float) -> torch.Tensor:
    """D3Q15 weights: 1 - 3 d0 + 2 d0^2, (d0 - d0^2) / 2, d0^2 / 8."""
    return torch.tensor([1.0 - 3.0 * d0 + 2.0 * d0 * d0] + [(d0 - d0 * d0) / 2.0] * 6
                        + [d0 * d0 / 8.0] * 8, dtype=DT)


def velocities(vel) -> torch.Tensor:
    return torch.tensor(vel, dtype=DT)


def hermite7(d0: float) -> torch.Tensor:
    """D3Q7 rows of reading R23, (7 moments, 7 velocities)."""
    cs2 = d0
    rows = [[1.0, cx, cy, cz, cx * cx - cs2, cy * cy - cs2, cz * cz - cs2] for (cx, cy, cz) in C7]
    return torch.tensor(rows, dtype=DT).T.contiguous()


def hermite15(d0: float) -> torch.Tensor:
    """D3Q15 rows of reading R23, (15 moments, 15 velocities)."""
    cs2 = d0
    rows = []
    for (cx, cy, cz) in C15:
        c2 = cx * cx + cy * cy + cz * cz
        rows.append([1.0, cx, cy, cz,
                     cx * cx - cs2, cy * cy - cs2, cz * cz - cs2,
                     cx * cy, cy * cz, cz * cx,
                     cx * (cy * cy - cs2), cy * (cz * cz - cs2), cz * (cx * cx - cs2),
                     cx * cy * cz,
                     cx * cx * cy * cy * cz * cz - cs2 * c2 + 2.0 * cs2 * cs2])
    return torch.tensor(rows, dtype=DT).T.contiguous()


def rates7(s0, s1, s21):
    """diag(S) of D3Q7: (s0, s1, s1, s1, s21, s21, s21), Sec. 3."""
    return [s0, s1, s1, s1, s21, s21, s21]


def rates15(s0, s1, s21, s22, s3, s4):
    """diag(S) of D3Q15: (s0, s1 x3, s21 x3, s22 x3, s3 x4, s4), Sec. 3."""
    return [s0] + [s1] * 3 + [s21] * 3 + [s22] * 3 + [s3] * 4 + [s4]


def collision_matrix(H: torch.Tensor, s) -> torch.Tensor:
    """Lambda = H^-1 S H (Sec. 3)."""
    return torch.linalg.inv(H) @ torch.diag(torch.tensor(s, dtype=DT)) @ H


def pressure_constants(d0: float, s21):
    """K = 1 - 2 d0 and H = K (3 - 7 d0)(s21 - 2) / 2, the three-dimensional
    constants printed below Eq. 19."""
    K = 1.0 - 2.0 * d0
    return K, K * (3.0 - 7.0 * d0) * (s21 - 2.0) / 2.0


# ----------------------------------------------------------------------------
# neighbour access and stencils (readings R24, R27)
# ----------------------------------------------------------------------------

def nb(a, dx, dy, dz):
    """a(x + dx, y + dy, z + dz) on the periodic box (last three dims z, y, x)."""
    return torch.roll(a, shifts=(-dz, -dy, -dx), dims=(-3, -2, -1))


def grad(chi, w, cs2):
    """Isotropic gradient sum_p w_p c_p chi(x + c_p) / cs2 (D3Q15 weights)."""
    g = [torch.zeros_like(chi) for _ in range(3)]
    for p, c in enumerate(C15):
        if p == 0:
            continue
        v = nb(chi, *c) * (w[p] / cs2)
        for a in range(3):
            if c[a]:
                g[a] = g[a] + c[a] * v
    return tuple(g)


def div_psi_grad(psi, C, w, cs2):
    """div(psi grad C) = sum_p 2 w_p (psi(x) + psi(x + c_p)) / 2
    (C(x + c_p) - C(x)) / cs2."""
    out = torch.zeros_like(C)
    for p, c in enumerate(C15):
        if p == 0:
            continue
        psi_mid = 0.5 * (psi + nb(psi, *c))
        out = out + 2.0 * w[p] * psi_mid * (nb(C, *c) - C) / cs2
    return out


def stream(post, vel):
    """Pull streaming: new_p(x) = post_p(x - c_p), periodic; ``post`` is
    (..., Q, nz, ny, nx)."""
    out = [nb(post[..., p, :, :, :], -c[0], -c[1], -c[2]) for p, c in enumerate(vel)]
    return torch.stack(out, dim=-4)


# ----------------------------------------------------------------------------
# model pieces, Sec. 2
# ----------------------------------------------------------------------------

def g_prime(C):
    """g'(C) for g(C) = C^2 (C - 1)^2 (Sec. 2.1)."""
    return 2.0 * C * (C - 1.0) ** 2 + 2.0 * C * C * (C - 1.0)


def pair_cosines(cos_iN, sigma):
    """cos(theta_jq) of every pair from the N-1 angles theta_iN (Eq. 2.9,
    sigma_NN = 0)."""
    N = len(sigma)
    cN = list(cos_iN) + [torch.zeros_like(cos_iN[0])]
    out = [[None] * N for _ in range(N)]
    for j in range(N):
        for q in range(N):
            if j != q:
                out[j][q] = (sigma[j][N - 1] * cN[j] - sigma[q][N - 1] * cN[q]) / sigma[j][q]
    return out


def chemical_potentials(C, psi, cos_pairs, prm, w, cs2):
    """psi mu_i (i = 1..N) by Eq. 2.14 with beta_ij = 3 sigma_ij / epsilon,
    and mu_i = psi mu_i / psi."""
    N = len(C)
    sigma, eps = prm["sigma"], prm["width"]
    L = [div_psi_grad(psi, C[j], w, cs2) for j in range(N)]
    gp = grad(psi, w, cs2)
    agp = torch.sqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2])
    psi_mu = []
    for i in range(N):
        acc = torch.zeros_like(psi)
        for j in range(N):
            beta = 3.0 * sigma[i][j] / eps
            acc = acc + 2.0 * beta * psi * (g_prime(C[i]) - g_prime(C[i] + C[j]))
            acc = acc + 0.75 * eps * sigma[i][j] * L[j]
            inner = torch.zeros_like(psi)
            for q in range(N):
                if q != j:
                    inner = inner + cos_pairs[j][q] * C[j] * C[q]
            acc = acc + 3.0 * sigma[i][j] * inner * agp
        psi_mu.append(acc)
    return psi_mu, [pm / psi for pm in psi_mu], gp


def mobility(C, m0):
    """M_ij = -m0 C_i C_j (i != j), M_ii = -sum_{j != i} M_ij (Eq. 2.5)."""
    N = len(C)
    M = [[None] * N for _ in range(N)]
    for i in range(N):
        for j in range(N):
            if i != j:
                M[i][j] = -m0 * C[i] * C[j]
    for i in range(N):
        M[i][i] = -sum(M[i][j] for j in range(N) if j != i)
    return M


# ----------------------------------------------------------------------------
# equilibria and sources, Sec. 3
# ----------------------------------------------------------------------------

def f_equilibrium(psiC, psi_mu, u, eta, w, cs2):
    """f^{i,eq}_p of Eq. 3.5 on D3Q7 -> (7, nz, ny, nx)."""
    out = []
    for p, c in enumerate(C7):
        if p == 0:
            out.append((w[0] - 1.0) * eta * psi_mu + psiC)
        else:
            cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
            out.append(w[p] * eta * psi_mu + w[p] * psiC * cu / cs2)
    return torch.stack(out)


def f_source(V, w, cs2):
    """F^i_p = w_p c_p . V / cs2 (Eq. 3.6) on D3Q7."""
    return torch.stack([w[p] * (c[0] * V[0] + c[1] * V[1] + c[2] * V[2]) / cs2
                        for p, c in enumerate(C7)])


PAIRS = ((0, 1), (1, 2), (2, 0))      # xy, yz, zx


def s_vector(psi, rho, u, mC, w, cs2, c2=1.0):
    """s_p below Eq. 3.10 on D3Q15 (off-diagonal pairs counted once, R3)."""
    diag = [psi * rho * u[a] * u[a] + psi * mC[a] * u[a] for a in range(3)]
    off = [psi * rho * u[a] * u[b] + 0.5 * (psi * mC[a] * u[b] + psi * u[a] * mC[b])
           for (a, b) in PAIRS]
    out = []
    for p, c in enumerate(C15):
        t = (c[0] * u[0] + c[1] * u[1] + c[2] * u[2]) * psi * rho / cs2
        for a in range(3):
            t = t + diag[a] * (c[a] * c[a] - cs2) / (c2 * cs2 - cs2 * cs2)
        for k, (a, b) in enumerate(PAIRS):
            if c[a] * c[b]:
                t = t + off[k] * (c[a] * c[b]) / (cs2 * cs2)
        out.append(w[p] * t)
    return torch.stack(out)


def g_equilibrium(psiP, s, rho0, w, cs2):
    """g^eq_p of Eq. 3.8 on D3Q15."""
    out = []
    for p in range(15):
        if p == 0:
            out.append((w[0] - 1.0) * psiP / cs2 + rho0 + s[0])
        else:
            out.append(w[p] * psiP / cs2 + s[p])
    return torch.stack(out)


def g_source(a0, F, M2G, w, cs2, c2=1.0):
    """G_p of Eq. 3.10 on D3Q15; ``M2G`` = (xx, yy, zz, xy, yz, zx)."""
    out = []
    for p, c in enumerate(C15):
        t = a0 + (c[0] * F[0] + c[1] * F[1] + c[2] * F[2]) / cs2
        for a in range(3):
            t = t + M2G[a] * (c[a] * c[a] - cs2) / (c2 * cs2 - cs2 * cs2)
        for k, (a, b) in enumerate(PAIRS):
            if c[a] * c[b]:
                t = t + M2G[3 + k] * (c[a] * c[b]) / (cs2 * cs2)
        out.append(w[p] * t)
    return torch.stack(out)


def derived_rates(prm):
    """Per-phase s_1 from m0 = (1/s1 - 1/2) eta_i cs2 (Eq. 17)."""
    return [1.0 / (prm["m0"] / (eta * prm["d0"]) + 0.5) for eta in prm["eta"]]


def flow_shear_rates(nu, d0, c2=1.0):
    """s21, s22 from nu by Eq. 16."""
    cs2 = d0 * c2
    return 1.0 / (2.0 * nu / (c2 - cs2) + 0.5), 1.0 / (nu / cs2 + 0.5)


# ----------------------------------------------------------------------------
# the step
# ----------------------------------------------------------------------------

class Oracle3D:
    """State and time stepping of the three-dimensional DD-CCLB method.

    ``params``: nx, ny, nz, nphase, rho, nu, sigma, width, eps0, d0, m0, eta
    (N-1), s_f = (s0, s21) of the D3Q7 phase lattice, s_g = (s0, s1, s3, s4)
    of the D3Q15 flow lattice, rho0, body_force (3).  Fields: ``f``
    (N-1, 7, nz, ny, nx), ``g`` (15, nz, ny, nx), lagged ``a`` (3: xy, yz,
    zx), ``psiCu`` (N-1, 3), ``T`` (6: xx, yy, zz, xy, yz, zx), ``psimu``.
    """

    def __init__(self, params, psi, C0, cos_theta, cos_theta_field=None, frozen_flow=False):
        prm = dict(params)
        self.prm = prm
        self.N = int(prm["nphase"])
        self.shape = (int(prm["nz"]), int(prm["ny"]), int(prm["nx"]))
        self.d0 = float(prm["d0"])
        self.cs2 = self.d0
        self.w7 = weights7(self.d0)
        self.w15 = weights15(self.d0)
        self.frozen = bool(frozen_flow)
        self.psi = torch.as_tensor(psi, dtype=DT)
        if cos_theta_field is not None:
            ct = torch.as_tensor(cos_theta_field, dtype=DT)
            self.cos_iN = [ct[i] for i in range(self.N - 1)]
        else:
            self.cos_iN = [torch.full(self.shape, float(cos_theta[i]), dtype=DT)
                           for i in range(self.N - 1)]
        H7 = hermite7(self.d0)
        sf = prm["s_f"]
        self.Lam_f = [collision_matrix(H7, rates7(sf[0], s1, sf[1])) for s1 in derived_rates(prm)]
        self.H = hermite15(self.d0)
        self.Hinv = torch.linalg.inv(self.H)
        self.init_state(torch.as_tensor(C0, dtype=DT))

    def volume_fractions(self, f):
        """phi C_i = sum_p f^i_p, C_i = phi C_i / phi, C_N = 1 - sum."""
        psiC = [f[i].sum(dim=0) for i in range(self.N - 1)]
        C = [pc / self.psi for pc in psiC]
        return psiC, C + [1.0 - sum(C)]

    def init_state(self, C0):
        """f = f^eq(C0, mu(C0), u = 0), g = g^eq(P = 0, u = 0), lagged zero
        (reading R13)."""
        N, z = self.N, torch.zeros(self.shape, dtype=DT)
        C = [C0[i] for i in range(N - 1)]
        C = C + [1.0 - sum(C)]
        cp = pair_cosines(self.cos_iN, self.prm["sigma"])
        psi_mu, _, _ = chemical_potentials(C, self.psi, cp, self.prm, self.w15, self.cs2)
        self.f = torch.stack([f_equilibrium(self.psi * C[i], psi_mu[i], (z, z, z),
                                            self.prm["eta"][i], self.w7, self.cs2)
                              for i in range(N - 1)])
        self.g = g_equilibrium(z, torch.zeros((15,) + self.shape, dtype=DT),
                               self.prm["rho0"], self.w15, self.cs2)
        self.P = z.clone()
        self.a = torch.zeros((3,) + self.shape, dtype=DT)
        self.psiCu = torch.zeros((N - 1, 3) + self.shape, dtype=DT)
        self.T = torch.zeros((6,) + self.shape, dtype=DT)
        self.psimu = z.clone()
        self.steps = 0

    def fields(self):
        """Everything the step computes before collision."""
        prm, w, cs2, N, psi = self.prm, self.w15, self.cs2, self.N, self.psi
        psiC, C = self.volume_fractions(self.f)
        rho = sum(C[i] * prm["rho"][i] for i in range(N))
        nu = sum(C[i] * prm["nu"][i] for i in range(N))
        s21, s22 = flow_shear_rates(nu, self.d0)
        cp = pair_cosines(self.cos_iN, prm["sigma"])
        psi_mu, mu, gpsi = chemical_potentials(C, psi, cp, prm, w, cs2)
        gradC = [grad(C[j], w, cs2) for j in range(N)]
        gradmu = [grad(mu[j], w, cs2) for j in range(N)]
        m0 = prm["m0"]
        M = mobility(C, m0)
        S = []
        for i in range(N - 1):
            comp = []
            for a in range(3):
                v = (psi * M[i][i] - psi * m0) / m0 * gradmu[i][a]
                for j in range(N):
                    if j != i:
                        v = v + psi * M[i][j] / m0 * gradmu[j][a]
                comp.append(v)
            S.append(comp)
        mC = []
        for a in range(3):
            v = torch.zeros_like(psi)
            for i in range(N):
                for j in range(N):
                    v = v - prm["rho"][i] * M[i][j] * gradmu[j][a]
            mC.append(v)
        # F' = sum psi mu_i grad C_i - div A (lagged, R25) + psi rho b
        F = [sum(psi_mu[i] * gradC[i][a] for i in range(N)) for a in range(3)]
        # A_jk = psi (m^C_j u_k - u_j m^C_k) / 2 with a_xy = A_xy, a_yz = A_yz,
        # a_zx = A_zx; -(div A)_k = -sum_j d_j A_jk
        gxy, gyz, gzx = (grad(self.a[k], w, cs2) for k in range(3))
        F[0] = F[0] + gxy[1] - gzx[2]           # -(d_y A_yx + d_z A_zx)
        F[1] = F[1] - gxy[0] + gyz[2]           # -(d_x A_xy + d_z A_zy)
        F[2] = F[2] + gzx[0] - gyz[1]           # -(d_x A_xz + d_y A_yz)
        b = prm["body_force"]
        F = [F[a] + psi * rho * b[a] for a in range(3)]
        damp = (1.0 - psi) / prm["eps0"] ** 3
        grad_rho = grad(rho, w, cs2)
        grad_psirho = grad(psi * rho, w, cs2)
        K, Hc = pressure_constants(self.d0, s21)
        sg0 = prm["s_g"][0]
        A = 0.5 + K * (1.0 - self.d0) * (2.0 - sg0) / (2.0 * sg0)
        cP = cs2 / (1.0 - w[0])
        sum_g = self.g[1:].sum(dim=0)
        if self.frozen:
            u = [torch.zeros_like(psi) for _ in range(3)]
            P = self.P
        else:
            J = [sum(c[a] * self.g[p] for p, c in enumerate(C15) if c[a]) for a in range(3)]
            den = psi * rho + 0.5 * damp
            u0 = [(J[a] + 0.5 * F[a]) / den for a in range(3)]
            e = [0.5 * gpsi[a] / den for a in range(3)]
            kk = K / 2.0 - w[0] / (1.0 - cs2)
            bv = [A * psi * grad_rho[a] + kk * psi * mC[a] + Hc / s21 * grad_psirho[a]
                  for a in range(3)]
            gam = kk * psi * rho
            G0 = sum_g - K / 2.0 * self.psimu

            def dot(x, y):
                return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]
            qa = cP * gam * dot(e, e)
            qb = cP * (dot(bv, e) + 2.0 * gam * dot(u0, e)) - psi
            qc = cP * (G0 + dot(bv, u0) + gam * dot(u0, u0))
            root = torch.sqrt(torch.clamp(qb * qb - 4.0 * qa * qc, min=0.0))
            P = -2.0 * qc / torch.where(qb < 0, qb - root, qb + root)
            u = [u0[a] + P * e[a] for a in range(3)]
            F = [F[a] + P * gpsi[a] for a in range(3)]
        F = [F[a] - damp * u[a] for a in range(3)]
        u_grad_rho = u[0] * grad_rho[0] + u[1] * grad_rho[1] + u[2] * grad_rho[2]
        psimu = psi * (rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
                       + mC[0] * u[0] + mC[1] * u[1] + mC[2] * u[2])
        return dict(psiC=psiC, C=C, rho=rho, s21=s21, s22=s22, psi_mu=psi_mu, mu=mu,
                    grad_psi=gpsi, S=S, mC=mC, F=F, u=u, P=P, psiP=psi * P,
                    u_grad_rho=u_grad_rho, grad_psirho=grad_psirho, psimu=psimu)

    def step(self, n=1):
        for _ in range(int(n)):
            self._step()

    def _step(self):
        prm, cs2, N, psi = self.prm, self.cs2, self.N, self.psi
        fl = self.fields()
        u = fl["u"]
        f_post, new_psiCu = [], []
        for i in range(N - 1):
            eta = prm["eta"][i]
            psiCu = [fl["psiC"][i] * u[a] for a in range(3)]
            V = [psiCu[a] - self.psiCu[i, a]
                 + cs2 * eta * (fl["mu"][i] * fl["grad_psi"][a] - fl["S"][i][a]) for a in range(3)]
            feq = f_equilibrium(fl["psiC"][i], fl["psi_mu"][i], u, eta, self.w7, cs2)
            Fi = f_source(V, self.w7, cs2)
            Lam = self.Lam_f[i]
            fi = self.f[i]
            post = (fi - torch.einsum("pq,q...->p...", Lam, fi - feq) + Fi
                    - 0.5 * torch.einsum("pq,q...->p...", Lam, Fi))
            f_post.append(post)
            new_psiCu.append(torch.stack(psiCu))
        self.f = stream(torch.stack(f_post), C7)
        self.psiCu = torch.stack(new_psiCu)
        if not self.frozen:
            mC, rho = fl["mC"], fl["rho"]
            s = s_vector(psi, rho, u, mC, self.w15, cs2)
            geq = g_equilibrium(fl["psiP"], s, prm["rho0"], self.w15, cs2)
            T = [psi * mC[a] * u[a] for a in range(3)]
            T += [0.5 * (psi * mC[a] * u[b] + psi * u[a] * mC[b]) for (a, b) in PAIRS]
            T = torch.stack(T)
            dT = T - self.T
            gpr = fl["grad_psirho"]
            ugpr = u[0] * gpr[0] + u[1] * gpr[1] + u[2] * gpr[2]
            M2G = [dT[a] + 2.0 * cs2 * u[a] * gpr[a] + (1.0 - 3.0 * cs2) * ugpr for a in range(3)]
            M2G += [dT[3 + k] + cs2 * (u[a] * gpr[b] + gpr[a] * u[b]) for k, (a, b) in enumerate(PAIRS)]
            G = g_source(psi * fl["u_grad_rho"], fl["F"], M2G, self.w15, cs2)
            sg = prm["s_g"]
            one = torch.ones_like(psi)
            rates = torch.stack([sg[0] * one] + [sg[1] * one] * 3 + [fl["s21"]] * 3
                                + [fl["s22"]] * 3 + [sg[2] * one] * 4 + [sg[3] * one])

            def lam_g(v):
                m = torch.einsum("ap,p...->a...", self.H, v)
                return torch.einsum("pa,a...->p...", self.Hinv, rates * m)
            g_post = self.g - lam_g(self.g - geq) + G - 0.5 * lam_g(G)
            self.g = stream(g_post, C15)
            self.a = torch.stack([0.5 * psi * (mC[a] * u[b] - u[a] * mC[b]) for (a, b) in PAIRS])
            self.T = T
            self.P = fl["P"]
            self.psimu = fl["psimu"]
        self.steps += 1

    def mass(self):
        """Per-phase sum_x sum_p f^i_p (= sum_x psi C_i)."""
        return self.f.sum(dim=(1, 2, 3, 4))

    def macroscopic(self):
        """C_1..C_N, rho, u (3), P and mu_1..mu_N of the current state, as
        the next step computes them."""
        fl = self.fields()
        return dict(C=torch.stack(fl["C"]), rho=fl["rho"], ux=fl["u"][0], uy=fl["u"][1],
                    uz=fl["u"][2], P=fl["P"], mu=torch.stack(fl["mu"]))
