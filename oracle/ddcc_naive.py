"""Second, independent transcription of one DD-CCLB time step (test
infrastructure).

Only the tests may import this module.  It restates Sec. 3 of the paper a
second time, node by node, in plain Python floats and small numpy matrices,
sharing no code with ``ddcc_oracle`` (the whole-grid torch transcription)
and none with the CUDA path.  The two transcriptions take the same readings
of the paper (R1-R14: beta_ij = 3 sigma_ij / eps, the Hermite rows, the
off-diagonal pair counted once, the lagged antisymmetric flux with u and P
solved together, the isotropic stencils, mirror ghosts and halfway
bounce-back at outer walls), but are written differently on purpose:

* the collision is the full 9 x 9 matrix Lambda = H^-1 S H per node, with
  H evaluated from the Hermite polynomials at each velocity and the inverse
  taken by a linear solve;
* the equilibria and sources are summed over the tensor indices alpha,
  beta as the paper prints them (Eqs. 3.5, 3.6, 3.8, 3.10);
* the coupled velocity / Eq. 19 pressure is found by Newton's method on P
  from the root of the linearised problem (the root the reading takes);
* streaming pushes every post-collision population to its neighbour, with
  bounce-back into the opposite direction at an outer wall.

It is meant for grids of a few dozen nodes: it is very slow.
"""
from __future__ import annotations

import math

import numpy as np

# D2Q9 (Sec. 3): p = 0 rest; 1..4 (+-c, 0), (0, +-c); 5..8 (+-c, +-c)
CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def d2q9_weight(p: int, d0: float) -> float:
    """omega_p(d0) of Sec. 3: 1 - 2 d0 + d0^2, (d0 - d0^2)/2, d0^2/4."""
    if p == 0:
        return 1.0 - 2.0 * d0 + d0 * d0
    if p <= 4:
        return (d0 - d0 * d0) / 2.0
    return d0 * d0 / 4.0


def hermite_row_values(cx: int, cy: int, cs2: float):
    """The nine Hermite polynomials (reading R2), in the order of S."""
    hx2, hy2 = cx * cx - cs2, cy * cy - cs2
    return [1.0, cx, cy, hx2, hy2, cx * cy, hx2 * cy, cx * hy2, hx2 * hy2]


def collision(d0: float, rates) -> np.ndarray:
    """Lambda = H^-1 diag(rates) H (Sec. 3)."""
    H = np.array([hermite_row_values(CX[p], CY[p], d0) for p in range(9)]).T
    return np.linalg.solve(H, np.diag(rates) @ H)


class NaiveStep:
    """Node-by-node DD-CCLB state.  ``C0`` holds the N-1 evolved volume
    fractions, ``cos_field`` the N-1 per-node cos(theta_iN) (or None with
    ``cos_uniform``)."""

    def __init__(self, prm, psi, C0, cos_uniform, cos_field=None):
        self.p = prm
        self.N = int(prm["nphase"])
        self.nx, self.ny = int(prm["nx"]), int(prm["ny"])
        self.perx, self.pery = bool(prm["periodic_x"]), bool(prm["periodic_y"])
        self.d0 = float(prm["d0"])
        self.cs2 = self.d0
        self.w = [d2q9_weight(p, self.d0) for p in range(9)]
        self.psi = np.array(psi, dtype=np.float64)
        N = self.N
        if cos_field is not None:
            self.cosN = np.array(cos_field, dtype=np.float64)
        else:
            self.cosN = np.empty((N - 1, self.ny, self.nx))
            for i in range(N - 1):
                self.cosN[i] = float(cos_uniform[i])
        sf = prm["s_f"]
        self.lam_f = []
        for eta in prm["eta"]:
            s1 = 1.0 / (prm["m0"] / (eta * self.cs2) + 0.5)          # Eq. 17
            self.lam_f.append(collision(self.d0, [sf[0], s1, s1, sf[1], sf[1], sf[2], sf[3], sf[3], sf[4]]))
        self.init(np.array(C0, dtype=np.float64))

    # -- neighbours ----------------------------------------------------------

    def _ix(self, i, n, periodic):
        if 0 <= i < n:
            return i, True
        if periodic:
            return i % n, True
        return (-i - 1 if i < 0 else 2 * n - i - 1), False    # mirror ghost

    def at(self, a, x, y, dx, dy):
        """a at (x + dx, y + dy): periodic image, or the mirror ghost node."""
        xi, _ = self._ix(x + dx, self.nx, self.perx)
        yi, _ = self._ix(y + dy, self.ny, self.pery)
        return a[..., yi, xi]

    def grad(self, a, x, y):
        """Isotropic gradient (reading R7): sum_p w_p c_p a(x + c_p) / cs2."""
        gx = gy = 0.0
        for p in range(1, 9):
            v = self.w[p] * self.at(a, x, y, CX[p], CY[p]) / self.cs2
            gx += CX[p] * v
            gy += CY[p] * v
        return gx, gy

    def div_psi_grad(self, c, x, y):
        """div(psi grad c) with the mid-link psi (reading R7)."""
        s = 0.0
        for p in range(1, 9):
            pm = 0.5 * (self.psi[y, x] + self.at(self.psi, x, y, CX[p], CY[p]))
            s += 2.0 * self.w[p] * pm * (self.at(c, x, y, CX[p], CY[p]) - c[y, x]) / self.cs2
        return s

    # -- model ---------------------------------------------------------------

    @staticmethod
    def gp(c):
        """g'(C) for g(C) = C^2 (1 - C)^2."""
        return 2.0 * c * (1.0 - c) ** 2 - 2.0 * c * c * (1.0 - c)

    def cos_pair(self, j, q, x, y):
        """cos(theta_jq) from the angles theta_iN by Eq. 2.9 (reading R10)."""
        N, sig = self.N, self.p["sigma"]
        cj = self.cosN[j, y, x] if j < N - 1 else 0.0
        cq = self.cosN[q, y, x] if q < N - 1 else 0.0
        return (sig[j][N - 1] * cj - sig[q][N - 1] * cq) / sig[j][q]

    def chem(self, C):
        """psi mu_i (Eq. 2.14) and mu_i on the whole grid."""
        N, p = self.N, self.p
        sig, eps = p["sigma"], p["width"]
        pmu = np.zeros((N, self.ny, self.nx))
        for y in range(self.ny):
            for x in range(self.nx):
                gpx, gpy = self.grad(self.psi, x, y)
                ag = math.sqrt(gpx * gpx + gpy * gpy)
                ps = self.psi[y, x]
                L = [self.div_psi_grad(C[j], x, y) for j in range(N)]
                for i in range(N):
                    v = 0.0
                    for j in range(N):
                        beta = 3.0 * sig[i][j] / eps                     # reading R1
                        v += 2.0 * beta * ps * (self.gp(C[i, y, x]) - self.gp(C[i, y, x] + C[j, y, x]))
                        v += 0.75 * eps * sig[i][j] * L[j]
                        inner = 0.0
                        for q in range(N):
                            if q != j:
                                inner += self.cos_pair(j, q, x, y) * C[j, y, x] * C[q, y, x]
                        v += 3.0 * sig[i][j] * inner * ag
                    pmu[i, y, x] = v
        return pmu, pmu / self.psi[None]

    def fractions(self):
        N = self.N
        C = np.empty((N, self.ny, self.nx))
        psiC = self.f.sum(axis=1)
        C[:N - 1] = psiC / self.psi[None]
        C[N - 1] = 1.0 - C[:N - 1].sum(axis=0)
        return psiC, C

    def init(self, C0):
        """Reading R13: f = f^eq(C0, mu(C0), u = 0), g = g^eq(P = 0, u = 0),
        lagged fields zero."""
        N = self.N
        C = np.empty((N, self.ny, self.nx))
        C[:N - 1] = C0
        C[N - 1] = 1.0 - C0.sum(axis=0)
        pmu, _ = self.chem(C)
        self.f = np.zeros((N - 1, 9, self.ny, self.nx))
        for i in range(N - 1):
            eta = self.p["eta"][i]
            for q in range(9):
                self.f[i, q] = self.w[q] * eta * pmu[i] + (self.psi * C[i] - eta * pmu[i] if q == 0 else 0.0)
        self.g = np.zeros((9, self.ny, self.nx))
        self.g[0] = self.p["rho0"]
        self.a = np.zeros((self.ny, self.nx))
        self.pcu = np.zeros((N - 1, 2, self.ny, self.nx))
        self.T = np.zeros((3, self.ny, self.nx))
        self.pmu_lag = np.zeros((self.ny, self.nx))

    # -- equilibria and sources (Sec. 3) -----------------------------------

    def g_eq(self, q, psiP, psi, rho, u, mC):
        """Eq. 3.8 with s_p; the alpha-bar sum counts the xy pair once."""
        w, cs2 = self.w[q], self.cs2
        c = (CX[q], CY[q])
        s = sum(c[al] * psi * rho * u[al] for al in range(2)) / cs2
        for al in range(2):
            s += (psi * rho * u[al] * u[al] + psi * mC[al] * u[al]) * (c[al] * c[al] - cs2) / (cs2 - cs2 * cs2)
        s += (psi * rho * u[0] * u[1] + 0.5 * (psi * mC[0] * u[1] + psi * u[0] * mC[1])) * c[0] * c[1] / (cs2 * cs2)
        s *= w
        if q == 0:
            return (w - 1.0) * psiP / cs2 + self.p["rho0"] + s
        return w * psiP / cs2 + s

    def G_src(self, q, a0, F, M2):
        """Eq. 3.10; M2 = (M_xx, M_yy, M_xy)."""
        w, cs2 = self.w[q], self.cs2
        c = (CX[q], CY[q])
        t = a0 + (c[0] * F[0] + c[1] * F[1]) / cs2
        t += (M2[0] * (c[0] * c[0] - cs2) + M2[1] * (c[1] * c[1] - cs2)) / (cs2 - cs2 * cs2)
        t += M2[2] * c[0] * c[1] / (cs2 * cs2)
        return w * t

    # -- one step ------------------------------------------------------------

    def step(self, n=1):
        for _ in range(int(n)):
            self._step()

    def _step(self):
        p, N, cs2, nx, ny = self.p, self.N, self.cs2, self.nx, self.ny
        d0, w = self.d0, self.w
        rho_i, nu_i, m0 = p["rho"], p["nu"], p["m0"]
        psiC, C = self.fractions()
        pmu, mu = self.chem(C)
        rho = np.einsum("i,iyx->yx", np.array(rho_i), C)
        nu = np.einsum("i,iyx->yx", np.array(nu_i), C)
        psirho = self.psi * rho
        sg0, sg1, sg3, sg4 = p["s_g"]
        K = 1.0 - d0                                                   # 2D, below Eq. 19
        fpost = np.empty_like(self.f)
        gpost = np.empty_like(self.g)
        a_new = np.empty_like(self.a)
        pcu_new = np.empty_like(self.pcu)
        T_new = np.empty_like(self.T)
        pmu_new = np.empty_like(self.pmu_lag)
        eps0 = p["eps0"]
        for y in range(ny):
            for x in range(nx):
                ps = self.psi[y, x]
                Cn = C[:, y, x]
                gC = [self.grad(C[j], x, y) for j in range(N)]
                gm = [self.grad(mu[j], x, y) for j in range(N)]
                gps = self.grad(self.psi, x, y)
                grho = self.grad(rho, x, y)
                gpr = self.grad(psirho, x, y)
                # Eq. 2.5
                M = np.zeros((N, N))
                for i in range(N):
                    for j in range(N):
                        if i != j:
                            M[i, j] = -m0 * Cn[i] * Cn[j]
                    M[i, i] = -sum(M[i, j] for j in range(N) if j != i)
                # m^C = -sum_ij rho_i M_ij grad mu_j (Sec. 2.2)
                mC = [-sum(rho_i[i] * M[i, j] * gm[j][al] for i in range(N) for j in range(N))
                      for al in range(2)]
                # force without P grad psi and damping; a lagged (reading R4)
                dax, day = self.grad(self.a, x, y)
                r = rho[y, x]
                F0 = [sum(pmu[i, y, x] * gC[i][al] for i in range(N)) + ps * r * p["body_force"][al]
                      for al in range(2)]
                F0[0] += day
                F0[1] -= dax
                J = [sum(CX[q] * self.g[q, y, x] for q in range(9)),
                     sum(CY[q] * self.g[q, y, x] for q in range(9))]
                damp = (1.0 - ps) / eps0 ** 3
                s21 = 1.0 / (2.0 * nu[y, x] / (1.0 - cs2) + 0.5)          # Eq. 16
                s22 = 1.0 / (nu[y, x] / cs2 + 0.5)
                H = K * (1.0 - 2.0 * d0) * (s21 - 2.0)
                Acoef = 0.5 + K * (1.0 - d0) * (2.0 - sg0) / (2.0 * sg0)
                sum_g = sum(self.g[q, y, x] for q in range(1, 9))

                def velocity(P):
                    # psi rho u = J + F / 2, F = F0 + P grad psi - damp u (Sec. 3)
                    den = ps * r + 0.5 * damp
                    return [(J[al] + 0.5 * (F0[al] + P * gps[al])) / den for al in range(2)]

                def eq19_residual(P):
                    u = velocity(P)
                    mu_dot = ps * (r * (u[0] ** 2 + u[1] ** 2) + mC[0] * u[0] + mC[1] * u[1])
                    s_rest = -w[0] * mu_dot / (1.0 - cs2)                 # s_p at p = 0
                    rhs = (sum_g + Acoef * ps * (u[0] * grho[0] + u[1] * grho[1])
                           + 0.5 * K * (mu_dot - self.pmu_lag[y, x])
                           + H / s21 * (u[0] * gpr[0] + u[1] * gpr[1]) + s_rest)
                    return ps * P - cs2 / (1.0 - w[0]) * rhs

                # Newton from the root of the problem linearised at P = 0
                r0 = eq19_residual(0.0)
                h = 1e-3 * max(1.0, abs(r0))
                slope = (eq19_residual(h) - eq19_residual(-h)) / (2 * h)
                curv = (eq19_residual(h) - 2 * r0 + eq19_residual(-h)) / (h * h)
                P = -r0 / slope
                for _ in range(60):
                    res = eq19_residual(P)
                    d = slope + curv * P                                  # R is quadratic in P
                    dP = -res / d
                    P += dP
                    if abs(dP) <= 1e-17 * max(1.0, abs(P)):
                        break
                u = velocity(P)
                F = [F0[al] + P * gps[al] - damp * u[al] for al in range(2)]
                # ---- phase populations (Eqs. 3.1, 3.5-3.7)
                for i in range(N - 1):
                    eta = p["eta"][i]
                    pcu = [psiC[i, y, x] * u[al] for al in range(2)]
                    S = [((ps * M[i, i] - ps * m0) / m0) * gm[i][al]
                         + sum(ps * M[i, j] / m0 * gm[j][al] for j in range(N) if j != i) for al in range(2)]
                    V = [(pcu[al] - self.pcu[i, al, y, x]) + cs2 * eta * (mu[i, y, x] * gps[al] - S[al])
                         for al in range(2)]
                    feq = np.empty(9)
                    Fi = np.empty(9)
                    for q in range(9):
                        if q == 0:
                            feq[q] = (w[0] - 1.0) * eta * pmu[i, y, x] + psiC[i, y, x]
                        else:
                            feq[q] = w[q] * eta * pmu[i, y, x] + w[q] * (CX[q] * pcu[0] + CY[q] * pcu[1]) / cs2
                        Fi[q] = w[q] * (CX[q] * V[0] + CY[q] * V[1]) / cs2
                    fl = self.f[i, :, y, x]
                    Lf = self.lam_f[i]
                    fpost[i, :, y, x] = fl - Lf @ (fl - feq) + Fi - 0.5 * (Lf @ Fi)
                    pcu_new[i, :, y, x] = pcu
                # ---- flow populations (Eqs. 3.2, 3.8, 3.10)
                Tn = [ps * mC[0] * u[0], ps * mC[1] * u[1], 0.5 * (ps * mC[0] * u[1] + ps * u[0] * mC[1])]
                ugpr = u[0] * gpr[0] + u[1] * gpr[1]
                M2 = [(Tn[0] - self.T[0, y, x]) + cs2 * 2.0 * u[0] * gpr[0] + (1.0 - 3.0 * cs2) * ugpr,
                      (Tn[1] - self.T[1, y, x]) + cs2 * 2.0 * u[1] * gpr[1] + (1.0 - 3.0 * cs2) * ugpr,
                      (Tn[2] - self.T[2, y, x]) + cs2 * (u[0] * gpr[1] + gpr[0] * u[1])]
                a0 = ps * (u[0] * grho[0] + u[1] * grho[1])
                geq = np.array([self.g_eq(q, ps * P, ps, r, u, mC) for q in range(9)])
                Gq = np.array([self.G_src(q, a0, F, M2) for q in range(9)])
                Lg = collision(d0, [sg0, sg1, sg1, s21, s21, s22, sg3, sg3, sg4])
                gl = self.g[:, y, x]
                gpost[:, y, x] = gl - Lg @ (gl - geq) + Gq - 0.5 * (Lg @ Gq)
                a_new[y, x] = 0.5 * ps * (mC[0] * u[1] - u[0] * mC[1])
                T_new[:, y, x] = Tn
                pmu_new[y, x] = ps * (r * (u[0] ** 2 + u[1] ** 2) + mC[0] * u[0] + mC[1] * u[1])
        # ---- streaming: push to x + c_p, or bounce back at an outer wall
        self.f = np.empty_like(fpost)
        self.g = np.empty_like(gpost)
        for y in range(ny):
            for x in range(nx):
                for q in range(9):
                    tx, okx = self._ix(x + CX[q], nx, self.perx)
                    ty, oky = self._ix(y + CY[q], ny, self.pery)
                    if okx and oky:
                        self.f[:, q, ty, tx] = fpost[:, q, y, x]
                        self.g[q, ty, tx] = gpost[q, y, x]
                    else:
                        self.f[:, OPP[q], y, x] = fpost[:, q, y, x]
                        self.g[OPP[q], y, x] = gpost[q, y, x]
        self.a, self.pcu, self.T, self.pmu_lag = a_new, pcu_new, T_new, pmu_new

    def mass(self):
        return self.f.sum(axis=(1, 2, 3))
