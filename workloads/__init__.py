"""Seeded synthetic inputs for the DD-CCLB step.

This module is shared by the CUDA path (through the Python binding, tests and
``bench.py``) and by the CPU oracle.  It holds geometry and parameter sets
only, never any arithmetic of the lattice Boltzmann method itself: it builds

* the smooth solid characteristic function psi (phi in the paper, Sec. 2.3):
  1 in the fluid, 0 in the solid, 1/2 on the wall, from a signed distance d
  as psi = 1/2 (1 + tanh(d / (sqrt(2) xi))), clamped below at psi_min;
* the initial volume fractions C_i of the N-1 evolved phases from tanh
  droplet profiles C = 1/2 (1 + tanh(2 (R - r) / W)) (the interface profile
  of the free energy in Eq. 2.1 with width W = epsilon);
* the contact angles theta_iN, uniform or as a per-node field;
* the physical parameters of each workload (densities, viscosities,
  surface tensions, widths, relaxation rates) in lattice units.

Every problem is a plain dict (``params``) plus numpy arrays, all float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MAX_PHASES = 4

# Three- and four-phase workloads take the paper's multiphase settings
# (Secs. 4.2-4.3): interface width 8 and a small eta (m0 = 0.01 at
# s1 = 1/0.8).  The constant-mobility split of Sec. 3 leaves a residual at
# triple regions that drives the derived phase below zero; it grows with m0
# and with 1/epsilon, and these settings keep it bounded.
TERNARY_WIDTH = 8.0
TERNARY_ETA = 0.1


@dataclass
class Problem:
    """One synthetic workload: parameters and initial fields (float64)."""

    name: str
    params: dict
    psi: np.ndarray                   # (ny, nx)
    C0: np.ndarray                    # (N-1, ny, nx) initial C_i, i < N
    cos_theta: np.ndarray             # (N-1,) uniform cos(theta_iN) ...
    cos_theta_field: np.ndarray | None = None   # ... or (N-1, ny, nx)
    steps: int = 0                    # step count of the workload
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return int(self.params["nx"]) * int(self.params["ny"])


def base_params(nx, ny, nphase, *, periodic_x=1, periodic_y=1, rho=None,
                nu=None, sigma=0.01, width=4.0, xi=1.0, d0=1.0 / 3.0, tau=0.8,
                eta=1.0, body_force=(0.0, 0.0), psi_min=1e-6):
    """Physical parameters in lattice units (dx = dt = c = 1).

    ``tau`` fixes the phase-LB rate s_1 = 1/tau for the given eta, i.e. the
    mobility m0 = (tau - 1/2) eta d0 (Eq. 17); the same tau is used as the
    shear rate of the flow LB, nu = (tau - 1/2) d0 (Eq. 16).  The remaining
    rates follow the single-droplet set-up of Sec. 4.1: s0 = 1 and 1.2 for
    every other rate.  ``sigma`` is a scalar (all pairs) or an N x N matrix.
    The solid diffuse-layer width is eps0 = 2 sqrt(2) xi, the width at which
    1/2 (1 + tanh(d / (sqrt 2 xi))) equals the paper's 1/2 + 1/2 tanh(2 d / eps0).
    """
    N = int(nphase)
    if not 2 <= N <= MAX_PHASES:
        raise ValueError("nphase must be in [2, 4]")
    rho = [1.0] * N if rho is None else [float(r) for r in rho]
    nu_default = (tau - 0.5) * d0
    nu = [nu_default] * N if nu is None else [float(v) for v in nu]
    if np.isscalar(sigma):
        sig = np.full((N, N), float(sigma))
        np.fill_diagonal(sig, 0.0)
    else:
        sig = np.asarray(sigma, dtype=np.float64)
    eta_l = [float(eta)] * (N - 1) if np.isscalar(eta) else [float(e) for e in eta]
    m0 = (tau - 0.5) * eta_l[0] * d0
    return {
        "nx": int(nx), "ny": int(ny), "nphase": N,
        "periodic_x": int(periodic_x), "periodic_y": int(periodic_y),
        "rho": rho, "nu": nu, "sigma": sig.tolist(),
        "width": float(width), "eps0": 2.0 * math.sqrt(2.0) * float(xi),
        "d0": float(d0), "m0": float(m0), "eta": eta_l,
        # phase LB: s0, s21, s22, s3, s4 (s1 per phase from m0 and eta_i)
        "s_f": [1.0, 1.2, 1.2, 1.2, 1.2],
        # flow LB: s0, s1, s3, s4 (s21, s22 per node from nu)
        "s_g": [1.0, 1.2, 1.2, 1.2],
        "rho0": 1.0,
        "body_force": [float(body_force[0]), float(body_force[1])],
        "psi_min": float(psi_min),
    }


# ----------------------------------------------------------------------------
# geometry helpers
# ----------------------------------------------------------------------------

def _grid(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def _min_image(d, L, periodic):
    if periodic:
        d = d - L * np.round(d / L)
    return d


def _axes(periodic):
    """(periodic_x, periodic_y) from a bool or a pair."""
    if isinstance(periodic, (tuple, list)):
        return bool(periodic[0]), bool(periodic[1])
    return bool(periodic), bool(periodic)


# Solid diffuse-layer width of the complex-geometry workloads: eps0 = 6 lattice
# units, the paper's choice next to an interface width of 8 (Sec. 4.5; Sec. 4.4
# takes eps0 = eps = 5).  On the solid side psi falls by exp(4 / eps0) per node;
# with eps0 = 2 sqrt 2 (xi = 1) that is a factor 4.1 and the solid interior of
# the 4096^2 imbibition case develops a grid-scale mode that overflows after
# ~1000 steps, while eps0 = 6 (factor 1.95) runs 4000 steps cleanly.
SOLID_XI = 3.0 / math.sqrt(2.0)

# Surface tensions of the three-phase lens and emulsion, each drawn from
# {0.005, 0.01, 0.015}: sigma_12 = 0.015, sigma_13 = sigma_23 = 0.01.  The
# assignment that uses all three values is a degenerate Neumann triangle
# (0.015 = 0.005 + 0.01, zero spreading coefficient); with it the lens point
# of the 256^2 lens overflows after ~2000 steps in both precisions, while
# this triangle runs 10^4 steps (lens) and 2 x 10^4 steps (emulsion).
LENS_SIGMA = [[0.0, 0.015, 0.01], [0.015, 0.0, 0.01], [0.01, 0.01, 0.0]]


def psi_from_distance(d, xi=1.0, psi_min=1e-6):
    """psi = 1/2 (1 + tanh(d / (sqrt 2 xi))), d > 0 in the fluid."""
    psi = 0.5 * (1.0 + np.tanh(d / (math.sqrt(2.0) * xi)))
    return np.maximum(psi, psi_min)


def drop_profile(r, R, W):
    """Tanh volume-fraction profile of a drop of radius R, width W."""
    return 0.5 * (1.0 + np.tanh(2.0 * (R - r) / W))


def _normalise(C):
    """Scale overlapping drops so that sum_{i<N} C_i <= 1 at every node."""
    s = C.sum(axis=0)
    scale = np.where(s > 1.0, 1.0 / np.maximum(s, 1e-300), 1.0)
    return C * scale[None]


def _place_circles(rng, nx, ny, n_max, rmin, rmax, gap, periodic, avoid=(),
                   target_fraction=None, max_tries=200000):
    """Random non-overlapping circles (rejection sampling).

    Returns an array (k, 3) of (cx, cy, r).  ``avoid`` is a list of
    (cx, cy, R) discs the circles must clear by ``gap``.  With
    ``target_fraction`` circles are added until their area reaches that
    fraction of the domain (or n_max circles)."""
    px, py = _axes(periodic)
    circles = []
    area = 0.0
    cell = 2.0 * rmax + gap
    gx, gy = max(1, int(nx // cell)), max(1, int(ny // cell))
    buckets = {}
    tries = 0
    while len(circles) < n_max and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        ok = True
        for (ax, ay, aR) in avoid:
            dx = _min_image(cx - ax, nx, px)
            dy = _min_image(cy - ay, ny, py)
            if dx * dx + dy * dy < (r + aR + gap) ** 2:
                ok = False
                break
        if not ok:
            continue
        bx, by = int(cx / nx * gx), int(cy / ny * gy)
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                key = ((bx + ox) % gx, (by + oy) % gy)
                for (qx, qy, qr) in buckets.get(key, ()):
                    dx = _min_image(cx - qx, nx, px)
                    dy = _min_image(cy - qy, ny, py)
                    if dx * dx + dy * dy < (r + qr + gap) ** 2:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        circles.append((cx, cy, r))
        buckets.setdefault((bx, by), []).append((cx, cy, r))
        area += math.pi * r * r
        if target_fraction is not None and area >= target_fraction * nx * ny:
            break
    return np.array(circles, dtype=np.float64).reshape(-1, 3)


def circles_distance(circles, nx, ny, periodic=True, reach=10.0, owner=False):
    """Signed distance to the union of solid circles (positive in fluid).

    Only the band within ``reach`` of a circle is resolved exactly; farther
    nodes get +reach, where psi has already saturated to 1.  With ``owner``
    the index of the nearest circle is returned too (-1 where none is within
    reach)."""
    px, py = _axes(periodic)
    d = np.full((ny, nx), reach, dtype=np.float64)
    own = np.full((ny, nx), -1, dtype=np.int64) if owner else None
    for k, (cx, cy, r) in enumerate(circles):
        ext = int(math.ceil(r + reach)) + 1
        xs = np.arange(int(math.floor(cx)) - ext, int(math.floor(cx)) + ext + 1)
        ys = np.arange(int(math.floor(cy)) - ext, int(math.floor(cy)) + ext + 1)
        if px:
            xi_u = np.unique(xs % nx)
            dx = _min_image(xi_u - cx, nx, True)
        else:
            xi_u = xs[(xs >= 0) & (xs < nx)]
            dx = xi_u - cx
        if py:
            yi_u = np.unique(ys % ny)
            dy = _min_image(yi_u - cy, ny, True)
        else:
            yi_u = ys[(ys >= 0) & (ys < ny)]
            dy = yi_u - cy
        dist = np.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2) - r
        sub = d[np.ix_(yi_u, xi_u)]
        better = dist < sub
        d[np.ix_(yi_u, xi_u)] = np.where(better, dist, sub)
        if owner:
            osub = own[np.ix_(yi_u, xi_u)]
            own[np.ix_(yi_u, xi_u)] = np.where(better, k, osub)
    return (d, own) if owner else d


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def config1_droplet_wall(nx=64, ny=64, R=16.0, wall=12.0, theta_deg=60.0,
                         nphase=2, absent_phase=None):
    """Semicircular droplet on a flat wall embedded by psi (Sec. 4.1 style).

    64x64, x periodic, walls in y, wall plane y_w = 12, xi = 1, drop radius
    16 centred on the wall plane, W = 4, rho ratio 1, tau = 0.8,
    sigma = 0.01, theta = 60 deg, 1000 steps.

    With ``nphase=3`` the same drop is set up as a ternary system whose
    phase ``absent_phase`` (2 or 3) is absent, the reduction-consistency
    case of Table 1: the drop is phase 1, the present ambient phase keeps
    the pair's surface tension and the absent phase gets theta = 90 deg
    against phase N (or phase 2), so that Eq. 2.9 returns theta_12 = theta.
    """
    x, y = _grid(nx, ny)
    psi = psi_from_distance(y - wall)
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - wall) ** 2)
    c1 = drop_profile(r, R, 4.0)
    ct = math.cos(math.radians(theta_deg))
    if nphase == 2:
        C0 = c1[None]
        cos_theta = np.array([ct])
    elif nphase == 3:
        if absent_phase == 3:
            # C1 drop, C2 ambient, C3 == 0 (the derived phase)
            C0 = np.stack([c1, 1.0 - c1])
            # theta_13 = theta, theta_23 = 90 => cos theta_12 = cos theta
            cos_theta = np.array([ct, 0.0])
        elif absent_phase == 2:
            # C1 drop, C2 == 0, C3 ambient
            C0 = np.stack([c1, np.zeros_like(c1)])
            # theta_13 = theta; theta_23 arbitrary (phase 2 absent)
            cos_theta = np.array([ct, 0.0])
        else:
            raise ValueError("absent_phase must be 2 or 3")
    else:
        raise ValueError("nphase must be 2 or 3")
    params = base_params(nx, ny, nphase, periodic_x=1, periodic_y=0,
                         sigma=0.01, width=4.0, xi=1.0, tau=0.8)
    return Problem("droplet_wall_64x64_N%d" % nphase, params, psi, C0,
                   cos_theta, None, steps=1000,
                   note="semicircular drop R=16 on a psi-embedded flat wall")


def config10_table1_drop(theta_deg=60.0, nphase=3, nx=256, ny=128, R=50.0, wall=12.0, width=8.0,
                         d0=0.4, m0=0.01):
    """The Table 1 set-up of Sec. 4.1 at its own drop size: a semicircular
    drop of radius 50 on a flat wall, computed as a ternary system with one
    phase absent (``nphase=3``: the drop is phase 1, the ambient phase 3,
    phase 2 absent, C_2 = 0) or as the two-phase system (``nphase=2``), with
    the printed d0 = 0.4, m0 = 0.01, relaxation rates (s1^f = 10/19, 1 for
    s0 and 1.2 for the others) and solid layer eps0 = 4 (xi = sqrt 2),
    nu = 0.1.  In lattice units, with one density for all phases (the
    printed 1 : 0.01 overflows in this reading of the pressure scheme),
    sigma = 0.01 and an interface width of 8 instead of 5 (with 5 the angle
    is still 5 deg from equilibrium after 4 x 10^4 steps).  The absent phase
    is one of the evolved phases: with the derived phase C_N absent the
    constant-mobility split drives C_N away from zero at the interface and
    the ternary run overflows within 10^4 - 2 x 10^4 steps (reading R16)."""
    x, y = _grid(nx, ny)
    xi = math.sqrt(2.0)
    psi = psi_from_distance(y - wall, xi=xi)
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - wall) ** 2)
    c1 = drop_profile(r, R, width)
    ct = math.cos(math.radians(theta_deg))
    s1 = 10.0 / 19.0 if abs(d0 - 0.4) < 1e-12 else 1.0 / 0.8
    eta = m0 / ((1.0 / s1 - 0.5) * d0)
    if nphase == 2:
        C0 = c1[None]
        cos_theta = np.array([ct])
    elif nphase == 3:
        C0 = np.stack([c1, np.zeros_like(c1)])  # C_2 = 0, C_3 = 1 - C_1
        cos_theta = np.array([ct, 0.0])         # theta_13 = theta; theta_23 plays no part
    else:
        raise ValueError("nphase must be 2 or 3")
    params = base_params(nx, ny, nphase, periodic_x=1, periodic_y=0, sigma=0.01, width=width, xi=xi,
                         d0=d0, tau=0.5 + 0.1 / d0, eta=eta)
    params["m0"] = m0
    params["s_f"] = [1.0, 1.2, 1.2, 1.2, 1.2]
    params["s_g"] = [1.0, 1.2, 1.2, 1.2]
    return Problem("table1_drop_%dx%d_N%d_theta%d" % (nx, ny, nphase, int(theta_deg)), params, psi, C0,
                   cos_theta, None, steps=40000,
                   note="Table 1 set-up: semicircular drop R=50 on a psi-embedded flat wall")


def config8_ternary_compound_drop(theta13_deg=90.0, theta23_deg=90.0, nx=300, ny=170, R=60.0,
                                  wall=16.0, sigma=0.005, m0=0.01, tau=0.8, d0=1.0 / 3.0,
                                  tau_f=None, rho=None, nu=0.1):
    """Sec. 4.2 / Table 2: a semicircular compound drop of radius R on a flat
    wall embedded by psi (eps0 = 6, as the paper's 0.6 / 0.1), split at its
    axis into phase 1 (left quarter disc) and phase 2 (right quarter disc),
    surrounded by phase 3; x periodic, y walled, nx x ny = 300 x 170,
    sigma_ij = 0.005, eps = 8, m0 = 0.01.  The equilibrium shape depends on
    the surface tensions, angles and volumes only, so the phases share one
    density and viscosity here (the paper's 100 : 50 : 1 densities change
    the path to equilibrium, not the equilibrium)."""
    x, y = _grid(nx, ny)
    psi = psi_from_distance(y - wall, xi=SOLID_XI)
    xc = nx / 2.0
    r = np.sqrt((x - xc) ** 2 + (y - wall) ** 2)
    W_ = TERNARY_WIDTH
    drop = drop_profile(r, R, W_)
    left = 0.5 * (1.0 - np.tanh(2.0 * (x - xc) / W_))
    C0 = np.stack([drop * left, drop * (1.0 - left)])
    params = base_params(nx, ny, 3, periodic_x=1, periodic_y=0, sigma=sigma, width=W_,
                         xi=SOLID_XI, tau=tau, eta=1.0, d0=d0, rho=rho, nu=[nu] * 3)
    # the phase LB's s1 = 1 / tau_f (Eq. 17 gives eta from m0)
    tf = tau if tau_f is None else tau_f
    params["m0"] = float(m0)
    params["eta"] = [m0 / ((tf - 0.5) * params["d0"])] * 2
    ct = np.cos(np.radians([theta13_deg, theta23_deg]))
    return Problem("ternary_compound_drop_%dx%d_t13_%g" % (nx, ny, theta13_deg), params, psi, C0, ct,
                   None, steps=100000, note="compound drop on a flat wall (Sec. 4.2, Table 2)",
                   extra={"R": R, "wall": wall, "xc": xc})


def config11_quaternary_compound_drop(theta34_deg=90.0, nx=500, ny=200, R=60.0, wall=16.0, sigma=0.005,
                                      m0=0.01, tau=0.8, d0=1.0 / 3.0, nu=0.1):
    """Sec. 4.3 / Table 3: three semicircular drops of radius R on a flat wall
    embedded by psi (eps0 = 6), side by side and touching (phases 1, 2, 3
    from left to right, centres 2R apart), surrounded by phase 4; x periodic,
    y walled, nx x ny = 500 x 200 (the paper's lattice), sigma_ij = 0.005,
    theta_14 = theta_24 = 90 deg (so theta_12 = 90 deg by Eq. 2.9), eps = 8,
    m0 = 0.01.  As for Table 2 the phases share one density and viscosity:
    the equilibrium shape depends on the tensions, angles and volumes only."""
    x, y = _grid(nx, ny)
    psi = psi_from_distance(y - wall, xi=SOLID_XI)
    xc = nx / 2.0
    W_ = TERNARY_WIDTH
    drops = [drop_profile(np.sqrt((x - (xc + dx)) ** 2 + (y - wall) ** 2), R, W_)
             for dx in (-2.0 * R, 0.0, 2.0 * R)]
    C0 = _normalise(np.stack(drops))
    params = base_params(nx, ny, 4, periodic_x=1, periodic_y=0, sigma=sigma, width=W_,
                         xi=SOLID_XI, tau=tau, eta=1.0, d0=d0, nu=[nu] * 4)
    params["m0"] = float(m0)
    params["eta"] = [m0 / ((tau - 0.5) * params["d0"])] * 3
    ct = np.cos(np.radians([90.0, 90.0, theta34_deg]))
    return Problem("quaternary_compound_drop_%dx%d_t34_%g" % (nx, ny, theta34_deg), params, psi, C0, ct,
                   None, steps=200000, note="quaternary compound drop on a flat wall (Sec. 4.3, Table 3)",
                   extra={"R": R, "wall": wall, "xc": xc})


def config2_lens(nx=256, ny=256, seed=2, n_circles=20, xi=SOLID_XI, sigma=None):
    """Three-phase liquid lens over 20 random solid circles, 256^2 periodic.

    Drops of radius 40 (phases 1 and 2) centred at (88, 128) and (168, 128)
    touch at a lens point inside phase 3.  Circles r ~ U[8, 20] with a gap
    of 4, seed 2, kept clear of the drops.  rho = 1:2:3, sigma_ij from
    LENS_SIGMA, theta_13 = 45, theta_23 = 135 deg; solid layer eps0 = 6
    (SOLID_XI).
    """
    rng = np.random.default_rng(seed)
    sx, sy = nx / 256.0, ny / 256.0
    R = 40.0 * min(sx, sy)
    drops = [(88.0 * sx, 128.0 * sy, R), (168.0 * sx, 128.0 * sy, R)]
    circles = _place_circles(rng, nx, ny, n_circles, 8.0 * min(sx, sy),
                             20.0 * min(sx, sy), 4.0, True, avoid=drops)
    d = circles_distance(circles, nx, ny, periodic=True)
    psi = psi_from_distance(d, xi=xi)
    x, y = _grid(nx, ny)
    C = []
    for (cx, cy, rr) in drops:
        dx = _min_image(x - cx, nx, True)
        dy = _min_image(y - cy, ny, True)
        C.append(drop_profile(np.sqrt(dx * dx + dy * dy), rr, TERNARY_WIDTH))
    C0 = _normalise(np.stack(C))
    if sigma is None:
        sigma = LENS_SIGMA
    params = base_params(nx, ny, 3, rho=[1.0, 2.0, 3.0], sigma=sigma,
                         width=TERNARY_WIDTH, xi=xi, tau=0.8, eta=TERNARY_ETA)
    cos_theta = np.array([math.cos(math.radians(45.0)),
                          math.cos(math.radians(135.0))])
    return Problem("lens_%dx%d_N3" % (nx, ny), params, psi, C0, cos_theta,
                   None, steps=10000, extra={"circles": circles},
                   note="two R=40 drops touching at a lens over 20 circles")


def config3_emulsion(nx=1024, ny=1024, seed=3, porosity=0.6, n_drops=40, xi=SOLID_XI,
                     sigma=None):
    """40-drop emulsion in a random-circle matrix at porosity 0.6, 1024^2.

    Circles r ~ U[8, 20] (gap 4) are added until their area is 40% of the
    domain; drops R ~ U[10, 30] are placed in pore space (clear of circles
    and of each other), alternating phases 1 and 2 inside phase 3.  Same
    fluid parameters as the lens case plus a body force 1e-6 along x; solid
    layer eps0 = 6 (SOLID_XI)."""
    rng = np.random.default_rng(seed)
    s = nx / 1024.0
    circles = _place_circles(rng, nx, ny, 100000, 8.0 * s, 20.0 * s, 4.0 * s,
                             True, target_fraction=1.0 - porosity)
    d = circles_distance(circles, nx, ny, periodic=True)
    psi = psi_from_distance(d, xi=xi)
    drops = []
    tries = 0
    while len(drops) < n_drops and tries < 200000:
        tries += 1
        R = rng.uniform(10.0, 30.0) * s
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        ok = True
        for (qx, qy, qr) in circles:
            dx = _min_image(cx - qx, nx, True)
            dy = _min_image(cy - qy, ny, True)
            if dx * dx + dy * dy < (R + qr) ** 2:
                ok = False
                break
        if ok:
            for (qx, qy, qr) in drops:
                dx = _min_image(cx - qx, nx, True)
                dy = _min_image(cy - qy, ny, True)
                if dx * dx + dy * dy < (R + qr) ** 2:
                    ok = False
                    break
        if ok:
            drops.append((cx, cy, R))
    C0 = _drops_field(drops, nx, ny, 3, periodic=True, W=TERNARY_WIDTH)
    if sigma is None:
        sigma = LENS_SIGMA
    params = base_params(nx, ny, 3, rho=[1.0, 2.0, 3.0], sigma=sigma,
                         width=TERNARY_WIDTH, xi=xi, tau=0.8, eta=TERNARY_ETA,
                         body_force=(1e-6, 0.0))
    cos_theta = np.array([math.cos(math.radians(45.0)),
                          math.cos(math.radians(135.0))])
    return Problem("emulsion_%dx%d_N3" % (nx, ny), params, psi, C0, cos_theta,
                   None, steps=20000, extra={"circles": circles, "drops": drops},
                   note="40-drop emulsion in a porous matrix, porosity 0.6")


def _drops_field(drops, nx, ny, nphase, periodic=True, W=4.0):
    """Volume fractions of drops cycling over phases 1..N-1 (window-local)."""
    px, py = _axes(periodic)
    C = np.zeros((nphase - 1, ny, nx))
    for k, (cx, cy, R) in enumerate(drops):
        ph = k % (nphase - 1)
        ext = int(math.ceil(R + 3 * W)) + 1
        xs = np.arange(int(cx) - ext, int(cx) + ext + 1)
        ys = np.arange(int(cy) - ext, int(cy) + ext + 1)
        if px:
            xw_u = np.unique(xs % nx)
            dx = _min_image(xw_u - cx, nx, True)
        else:
            xw_u = xs[(xs >= 0) & (xs < nx)]
            dx = xw_u - cx
        if py:
            yw_u = np.unique(ys % ny)
            dy = _min_image(yw_u - cy, ny, True)
        else:
            yw_u = ys[(ys >= 0) & (ys < ny)]
            dy = yw_u - cy
        prof = drop_profile(np.sqrt(dy[:, None] ** 2 + dx[None, :] ** 2), R, W)
        sub = C[ph][np.ix_(yw_u, xw_u)]
        C[ph][np.ix_(yw_u, xw_u)] = np.maximum(sub, prof)
    return _normalise(C)


def config4_imbibition(nx=4096, ny=4096, seed=4, n_circles=2000,
                       drop_fraction=0.15, xi=SOLID_XI, psi_min=1e-6):
    """Four-phase imbibition in a porous medium of 2000 circles, 4096^2.

    Circles r ~ U[20, 40] (gap 4, ~34% solid), each with its own contact
    angles theta_iN ~ U[30, 150] deg (i = 1..3); every node takes the
    angles of its nearest circle.  Drops R ~ U[15, 60] cycle over phases
    1..3 until they fill ~15% of the domain.  rho = (1, 0.8, 0.5, 0.1) and
    sigma_ij = 0.005 (Sec. 4.3), tau = 0.8, solid layer eps0 = 6 (SOLID_XI).
    Smaller grids scale the circle count and radii with the domain."""
    rng = np.random.default_rng(seed)
    s = nx / 4096.0
    n_c = max(1, int(round(n_circles * s * s)))
    rmin, rmax = max(20.0 * s, 3.0), max(40.0 * s, 5.0)
    circles = _place_circles(rng, nx, ny, n_c, rmin, rmax, 4.0, True)
    d, own = circles_distance(circles, nx, ny, periodic=True, owner=True)
    psi = psi_from_distance(d, xi=xi, psi_min=psi_min)
    th = rng.uniform(30.0, 150.0, size=(len(circles), 3))
    cos_c = np.cos(np.radians(th))
    cos_field = np.zeros((3, ny, nx))
    has = own >= 0
    for i in range(3):
        cos_field[i][has] = cos_c[own[has], i]
    drops = []
    area = 0.0
    tries = 0
    dmin, dmax = max(15.0 * s, 3.0), max(60.0 * s, 6.0)
    while area < drop_fraction * nx * ny and tries < 500000:
        tries += 1
        R = rng.uniform(dmin, dmax)
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        if d[int(cy) % ny, int(cx) % nx] <= 0.0:
            continue                       # drop centres lie in pore space
        drops.append((cx, cy, R))
        area += math.pi * R * R
    C0 = _drops_field(drops, nx, ny, 4, periodic=True, W=TERNARY_WIDTH)
    params = base_params(nx, ny, 4, rho=[1.0, 0.8, 0.5, 0.1], sigma=0.005,
                         width=TERNARY_WIDTH, xi=xi, tau=0.8, eta=TERNARY_ETA, psi_min=psi_min)
    return Problem("imbibition_%dx%d_N4" % (nx, ny), params, psi, C0,
                   cos_c.mean(axis=0), cos_field, steps=5000,
                   extra={"circles": circles},
                   note="droplets imbibing a porous medium, theta per circle")


def config5_wavy_wall(nx=256, ny=256, theta_deg=60.0, R=30.0, x_drop=100.0, xi=SOLID_XI):
    """Droplet on a sinusoidal wall (amplitude 8, wavelength 64), 256^2.

    x periodic, walls in y, wall y_w(x) = 48 + 8 sin(2 pi x / 64), psi from
    the vertical distance y - y_w(x); drop radius 30 centred on the wall at
    x = 100; a uniform theta = 60 deg given as a per-node field; solid layer
    eps0 = 6 (SOLID_XI)."""
    s = nx / 256.0
    x, y = _grid(nx, ny)
    yw = 48.0 * s + 8.0 * s * np.sin(2.0 * np.pi * x / (64.0 * s))
    psi = psi_from_distance(y - yw, xi=xi)
    xd = x_drop * s
    yd = 48.0 * s + 8.0 * s * math.sin(2.0 * math.pi * xd / (64.0 * s))
    dx = _min_image(x - xd, nx, True)
    r = np.sqrt(dx * dx + (y - yd) ** 2)
    C0 = drop_profile(r, R * s, 4.0)[None]
    ct = math.cos(math.radians(theta_deg))
    cos_field = np.full((1, ny, nx), ct)
    params = base_params(nx, ny, 2, periodic_x=1, periodic_y=0, sigma=0.01,
                         width=4.0, xi=xi, tau=0.8)
    return Problem("wavy_wall_%dx%d_N2" % (nx, ny), params, psi, C0,
                   np.array([ct]), cos_field, steps=2000,
                   note="drop on a sinusoidal wall, theta field 60 deg")


def config6_wavy_channel(L=150, theta13=(120.0, 120.0), theta23=(60.0, 60.0), u_mean=0.003):
    """Compound drop driven through a wavy channel (Sec. 4.5), L x L.

    Two solids with their own characteristic functions,
    psi_1 = 1/2 + 1/2 tanh(2 (y - L/4 - B(x)) / eps0) (bottom wall) and
    psi_2 = 1/2 - 1/2 tanh(2 (y - 3L/4 - U(x)) / eps0) (top wall), with
    U(x) = -B(x) = 0.05 L sqrt(x/L) sin(3 pi x / L) and eps0 = 6; angles
    theta^k_13, theta^k_23 per wall k.  A concentric drop, inner radius L/5
    (phase 1) and outer radius L/3 (phase 2), at (L/2, L/2) in phase 3;
    rho = (1, 1, 0.1), sigma_ij = 0.004, m0 = 0.01, eps = 8, d0 = 0.3.  Two
    drives: ``params`` (periodic x) carries a body force giving the mean
    velocity u_mean (plane Poiseuille: b = 12 nu u_mean / H^2, H = L/2);
    ``extra["open_x"]`` is the paper's parabolic inflow/outflow profile, for
    a run with open x ends (periodic_x = 0, no body force)."""
    x, y = _grid(L, L)
    U = 0.05 * L * np.sqrt(x / L) * np.sin(3.0 * np.pi * x / L)
    B = -U
    eps0 = 6.0
    psi1 = np.maximum(0.5 + 0.5 * np.tanh(2.0 * (y - L / 4.0 - B) / eps0), 1e-6)
    psi2 = np.maximum(0.5 - 0.5 * np.tanh(2.0 * (y - 3.0 * L / 4.0 - U) / eps0), 1e-6)
    r = np.sqrt((x - L / 2.0) ** 2 + (y - L / 2.0) ** 2)
    c1 = drop_profile(r, L / 5.0, TERNARY_WIDTH)
    c2 = drop_profile(r, L / 3.0, TERNARY_WIDTH) * (1.0 - c1)
    C0 = _normalise(np.stack([c1, c2]))
    d0, tau = 0.3, 0.8
    nu = (tau - 0.5) * d0
    H = L / 2.0
    body = 12.0 * nu * u_mean / (H * H)
    params = base_params(L, L, 3, periodic_x=1, periodic_y=0, rho=[1.0, 1.0, 0.1], sigma=0.004,
                         width=TERNARY_WIDTH, xi=eps0 / (2.0 * math.sqrt(2.0)), d0=d0, tau=tau,
                         eta=TERNARY_ETA, body_force=(body, 0.0))
    # m0 = 0.01 (Sec. 4.5): eta from Eq. 17 at s1 = 1 / tau
    params["eta"] = [0.01 / ((tau - 0.5) * d0)] * 2
    params["m0"] = 0.01
    walls = []
    for k, (p_k) in enumerate((psi1, psi2)):
        walls.append((p_k, np.array([math.cos(math.radians(theta13[k])),
                                     math.cos(math.radians(theta23[k]))])))
    # the paper's inflow / outflow: a parabolic profile of mean u_mean across
    # the gap between the walls at x = 0 (B(0) = U(0) = 0), ambient phase in
    ys = np.arange(L) + 0.0
    gap = np.clip((ys - L / 4.0) * (3.0 * L / 4.0 - ys), 0.0, None)
    u_in = 6.0 * u_mean * gap / (L / 2.0) ** 2
    open_x = (u_in, np.zeros((2, L)))
    return Problem("wavy_channel_%dx%d_N3" % (L, L), params, psi1 * psi2, C0, None, None,
                   steps=20000, extra={"walls": walls, "open_x": open_x},
                   note="compound drop through a wavy channel, two walls with their own angles")


def random_problem(nx, ny, nphase, seed, *, periodic_x=1, periodic_y=1,
                   theta_field=False, n_circles=None, n_drops=None,
                   rho=None, nu=None, sigma=None, body_force=(0.0, 0.0),
                   d0=1.0 / 3.0, tau=0.8, width=4.0):
    """Small random problem for parity tests on ragged grids.

    Random solid circles (radius >= 4, psi with xi = 1), a wall plane near
    the bottom when y is not periodic, drops of radius >= 1.5 W cycling over
    the evolved phases, random per-phase densities, viscosities and surface
    tensions unless given, and contact angles in [45, 135] deg: uniform, or
    per circle as a field (each node takes the angles of its nearest
    circle, the wall plane its own)."""
    rng = np.random.default_rng(seed)
    N = int(nphase)
    L = min(nx, ny)
    per = (bool(periodic_x), bool(periodic_y))
    nc = n_circles if n_circles is not None else max(1, (nx * ny) // 900)
    circles = _place_circles(rng, nx, ny, nc, max(4.0, L / 10), max(5.0, L / 7),
                             3.0, per)
    d, own = circles_distance(circles, nx, ny, periodic=per, owner=True)
    x, y = _grid(nx, ny)
    if not periodic_y:
        yw = 0.2 * ny
        plane = y - yw
        own = np.where(plane < d, len(circles), own)
        d = np.minimum(d, plane)              # a wall plane near the bottom
    psi = psi_from_distance(d)
    nd = n_drops if n_drops is not None else max(N - 1, (nx * ny) // 500)
    Rmin, Rmax = 1.5 * width, max(1.5 * width + 1.0, L / 4)
    drops = [(rng.uniform(0, nx), rng.uniform(0.3 * ny, 0.9 * ny),
              rng.uniform(Rmin, Rmax)) for _ in range(nd)]
    C0 = _drops_field(drops, nx, ny, N, periodic=per, W=width)
    if rho is None:
        rho = list(rng.uniform(0.5, 2.0, size=N))
    if nu is None:
        nu = list(rng.uniform(0.05, 0.15, size=N))
    if sigma is None:
        sg = rng.uniform(0.006, 0.012, size=(N, N))
        sigma = np.triu(sg, 1) + np.triu(sg, 1).T
    params = base_params(nx, ny, N, periodic_x=periodic_x, periodic_y=periodic_y,
                         rho=rho, nu=nu, sigma=sigma, width=width, xi=1.0,
                         d0=d0, tau=tau, body_force=body_force)
    # the ternary and quaternary settings of Secs. 4.2-4.3: a small mobility
    # and a small eta keep the derived phase from undershooting at triple
    # regions (the constant-m0 split of Sec. 3 leaves a residual there)
    if N > 2:
        params["m0"] = 0.01
        params["eta"] = list(rng.uniform(0.08, 0.15, size=N - 1))
    else:
        params["eta"] = list(rng.uniform(0.8, 1.2, size=N - 1))
    n_owner = len(circles) + 1
    ang = rng.uniform(45.0, 135.0, size=(n_owner, N - 1))
    ct = np.cos(np.radians(ang.mean(axis=0)))
    cf = None
    if theta_field:
        cf = np.empty((N - 1, ny, nx))
        o = np.where(own >= 0, own, n_owner - 1)
        for i in range(N - 1):
            cf[i] = np.cos(np.radians(ang[o, i]))
    return Problem("random_%dx%d_N%d_s%d" % (nx, ny, N, seed), params, psi, C0,
                   ct, cf, steps=0, note="random parity case")


def random_small(nphase, seed, *, nx=8, ny=8, periodic_y=1):
    """Small grid with every input drawn at random, node by node, for
    brute-force agreement tests: psi in [0.3, 1], volume fractions from a
    flat Dirichlet distribution, per-node contact angles, random densities,
    viscosities, surface tensions, d0, eta and relaxation rates, and a body
    force, so that every term of the step is active from the first step."""
    rng = np.random.default_rng(seed)
    N = int(nphase)
    sg = rng.uniform(0.02, 0.06, size=(N, N))
    sigma = np.triu(sg, 1) + np.triu(sg, 1).T
    params = base_params(nx, ny, N, periodic_y=periodic_y,
                         rho=list(rng.uniform(0.5, 3.0, size=N)),
                         nu=list(rng.uniform(0.05, 0.2, size=N)), sigma=sigma, width=3.0,
                         xi=1.0, d0=float(rng.uniform(0.3, 0.45)),
                         body_force=(1e-4, -5e-5))
    params["m0"] = 0.05
    params["eta"] = list(rng.uniform(0.5, 1.5, size=N - 1))
    params["s_f"] = list(rng.uniform(0.8, 1.6, size=5))
    params["s_g"] = list(rng.uniform(0.8, 1.6, size=4))
    psi = rng.uniform(0.3, 1.0, size=(ny, nx))
    C = rng.dirichlet(np.ones(N), size=(ny, nx))            # (ny, nx, N)
    C0 = np.ascontiguousarray(np.moveaxis(C[..., :N - 1], -1, 0))
    cf = rng.uniform(-0.8, 0.8, size=(N - 1, ny, nx))
    return Problem("random_small_%dx%d_N%d_s%d" % (nx, ny, N, seed), params, psi, C0,
                   cf.mean(axis=(1, 2)), cf, steps=50, note="brute-force agreement case")


def config(k, **kw):
    """Workload k = 1..5 at full size (keyword overrides allowed)."""
    return {1: config1_droplet_wall, 2: config2_lens, 3: config3_emulsion,
            4: config4_imbibition, 5: config5_wavy_wall}[k](**kw)


# ----------------------------------------------------------------------------
# three-dimensional workloads (D3Q7 phase / D3Q15 flow lattices)
# ----------------------------------------------------------------------------

def base_params_3d(nx, ny, nz, nphase, *, rho=None, nu=None, sigma=0.01, width=4.0,
                   xi=1.0, d0=1.0 / 3.0, tau=0.8, eta=1.0, body_force=(0.0, 0.0, 0.0),
                   psi_min=1e-6):
    """Parameters of a periodic 3D box; as ``base_params`` with the D3Q7
    phase rates (s0, s21) and the D3Q15 flow rates (s0, s1, s3, s4).

    The flow's fourth-order rate is s4 = 0.8, not the 1.2 of Secs. 4.1-4.4:
    with s0 = 1 and s4 = 1.2 the pressure of Eq. 19, formed from the moving
    populations only, has a checkerboard mode (-1)^(x+y+z) on D3Q15 that
    grows by a factor 1.34-1.35 per step (every D3Q15 velocity changes the
    parity of x+y+z, so the two sublattices meet only in the collision);
    with s4 = 0.8 the linearised bulk update has no mode outside the unit
    circle.  s4 relaxes a ghost moment that does not enter the Navier-Stokes
    limit."""
    prm = base_params(nx, ny, nphase, rho=rho, nu=nu, sigma=sigma, width=width, xi=xi,
                      d0=d0, tau=tau, eta=eta, psi_min=psi_min)
    prm.pop("periodic_x")
    prm.pop("periodic_y")
    prm["nz"] = int(nz)
    prm["s_f"] = [1.0, 1.2]
    prm["s_g"] = [1.0, 1.2, 1.2, 0.8]
    prm["body_force"] = [float(v) for v in body_force]
    return prm


def _grid3(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz) + 0.0, np.arange(ny) + 0.0, np.arange(nx) + 0.0,
                          indexing="ij")
    return x, y, z


def _dist3(x, y, z, c, shape):
    """Periodic (minimum-image) distance from every node to point c."""
    nz, ny, nx = shape
    dx = np.abs(x - c[0])
    dy = np.abs(y - c[1])
    dz = np.abs(z - c[2])
    dx = np.minimum(dx, nx - dx)
    dy = np.minimum(dy, ny - dy)
    dz = np.minimum(dz, nz - dz)
    return np.sqrt(dx * dx + dy * dy + dz * dz)


def config7_sphere(L=256, N=3, Rs=None, R0=None, theta_deg=(90.0, 90.0), xi=SOLID_XI,
                   width=TERNARY_WIDTH, sigma=0.01):
    """Sec. 4.4: a hemispherical compound drop of radius R0 sitting on a
    solid sphere of radius Rs at the centre of a periodic L^3 box; the drop
    is split into phase 1 (x < centre) and phase 2 (x >= centre), both with
    the same density, viscosity and wettability, immersed in phase 3.
    Arrays are (L, L, L) in (z, y, x) order."""
    Rs = 0.2 * L if Rs is None else Rs
    R0 = 0.3 * L if R0 is None else R0
    x, y, z = _grid3(L, L, L)
    c = (L / 2 - 0.3, L / 2 - 0.2, L / 2 - 0.1)
    rs = _dist3(x, y, z, c, (L, L, L))
    psi = psi_from_distance(rs - Rs, xi=xi)
    # hemisphere above the sphere's equator (y >= centre)
    drop = drop_profile(rs, R0, width) * (0.5 * (1.0 + np.tanh(2.0 * (y - c[1]) / width)))
    left = 0.5 * (1.0 - np.tanh(2.0 * (x - c[0]) / width))
    C0 = np.zeros((N - 1, L, L, L))
    C0[0] = drop * left
    if N > 2:
        C0[1] = drop * (1.0 - left)
    # d0 = 0.4 and s0 = s21 = 1 of the phase lattice as in Sec. 4.4 (the
    # D3Q7 rest weight 1 - 3 d0 is then negative, as it is there)
    params = base_params_3d(L, L, L, N, sigma=sigma, width=width, xi=xi, eta=TERNARY_ETA, d0=0.4)
    params["s_f"] = [1.0, 1.0]
    params["m0"] = 0.01
    ct = np.cos(np.radians(np.asarray(theta_deg[:N - 1], dtype=np.float64)))
    return Problem("sphere_%d^3_N%d" % (L, N), params, psi, C0, ct, None, steps=1000,
                   note="compound drop on a solid sphere (Sec. 4.4), periodic box")


def random_problem_3d(nx, ny, nz, nphase, seed, *, theta_field=False, n_spheres=None,
                      n_drops=None, width=4.0, d0=1.0 / 3.0, tau=0.8):
    """Small random 3D problem for parity tests: random solid spheres
    (psi with xi = 1), drops cycling over the evolved phases, random
    densities, viscosities and surface tensions, and contact angles in
    [45, 135] deg, uniform or per sphere (each node takes the angles of
    its nearest sphere)."""
    rng = np.random.default_rng(seed)
    N = int(nphase)
    shape = (nz, ny, nx)
    x, y, z = _grid3(nx, ny, nz)
    L = min(nx, ny, nz)
    ns = n_spheres if n_spheres is not None else max(1, (nx * ny * nz) // 4000)
    d = np.full(shape, 1e9)
    own = np.zeros(shape, dtype=np.int64)
    for k in range(ns):
        c = rng.uniform(0, [nx, ny, nz])
        dk = _dist3(x, y, z, c, shape) - rng.uniform(max(2.5, L / 8), max(3.5, L / 5))
        own = np.where(dk < d, k, own)
        d = np.minimum(d, dk)
    psi = psi_from_distance(d)
    nd = n_drops if n_drops is not None else max(N - 1, (nx * ny * nz) // 2000)
    C0 = np.zeros((N - 1,) + shape)
    for k in range(nd):
        c = rng.uniform(0, [nx, ny, nz])
        R = rng.uniform(1.2 * width, max(1.2 * width + 1.0, L / 3))
        C0[k % (N - 1)] = np.maximum(C0[k % (N - 1)],
                                     drop_profile(_dist3(x, y, z, c, shape), R, width))
    C0 = _normalise(C0)
    rho = list(rng.uniform(0.5, 2.0, size=N))
    nu = list(rng.uniform(0.05, 0.15, size=N))
    sg = rng.uniform(0.006, 0.012, size=(N, N))
    sigma = np.triu(sg, 1) + np.triu(sg, 1).T
    params = base_params_3d(nx, ny, nz, N, rho=rho, nu=nu, sigma=sigma, width=width,
                            d0=d0, tau=tau)
    if N > 2:
        params["m0"] = 0.01
        params["eta"] = list(rng.uniform(0.08, 0.15, size=N - 1))
    else:
        params["eta"] = list(rng.uniform(0.8, 1.2, size=N - 1))
    ang = rng.uniform(45.0, 135.0, size=(ns, N - 1))
    ct = np.cos(np.radians(ang.mean(axis=0)))
    cf = None
    if theta_field:
        cf = np.stack([np.cos(np.radians(ang[own, i])) for i in range(N - 1)])
    return Problem("random3d_%dx%dx%d_N%d_s%d" % (nx, ny, nz, N, seed), params, psi, C0,
                   ct, cf, steps=0, note="random 3D parity case")


def config9_drop_on_sphere(L=128, Rs=15.0, R0=30.0, theta_deg=90.0, width=4.0, sigma=0.01,
                           xi=SOLID_XI):
    """Sec. 4.4 with one drop: a hemispherical drop of radius R0 placed on a
    solid sphere of radius Rs at the centre of a periodic L^3 box (the
    paper's compound drop of two fluids with equal properties and angles
    behaves as one drop).  d0 = 0.4 and the phase rates s0 = s21 = 1 as in
    Sec. 4.4; flow rates as ``base_params_3d``."""
    x, y, z = _grid3(L, L, L)
    c = (L / 2 - 0.3, L / 2 - 0.2, L / 2 - 0.1)
    rs = _dist3(x, y, z, c, (L, L, L))
    psi = psi_from_distance(rs - Rs, xi=xi)
    drop = drop_profile(rs, R0, width) * (0.5 * (1.0 + np.tanh(2.0 * (y - c[1]) / width)))
    params = base_params_3d(L, L, L, 2, sigma=sigma, width=width, xi=xi, d0=0.4)
    params["s_f"] = [1.0, 1.0]
    ct = np.array([math.cos(math.radians(theta_deg))])
    return Problem("drop_on_sphere_%d^3_t%g" % (L, theta_deg), params, psi, drop[None], ct, None,
                   steps=50000, note="drop on a solid sphere (Sec. 4.4), periodic box",
                   extra={"Rs": Rs, "centre": c, "R0": R0})
