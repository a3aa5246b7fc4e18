"""The gradient reference of the GPU adjoint tests -- reverse-mode autograd
through the FP64 oracle -- pinned against central finite differences of the
oracle itself on a tiny walled grid (objective: phase-1 x-centroid)."""
import numpy as np
import torch

import workloads as W
from oracle import Oracle


def _problem(nx=12, ny=10, N=2, seed=3):
    rng = np.random.default_rng(seed)
    x, y = np.meshgrid(np.arange(nx) + 0.0, np.arange(ny) + 0.0)
    d = np.minimum(y - 2.3, np.hypot(x - 7.4, y - 6.2) - 2.1)
    psi = W.psi_from_distance(d, xi=W.SOLID_XI)
    C0 = W.drop_profile(np.hypot(x - 3.6, y - 2.3), 3.2, 3.0)[None]
    params = W.base_params(nx, ny, N, periodic_x=1, periodic_y=0, sigma=0.02, width=3.0,
                           xi=W.SOLID_XI, tau=0.8)
    cf = rng.uniform(-0.6, 0.6, size=(N - 1, ny, nx))
    return params, psi, C0, cf


def _J(params, psi, C0, cf, T):
    o = Oracle(params, psi, C0, None, cf)
    o.step(T)
    m = o.f[0].sum(dim=0)
    xs = torch.arange(params["nx"], dtype=torch.float64)
    return (m * xs[None, :]).sum() / m.sum()


def test_autograd_reference_matches_central_differences():
    params, psi, C0, cf = _problem()
    T = 6
    psi_t = torch.tensor(psi, requires_grad=True)
    cf_t = torch.tensor(cf, requires_grad=True)
    J = _J(params, psi_t, C0, cf_t, T)
    J.backward()
    gc, gp = cf_t.grad.numpy(), psi_t.grad.numpy()
    assert np.isfinite(gc).all() and np.isfinite(gp).all()
    h = 1e-4
    rng = np.random.default_rng(0)
    for (y, x) in [tuple(v) for v in rng.integers(0, [10, 12], size=(4, 2))] + [(2, 4), (3, 3)]:
        for kind in ("cos", "psi"):
            vals = []
            for s in (1.0, -1.0):
                p2, c2 = psi.copy(), cf.copy()
                if kind == "cos":
                    c2[0, y, x] += s * h
                else:
                    p2[y, x] += s * h
                with torch.no_grad():
                    vals.append(_J(params, p2, C0, c2, T).item())
            g_fd = (vals[0] - vals[1]) / (2 * h)
            g = gc[0, y, x] if kind == "cos" else gp[y, x]
            scale = max(abs(g_fd), 1e-4 * max(np.abs(gc).max(), np.abs(gp).max()))
            assert abs(g - g_fd) <= 1e-5 * scale, (kind, (y, x), g, g_fd)
