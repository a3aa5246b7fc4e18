"""Oracle pins for the open (inflow/outflow) x boundaries (reading R22 of
Sec. 4.5's parabolic inflow and outflow)."""
import numpy as np
import torch

import workloads as W
from oracle import Oracle


def _channel(nx, ny, umax):
    prm = W.base_params(nx, ny, 2, periodic_x=0, periodic_y=0, sigma=0.01, width=4.0, tau=0.8)
    y = np.arange(ny) + 0.5          # halfway bounce-back walls at y = 0 and y = ny
    u_in = 4.0 * umax * y * (ny - y) / ny ** 2
    return prm, u_in


def test_fluid_at_rest_stays_at_rest():
    prm, _ = _channel(20, 12, 0.0)
    o = Oracle(prm, np.ones((12, 20)), np.zeros((1, 12, 20)), np.array([0.2]),
               open_x=(np.zeros(12), np.zeros((1, 12))))
    o.step(50)
    m = o.macroscopic()
    for k in ("ux", "uy", "P"):
        assert torch.abs(m[k]).max().item() == 0.0, k


def test_plane_poiseuille_through_open_ends():
    """A parabolic inflow between bounce-back walls keeps its profile down the
    channel (fully developed) and the flux through every section equals the
    inflow flux."""
    nx, ny, umax = 48, 16, 0.02
    prm, u_in = _channel(nx, ny, umax)
    o = Oracle(prm, np.ones((ny, nx)), np.zeros((1, ny, nx)), np.array([0.0]),
               open_x=(u_in, np.zeros((1, ny))))
    o.step(3000)
    m = o.macroscopic()
    ux = m["ux"].numpy()
    mid = ux[:, nx // 2]
    assert np.abs(mid - u_in).max() <= 0.03 * umax
    flux = ux.sum(axis=0)
    assert np.abs(flux[2:-2] / u_in.sum() - 1.0).max() <= 0.02
    assert np.abs(m["uy"].numpy()).max() <= 0.03 * umax


def test_inflow_composition_enters():
    """Phase 1 fed at the inlet fills the channel from the left."""
    nx, ny, umax = 40, 12, 0.05
    prm, u_in = _channel(nx, ny, umax)
    o = Oracle(prm, np.ones((ny, nx)), np.zeros((1, ny, nx)), np.array([0.0]),
               open_x=(u_in, np.ones((1, ny))))
    o.step(400)
    C = o.macroscopic()["C"][0].numpy()
    assert C[:, 1:4].mean() > 0.9
    assert C[:, -4:].mean() < C[:, 1:4].mean()
