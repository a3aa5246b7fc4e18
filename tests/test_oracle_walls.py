"""Oracle pins for solids given by several characteristic functions (Sec. 4.5:
psi = psi_1 psi_2, wetting term sum_k cos(theta^k_jq) |grad psi_k|)."""
import math

import numpy as np
import torch

import workloads as W
from oracle import Oracle


def _channel(nx=40, ny=36, N=3, seed=1):
    rng = np.random.default_rng(seed)
    x, y = np.meshgrid(np.arange(nx) + 0.0, np.arange(ny) + 0.0)
    xi = W.SOLID_XI
    psi1 = W.psi_from_distance(y - 7.3 - 2.0 * np.sin(2 * np.pi * x / nx), xi=xi)
    psi2 = W.psi_from_distance(28.6 + 1.5 * np.cos(2 * np.pi * x / nx) - y, xi=xi)
    C0 = np.zeros((N - 1, ny, nx))
    C0[0] = W.drop_profile(np.hypot(x - 14.2, y - 9.0), 6.0, 4.0)
    if N > 2:
        C0[1] = W.drop_profile(np.hypot(x - 27.1, y - 26.0), 5.0, 4.0) * (1 - C0[0])
    prm = W.base_params(nx, ny, N, periodic_x=1, periodic_y=0, sigma=0.01, width=4.0, xi=xi,
                        tau=0.8, eta=0.5)
    cos1 = rng.uniform(-0.7, 0.7, size=(N - 1, ny, nx))
    cos2 = rng.uniform(-0.7, 0.7, size=(N - 1, ny, nx))
    return prm, psi1, psi2, C0, cos1, cos2


def _fields(o):
    m = o.macroscopic()
    return {k: v.numpy() for k, v in m.items()}


def test_flat_second_function_reduces_to_one_solid():
    """psi_2 = 1 has no gradient: the run equals the single-psi run of psi_1
    with its angle field, bit for bit."""
    prm, psi1, psi2, C0, cos1, cos2 = _channel()
    a = Oracle(prm, psi1, C0, None, cos1)
    b = Oracle(prm, None, C0, None, walls=[(psi1, cos1), (np.ones_like(psi1), cos2)])
    a.step(30)
    b.step(30)
    fa, fb = _fields(a), _fields(b)
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_order_of_the_solids_does_not_matter():
    prm, psi1, psi2, C0, cos1, cos2 = _channel()
    a = Oracle(prm, None, C0, None, walls=[(psi1, cos1), (psi2, cos2)])
    b = Oracle(prm, None, C0, None, walls=[(psi2, cos2), (psi1, cos1)])
    a.step(30)
    b.step(30)
    fa, fb = _fields(a), _fields(b)
    for k in fa:
        assert np.abs(fa[k] - fb[k]).max() <= 1e-13, k


def test_neutral_walls_add_no_wetting():
    """theta = 90 deg on every solid (cos = 0) gives the same step as a single
    psi = psi_1 psi_2 with a 90-degree field: the wetting term vanishes."""
    prm, psi1, psi2, C0, cos1, cos2 = _channel(N=2)
    zero = np.zeros_like(cos1)
    a = Oracle(prm, psi1 * psi2, C0, None, zero)
    b = Oracle(prm, None, C0, None, walls=[(psi1, zero), (psi2, zero)])
    a.step(30)
    b.step(30)
    fa, fb = _fields(a), _fields(b)
    for k in fa:
        assert np.abs(fa[k] - fb[k]).max() <= 1e-14, k


def test_walls_conserve_mass():
    prm, psi1, psi2, C0, cos1, cos2 = _channel()
    o = Oracle(prm, None, C0, None, walls=[(psi1, cos1), (psi2, cos2)])
    m0 = o.mass()
    o.step(100)
    assert (torch.abs(o.mass() - m0) / torch.abs(m0)).max().item() <= 1e-13
