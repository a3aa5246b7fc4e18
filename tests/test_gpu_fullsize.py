"""GPU parity at the benchmark's own size: the 4096 x 4096, N = 4 porous
imbibition with per-circle contact angles, stepped on the default fused
tile path (the launch configuration ``bench.py`` times), compared element by
element with the FP64 oracle on cropped windows after two steps.

The oracle steps a periodic crop of the initial fields with a margin of 10
nodes on every side; information moves at most three nodes per step (two
stencil hops and streaming), so after two steps the inner window is exact.
The windows sit on a contact line (a drop meeting a solid circle), on a
free drop interface, on a bare solid wall, and across the periodic seam
(0, 0).  Bars: FP64 1e-10 (C_i on psi >= 0.01, u everywhere); FP32 the
stated FP32 error after two steps, 2e-6 in C_i on psi >= 0.5 and 2e-7 in u.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import Oracle

N_WIN, MARGIN, STEPS = 24, 10, 2


@pytest.fixture(scope="module")
def ddcc():  # noqa: D401
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10314_gb300 import build as B
    B.build()
    import paper_2311_10314_gb300 as D
    return D


def _crop(a, y0, x0, n):
    ny, nx = a.shape[-2:]
    return a[..., (np.arange(y0, y0 + n) % ny)[:, None], (np.arange(x0, x0 + n) % nx)[None, :]]


def windows(pb, n=N_WIN):
    """Lower-left corners of the compared windows, chosen from the initial
    fields: the strongest contact line, the strongest drop interface in open
    fluid, the steepest bare solid wall, and the periodic seam."""
    psi, C0 = pb.psi, pb.C0
    gy, gx = np.gradient(psi)
    ag = np.hypot(gx, gy)
    mix = (C0 * (1.0 - C0)).max(axis=0)
    picks = [ag * mix, mix * (psi > 0.99), ag * (C0.sum(axis=0) < 1e-3)]
    out = []
    for score in picks:
        y, x = np.unravel_index(int(np.argmax(score)), score.shape)
        out.append((int(y) - n // 2, int(x) - n // 2))
    out.append((-n // 2, -n // 2))
    return out


@pytest.fixture(scope="module")
def imbibition_full(ddcc):
    pb = W.config4_imbibition()
    got = {}
    for prec in (ddcc.DDCC_FP64, ddcc.DDCC_FP32):
        sim = ddcc.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=prec)
        assert sim.path == "tile"
        sim.step(STEPS)
        f = sim.fields()
        got[prec] = {k: f[k] for k in ("C", "ux", "uy")}
        got[prec]["mass"] = sim.mass()
        sim.close()
        del sim
        torch.cuda.empty_cache()
    refs = []
    side = N_WIN + 2 * MARGIN
    for (y0, x0) in windows(pb):
        prm = dict(pb.params)
        prm["nx"] = prm["ny"] = side
        ys, xs = y0 - MARGIN, x0 - MARGIN
        o = Oracle(prm, _crop(pb.psi, ys, xs, side), _crop(pb.C0, ys, xs, side), pb.cos_theta,
                   _crop(pb.cos_theta_field, ys, xs, side))
        o.step(STEPS)
        inner = (Ellipsis, slice(MARGIN, MARGIN + N_WIN), slice(MARGIN, MARGIN + N_WIN))
        m = o.macroscopic()
        refs.append({k: m[k].numpy()[inner] for k in ("C", "ux", "uy")})
    return pb, got, refs


def test_windows_cover_the_features():
    pb = W.config4_imbibition()
    ws = windows(pb)
    psi = [_crop(pb.psi, y0, x0, N_WIN) for (y0, x0) in ws]
    C = [_crop(pb.C0, y0, x0, N_WIN) for (y0, x0) in ws]
    # contact line: solid, and a drop interface (C crosses 1/2)
    assert psi[0].min() < 0.5 and C[0].max() > 0.6 and (C[0] * (1 - C[0])).max() > 0.2
    # free interface: no solid, a drop interface
    assert psi[1].min() > 0.9 and (C[1] * (1 - C[1])).max() > 0.2
    # bare wall: solid, no drop
    assert psi[2].min() < 0.5 and C[2].max() < 1e-2
    assert len(set(ws)) == 4


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol_c,tol_u,bulk", [(0, 1e-10, 1e-10, 0.01), (1, 2e-6, 2e-7, 0.5)])
def test_imbibition_full_size_windows(imbibition_full, precision, tol_c, tol_u, bulk):
    pb, got, refs = imbibition_full
    g = got[precision]
    for (y0, x0), ref in zip(windows(pb), refs):
        mask = _crop(pb.psi, y0, x0, N_WIN) >= bulk
        dC = np.abs(ref["C"] - _crop(g["C"], y0, x0, N_WIN))[:, mask]
        assert dC.max() <= tol_c, ("C", (y0, x0), dC.max())
        for k in ("ux", "uy"):
            err = np.abs(ref[k] - _crop(g[k], y0, x0, N_WIN)).max()
            assert err <= tol_u, (k, (y0, x0), err)
    assert np.isfinite(g["mass"]).all()
