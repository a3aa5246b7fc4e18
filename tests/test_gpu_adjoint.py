"""GPU adjoint: gradients of a phase x-centroid after T steps with respect to
the per-node contact-angle field cos(theta_iN)(x) and psi(x), through the C
ABI (ddcc_adjoint_step / ddcc_adjoint_initial / ddcc_objective_centroid).

Bars:
  * against reverse-mode autograd through the FP64 oracle (small grids, every
    node): max |g - g_ref| <= 1e-8 max |g_ref| (FP64 adjoint);
  * against central finite differences of the FP64 forward (h = 1e-4) on the
    256^2 wavy-wall drop after 2000 steps, checkpoint every 100 steps, at 16
    seeded nodes (8 for theta, 8 for psi) where |grad psi| > 1e-2 and
    C_1 C_2 > 1e-3: |g - g_FD| <= 1e-4 max(|g_FD|, 1e-8 max |g|);
  * the FP32 adjoint against the FP64 adjoint (stated FP32 gradient error);
  * the gradients do not depend on the checkpoint interval, nor on one- or
    two-level checkpointing (bit for bit);
  * the four-phase 4096^2 imbibition workload fits on one GPU with two-level
    checkpointing and its FP32 gradients are finite.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10314_gb300 import build as B
    B.build()
    import paper_2311_10314_gb300 as D
    from paper_2311_10314_gb300 import adjoint as A
    return D, A


def _wall_drop_problem(nx, ny, N, seed):
    """Drop(s) on a psi-embedded wall plus one solid circle, x periodic, y
    walled; psi varies at every node (no flat region), a random theta field."""
    rng = np.random.default_rng(seed)
    x, y = np.meshgrid(np.arange(nx) + 0.0, np.arange(ny) + 0.0)
    cx, cy, R = 0.63 * nx + 0.37, 0.58 * ny + 0.21, 3.1
    d = np.minimum(y - 3.3, np.hypot(x - cx, y - cy) - R)
    psi = W.psi_from_distance(d, xi=W.SOLID_XI)
    C0 = np.zeros((N - 1, ny, nx))
    C0[0] = W.drop_profile(np.hypot(x - 0.3 * nx, y - 3.3), 5.5, 4.0)
    if N > 2:
        C0[1] = W.drop_profile(np.hypot(x - 0.3 * nx - 9.0, y - 3.3), 4.5, 4.0) * (1 - C0[0])
    params = W.base_params(nx, ny, N, periodic_x=1, periodic_y=0, sigma=0.01, width=4.0,
                           xi=W.SOLID_XI, tau=0.8, eta=1.0 if N == 2 else 0.5)
    if N > 2:
        params["rho"] = [1.0, 2.0, 1.5]
    cos_field = rng.uniform(-0.6, 0.6, size=(N - 1, ny, nx))
    return params, psi, C0, cos_field


def _oracle_gradient(params, psi, C0, cos_field, T, phase=0):
    psi_t = torch.tensor(psi, dtype=torch.float64, requires_grad=True)
    cf_t = torch.tensor(cos_field, dtype=torch.float64, requires_grad=True)
    o = Oracle(params, psi_t, C0, None, cf_t)
    o.step(T)
    m = o.f[phase].sum(dim=0)
    xs = torch.arange(params["nx"], dtype=torch.float64)
    J = (m * xs[None, :]).sum() / m.sum()
    J.backward()
    return J.item(), cf_t.grad.numpy(), psi_t.grad.numpy()


@pytest.mark.parametrize("N,T,ckpt", [(2, 30, 7), (3, 24, 10)])
def test_adjoint_matches_autograd_through_oracle(ddcc, N, T, ckpt):
    D, A = ddcc
    params, psi, C0, cf = _wall_drop_problem(26, 22, N, seed=N)
    J_ref, gc_ref, gp_ref = _oracle_gradient(params, psi, C0, cf, T)
    J, gc, gp = A.centroid_gradient(params, psi, C0, cf, T, ckpt=ckpt, precision=D.DDCC_FP64)
    assert abs(J - J_ref) <= 1e-10 * abs(J_ref)
    assert np.isfinite(gc).all() and np.isfinite(gp).all()
    ec = np.abs(gc - gc_ref).max() / np.abs(gc_ref).max()
    ep = np.abs(gp - gp_ref).max() / np.abs(gp_ref).max()
    assert ec <= 1e-8 and ep <= 1e-8, (ec, ep)


def test_adjoint_checkpoint_interval_does_not_change_gradient(ddcc):
    D, A = ddcc
    params, psi, C0, cf = _wall_drop_problem(40, 30, 2, seed=5)
    out = [A.centroid_gradient(params, psi, C0, cf, 45, ckpt=c, precision=D.DDCC_FP64) for c in (1, 9, 45, 100)]
    # two-level checkpointing: sub-segments of 3 and 4 steps in 9- and
    # 45-step segments (ragged last sub-segments), and one-level forced
    out += [A.centroid_gradient(params, psi, C0, cf, 45, ckpt=c, precision=D.DDCC_FP64, sub=b)
            for c, b in ((9, 4), (45, 3), (45, 45))]
    for J, gc, gp in out[1:]:
        assert J == out[0][0]
        assert np.array_equal(gc, out[0][1]) and np.array_equal(gp, out[0][2])


@pytest.fixture(scope="module")
def wavy_adjoint(ddcc):
    D, A = ddcc
    pb = W.config5_wavy_wall()
    J, gc, gp = A.centroid_gradient(pb.params, pb.psi, pb.C0, pb.cos_theta_field, 2000, ckpt=100,
                                    precision=D.DDCC_FP64)
    return pb, J, gc, gp


def _select_nodes(pb, C_end, rng, k):
    gy, gx = np.gradient(pb.psi)
    gpsi = np.hypot(gx, gy)
    c0 = pb.C0[0]
    mix = np.maximum(c0 * (1 - c0), C_end * (1 - C_end))
    ok = (gpsi > 1e-2) & (mix > 1e-3) & (pb.psi > 0.02) & (pb.psi < 0.98)
    cand = np.argwhere(ok)
    assert len(cand) >= k
    return [tuple(v) for v in cand[rng.choice(len(cand), size=k, replace=False)]]


def test_adjoint_against_central_differences_wavy_wall(ddcc, wavy_adjoint):
    D, A = ddcc
    pb, J, gc, gp = wavy_adjoint
    sim = D.Sim(pb.params, pb.psi, pb.C0, cos_theta_field=pb.cos_theta_field, precision=D.DDCC_FP64)
    sim.step(2000)
    C_end = sim.read(D.FIELD_C)
    sim.close()
    rng = np.random.default_rng(2000)
    nodes = _select_nodes(pb, C_end, rng, 16)
    h = 1e-4
    gmax = {"cos": np.abs(gc).max(), "psi": np.abs(gp).max()}
    for n, (y, x) in enumerate(nodes):
        kind = "cos" if n < 8 else "psi"
        vals = []
        for s in (1.0, -1.0):
            cf = pb.cos_theta_field.copy()
            psi = pb.psi.copy()
            if kind == "cos":
                cf[0, y, x] += s * h
            else:
                psi[y, x] += s * h
            vals.append(A.centroid(pb.params, psi, pb.C0, cf, 2000, precision=D.DDCC_FP64))
        g_fd = (vals[0] - vals[1]) / (2 * h)
        g = gc[0, y, x] if kind == "cos" else gp[y, x]
        denom = max(abs(g_fd), 1e-8 * gmax[kind])
        assert abs(g - g_fd) <= 1e-4 * denom, (kind, (y, x), g, g_fd)


def test_fp32_adjoint_against_fp64(ddcc, wavy_adjoint):
    """The FP32 adjoint of the same 2000-step wavy-wall run: max error
    relative to the FP64 gradient's max, per field (stated FP32 error)."""
    D, A = ddcc
    pb, J, gc, gp = wavy_adjoint
    J32, gc32, gp32 = A.centroid_gradient(pb.params, pb.psi, pb.C0, pb.cos_theta_field, 2000,
                                          ckpt=100, precision=D.DDCC_FP32)
    assert abs(J32 - J) <= 1e-5 * abs(J)
    ec = np.abs(gc32 - gc).max() / np.abs(gc).max()
    ep = np.abs(gp32 - gp).max() / np.abs(gp).max()
    assert ec <= 1e-2 and ep <= 1e-2, (ec, ep)


def test_rollout_autograd_function(ddcc):
    D, A = ddcc
    params, psi, C0, cf = _wall_drop_problem(26, 22, 2, seed=7)
    cf_t = torch.tensor(cf, dtype=torch.float64, requires_grad=True)
    psi_t = torch.tensor(psi, dtype=torch.float64, requires_grad=True)
    J = A.rollout(cf_t, psi_t, params, C0, 20, ckpt=6)
    (3.0 * J).backward()
    J2, gc, gp = A.centroid_gradient(params, psi, C0, cf, 20, ckpt=6)
    assert math.isclose(J.item(), J2, rel_tol=0, abs_tol=0)
    assert np.allclose(cf_t.grad.numpy(), 3.0 * gc, rtol=0, atol=0)
    assert np.allclose(psi_t.grad.numpy(), 3.0 * gp, rtol=0, atol=0)


def test_adjoint_fits_at_4096(ddcc):
    """The 4096^2 N = 4 imbibition (3.2 GB per FP32 state): T = 60 with a
    checkpoint every 30 steps would hold 2 + 30 states one-level; forced
    two-level with sub = 6 it holds 2 + 5 + 6.  J finite, gradients finite
    and non-zero where the phases meet the solid."""
    D, A = ddcc
    pb = W.config4_imbibition()
    J, gc, gp = A.centroid_gradient(pb.params, pb.psi, pb.C0, pb.cos_theta_field, 60, ckpt=30,
                                    precision=D.DDCC_FP32, sub=6)
    assert math.isfinite(J)
    assert np.isfinite(gc).all() and np.isfinite(gp).all()
    assert np.abs(gc).max() > 0 and np.abs(gp).max() > 0



@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pipelined_sweep_is_bit_identical(ddcc, precision):
    """The pipelined reverse sweep (each segment reversed while the one
    before it is recomputed on a second stream, the segments replayed as
    graphs from the fifth call on) gives the gradients of the plain sweep
    bit for bit: 256^2 wavy wall, T = 400 in segments of 50."""
    D, A = ddcc
    prec = D.DDCC_FP32 if precision == "fp32" else D.DDCC_FP64
    pb = W.config5_wavy_wall()
    out = []
    for pipe in (True, False):
        run = A.CheckpointedRun(pb.params, pb.psi, pb.C0, pb.cos_theta_field, 400, ckpt=50, precision=prec,
                                pipeline=pipe)
        try:
            assert run.pipe == pipe
            out.append((run.J,) + tuple(run.reverse()))
        finally:
            run.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    assert np.abs(out[0][1]).max() > 0 and np.abs(out[0][2]).max() > 0
