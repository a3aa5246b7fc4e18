"""GPU parity of the three-dimensional path (D3Q7 phase, D3Q15 flow) through
the C ABI of include/ddcc3d.h, against the FP64 CPU oracle.

* FP64, element by element after 30 steps on ragged boxes that span several
  thread blocks along every axis, N = 2..4, uniform angles and per-node
  angle fields: C on psi >= 0.01, u, P and mu within 1e-10; both step paths
  (the fused z-marching kernel, whose small boxes run in many z chunks, and
  the three separate kernels);
* the fused and the three-kernel step agree with each other to round-off on
  a box of several columns and z chunks;
* FP32 against the same oracle: C within 2e-5, u within 1e-6 (including
  boxes one quad wide and with ragged quads for the vectorised kernel);
* the smallest box the ABI accepts (3 x 3 x 3) and a fluid at rest;
* conservation on the GPU: sum_x psi C_i drifts by <= 1e-13 (FP64) and
  <= 1e-6 (FP32, FP64 reduction) relative over 500 steps, on random solids
  (N = 2) and the Sec. 4.4 sphere at 48^3 (N = 3);
* the Sec. 4.4 sphere workload at its full size (256^3, N = 3) in the
  launch configuration the benchmark times: one step on the GPU, compared
  with the oracle on cropped windows (a periodic crop with a margin of 10
  nodes reproduces the interior exactly for two steps and the read-out,
  whose dependence radius is 9 nodes);
* the Laplace law of a static drop in 3D: Delta P = 2 sigma / R within 4%.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle.ddcc_oracle3d import Oracle3D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_10314_gb300 import build as B
    B.build()
    import paper_2311_10314_gb300 as D
    return D


_ORACLE = {}


def _pair(D, pb, steps, precision, path="fused"):
    key = (pb.name, int(pb.params["nphase"]), pb.psi.shape, float(pb.psi.sum()), steps)
    if key not in _ORACLE:
        o = Oracle3D(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field)
        o.step(steps)
        _ORACLE[key] = {k: v.numpy() for k, v in o.macroscopic().items()}
    ref = _ORACLE[key]
    sim = D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision,
                  path=path)
    sim.step(steps)
    got = sim.fields()
    sim.close()
    return ref, got


CASES = [((9, 10, 11), 2, 1, True), ((8, 12, 10), 3, 2, False), ((10, 9, 12), 4, 3, True),
         ((11, 13, 70), 3, 4, True)]


@pytest.mark.parametrize("path", ["fused", "split"])
@pytest.mark.parametrize("shape,N,seed,tf", CASES)
def test_fp64_matches_oracle(D, shape, N, seed, tf, path):
    nz, ny, nx = shape
    pb = W.random_problem_3d(nx, ny, nz, N, seed=seed, theta_field=tf)
    ref, got = _pair(D, pb, 30, D.DDCC_FP64, path)
    fl = pb.psi >= 0.01
    assert np.abs(ref["C"] - got["C"])[:, fl].max() <= 1e-10
    for k in ("ux", "uy", "uz", "P"):
        assert np.abs(ref[k] - got[k]).max() <= 1e-10, k
    assert np.abs(ref["mu"] - got["mu"])[:, fl].max() <= 1e-10


# FP32 boxes with nx a multiple of 4 take the four-nodes-per-thread chemical
# potential kernel: one quad wide (4 x 3 x 5), and a 36-wide box whose last
# block has lanes beyond the box
FP32_CASES = CASES[:3] + [((5, 3, 4), 2, 5, True), ((7, 6, 36), 3, 6, True)]


@pytest.mark.parametrize("path", ["fused", "split"])
@pytest.mark.parametrize("shape,N,seed,tf", FP32_CASES)
def test_fp32_matches_oracle(D, shape, N, seed, tf, path):
    nz, ny, nx = shape
    pb = W.random_problem_3d(nx, ny, nz, N, seed=seed, theta_field=tf)
    ref, got = _pair(D, pb, 30, D.DDCC_FP32, path)
    fl = pb.psi >= 0.01
    assert np.abs(ref["C"] - got["C"])[:, fl].max() <= 2e-5
    for k in ("ux", "uy", "uz"):
        assert np.abs(ref[k] - got[k]).max() <= 1e-6, k


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
@pytest.mark.parametrize("N", [2, 4])
def test_fused_matches_split(D, precision, tol, N):
    """The fused step against the three kernels: 72 x 20 x 40 nodes (three
    columns of 32 in x, a ragged one; three rows of 8 in y, a ragged one;
    several z chunks), 25 steps, per-node angles; every field of the
    read-out within tol of its own scale."""
    pb = W.random_problem_3d(72, 20, 40, N, seed=10 + N, theta_field=True)
    out = {}
    for path in ("fused", "split"):
        sim = D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision,
                      path=path)
        sim.step(25)
        out[path] = sim.fields()
        sim.close()
    for k in ("C", "ux", "uy", "uz", "P", "mu"):
        a, b = out["fused"][k], out["split"][k]
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-3), k


@pytest.mark.parametrize("N", [2, 3])
def test_smallest_box(D, N):
    rng = np.random.default_rng(N)
    prm = W.base_params_3d(3, 3, 3, N, sigma=0.01, width=3.0, eta=0.5)
    psi = rng.uniform(0.2, 1.0, size=(3, 3, 3))
    C0 = rng.uniform(0.0, 0.9 / (N - 1), size=(N - 1, 3, 3, 3))
    cf = rng.uniform(-0.7, 0.7, size=(N - 1, 3, 3, 3))
    pb = W.Problem("tiny", prm, psi, C0, None, cf)
    ref, got = _pair(D, pb, 40, D.DDCC_FP64)
    assert np.abs(ref["C"] - got["C"]).max() <= 1e-10
    assert np.abs(ref["ux"] - got["ux"]).max() <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_fluid_at_rest_stays_at_rest(D, precision):
    shape = (12, 10, 16)
    prm = W.base_params_3d(16, 10, 12, 2)
    sim = D.Sim3D(prm, np.ones(shape), np.zeros((1,) + shape), np.array([0.3]), precision=precision)
    sim.step(100)
    f = sim.fields()
    sim.close()
    for k in ("ux", "uy", "uz", "P"):
        assert np.abs(f[k]).max() == 0.0, k


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-6)])
@pytest.mark.parametrize("case", ["random_N2", "sphere_N3"])
def test_mass_conserved(D, precision, tol, case):
    if case == "random_N2":
        pb = W.random_problem_3d(40, 36, 33, 2, seed=8, theta_field=True)
    else:
        pb = W.config7_sphere(L=48)
    sim = D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=precision)
    m0 = sim.mass()
    sim.step(500)
    m1 = sim.mass()
    sim.close()
    assert (np.abs(m1 - m0) / m0).max() <= tol


def _crop(a, z0, y0, x0, n):
    idx = np.ix_(*[np.arange(c, c + n) % a.shape[k - 3] for k, c in enumerate((z0, y0, x0))])
    return a[(Ellipsis,) + idx]


def _sphere_windows(L):
    c = L // 2
    # at the sphere's top under the drop, at the drop's free interface, at
    # the phase 1 / phase 2 boundary inside the drop, and in the bulk
    return [(c - 8, c + int(0.2 * L) - 8, c - 8), (c - 8, c + int(0.3 * L) - 8, c + 10),
            (c - 8, c + 52, c - 8), (10, 10, 10)]


@pytest.fixture(scope="module")
def sphere_full(D):
    pb = W.config7_sphere()
    out = {}
    for prec in (0, 1):
        sim = D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, precision=prec)
        sim.step(2)
        out[prec] = sim.fields()
        out[prec]["mass"] = sim.mass()
        sim.close()
    n, m = 16, 10
    refs = []
    for (z0, y0, x0) in _sphere_windows(pb.params["nx"]):
        s = (z0 - m, y0 - m, x0 - m)
        prm = dict(pb.params)
        prm["nx"] = prm["ny"] = prm["nz"] = n + 2 * m
        o = Oracle3D(prm, _crop(pb.psi, *s, n + 2 * m), _crop(pb.C0, *s, n + 2 * m), pb.cos_theta)
        o.step(2)
        inner = (Ellipsis,) + (slice(m, m + n),) * 3
        refs.append({k: v.numpy()[inner] for k, v in o.macroscopic().items()})
    return pb, out, refs, n


@pytest.mark.parametrize("precision,tol_c,tol_u", [(0, 1e-11, 1e-12), (1, 2e-6, 2e-7)])
def test_sphere_full_size_windows(D, sphere_full, precision, tol_c, tol_u):
    pb, out, refs, n = sphere_full
    got = out[precision]
    for (z0, y0, x0), ref in zip(_sphere_windows(pb.params["nx"]), refs):
        for k, tol in (("C", tol_c), ("ux", tol_u), ("uy", tol_u), ("uz", tol_u)):
            err = np.abs(ref[k] - _crop(got[k], z0, y0, x0, n)).max()
            assert err <= tol, (k, (z0, y0, x0), err)
    assert np.isfinite(got["mass"]).all()


def test_laplace_law_3d(D):
    """Static drops (psi = 1) of R = 10 and 14 in a 64^3 box, 8000 steps,
    pressure averaged over the last 2000: Delta P R / (2 sigma) within 4%."""
    L, sigma, Wd = 64, 0.01, 4.0
    prm = W.base_params_3d(L, L, L, 2, sigma=sigma, width=Wd)
    z, y, x = np.meshgrid(*(np.arange(L) + 0.0,) * 3, indexing="ij")
    r = np.sqrt((x - L / 2 + 0.3) ** 2 + (y - L / 2 + 0.2) ** 2 + (z - L / 2 + 0.1) ** 2)
    for R in (10.0, 14.0):
        sim = D.Sim3D(prm, np.ones((L, L, L)), W.drop_profile(r, R, Wd)[None], np.array([0.0]),
                      precision=D.DDCC_FP64)
        sim.step(6000)
        inside, outside = r < R - 2 * Wd, r > R + 2 * Wd
        vals = []
        for _ in range(20):
            sim.step(100)
            P = sim.read(D._lib.FIELD_P)
            vals.append(P[inside].mean() - P[outside].mean())
        sim.close()
        ratio = float(np.mean(vals)) * R / (2 * sigma)
        assert abs(ratio - 1.0) < 0.04, (R, ratio)


def sphere_contact_angle(C, pb):
    """Contact angle of a drop on a solid sphere: fit a sphere (algebraic
    least squares) to the C = 1/2 crossings along grid lines where
    psi > 0.99 at both ends, then take the angle between the drop's and the
    solid's outward normals on their intersection circle,
    cos(theta) = (R_l^2 + R_s^2 - d^2) / (2 R_l R_s), d the distance of the
    centres (theta measured inside the drop)."""
    import math
    pts = []
    for axis in range(3):
        a = np.moveaxis(C, axis, -1) - 0.5
        q = np.moveaxis(pb.psi, axis, -1)
        s0, s1 = a[..., :-1], a[..., 1:]
        m = ((s0 >= 0) != (s1 >= 0)) & (q[..., :-1] > 0.99) & (q[..., 1:] > 0.99)
        idx = np.argwhere(m).astype(float)
        idx[:, -1] += s0[m] / (s0[m] - s1[m])
        order = [k for k in range(3) if k != axis] + [axis]
        P = np.empty_like(idx)
        for k, ax in enumerate(order):
            P[:, ax] = idx[:, k]
        pts.append(P)
    P = np.concatenate(pts)[:, ::-1]                 # (x, y, z)
    A = np.c_[2 * P, np.ones(len(P))]
    sol = np.linalg.lstsq(A, (P ** 2).sum(1), rcond=None)[0]
    Rl = math.sqrt(sol[3] + (sol[:3] ** 2).sum())
    d = np.linalg.norm(sol[:3] - np.asarray(pb.extra["centre"]))
    Rs = pb.extra["Rs"]
    return math.degrees(math.acos(max(-1.0, min(1.0, (Rl ** 2 + Rs ** 2 - d ** 2) / (2 * Rl * Rs)))))


def test_sphere_angle_fit_on_exact_caps():
    """The fit itself, on tanh caps of a known angle (no GPU needed, but
    kept beside its use)."""
    import math
    for th in (60.0, 90.0, 120.0):
        pb = W.config9_drop_on_sphere(theta_deg=th)
        L = pb.params["nx"]
        x, y, z = W._grid3(L, L, L)
        Rl, Rs = 25.0, pb.extra["Rs"]
        d = math.sqrt(Rl ** 2 + Rs ** 2 - 2 * Rl * Rs * math.cos(math.radians(th)))
        c = pb.extra["centre"]
        C = W.drop_profile(W._dist3(x, y, z, (c[0], c[1] + d, c[2]), (L, L, L)), Rl, 4.0)
        assert abs(sphere_contact_angle(C, pb) - th) < 0.1


@pytest.mark.parametrize("theta,tol", [(60.0, 2.0), (90.0, 2.5), (120.0, 6.5)])
def test_contact_angle_on_sphere(D, theta, tol):
    """Sec. 4.4 with one drop: a hemispherical drop (R0 = 30) on a solid
    sphere (R_s = 15, eps0 = 6) in a 128^3 box settles at the prescribed
    angle (FP32, 1.2 10^5 steps).  Measured: 60.3, 91.5, 125.3 deg; the
    120-degree error shrinks with eps0 / R_s (122.2 deg at eps0 = 2.8,
    123.1 deg at R_s = 20), a diffuse-domain effect."""
    pb = W.config9_drop_on_sphere(theta_deg=theta)
    sim = D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, precision=D.DDCC_FP32)
    m0 = sim.mass()
    sim.step(120000)
    C = sim.read(D.FIELD_C)
    m1 = sim.mass()
    sim.close()
    assert abs(sphere_contact_angle(C, pb) - theta) <= tol
    assert abs(m1[0] - m0[0]) / m0[0] <= 1e-7


@pytest.mark.parametrize("bad", [0.0, 1.5, float("nan")])
def test_create_rejects_psi_outside_unit_interval(D, bad):
    """One psi value outside (0, 1] anywhere in the box gives DDCC_ERR_PARAM
    from create; the box without it is accepted."""
    from paper_2311_10314_gb300 import _lib
    pb = W.random_problem_3d(20, 18, 16, 2, seed=9)
    for where in (0, 4100, -1):
        psi = pb.psi.copy()
        psi.reshape(-1)[where] = bad
        with pytest.raises(_lib.DdccError) as ei:
            D.Sim3D(pb.params, psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=D.DDCC_FP32)
        assert ei.value.status == _lib.DDCC_ERR_PARAM
    D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=D.DDCC_FP32).close()
