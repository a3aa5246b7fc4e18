"""ctypes binding of libddcc.so: the C ABIs of include/ddcc.h and
include/ddcc3d.h, same names.

This module only marshals arguments.  It raises ``RuntimeError`` when the
shared library has not been built (``python -m paper_2311_10314_gb300.build``
or ``__graft_entry__.build()``): there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddcc.so")

MAX_PHASES = 4
DDCC_OK = 0
DDCC_ERR_PARAM = -1
DDCC_ERR_WORKSPACE = -2
DDCC_ERR_CUDA = -3
DDCC_ERR_NONFINITE = -4
DDCC_ERR_NOMEM = -5
DDCC_ERR_UNSUPPORTED = -6
DDCC_FP64 = 0
DDCC_FP32 = 1
FIELD_C = 0
FIELD_RHO = 8
FIELD_UX = 9
FIELD_UY = 10
FIELD_P = 11
FIELD_MU = 12
FIELD_PSI = 20

# every symbol include/ddcc.h declares
EXPORTED = (
    "ddcc_workspace_bytes", "ddcc_create", "ddcc_step", "ddcc_read", "ddcc_mass",
    "ddcc_state_bytes", "ddcc_save_state", "ddcc_load_state", "ddcc_step_count",
    "ddcc_destroy", "ddcc_status_string", "ddcc_version", "ddcc_profile", "ddcc_kernel_times",
    "ddcc_phase_mass_noalloc", "ddcc_step_path", "ddcc_adjoint_bytes", "ddcc_adjoint_step",
    "ddcc_adjoint_initial", "ddcc_objective_centroid", "ddcc_step_between", "ddcc_create_walls",
    "ddcc_set_inflow", "ddcc_adjoint_segment", "ddcc_adjoint_segment_pipelined",
    "ddcc_selftest_bounded_wait", "ddcc_measure_fp64_peak", "ddcc_rows_bytes", "ddcc_get_rows", "ddcc_set_rows",
)
# every symbol include/ddcc3d.h declares
EXPORTED_3D = (
    "ddcc3d_workspace_bytes", "ddcc3d_create", "ddcc3d_step", "ddcc3d_read", "ddcc3d_mass",
    "ddcc3d_step_count", "ddcc3d_profile", "ddcc3d_kernel_times", "ddcc3d_destroy",
)
FIELD_UZ = 21
KERNEL_KINDS_3D = ("order_param", "chem_pot", "update", "fused_step")
DDCC3D_FLAG_SPLIT = 1
DDCC3D_FLAG_FUSED = 2
NOALLOC_MAX_ROWS = 16384
KERNEL_KINDS = ("order_param", "collide_stream", "row_sweep", "ghost_fill")
DDCC_ERR_TIMEOUT = -7
DDCC_FLAG_TILE = 1
DDCC_FLAG_SWEEP = 2
DDCC_FLAG_OPEN_X = 4
DDCC_PATH_TILE = 1
DDCC_PATH_SWEEP = 2
GHOST_X, GHOST_Y = 4, 6


class ddcc_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nphase", C.c_int32),
        ("periodic_x", C.c_int32), ("periodic_y", C.c_int32), ("precision", C.c_int32),
        ("rho", C.c_double * MAX_PHASES), ("nu", C.c_double * MAX_PHASES),
        ("sigma", (C.c_double * MAX_PHASES) * MAX_PHASES),
        ("width", C.c_double), ("eps0", C.c_double), ("d0", C.c_double), ("m0", C.c_double),
        ("eta", C.c_double * MAX_PHASES), ("s_f", C.c_double * 5), ("s_g", C.c_double * 4),
        ("rho0", C.c_double), ("body_force", C.c_double * 2), ("flags", C.c_uint32),
    ]


class ddcc3d_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nphase", C.c_int32),
        ("precision", C.c_int32), ("reserved", C.c_int32),
        ("rho", C.c_double * MAX_PHASES), ("nu", C.c_double * MAX_PHASES),
        ("sigma", (C.c_double * MAX_PHASES) * MAX_PHASES),
        ("width", C.c_double), ("eps0", C.c_double), ("d0", C.c_double), ("m0", C.c_double),
        ("eta", C.c_double * MAX_PHASES), ("s_f", C.c_double * 2), ("s_g", C.c_double * 4),
        ("rho0", C.c_double), ("body_force", C.c_double * 3), ("flags", C.c_uint32),
    ]


class DdccError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s failed: %s (%d)" % (what, status_string(status), status))
        self.status = status


_lib = None


def load():
    """Load libddcc.so (once); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libddcc.so is not built (expected at %s); run "
            "`python -m paper_2311_10314_gb300.build` first" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER(ddcc_params)
    vp = C.c_void_p
    dp = C.POINTER(C.c_double)
    lib.ddcc_workspace_bytes.argtypes = [P]
    lib.ddcc_workspace_bytes.restype = C.c_size_t
    lib.ddcc_create.argtypes = [P, vp, C.c_size_t, vp, dp, dp, dp, dp, C.POINTER(vp)]
    lib.ddcc_create.restype = C.c_int
    lib.ddcc_step.argtypes = [vp, C.c_int64]
    lib.ddcc_step.restype = C.c_int
    lib.ddcc_read.argtypes = [vp, C.c_int, dp]
    lib.ddcc_read.restype = C.c_int
    lib.ddcc_mass.argtypes = [vp, dp]
    lib.ddcc_mass.restype = C.c_int
    lib.ddcc_state_bytes.argtypes = [vp]
    lib.ddcc_state_bytes.restype = C.c_size_t
    lib.ddcc_save_state.argtypes = [vp, vp, C.c_int]
    lib.ddcc_save_state.restype = C.c_int
    lib.ddcc_load_state.argtypes = [vp, vp, C.c_int]
    lib.ddcc_load_state.restype = C.c_int
    lib.ddcc_step_count.argtypes = [vp]
    lib.ddcc_step_count.restype = C.c_int64
    lib.ddcc_destroy.argtypes = [vp]
    lib.ddcc_destroy.restype = None
    lib.ddcc_status_string.argtypes = [C.c_int]
    lib.ddcc_status_string.restype = C.c_char_p
    lib.ddcc_version.argtypes = []
    lib.ddcc_version.restype = C.c_int
    lib.ddcc_profile.argtypes = [vp, C.c_int]
    lib.ddcc_profile.restype = C.c_int
    lib.ddcc_kernel_times.argtypes = [vp, dp, C.POINTER(C.c_int64), C.c_int]
    lib.ddcc_kernel_times.restype = C.c_int
    lib.ddcc_phase_mass_noalloc.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64,
                                            C.c_int64, vp, vp]
    lib.ddcc_phase_mass_noalloc.restype = C.c_int
    lib.ddcc_step_path.argtypes = [vp]
    lib.ddcc_step_path.restype = C.c_int
    lib.ddcc_adjoint_bytes.argtypes = [vp]
    lib.ddcc_adjoint_bytes.restype = C.c_size_t
    lib.ddcc_adjoint_step.argtypes = [vp, vp, vp, vp, vp, C.c_size_t, vp, vp]
    lib.ddcc_adjoint_step.restype = C.c_int
    lib.ddcc_adjoint_initial.argtypes = [vp, dp, vp, vp, C.c_size_t, vp, vp]
    lib.ddcc_adjoint_initial.restype = C.c_int
    lib.ddcc_objective_centroid.argtypes = [vp, C.c_int, vp, C.c_size_t, dp, vp]
    lib.ddcc_objective_centroid.restype = C.c_int
    lib.ddcc_step_between.argtypes = [vp, vp, vp]
    lib.ddcc_step_between.restype = C.c_int
    lib.ddcc_create_walls.argtypes = [C.POINTER(ddcc_params), vp, C.c_size_t, vp, C.c_int, dp, dp, dp,
                                      C.POINTER(vp)]
    lib.ddcc_create_walls.restype = C.c_int
    lib.ddcc_set_inflow.argtypes = [vp, dp, dp]
    lib.ddcc_set_inflow.restype = C.c_int
    lib.ddcc_adjoint_segment.argtypes = [vp, C.POINTER(vp), C.c_int, vp, vp, vp, C.c_size_t, vp, vp,
                                         C.POINTER(C.c_int)]
    lib.ddcc_adjoint_segment.restype = C.c_int
    lib.ddcc_adjoint_segment_pipelined.argtypes = [vp, C.POINTER(vp), C.c_int, C.POINTER(vp), C.c_int, vp, vp,
                                                   vp, C.c_size_t, vp, vp, C.POINTER(C.c_int)]
    lib.ddcc_adjoint_segment_pipelined.restype = C.c_int
    lib.ddcc_selftest_bounded_wait.argtypes = [vp, vp, C.c_int]
    lib.ddcc_selftest_bounded_wait.restype = C.c_int
    lib.ddcc_measure_fp64_peak.argtypes = [vp, vp, dp]
    lib.ddcc_measure_fp64_peak.restype = C.c_int
    lib.ddcc_rows_bytes.argtypes = [vp, C.c_int]
    lib.ddcc_rows_bytes.restype = C.c_size_t
    lib.ddcc_get_rows.argtypes = [vp, C.c_int, C.c_int, vp]
    lib.ddcc_get_rows.restype = C.c_int
    lib.ddcc_set_rows.argtypes = [vp, C.c_int, C.c_int, vp]
    lib.ddcc_set_rows.restype = C.c_int
    P3 = C.POINTER(ddcc3d_params)
    lib.ddcc3d_workspace_bytes.argtypes = [P3]
    lib.ddcc3d_workspace_bytes.restype = C.c_size_t
    lib.ddcc3d_create.argtypes = [P3, vp, C.c_size_t, vp, dp, dp, dp, dp, C.POINTER(vp)]
    lib.ddcc3d_create.restype = C.c_int
    lib.ddcc3d_step.argtypes = [vp, C.c_int64]
    lib.ddcc3d_step.restype = C.c_int
    lib.ddcc3d_read.argtypes = [vp, C.c_int, dp]
    lib.ddcc3d_read.restype = C.c_int
    lib.ddcc3d_mass.argtypes = [vp, dp]
    lib.ddcc3d_mass.restype = C.c_int
    lib.ddcc3d_step_count.argtypes = [vp]
    lib.ddcc3d_step_count.restype = C.c_int64
    lib.ddcc3d_profile.argtypes = [vp, C.c_int]
    lib.ddcc3d_profile.restype = C.c_int
    lib.ddcc3d_kernel_times.argtypes = [vp, dp, C.POINTER(C.c_int64), C.c_int]
    lib.ddcc3d_kernel_times.restype = C.c_int
    lib.ddcc3d_destroy.argtypes = [vp]
    lib.ddcc3d_destroy.restype = None
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().ddcc_status_string(int(status)).decode()


def make_params(prm: dict, precision: int = DDCC_FP64, flags: int = 0) -> ddcc_params:
    """Fill ddcc_params from a parameter dict (keys as in ``workloads``)."""
    p = ddcc_params()
    N = int(prm["nphase"])
    p.nx, p.ny, p.nphase = int(prm["nx"]), int(prm["ny"]), N
    p.periodic_x, p.periodic_y = int(prm["periodic_x"]), int(prm["periodic_y"])
    p.precision = int(precision)
    for i in range(N):
        p.rho[i] = float(prm["rho"][i])
        p.nu[i] = float(prm["nu"][i])
        for j in range(N):
            p.sigma[i][j] = float(prm["sigma"][i][j])
    for i in range(N - 1):
        p.eta[i] = float(prm["eta"][i])
    p.width, p.eps0, p.d0, p.m0 = (float(prm[k]) for k in ("width", "eps0", "d0", "m0"))
    for k in range(5):
        p.s_f[k] = float(prm["s_f"][k])
    for k in range(4):
        p.s_g[k] = float(prm["s_g"][k])
    p.rho0 = float(prm.get("rho0", 1.0))
    p.body_force[0], p.body_force[1] = (float(v) for v in prm.get("body_force", (0.0, 0.0)))
    p.flags = int(flags)
    return p


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def ddcc_workspace_bytes(params: ddcc_params) -> int:
    return int(load().ddcc_workspace_bytes(C.byref(params)))


def ddcc_create(params, dev_workspace: int, nbytes: int, stream: int, psi, cos_theta_field,
                cos_theta_uniform, C0):
    """Returns the handle (an opaque int)."""
    lib = load()
    psi, cf, cu, c0 = _f64(psi), _f64(cos_theta_field), _f64(cos_theta_uniform), _f64(C0)
    h = C.c_void_p()
    st = lib.ddcc_create(C.byref(params), C.c_void_p(dev_workspace), C.c_size_t(nbytes),
                         C.c_void_p(stream), _dptr(psi), _dptr(cf), _dptr(cu), _dptr(c0),
                         C.byref(h))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_create")
    return h.value


def ddcc_create_walls(params, dev_workspace: int, nbytes: int, stream: int, wall_psi, wall_cos_theta, C0):
    """Handle for a solid of several parts: wall_psi (K, ny, nx), wall_cos_theta
    (K, N-1, ny, nx) host float64 arrays."""
    lib = load()
    wp, wc, c0 = _f64(wall_psi), _f64(wall_cos_theta), _f64(C0)
    h = C.c_void_p()
    st = lib.ddcc_create_walls(C.byref(params), C.c_void_p(dev_workspace), C.c_size_t(nbytes),
                               C.c_void_p(stream), C.c_int(int(wp.shape[0])), _dptr(wp), _dptr(wc),
                               _dptr(c0), C.byref(h))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_create_walls")
    return h.value


def ddcc_step(h, nsteps: int):
    st = load().ddcc_step(C.c_void_p(h), C.c_int64(int(nsteps)))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_step")


def ddcc_read(h, field: int, out: np.ndarray):
    assert out.dtype == np.float64 and out.flags.c_contiguous
    st = load().ddcc_read(C.c_void_p(h), C.c_int(int(field)), _dptr(out))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_read")
    return out


def ddcc_mass(h, nphase: int) -> np.ndarray:
    out = np.zeros(max(nphase - 1, 1), dtype=np.float64)
    st = load().ddcc_mass(C.c_void_p(h), _dptr(out))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_mass")
    return out[: nphase - 1]


def ddcc_state_bytes(h) -> int:
    return int(load().ddcc_state_bytes(C.c_void_p(h)))


def ddcc_save_state(h, buf_ptr: int, on_device: bool):
    st = load().ddcc_save_state(C.c_void_p(h), C.c_void_p(buf_ptr), C.c_int(1 if on_device else 0))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_save_state")


def ddcc_load_state(h, buf_ptr: int, on_device: bool):
    st = load().ddcc_load_state(C.c_void_p(h), C.c_void_p(buf_ptr), C.c_int(1 if on_device else 0))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_load_state")


def ddcc_step_count(h) -> int:
    return int(load().ddcc_step_count(C.c_void_p(h)))


def ddcc_destroy(h):
    if h:
        load().ddcc_destroy(C.c_void_p(h))


def ddcc_version() -> int:
    return int(load().ddcc_version())


def ddcc_profile(h, enable: bool):
    st = load().ddcc_profile(C.c_void_p(h), C.c_int(1 if enable else 0))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_profile")


def ddcc_kernel_times(h):
    """{kind: (total_ms, launches)} recorded since the last call."""
    ms = (C.c_double * 8)()
    cnt = (C.c_int64 * 8)()
    n = load().ddcc_kernel_times(C.c_void_p(h), ms, cnt, 8)
    if n < 0:
        raise DdccError(n, "ddcc_kernel_times")
    return {KERNEL_KINDS[k]: (float(ms[k]), int(cnt[k])) for k in range(n)}


def ddcc_phase_mass_noalloc(dev_populations: int, precision: int, nphase: int, nx: int, ny: int,
                            row_stride: int, plane_stride: int, dev_out: int, stream: int):
    """Status code of the allocation-free per-phase mass reduction."""
    return int(load().ddcc_phase_mass_noalloc(
        C.c_void_p(dev_populations), C.c_int(precision), C.c_int(nphase), C.c_int(nx),
        C.c_int(ny), C.c_int64(row_stride), C.c_int64(plane_stride), C.c_void_p(dev_out),
        C.c_void_p(stream)))


def ddcc_step_path(h) -> int:
    return int(load().ddcc_step_path(C.c_void_p(h)))


def state_layout(nx: int, ny: int, nphase: int, elem_bytes: int):
    """(offset of node (0, 0) of the first population plane in a saved
    state, row stride, plane stride) in elements, as documented in ddcc.h."""
    pitch = (nx + 2 * GHOST_X + 31) // 32 * 32
    plane_bytes = (pitch * (ny + 2 * GHOST_Y) * elem_bytes + 255) // 256 * 256
    org = GHOST_Y * pitch + GHOST_X
    return 256 // elem_bytes + org, pitch, plane_bytes // elem_bytes


def ddcc_adjoint_bytes(h) -> int:
    return int(load().ddcc_adjoint_bytes(C.c_void_p(h)))


def ddcc_adjoint_step(h, state_n: int, adj_next: int, adj_out: int, scratch: int, scratch_bytes: int,
                      dJ_dcos: int, dJ_dpsi: int):
    st = load().ddcc_adjoint_step(C.c_void_p(h), C.c_void_p(state_n), C.c_void_p(adj_next),
                                  C.c_void_p(adj_out), C.c_void_p(scratch), C.c_size_t(scratch_bytes),
                                  C.c_void_p(dJ_dcos), C.c_void_p(dJ_dpsi))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_adjoint_step")


def ddcc_adjoint_initial(h, C0, adj0: int, scratch: int, scratch_bytes: int, dJ_dcos: int, dJ_dpsi: int):
    c0 = _f64(C0)
    st = load().ddcc_adjoint_initial(C.c_void_p(h), _dptr(c0), C.c_void_p(adj0), C.c_void_p(scratch),
                                     C.c_size_t(scratch_bytes), C.c_void_p(dJ_dcos), C.c_void_p(dJ_dpsi))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_adjoint_initial")


def ddcc_objective_centroid(h, phase: int, scratch: int, scratch_bytes: int, adj_seed: int = 0) -> float:
    out = np.zeros(1, dtype=np.float64)
    st = load().ddcc_objective_centroid(C.c_void_p(h), C.c_int(int(phase)), C.c_void_p(scratch),
                                        C.c_size_t(scratch_bytes), _dptr(out),
                                        C.c_void_p(adj_seed) if adj_seed else None)
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_objective_centroid")
    return float(out[0])


def ddcc_step_between(h, state_in: int, state_out: int) -> int:
    """Status code (DDCC_ERR_UNSUPPORTED when the handle's step path has no
    buffer-to-buffer step); other errors raise."""
    st = load().ddcc_step_between(C.c_void_p(h), C.c_void_p(state_in), C.c_void_p(state_out))
    if st not in (DDCC_OK, DDCC_ERR_UNSUPPORTED):
        raise DdccError(st, "ddcc_step_between")
    return int(st)


def ddcc_set_inflow(h, u_in, C_in):
    u, c = _f64(u_in), _f64(C_in)
    st = load().ddcc_set_inflow(C.c_void_p(h), _dptr(u), _dptr(c))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_set_inflow")


def ddcc_adjoint_segment(h, states, adj_cur: int, adj_other: int, scratch: int, scratch_bytes: int,
                         dJ_dcos: int, dJ_dpsi: int):
    """(status, result_in_other): DDCC_ERR_UNSUPPORTED is returned, other
    errors raise."""
    arr = (C.c_void_p * len(states))(*states)
    flag = C.c_int(0)
    st = load().ddcc_adjoint_segment(C.c_void_p(h), arr, C.c_int(len(states)), C.c_void_p(adj_cur),
                                     C.c_void_p(adj_other), C.c_void_p(scratch), C.c_size_t(scratch_bytes),
                                     C.c_void_p(dJ_dcos), C.c_void_p(dJ_dpsi), C.byref(flag))
    if st not in (DDCC_OK, DDCC_ERR_UNSUPPORTED):
        raise DdccError(st, "ddcc_adjoint_segment")
    return int(st), bool(flag.value)


def ddcc_adjoint_segment_pipelined(h, states, nxt, adj_cur: int, adj_other: int, scratch: int,
                                   scratch_bytes: int, dJ_dcos: int, dJ_dpsi: int):
    """(status, result_in_other) of the reverse of ``states`` with the
    recompute of ``nxt`` alongside: DDCC_ERR_UNSUPPORTED is returned, other
    errors raise."""
    a = (C.c_void_p * max(len(states), 1))(*states)
    b = (C.c_void_p * max(len(nxt), 1))(*nxt)
    flag = C.c_int(0)
    st = load().ddcc_adjoint_segment_pipelined(C.c_void_p(h), a, C.c_int(len(states)), b, C.c_int(len(nxt)),
                                               C.c_void_p(adj_cur), C.c_void_p(adj_other), C.c_void_p(scratch),
                                               C.c_size_t(scratch_bytes), C.c_void_p(dJ_dcos),
                                               C.c_void_p(dJ_dpsi), C.byref(flag))
    if st not in (DDCC_OK, DDCC_ERR_UNSUPPORTED):
        raise DdccError(st, "ddcc_adjoint_segment_pipelined")
    return int(st), bool(flag.value)


def ddcc_rows_bytes(h, nrows: int) -> int:
    return int(load().ddcc_rows_bytes(C.c_void_p(h), C.c_int(nrows)))


def ddcc_get_rows(h, y0: int, nrows: int, dev_buf: int) -> None:
    st = load().ddcc_get_rows(C.c_void_p(h), C.c_int(y0), C.c_int(nrows), C.c_void_p(dev_buf))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_get_rows")


def ddcc_set_rows(h, y0: int, nrows: int, dev_buf: int) -> None:
    st = load().ddcc_set_rows(C.c_void_p(h), C.c_int(y0), C.c_int(nrows), C.c_void_p(dev_buf))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_set_rows")


def ddcc_measure_fp64_peak(stream: int, dev_sink: int) -> float:
    """Measured FP64 FMA rate of the current device, TFLOP/s."""
    out = C.c_double(0.0)
    st = load().ddcc_measure_fp64_peak(C.c_void_p(stream), C.c_void_p(dev_sink), C.byref(out))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc_measure_fp64_peak")
    return float(out.value)


def ddcc_selftest_bounded_wait(stream: int, dev_flag: int, deliver: bool) -> int:
    """Status code: DDCC_ERR_TIMEOUT when the undelivered wait ran out."""
    return int(load().ddcc_selftest_bounded_wait(C.c_void_p(stream), C.c_void_p(dev_flag),
                                                 C.c_int(1 if deliver else 0)))


# ----------------------------------------------------------------------------
# three-dimensional stepper (include/ddcc3d.h)
# ----------------------------------------------------------------------------

def make_params_3d(prm: dict, precision: int = DDCC_FP64, flags: int = 0) -> ddcc3d_params:
    """Fill ddcc3d_params from a parameter dict (``workloads.base_params_3d``)."""
    p = ddcc3d_params()
    p.flags = int(flags)
    N = int(prm["nphase"])
    p.nx, p.ny, p.nz, p.nphase = int(prm["nx"]), int(prm["ny"]), int(prm["nz"]), N
    p.precision = int(precision)
    for i in range(N):
        p.rho[i] = float(prm["rho"][i])
        p.nu[i] = float(prm["nu"][i])
        for j in range(N):
            p.sigma[i][j] = float(prm["sigma"][i][j])
    for i in range(N - 1):
        p.eta[i] = float(prm["eta"][i])
    p.width, p.eps0, p.d0, p.m0 = (float(prm[k]) for k in ("width", "eps0", "d0", "m0"))
    for k in range(2):
        p.s_f[k] = float(prm["s_f"][k])
    for k in range(4):
        p.s_g[k] = float(prm["s_g"][k])
    p.rho0 = float(prm.get("rho0", 1.0))
    for a, v in enumerate(prm.get("body_force", (0.0, 0.0, 0.0))):
        p.body_force[a] = float(v)
    return p


def ddcc3d_workspace_bytes(params: ddcc3d_params) -> int:
    return int(load().ddcc3d_workspace_bytes(C.byref(params)))


def ddcc3d_create(params, dev_workspace: int, nbytes: int, stream: int, psi, cos_theta_field,
                  cos_theta_uniform, C0):
    """Returns the handle (an opaque int)."""
    lib = load()
    psi, cf, cu, c0 = _f64(psi), _f64(cos_theta_field), _f64(cos_theta_uniform), _f64(C0)
    h = C.c_void_p()
    st = lib.ddcc3d_create(C.byref(params), C.c_void_p(dev_workspace), C.c_size_t(nbytes),
                           C.c_void_p(stream), _dptr(psi), _dptr(cf), _dptr(cu), _dptr(c0),
                           C.byref(h))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc3d_create")
    return h.value


def ddcc3d_step(h, nsteps: int):
    st = load().ddcc3d_step(C.c_void_p(h), C.c_int64(int(nsteps)))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc3d_step")


def ddcc3d_read(h, field: int, out: np.ndarray):
    assert out.dtype == np.float64 and out.flags.c_contiguous
    st = load().ddcc3d_read(C.c_void_p(h), C.c_int(int(field)), _dptr(out))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc3d_read")
    return out


def ddcc3d_mass(h, nphase: int) -> np.ndarray:
    out = np.zeros(max(nphase - 1, 1), dtype=np.float64)
    st = load().ddcc3d_mass(C.c_void_p(h), _dptr(out))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc3d_mass")
    return out[: nphase - 1]


def ddcc3d_step_count(h) -> int:
    return int(load().ddcc3d_step_count(C.c_void_p(h)))


def ddcc3d_profile(h, enable: bool):
    st = load().ddcc3d_profile(C.c_void_p(h), C.c_int(1 if enable else 0))
    if st != DDCC_OK:
        raise DdccError(st, "ddcc3d_profile")


def ddcc3d_kernel_times(h):
    """{kind: (total_ms, launches)} recorded since the last call."""
    ms = (C.c_double * 4)()
    cnt = (C.c_int64 * 4)()
    n = load().ddcc3d_kernel_times(C.c_void_p(h), ms, cnt, 4)
    if n < 0:
        raise DdccError(n, "ddcc3d_kernel_times")
    return {KERNEL_KINDS_3D[k]: (float(ms[k]), int(cnt[k])) for k in range(n)}


def ddcc3d_destroy(h):
    if h:
        load().ddcc3d_destroy(C.c_void_p(h))
