"""The C ABI library builds for sm_103a, loads, and exports every symbol
include/ddcc.h and include/ddcc3d.h declare.  Host-only entry points are
exercised; nothing here launches a kernel."""
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_10314_gb300 import build as B
    B.build()
    from paper_2311_10314_gb300 import _lib
    return _lib


def _declared_functions(header="ddcc.h", prefix="ddcc_"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(%s[a-z0-9_]+)\s*\(" % prefix, text)))


def test_header_lists_the_binding_symbols():
    from paper_2311_10314_gb300 import _lib
    assert _declared_functions() == sorted(_lib.EXPORTED)
    assert _declared_functions("ddcc3d.h", "ddcc3d_") == sorted(_lib.EXPORTED_3D)


def test_exports_every_declared_symbol(lib):
    L = lib.load()
    for name in _declared_functions() + _declared_functions("ddcc3d.h", "ddcc3d_"):
        assert hasattr(L, name), name


def test_version_and_status_strings(lib):
    assert lib.ddcc_version() >= 100
    assert lib.status_string(0) == "ok"
    for code in (-1, -2, -3, -4, -5, -6):
        assert lib.status_string(code) not in ("ok", "unknown status")


def test_workspace_bytes_host_only(lib):
    pb = W.config1_droplet_wall()
    p64 = lib.make_params(pb.params, lib.DDCC_FP64)
    p32 = lib.make_params(pb.params, lib.DDCC_FP32)
    b64, b32 = lib.ddcc_workspace_bytes(p64), lib.ddcc_workspace_bytes(p32)
    assert b64 > 0 and b32 > 0 and b64 > b32
    # ~ (2 x 9(N-1) + 2 x 9 + 2 (2N+3) + ...) planes of 64 x 64 doubles
    assert b64 >= 8 * 64 * 64 * (2 * 9 + 2 * 9 + 2 * 7)


@pytest.mark.parametrize("field,value", [
    ("nphase", 5), ("nphase", 1), ("nx", 2), ("d0", 1.0), ("width", 0.0),
    ("m0", -1.0), ("precision", 7),
])
def test_invalid_params_rejected(lib, field, value):
    pb = W.config1_droplet_wall()
    p = lib.make_params(pb.params, lib.DDCC_FP64)
    setattr(p, field, value)
    assert lib.ddcc_workspace_bytes(p) == 0


def test_asymmetric_sigma_rejected(lib):
    pb = W.config2_lens(nx=64, ny=64)
    p = lib.make_params(pb.params, lib.DDCC_FP64)
    p.sigma[0][1] = 0.5
    assert lib.ddcc_workspace_bytes(p) == 0


def test_create_rejects_bad_workspace_without_gpu_work(lib):
    pb = W.config1_droplet_wall()
    p = lib.make_params(pb.params, lib.DDCC_FP64)
    with pytest.raises(lib.DdccError) as e:
        lib.ddcc_create(p, 0, 0, 0, pb.psi, None, pb.cos_theta, pb.C0)
    assert e.value.status == lib.DDCC_ERR_WORKSPACE


def test_workspace_bytes_3d_host_only(lib):
    prm = W.base_params_3d(20, 18, 16, 3)
    b64 = lib.ddcc3d_workspace_bytes(lib.make_params_3d(prm, lib.DDCC_FP64))
    b32 = lib.ddcc3d_workspace_bytes(lib.make_params_3d(prm, lib.DDCC_FP32))
    n = 20 * 18 * 16
    # 2 (7 (N-1) + 15) population planes, 2 (3N + 7) lagged planes, psi,
    # angles, C, mu: 98 planes at N = 3, plus a double staging plane
    assert b64 >= 8 * n * 98 + 8 * n and b32 >= 4 * n * 98 + 8 * n and b64 > b32


@pytest.mark.parametrize("field,value", [
    ("nphase", 5), ("nz", 2), ("d0", 0.5), ("d0", 0.0), ("width", 0.0), ("reserved", 1),
    ("flags", 3), ("flags", 4), ("precision", 3), ("nz", 131072), ("ny", 262144),
])
def test_invalid_params_3d_rejected(lib, field, value):
    p = lib.make_params_3d(W.base_params_3d(8, 8, 8, 2), lib.DDCC_FP64)
    assert lib.ddcc3d_workspace_bytes(p) > 0
    setattr(p, field, value)
    assert lib.ddcc3d_workspace_bytes(p) == 0


def test_create_3d_rejects_bad_workspace_without_gpu_work(lib):
    pb = W.random_problem_3d(8, 8, 8, 2, seed=1)
    p = lib.make_params_3d(pb.params, lib.DDCC_FP64)
    with pytest.raises(lib.DdccError) as e:
        lib.ddcc3d_create(p, 0, 0, 0, pb.psi, None, pb.cos_theta, pb.C0)
    assert e.value.status == lib.DDCC_ERR_WORKSPACE


def test_segment_calls_reject_bad_arguments_without_gpu_work(lib):
    """The reverse-segment entry points check their arguments on the host
    before touching the GPU: a null handle, negative or zero lengths."""
    import ctypes as C
    L = lib.load()
    vp = C.c_void_p
    flag = C.c_int(0)
    one = (vp * 1)(vp(256))
    for n, n_next in ((1, 1), (-1, 2), (2, -1)):
        st = L.ddcc_adjoint_segment_pipelined(None, one, n, one, n_next, vp(256), vp(512), vp(768),
                                              C.c_size_t(1 << 20), vp(1024), vp(2048), C.byref(flag))
        assert st == lib.DDCC_ERR_PARAM
    assert L.ddcc_adjoint_segment(None, one, 1, vp(256), vp(512), vp(768), C.c_size_t(1 << 20), vp(1024),
                                  vp(2048), C.byref(flag)) == lib.DDCC_ERR_PARAM
    assert L.ddcc_adjoint_segment(None, one, 0, vp(256), vp(512), vp(768), C.c_size_t(1 << 20), vp(1024),
                                  vp(2048), C.byref(flag)) == lib.DDCC_ERR_PARAM
