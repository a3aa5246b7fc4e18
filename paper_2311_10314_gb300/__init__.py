"""GB300-native DD-CCLB time stepper (arXiv 2311.10314) behind a C ABI.

``Sim`` owns one handle of libddcc.so (the D2Q9 stepper of include/ddcc.h),
``Sim3D`` one of its three-dimensional stepper (D3Q7 / D3Q15, include/ddcc3d.h):
the device workspace is a torch uint8 tensor on the current CUDA device, all
work runs on torch's current stream, and every step runs in the library's
sm_103a kernels.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (DDCC_FP32, DDCC_FP64, FIELD_C, FIELD_MU, FIELD_P, FIELD_PSI, FIELD_RHO,
                   FIELD_UX, FIELD_UY, DdccError, make_params)

__all__ = ["Sim", "Sim3D", "DDCC_FP32", "DDCC_FP64", "DdccError", "make_params"]


class Sim:
    """One DD-CCLB simulation on the current CUDA device.

    ``params`` is a parameter dict (see ``workloads.base_params``), ``psi``
    (ny, nx), ``C0`` (N-1, ny, nx), ``cos_theta`` (N-1,) uniform values or
    ``cos_theta_field`` (N-1, ny, nx); all float64 host arrays.  ``path``
    picks the step kernels: "tile" (default) or "sweep" (the TMA row sweep).
    ``walls`` = [(psi_k, cos_k), ...] gives a solid of several parts, each
    with its own characteristic function and angles (then ``psi`` and the
    angle arguments are ignored; psi = prod_k psi_k).
    """

    def __init__(self, params, psi, C0, cos_theta=None, cos_theta_field=None,
                 precision=DDCC_FP64, stream=None, path="tile", walls=None, open_x=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ddcc.Sim needs a CUDA device")
        _lib.load()
        self.params = dict(params)
        self.N = int(params["nphase"])
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self.precision = int(precision)
        if path not in ("tile", "sweep"):
            raise ValueError("path must be 'tile' or 'sweep'")
        flags = _lib.DDCC_FLAG_SWEEP if path == "sweep" else _lib.DDCC_FLAG_TILE
        if open_x is not None:
            flags |= _lib.DDCC_FLAG_OPEN_X
        self._p = make_params(params, precision, flags)
        nbytes = _lib.ddcc_workspace_bytes(self._p)
        if nbytes == 0:
            raise DdccError(_lib.DDCC_ERR_PARAM, "ddcc_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._ws_bytes = nbytes
        if walls is not None:
            # a solid of several parts: [(psi_k, cos_k), ...], cos_k the N-1
            # angles cos(theta^k_iN), uniform (N-1,) or per node (N-1, ny, nx)
            wp = np.stack([np.asarray(pk, dtype=np.float64) for pk, _ in walls])
            wc = np.stack([np.broadcast_to(np.asarray(ck, dtype=np.float64).reshape(
                self.N - 1, *([1, 1] if np.ndim(ck) == 1 else [self.ny, self.nx])),
                (self.N - 1, self.ny, self.nx)) for _, ck in walls])
            self.h = _lib.ddcc_create_walls(self._p, self._ws_ptr, nbytes, self.stream.cuda_stream,
                                            wp, wc, C0)
            if open_x is not None:
                _lib.ddcc_set_inflow(self.h, open_x[0], open_x[1])
            return
        cu = None if cos_theta is None else np.asarray(cos_theta, dtype=np.float64)
        if cos_theta_field is None and cu is None:
            raise ValueError("give cos_theta or cos_theta_field")
        self.h = _lib.ddcc_create(self._p, self._ws_ptr, nbytes, self.stream.cuda_stream,
                                  psi, cos_theta_field, cu, C0)
        if open_x is not None:
            # open_x = (u_in (ny,), C_in (N-1, ny)): inflow at x = 0, outflow at nx - 1
            _lib.ddcc_set_inflow(self.h, open_x[0], open_x[1])

    # -- stepping and read-out --------------------------------------------
    def step(self, n=1):
        _lib.ddcc_step(self.h, n)

    def read(self, field):
        out = np.empty((self.ny, self.nx), dtype=np.float64)
        return _lib.ddcc_read(self.h, field, out)

    def fields(self):
        """C (N, ny, nx), rho, ux, uy, P, mu (N, ny, nx) of the current state."""
        N = self.N
        return dict(C=np.stack([self.read(FIELD_C + i) for i in range(N)]),
                    rho=self.read(FIELD_RHO), ux=self.read(FIELD_UX), uy=self.read(FIELD_UY),
                    P=self.read(FIELD_P),
                    mu=np.stack([self.read(FIELD_MU + i) for i in range(N)]))

    def mass(self):
        return _lib.ddcc_mass(self.h, self.N)

    @property
    def path(self):
        """'sweep' or 'tile': the kernels ddcc_step runs for this handle."""
        return "sweep" if _lib.ddcc_step_path(self.h) == _lib.DDCC_PATH_SWEEP else "tile"

    @property
    def steps(self):
        return _lib.ddcc_step_count(self.h)

    def state_bytes(self):
        return _lib.ddcc_state_bytes(self.h)

    def save_state(self, buf=None):
        """Save to a torch uint8 CUDA tensor (allocated if ``buf`` is None)."""
        import torch
        if buf is None:
            buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device="cuda")
        _lib.ddcc_save_state(self.h, buf.data_ptr(), buf.is_cuda)
        return buf

    def load_state(self, buf):
        _lib.ddcc_load_state(self.h, buf.data_ptr(), buf.is_cuda)

    def close(self):
        if getattr(self, "h", None):
            _lib.ddcc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim3D:
    """One three-dimensional DD-CCLB simulation (periodic box) on the current
    CUDA device.  ``params`` from ``workloads.base_params_3d``; ``psi``
    (nz, ny, nx), ``C0`` (N-1, nz, ny, nx), ``cos_theta`` (N-1,) or
    ``cos_theta_field`` (N-1, nz, ny, nx); float64 host arrays.  ``path``
    "fused" (one kernel per step), "split" (three kernels) or "auto"
    (fused in FP32, split in FP64)."""

    def __init__(self, params, psi, C0, cos_theta=None, cos_theta_field=None,
                 precision=DDCC_FP64, stream=None, path="auto"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ddcc.Sim3D needs a CUDA device")
        _lib.load()
        self.params = dict(params)
        self.N = int(params["nphase"])
        self.shape = (int(params["nz"]), int(params["ny"]), int(params["nx"]))
        self.precision = int(precision)
        flags = {"auto": 0, "split": _lib.DDCC3D_FLAG_SPLIT, "fused": _lib.DDCC3D_FLAG_FUSED}
        if path not in flags:
            raise ValueError("path is 'auto', 'fused' or 'split'")
        self.path = path
        self._p = _lib.make_params_3d(params, precision, flags[path])
        nbytes = _lib.ddcc3d_workspace_bytes(self._p)
        if nbytes == 0:
            raise DdccError(_lib.DDCC_ERR_PARAM, "ddcc3d_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        self._ws_ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        cu = None if cos_theta is None else np.asarray(cos_theta, dtype=np.float64)
        if cos_theta_field is None and cu is None:
            raise ValueError("give cos_theta or cos_theta_field")
        self.h = _lib.ddcc3d_create(self._p, self._ws_ptr, nbytes, self.stream.cuda_stream,
                                    psi, cos_theta_field, cu, C0)

    def step(self, n=1):
        _lib.ddcc3d_step(self.h, n)

    def read(self, field):
        out = np.empty(self.shape, dtype=np.float64)
        return _lib.ddcc3d_read(self.h, field, out)

    def fields(self):
        """C (N, nz, ny, nx), rho, ux, uy, uz, P, mu (N, ...) of the current state."""
        N = self.N
        return dict(C=np.stack([self.read(FIELD_C + i) for i in range(N)]),
                    rho=self.read(FIELD_RHO), ux=self.read(FIELD_UX), uy=self.read(FIELD_UY),
                    uz=self.read(_lib.FIELD_UZ), P=self.read(FIELD_P),
                    mu=np.stack([self.read(FIELD_MU + i) for i in range(N)]))

    def mass(self):
        return _lib.ddcc3d_mass(self.h, self.N)

    @property
    def steps(self):
        return _lib.ddcc3d_step_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            _lib.ddcc3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
