"""Gradients of a phase centroid after T steps with respect to the per-node
contact-angle field and the solid characteristic function psi.

The reverse sweep runs the library's adjoint kernels (``ddcc_adjoint_step``
per step, ``ddcc_adjoint_initial`` for the initial state), with step
checkpointing: the forward pass keeps the state every ``ckpt`` steps, and
each segment is recomputed forward (its states kept in HBM) before it is
reversed.  ``rollout`` wraps this as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from . import Sim


class _Buffers:
    """Device buffers of one reverse sweep (torch uint8 tensors, 256-aligned)."""

    def __init__(self, sim, n_ckpt, seg):
        import torch
        self.sb = _lib.ddcc_state_bytes(sim.h)
        self.ab = _lib.ddcc_adjoint_bytes(sim.h)
        self._keep = []
        self.ckpt = [self._alloc(self.sb) for _ in range(n_ckpt)]
        self.seg = [self._alloc(self.sb) for _ in range(seg)]
        self.adj = [self._alloc(self.sb) for _ in range(2)]
        self.scratch = self._alloc(self.ab)
        N, ny, nx = sim.N, sim.ny, sim.nx
        self.dJ_dcos = torch.zeros((max(N - 1, 1), ny, nx), dtype=torch.float64, device="cuda")
        self.dJ_dpsi = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")

    def _alloc(self, nbytes):
        import torch
        t = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        self._keep.append(t)
        return (t.data_ptr() + 255) // 256 * 256


class CheckpointedRun:
    """Forward pass with a checkpoint at the start of every ``ckpt``-step
    segment; ``reverse`` then runs the adjoint sweep from the seed dJ/dstate."""

    def __init__(self, params, psi, C0, cos_theta_field, T, ckpt=100, precision=_lib.DDCC_FP64,
                 phase=0, path="tile"):
        self.T = int(T)
        self.ckpt = max(1, int(ckpt))
        self.phase = int(phase)
        self.C0 = np.asarray(C0, dtype=np.float64)
        self.sim = Sim(params, psi, C0, cos_theta_field=cos_theta_field, precision=precision, path=path)
        self.starts = list(range(0, self.T, self.ckpt))
        self.buf = _Buffers(self.sim, len(self.starts), min(self.ckpt, max(self.T, 1)))
        for k, t0 in enumerate(self.starts):
            _lib.ddcc_save_state(self.sim.h, self.buf.ckpt[k], True)
            self.sim.step(min(self.ckpt, self.T - t0))
        cur = self.buf.adj[0]
        self.J = _lib.ddcc_objective_centroid(self.sim.h, self.phase, self.buf.scratch, self.buf.ab, cur)

    def reverse(self):
        """dJ/dcos(theta_iN) (N-1, ny, nx) and dJ/dpsi (ny, nx), float64 numpy."""
        import torch
        sim, buf = self.sim, self.buf
        cur, nxt = buf.adj
        for k in range(len(self.starts) - 1, -1, -1):
            t0 = self.starts[k]
            n = min(self.ckpt, self.T - t0)
            # the whole segment in one library call where the step path allows
            st, flipped = _lib.ddcc_adjoint_segment(
                sim.h, [buf.ckpt[k]] + buf.seg[1:n], cur, nxt, buf.scratch, buf.ab,
                buf.dJ_dcos.data_ptr(), buf.dJ_dpsi.data_ptr())
            if st == _lib.DDCC_OK:
                if flipped:
                    cur, nxt = nxt, cur
                continue
            states = self._recompute(buf.ckpt[k], n)
            for s in range(n - 1, -1, -1):
                _lib.ddcc_adjoint_step(sim.h, states[s], cur, nxt, buf.scratch, buf.ab,
                                       buf.dJ_dcos.data_ptr(), buf.dJ_dpsi.data_ptr())
                cur, nxt = nxt, cur
        _lib.ddcc_adjoint_initial(sim.h, self.C0, cur, buf.scratch, buf.ab, buf.dJ_dcos.data_ptr(),
                                  buf.dJ_dpsi.data_ptr())
        torch.cuda.synchronize()
        return buf.dJ_dcos.cpu().numpy()[: sim.N - 1], buf.dJ_dpsi.cpu().numpy()

    def _recompute(self, ckpt_state, n):
        """The states of steps t0 .. t0+n-1 of a segment from its checkpoint:
        buffer to buffer when the step path allows it, else load/step/save."""
        sim, buf = self.sim, self.buf
        states = [ckpt_state] + buf.seg[1:n]
        for s in range(1, n):
            if _lib.ddcc_step_between(sim.h, states[s - 1], states[s]) != _lib.DDCC_OK:
                break
        else:
            return states
        _lib.ddcc_load_state(sim.h, ckpt_state, True)
        for s in range(1, n):
            sim.step(1)
            _lib.ddcc_save_state(sim.h, buf.seg[s], True)
        return states

    def close(self):
        if self.sim is not None:
            self.sim.close()
            self.sim = None
            self.buf = None


def centroid_gradient(params, psi, C0, cos_theta_field, T, ckpt=100, precision=_lib.DDCC_FP64,
                      phase=0, path="tile"):
    """J = sum_x x m_i(x) / sum_x m_i(x) (m_i = sum_p f^i_p, i = ``phase``)
    after T steps from the initial state of (psi, C0, cos_theta_field), and
    dJ/dcos(theta_iN)(x), dJ/dpsi(x) as float64 numpy arrays."""
    run = CheckpointedRun(params, psi, C0, cos_theta_field, T, ckpt, precision, phase, path)
    try:
        gc, gp = run.reverse()
        return run.J, gc, gp
    finally:
        run.close()


def centroid(params, psi, C0, cos_theta_field, T, precision=_lib.DDCC_FP64, phase=0, path="tile"):
    """The forward objective alone (no adjoint)."""
    sim = Sim(params, psi, C0, cos_theta_field=cos_theta_field, precision=precision, path=path)
    try:
        sim.step(int(T))
        import torch
        scratch = torch.empty(_lib.ddcc_adjoint_bytes(sim.h) + 256, dtype=torch.uint8, device="cuda")
        ptr = (scratch.data_ptr() + 255) // 256 * 256
        return _lib.ddcc_objective_centroid(sim.h, phase, ptr, _lib.ddcc_adjoint_bytes(sim.h), 0)
    finally:
        sim.close()


def rollout(cos_theta_field, psi, params, C0, T, ckpt=100, precision=_lib.DDCC_FP64, phase=0):
    """Differentiable J(cos_theta_field, psi) as a torch float64 scalar: the
    forward runs T steps with checkpoints, backward runs the adjoint sweep."""
    import torch

    class _Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, cos_f, psi_t):
            run = CheckpointedRun(params, psi_t.detach().cpu().numpy(), C0,
                                  cos_f.detach().cpu().numpy(), T, ckpt, precision, phase)
            ctx.run = run
            ctx.meta = (cos_f.dtype, cos_f.device, psi_t.dtype, psi_t.device)
            return torch.tensor(run.J, dtype=torch.float64, device=cos_f.device)

        @staticmethod
        def backward(ctx, gJ):
            run = ctx.run
            try:
                gc, gp = run.reverse()
            finally:
                run.close()
            cd, cdev, pd, pdev = ctx.meta
            return (gJ * torch.as_tensor(gc, dtype=cd, device=cdev),
                    gJ * torch.as_tensor(gp, dtype=pd, device=pdev))

    return _Rollout.apply(cos_theta_field, psi)
