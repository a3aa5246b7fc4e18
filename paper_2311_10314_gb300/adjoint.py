"""Gradients of a phase centroid after T steps with respect to the per-node
contact-angle field and the solid characteristic function psi.

The reverse sweep runs the library's adjoint kernels (``ddcc_adjoint_step``
per step, ``ddcc_adjoint_initial`` for the initial state), with step
checkpointing: the forward pass keeps the state every ``ckpt`` steps, and
each segment is recomputed forward (its states kept in HBM) before it is
reversed.  Where a whole segment of states does not fit in device memory
(a 4096^2 four-phase state is 3.2 GB in FP32), the checkpointing is two
level: a segment is first recomputed keeping only every ``sub``-th state,
then each sub-segment of ``sub`` steps is recomputed and reversed, so that
T/ckpt + ckpt/sub + sub states are held instead of T/ckpt + ckpt, for one
more forward step per reversed step.  The gradients are the same bit for
bit either way (the recompute is deterministic).  One-level sweeps that
have room for a second set of segment buffers are pipelined: each segment
is reversed while the next one (earlier in time) is recomputed into the
other set on a second stream (``ddcc_adjoint_segment_pipelined``), which
fills the GPU where the reverse kernels alone leave it idle; the
arithmetic and the gradients are unchanged.  ``rollout`` wraps this as a
``torch.autograd.Function``.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from . import Sim


class _Buffers:
    """Device buffers of one reverse sweep (torch uint8 tensors, 256-aligned):
    n_ckpt checkpoints, n_sub sub-segment checkpoints (two-level only), seg
    recomputed states and, for a pipelined sweep, a second set of seg2."""

    def __init__(self, sim, n_ckpt, seg, n_sub=0, seg2=0):
        import torch
        self.sb = _lib.ddcc_state_bytes(sim.h)
        self.ab = _lib.ddcc_adjoint_bytes(sim.h)
        self._keep = []
        self._view = {}
        self.ckpt = [self._alloc(self.sb) for _ in range(n_ckpt)]
        self.sub = [self._alloc(self.sb) for _ in range(n_sub)]
        self.seg = [self._alloc(self.sb) for _ in range(seg)]
        self.seg2 = [self._alloc(self.sb) for _ in range(seg2)]
        self.adj = [self._alloc(self.sb) for _ in range(2)]
        self.scratch = self._alloc(self.ab)
        N, ny, nx = sim.N, sim.ny, sim.nx
        self.dJ_dcos = torch.zeros((max(N - 1, 1), ny, nx), dtype=torch.float64, device="cuda")
        self.dJ_dpsi = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")

    def _alloc(self, nbytes):
        import torch
        t = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        self._keep.append(t)
        ptr = (t.data_ptr() + 255) // 256 * 256
        off = ptr - t.data_ptr()
        self._view[ptr] = t[off:off + nbytes]
        return ptr

    def copy_state(self, dst, src, stream):
        """Device copy of one saved state on the handle's stream."""
        import torch
        with torch.cuda.stream(stream):
            self._view[dst].copy_(self._view[src], non_blocking=True)


def _states_that_fit(sim, spare=0.9):
    """How many more states the current device has room for."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(free * spare) // (_lib.ddcc_state_bytes(sim.h) + 256)


class CheckpointedRun:
    """Forward pass with a checkpoint at the start of every ``ckpt``-step
    segment; ``reverse`` then runs the adjoint sweep from the seed dJ/dstate.
    ``sub``: None picks one-level checkpointing when a whole segment of
    states fits in device memory and two-level with sub = ceil(sqrt(ckpt))
    otherwise; an integer 1 <= sub < ckpt forces two-level with that
    sub-segment length; sub >= ckpt forces one level.  ``pipeline``: None
    pipelines a one-level sweep when two sets of segment buffers fit, False
    never, True whenever the sweep is one-level."""

    def __init__(self, params, psi, C0, cos_theta_field, T, ckpt=100, precision=_lib.DDCC_FP64,
                 phase=0, path="tile", sub=None, pipeline=None):
        self.T = int(T)
        self.ckpt = max(1, int(ckpt))
        self.phase = int(phase)
        self.C0 = np.asarray(C0, dtype=np.float64)
        self.sim = Sim(params, psi, C0, cos_theta_field=cos_theta_field, precision=precision, path=path)
        self.starts = list(range(0, self.T, self.ckpt))
        seg = min(self.ckpt, max(self.T, 1))
        room = _states_that_fit(self.sim) - len(self.starts) - 3
        if sub is None:
            sub = seg if seg <= room else int(np.ceil(np.sqrt(seg)))
        self.sub = max(1, min(int(sub), seg))
        if pipeline is None:
            pipeline = 2 * seg <= room
        self.pipe = bool(pipeline) and self.sub >= seg and seg > 1
        if self.sub < seg:
            n_sub = (seg + self.sub - 1) // self.sub
            self.buf = _Buffers(self.sim, len(self.starts), self.sub, n_sub)
        else:
            self.buf = _Buffers(self.sim, len(self.starts), seg, seg2=seg if self.pipe else 0)
        for k, t0 in enumerate(self.starts):
            _lib.ddcc_save_state(self.sim.h, self.buf.ckpt[k], True)
            self.sim.step(min(self.ckpt, self.T - t0))
        cur = self.buf.adj[0]
        self.J = _lib.ddcc_objective_centroid(self.sim.h, self.phase, self.buf.scratch, self.buf.ab, cur)

    def reverse(self):
        """dJ/dcos(theta_iN) (N-1, ny, nx) and dJ/dpsi (ny, nx), float64 numpy."""
        import torch
        sim, buf = self.sim, self.buf
        self._cur, self._nxt = buf.adj
        if self.pipe:
            self._reverse_pipelined()
        else:
            self._reverse_segments()
        cur = self._cur
        _lib.ddcc_adjoint_initial(sim.h, self.C0, cur, buf.scratch, buf.ab, buf.dJ_dcos.data_ptr(),
                                  buf.dJ_dpsi.data_ptr())
        torch.cuda.synchronize()
        return buf.dJ_dcos.cpu().numpy()[: sim.N - 1], buf.dJ_dpsi.cpu().numpy()

    def _reverse_pipelined(self):
        """All segments, last first, each reversed while the one before it
        is recomputed into the other buffer set.  Where the step path has
        no buffer-to-buffer step the library refuses the call before
        launching anything, and the segments not yet reversed go through
        ``_reverse_segment`` one by one."""
        sim, buf = self.sim, self.buf
        sets = (buf.seg, buf.seg2)
        K = len(self.starts)
        lens = [min(self.ckpt, self.T - t0) for t0 in self.starts]
        cur, nxt = self._cur, self._nxt
        for k in range(K, -1, -1):
            # reverse segment k (nothing at k = K), recompute segment k - 1;
            # the head copy is queued after the reverse of segment k + 1,
            # the last user of that buffer set
            rev = sets[k % 2][: lens[k]] if k < K else []
            ahead = []
            if k >= 1:
                ahead = sets[(k - 1) % 2][: lens[k - 1]]
                buf.copy_state(ahead[0], buf.ckpt[k - 1], sim.stream)
            st, flipped = _lib.ddcc_adjoint_segment_pipelined(
                sim.h, rev, ahead, cur, nxt, buf.scratch, buf.ab,
                buf.dJ_dcos.data_ptr(), buf.dJ_dpsi.data_ptr())
            if st != _lib.DDCC_OK:
                self._cur, self._nxt = cur, nxt
                for j in range(min(k, K - 1), -1, -1):
                    self._reverse_segment(buf.ckpt[j], lens[j])
                return
            if flipped:
                cur, nxt = nxt, cur
        self._cur, self._nxt = cur, nxt

    def _reverse_segments(self):
        sim, buf = self.sim, self.buf
        for k in range(len(self.starts) - 1, -1, -1):
            t0 = self.starts[k]
            n = min(self.ckpt, self.T - t0)
            if not buf.sub:
                self._reverse_segment(buf.ckpt[k], n)
                continue
            # two level: the sub-segment checkpoints of this segment, then
            # each sub-segment recomputed and reversed, last first
            _lib.ddcc_load_state(sim.h, buf.ckpt[k], True)
            heads = list(range(0, n, self.sub))
            for j, s0 in enumerate(heads):
                _lib.ddcc_save_state(sim.h, buf.sub[j], True)
                if j + 1 < len(heads):
                    sim.step(self.sub)
            for j in range(len(heads) - 1, -1, -1):
                self._reverse_segment(buf.sub[j], min(self.sub, n - heads[j]))

    def _reverse_segment(self, head, n):
        """Reverse the n steps that start from the state at head."""
        sim, buf = self.sim, self.buf
        cur, nxt = self._cur, self._nxt
        # the whole segment in one library call where the step path allows;
        # the head state is copied into the segment's own first buffer, so
        # every segment of a sweep passes the same buffers and the library
        # replays the segment as one CUDA graph after the first two
        buf.copy_state(buf.seg[0], head, sim.stream)
        st, flipped = _lib.ddcc_adjoint_segment(
            sim.h, buf.seg[:n], cur, nxt, buf.scratch, buf.ab,
            buf.dJ_dcos.data_ptr(), buf.dJ_dpsi.data_ptr())
        if st == _lib.DDCC_OK:
            if flipped:
                cur, nxt = nxt, cur
        else:
            states = self._recompute(head, n)
            for s in range(n - 1, -1, -1):
                _lib.ddcc_adjoint_step(sim.h, states[s], cur, nxt, buf.scratch, buf.ab,
                                       buf.dJ_dcos.data_ptr(), buf.dJ_dpsi.data_ptr())
                cur, nxt = nxt, cur
        self._cur, self._nxt = cur, nxt

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
                      phase=0, path="tile", sub=None, pipeline=None):
    """J = sum_x x m_i(x) / sum_x m_i(x) (m_i = sum_p f^i_p, i = ``phase``)
    after T steps from the initial state of (psi, C0, cos_theta_field), and
    dJ/dcos(theta_iN)(x), dJ/dpsi(x) as float64 numpy arrays (``sub`` as in
    ``CheckpointedRun``)."""
    run = CheckpointedRun(params, psi, C0, cos_theta_field, T, ckpt, precision, phase, path, sub, pipeline)
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
