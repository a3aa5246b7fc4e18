"""Decomposition of a y-periodic grid into y slabs, one per GPU.

The paper computes on one domain; this is how the step spreads over
several GPUs.  One step at node (x, y) reads the state within three rows of
y: the order parameters two rows out feed the chemical potential one row
out, whose gradient the node needs, and the populations streamed in come
from one row out.  So each rank runs the ordinary single-GPU step on its
own rows plus ``HALO`` = 3 extra rows on either side, treated as a periodic
grid of its own: after a step its own rows are exact, and only the three
edge rows on each side -- spoilt by the slab's own wrap -- must be replaced
by the neighbouring ranks' rows.  That exchange moves whole state rows
(every population and lagged plane, ``ddcc_get_rows`` / ``ddcc_set_rows``),
3 rows per side per step, point to point; the per-phase masses of the own
rows are reduced in FP64 on each rank and summed over ranks.  The extra
work is 6 rows per rank per step.

``SlabRun`` holds the decomposition logic and talks to a *stepper* (the
state of one extended slab) and an *exchange* (how rows reach the
neighbours); ``GpuSlab`` is the stepper on one GPU through the C ABI,
``TorchExchange`` the exchange over ``torch.distributed`` (NCCL with device
buffers, or gloo), and ``LocalSlabs`` holds every slab of a grid in one
process.
"""
from __future__ import annotations

import numpy as np

from . import _lib

HALO = 3


def slab_rows(ny: int, world: int, rank: int):
    """Own rows [y0, y1) of a rank: ny split as evenly as possible."""
    base, rem = divmod(int(ny), int(world))
    y0 = rank * base + min(rank, rem)
    return y0, y0 + base + (1 if rank < rem else 0)


def extend_rows(a, y0: int, y1: int, halo: int = HALO):
    """Rows y0 - halo .. y1 + halo - 1 of a (..., ny, nx) array, wrapping
    periodically in y."""
    a = np.asarray(a)
    ny = a.shape[-2]
    idx = np.arange(y0 - halo, y1 + halo) % ny
    return np.ascontiguousarray(np.take(a, idx, axis=-2))


class SlabRun:
    """One rank's slab: ``stepper`` holds the extended slab (own rows at
    local rows [HALO, HALO + n_own)), ``exchange`` delivers the neighbours'
    rows.  The halo rows are refreshed once at construction (they held the
    slab's own wrap until then) and after every step."""

    def __init__(self, stepper, n_own: int, exchange):
        if n_own < HALO:
            raise ValueError("each rank needs at least %d own rows" % HALO)
        self.stepper = stepper
        self.n_own = int(n_own)
        self.exchange = exchange
        self.refresh_halos()

    def refresh_halos(self):
        # own bottom rows go to the rank below (its top halo), own top rows to
        # the rank above (its bottom halo)
        down = self.stepper.get_rows(HALO, HALO)
        up = self.stepper.get_rows(self.n_own, HALO)
        from_below, from_above = self.exchange.swap(down, up)
        self.stepper.set_rows(0, HALO, from_below)
        self.stepper.set_rows(self.n_own + HALO, HALO, from_above)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.stepper.step(1)
            self.refresh_halos()

    def mass(self):
        """Per-phase FP64 mass of the whole grid (own rows, summed over
        ranks)."""
        return self.exchange.allreduce_sum(self.stepper.own_mass(HALO, self.n_own))

    def own_rows(self):
        """The rank's own state rows (the stepper's row layout)."""
        return self.stepper.get_rows(HALO, self.n_own)


class GpuSlab:
    """The extended slab on the current GPU: a ``Sim`` of rows
    y0 - HALO .. y1 + HALO - 1 of the global fields, periodic in y."""

    def __init__(self, params, psi, C0, cos_theta, cos_theta_field, y0: int, y1: int, precision, sim_cls):
        import torch
        if not int(params.get("periodic_y", 1)):
            raise ValueError("the y-slab decomposition needs a y-periodic grid")
        prm = dict(params)
        prm["ny"] = (y1 - y0) + 2 * HALO
        cf = None if cos_theta_field is None else extend_rows(cos_theta_field, y0, y1)
        self.sim = sim_cls(prm, extend_rows(psi, y0, y1), extend_rows(C0, y0, y1), cos_theta, cf,
                           precision=precision)
        self.N = self.sim.N
        self.nx = self.sim.nx
        self.precision = precision
        self._dtype = torch.float64 if precision == _lib.DDCC_FP64 else torch.float32
        self._out = torch.zeros(4, dtype=torch.float64, device="cuda")

    def step(self, n):
        self.sim.step(n)

    def _planes(self):
        return 9 * self.N + 2 * self.N + 3

    def get_rows(self, y0, n):
        import torch
        buf = torch.empty((self._planes(), n, self.nx), dtype=self._dtype, device="cuda")
        _lib.ddcc_get_rows(self.sim.h, y0, n, buf.data_ptr())
        return buf

    def set_rows(self, y0, n, buf):
        _lib.ddcc_set_rows(self.sim.h, y0, n, buf.contiguous().data_ptr())

    def own_mass(self, y0, n):
        import torch
        rows = self.get_rows(y0, n)
        st = _lib.ddcc_phase_mass_noalloc(rows.data_ptr(), self.precision, self.N, self.nx, n, self.nx,
                                          n * self.nx, self._out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
        if st != _lib.DDCC_OK:
            raise _lib.DdccError(st, "ddcc_phase_mass_noalloc")
        return self._out[: self.N - 1].cpu().numpy().copy()

    def close(self):
        self.sim.close()


class TorchExchange:
    """Rows to and from the neighbouring ranks over torch.distributed (ring
    of ranks, periodic in y); one rank exchanges with itself."""

    def __init__(self, rank: int, world: int, group=None):
        self.rank, self.world, self.group = int(rank), int(world), group

    def swap(self, down, up):
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return up.clone(), down.clone()
        below = (self.rank - 1) % self.world
        above = (self.rank + 1) % self.world
        from_below = torch.empty_like(up)
        from_above = torch.empty_like(down)
        # two phases, each a matched pair on every rank (with two ranks the
        # neighbour below is the neighbour above)
        for send, dst, recv, src in ((up, above, from_below, below), (down, below, from_above, above)):
            ops = [dist.P2POp(dist.isend, send.contiguous(), dst, self.group),
                   dist.P2POp(dist.irecv, recv, src, self.group)]
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        return from_below, from_above

    def allreduce_sum(self, local):
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return np.asarray(local, dtype=np.float64)
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor(np.asarray(local, dtype=np.float64), device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()


class LocalSlabs:
    """Every slab of one grid held in one process on the current GPU (for
    checking the decomposition against a single-domain run, and for a
    single GPU holding several slabs).  ``step`` steps every slab, then
    refreshes every halo from the neighbours' own rows, all read before any
    is written."""

    def __init__(self, params, psi, C0, cos_theta, cos_theta_field, world: int, precision, sim_cls):
        self.steppers, self.n_own = [], []
        ny = int(params["ny"])
        for r in range(int(world)):
            y0, y1 = slab_rows(ny, world, r)
            if y1 - y0 < HALO:
                raise ValueError("each slab needs at least %d own rows" % HALO)
            self.steppers.append(GpuSlab(params, psi, C0, cos_theta, cos_theta_field, y0, y1, precision,
                                         sim_cls))
            self.n_own.append(y1 - y0)
        self._refresh()

    def _refresh(self):
        w = len(self.steppers)
        got = []
        for r in range(w):
            below, above = (r - 1) % w, (r + 1) % w
            got.append((self.steppers[below].get_rows(self.n_own[below], HALO),
                        self.steppers[above].get_rows(HALO, HALO)))
        for r, (from_below, from_above) in enumerate(got):
            self.steppers[r].set_rows(0, HALO, from_below)
            self.steppers[r].set_rows(self.n_own[r] + HALO, HALO, from_above)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            for s in self.steppers:
                s.step(1)
            self._refresh()

    def mass(self):
        return np.sum([s.own_mass(HALO, n) for s, n in zip(self.steppers, self.n_own)], axis=0)

    def close(self):
        for s in self.steppers:
            s.close()
