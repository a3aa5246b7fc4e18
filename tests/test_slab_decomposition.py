"""The y-slab decomposition (``paper_2311_10314_gb300.slab``) on CPU ranks.

Each gloo rank runs the FP64 oracle on its extended slab (own rows plus
three rows a side, periodic of its own) through ``SlabRun`` and
``TorchExchange`` -- the same decomposition and exchange code the GPU
ranks run, with the oracle as the stepper.  After the steps, every rank's
own rows of every population and lagged field equal the single-domain
oracle's to round-off (1e-13 of each field's scale: the arithmetic is the
same node by node, but torch may sum in another order for another array
shape), and the FP64 masses summed over ranks equal the single-domain
masses to round-off.  With a halo of two rows instead of three the own
rows are off by far more than that.  Two and three ranks, with a per-node
angle field, a body force and density contrast; a rank's own-row count
both even and ragged.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleSlab:
    """The extended slab held by the FP64 oracle; rows in the library's
    plane order: f^1..f^{N-1} (9 each), g (9), a, psi C_i u (x, y per
    phase), T (xx, yy, xy), psi m.u."""

    def __init__(self, pb, y0, y1):
        from oracle import Oracle
        from paper_2311_10314_gb300 import slab
        prm = dict(pb.params)
        prm["ny"] = (y1 - y0) + 2 * slab.HALO
        cf = None if pb.cos_theta_field is None else slab.extend_rows(pb.cos_theta_field, y0, y1)
        self.o = Oracle(prm, slab.extend_rows(pb.psi, y0, y1), slab.extend_rows(pb.C0, y0, y1),
                        pb.cos_theta, cf)
        self.N = int(prm["nphase"])

    def step(self, n):
        self.o.step(n)

    def _fields(self):
        o = self.o
        return [o.f.reshape(-1, o.ny, o.nx), o.g, o.a[None], o.psiCu.reshape(-1, o.ny, o.nx), o.T,
                o.psimu[None]]

    def get_rows(self, y0, n):
        return torch.cat([f[:, y0:y0 + n] for f in self._fields()]).clone()

    def set_rows(self, y0, n, buf):
        k = 0
        for f in self._fields():
            f[:, y0:y0 + n] = buf[k:k + f.shape[0]]
            k += f.shape[0]

    def own_mass(self, y0, n):
        return self.o.f[:, :, y0:y0 + n].sum(dim=(1, 2, 3)).numpy()


def _problem():
    import workloads as W
    return W.random_problem(24, 20, 3, seed=5, theta_field=True, width=4.0, body_force=(2e-5, 0.0))


def _rank(rank, world, port, steps, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    torch.set_num_threads(1)
    import torch.distributed as dist
    from paper_2311_10314_gb300 import slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb = _problem()
    y0, y1 = slab.slab_rows(pb.params["ny"], world, rank)
    run = slab.SlabRun(OracleSlab(pb, y0, y1), y1 - y0, slab.TorchExchange(rank, world))
    m0 = run.mass()
    run.step(steps)
    m1 = run.mass()
    q.put((rank, y0, y1, run.own_rows().numpy(), m0, m1))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_match_single_domain(world):
    steps = 12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=600) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    from oracle import Oracle
    pb = _problem()
    ref = OracleSlab.__new__(OracleSlab)
    ref.o = Oracle(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field)
    ref.N = pb.params["nphase"]
    mref0 = ref.o.mass().numpy()
    ref.step(steps)
    for rank, y0, y1, rows, m0, m1 in out:
        want = ref.get_rows(y0, y1 - y0).numpy()
        # the same arithmetic node by node; torch may pick another summation
        # order for another array shape, so agreement is to round-off
        scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1)[:, None, None]
        err = np.abs(rows - want) / np.maximum(scale, 1e-300)
        assert err.max() <= 1e-13, (rank, err.max())
        assert np.allclose(m0, mref0, rtol=1e-14, atol=0)
        assert np.allclose(m1, ref.o.mass().numpy(), rtol=1e-14, atol=0)
    # the rows of the ranks tile the grid
    assert out[0][1] == 0 and out[-1][2] == pb.params["ny"]
    assert all(out[k][2] == out[k + 1][1] for k in range(world - 1))


def test_slab_rows_and_extension():
    from paper_2311_10314_gb300 import slab
    assert [slab.slab_rows(20, 3, r) for r in range(3)] == [(0, 7), (7, 14), (14, 20)]
    a = np.arange(5 * 4).reshape(5, 4)
    e = slab.extend_rows(a, 1, 3)
    assert e.shape == (2 + 2 * slab.HALO, 4)
    assert np.array_equal(e[:, 0], np.array([3, 4, 0, 1, 2, 3, 4, 0]) * 4)
