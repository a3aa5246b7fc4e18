"""The replica (N > 1) host logic of bench.py on CPU: two gloo ranks set up
from the torchrun environment, agree on the max-over-ranks time, pass the
barrier, and only rank 0 of the reference arm prints a line (2D imbibition
and 3D sphere workloads)."""
import io
import json
import os
import socket
import sys
import contextlib

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q, workload="imbibition"):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    t = bench.allreduce_max(1.5 + r, w)
    bench.barrier(w)
    buf = io.StringIO()

    class Args:
        size = 512 if workload == "imbibition" else 40
        steps = 1
        gpus = w
    Args.workload = workload
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args, w, r)
    dist.destroy_process_group()
    q.put((r, w, t, buf.getvalue()))


@pytest.mark.parametrize("workload", ["imbibition", "sphere3d"])
def test_two_gloo_ranks(workload):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, workload)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [2, 2]
    assert [o[2] for o in out] == [2.5, 2.5]
    assert out[1][3] == ""
    line = json.loads(out[0][3].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
