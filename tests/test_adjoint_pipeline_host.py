"""Host logic of the pipelined reverse sweep (``CheckpointedRun``), with the
library replaced by a recorder: no GPU.  The device-side ordering is the
library's (a fork and join on the handle's stream, GPU-tested for
bit-identical gradients); what is checked here is the sequence of calls the
sweep makes: segment k is reversed from the buffer set k % 2 while segment
k - 1 is recomputed into the other set from its checkpoint (copied into the
set's first buffer just before the call), the first call only recomputes,
the last only reverses, the adjoint buffers swap after odd segments, and a
refusal of the first call sends every segment through the one-by-one path.
"""
import pytest

from paper_2311_10314_gb300 import _lib
from paper_2311_10314_gb300 import adjoint as A


class _Sim:
    h = 7
    stream = None
    N = 2


class _Tensor:
    def __init__(self, p):
        self.p = p

    def data_ptr(self):
        return self.p


class _Buf:
    def __init__(self, K, seg, log):
        self.ckpt = [1000 + k for k in range(K)]
        self.seg = [2000 + i for i in range(seg)]
        self.seg2 = [3000 + i for i in range(seg)]
        self.adj = [10, 11]
        self.scratch, self.ab = 12, 1 << 20
        self.dJ_dcos, self.dJ_dpsi = _Tensor(13), _Tensor(14)
        self.sub = []
        self.log = log

    def copy_state(self, dst, src, stream):
        self.log.append(("copy", dst, src))


def _run(T, ckpt, log):
    r = A.CheckpointedRun.__new__(A.CheckpointedRun)
    r.T, r.ckpt = T, ckpt
    r.starts = list(range(0, T, ckpt))
    r.sim = _Sim()
    r.buf = _Buf(len(r.starts), ckpt, log)
    r._cur, r._nxt = r.buf.adj
    return r


@pytest.mark.parametrize("T,ckpt", [(400, 50), (230, 60), (50, 50), (61, 60)])
def test_pipelined_call_sequence(monkeypatch, T, ckpt):
    log = []
    calls = []

    def seg_pipe(h, states, nxt, cur, other, scratch, ab, dc, dp):
        assert not set(nxt[1:]) & set(states)
        calls.append((list(states), list(nxt), cur, other))
        log.append(("call", len(calls) - 1))
        return _lib.DDCC_OK, len(states) % 2 == 1

    monkeypatch.setattr(A._lib, "ddcc_adjoint_segment_pipelined", seg_pipe)
    r = _run(T, ckpt, log)
    r._reverse_pipelined()
    K = len(r.starts)
    lens = [min(ckpt, T - t0) for t0 in r.starts]
    sets = (r.buf.seg, r.buf.seg2)
    assert len(calls) == K + 1
    cur, other = 10, 11
    for i, (states, nxt, c, o) in enumerate(calls):
        k = K - i
        assert states == (sets[k % 2][: lens[k]] if k < K else [])
        assert nxt == (sets[(k - 1) % 2][: lens[k - 1]] if k >= 1 else [])
        assert (c, o) == (cur, other)
        if len(states) % 2:
            cur, other = other, cur
        if k >= 1:
            # the head of segment k - 1 is copied into its set right before the call
            j = log.index(("call", i))
            assert log[j - 1] == ("copy", sets[(k - 1) % 2][0], r.buf.ckpt[k - 1])
    assert (r._cur, r._nxt) == (cur, other)


def test_refused_first_call_reverses_segment_by_segment(monkeypatch):
    done = []
    monkeypatch.setattr(A._lib, "ddcc_adjoint_segment_pipelined",
                        lambda *a: (_lib.DDCC_ERR_UNSUPPORTED, False))
    r = _run(230, 60, [])
    monkeypatch.setattr(r, "_reverse_segment", lambda head, n: done.append((head, n)))
    r._reverse_pipelined()
    assert done == [(r.buf.ckpt[k], min(60, 230 - 60 * k)) for k in (3, 2, 1, 0)]
