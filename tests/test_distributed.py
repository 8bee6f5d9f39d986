"""The general strategy of the distributed prefix sum (chapter "Distributed
prefix sum", Section "General strategy") as host logic, on CPU ranks (gloo):
an exactly associative but non-commutative stand-in operator (interval
concatenation and an integer 2 x 2 matrix product) must give every rank the
serial fold's prefixes, for several rank counts and uneven or empty chunks.
The same chunk driver that runs the registration operator on GPUs
(SeriesChunk) runs here against a stand-in handle.  Not measured on more
than one GPU."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _elems(n, seed=0):
    rng = np.random.default_rng(seed)
    return [(k, k + 1, rng.integers(-2, 3, size=(2, 2))) for k in range(n)]


def _combine(a, b):
    assert a[1] == b[0], "chain mismatch"
    return (a[0], b[1], a[2] @ b[2])


def _worker(rank, world, port, n, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1712_02533_gb300 import distributed as D
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elems = _elems(n)
        a, b = D.chunk_bounds(n, world, rank)

        def send(obj, dst):
            t = torch.tensor([-1] * 6 if obj is None else [obj[0], obj[1], *obj[2].ravel().tolist()], dtype=torch.int64)
            dist.send(t, dst)

        def recv(src):
            t = torch.empty(6, dtype=torch.int64)
            dist.recv(t, src)
            v = t.tolist()
            return None if v[0] < 0 else (v[0], v[1], np.array(v[2:]).reshape(2, 2))

        got = D.distributed_scan(elems[a:b], rank, world, _combine, send, recv)
        want = D.serial_fold(elems, _combine)[a:b]
        ok = len(got) == len(want) and all(g[0] == w[0] and g[1] == w[1] and np.array_equal(g[2], w[2])
                                           for g, w in zip(got, want))
        # the chunk driver of the registration path, on a stand-in handle
        fake = _FakeSeries(elems, n)
        ch = D.SeriesChunk(fake, rank, world, kind=1, device="cpu")
        ch.run(D.local_ops_scan_fn(fake, 1))
        ok2 = all(fake.meta[e][:2] == (0, e + 1) and np.array_equal(fake.val[e], want[e - a][2]) for e in range(a, b))
        q.put((rank, ok, ok2, fake.batches))
    finally:
        dist.destroy_process_group()


class _FakeSeries:
    """Stand-in handle: slots hold (start, end) and an integer matrix encoded
    in the first four values of a field; function B multiplies matrices."""

    sides = [4]

    def __init__(self, elems, n):
        self.counts = [n + 1]
        self.elems = elems
        self.meta, self.val = {}, {}
        self.batches = 0

    def n_slots(self, series=0):
        return self.counts[0] - 1 + 3

    def apply_operator_batch(self, ops):
        self.batches += 1
        res = []
        for (_, left, right, dst, i, k) in ops:
            if left < 0:
                assert k == i + 1
                res.append((dst, (i, k), self.elems[i][2]))
            else:
                (a0, a1), (b0, b1) = self.meta[left], self.meta[right]
                assert a1 == b0 and a0 == i and b1 == k, "chain mismatch"
                res.append((dst, (i, k), self.val[left] @ self.val[right]))
        for dst, se, v in res:  # level-synchronous: all operands read first
            self.meta[dst], self.val[dst] = se, v

    def get_slot_device(self, slot, series=0):
        import torch
        f = torch.zeros((2, 5, 5), dtype=torch.float32)
        f.view(-1)[:4] = torch.tensor(self.val[slot].ravel(), dtype=torch.float32)
        return f

    def set_slot_device(self, slot, field, start, end, series=0):
        self.meta[slot] = (start, end)
        self.val[slot] = np.rint(field.reshape(-1)[:4].numpy()).astype(np.int64).reshape(2, 2)

    def copy_slot(self, src, dst, start, end, series=0):
        self.meta[dst], self.val[dst] = (start, end), self.val[src].copy()

    def schedule_ops(self, kind, n, chunks=1):
        from oracle import schedules as S
        return S.schedule(kind, n, chunks), 0


@pytest.mark.parametrize("world,n", [(2, 9), (4, 13), (4, 3), (3, 16)])
def test_general_strategy_equals_serial_fold_on_cpu_ranks(world, n):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
    assert all(ok for _, ok, _, _ in res), res
    assert all(ok2 for _, _, ok2, _ in res), res


def test_chunk_bounds_cover_the_series():
    from paper_1712_02533_gb300 import distributed as D
    for n in (1, 7, 399):
        for w in (1, 2, 3, 8):
            b = [D.chunk_bounds(n, w, r) for r in range(w)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(w - 1))
            sizes = [y - x for x, y in b]
            assert max(sizes) - min(sizes) <= 1


def test_global_stage_rounds_and_messages():
    """Kogge-Stone over P ranks: ceil(log2 P) rounds, every rank sends at most
    one partial per round (counted with an in-process transport)."""
    from paper_1712_02533_gb300 import distributed as D
    for world in (1, 2, 5, 8):
        totals = [(r, r + 1, np.array([[1, r], [0, 1]])) for r in range(world)]
        mail = {}
        sent = [0] * world
        # run the ranks round by round in lockstep: a rank's sends of round k
        # are delivered before its neighbours' receives of round k
        import threading
        out = [None] * world
        cv = threading.Condition()

        def send(r):
            def f(obj, dst):
                with cv:
                    mail.setdefault((r, dst), []).append(obj)
                    sent[r] += 1
                    cv.notify_all()
            return f

        def recv(r):
            def f(src):
                with cv:
                    cv.wait_for(lambda: mail.get((src, r)))
                    return mail[(src, r)].pop(0)
            return f

        ts = [threading.Thread(target=lambda r=r: out.__setitem__(r, D.global_exclusive_scan(
            totals[r], r, world, _combine, send(r), recv(r)))) for r in range(world)]
        for t in ts:
            t.start()
        for t in ts:
            t.join(timeout=30)
        rounds = int(np.ceil(np.log2(world))) if world > 1 else 0
        assert max(sent) <= rounds
        fold = D.serial_fold(totals, _combine)
        assert out[0] is None
        for r in range(1, world):
            assert out[r][:2] == (0, r) and np.array_equal(out[r][2], fold[r - 1][2])
