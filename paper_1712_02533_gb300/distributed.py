"""The general strategy of the distributed prefix sum across GPUs (chapter
"Distributed prefix sum", Section "General strategy", Algorithm "Distributed
parallel prefix sum").

One series is cut into P contiguous chunks of elements x_1..x_N (x_k =
phi_{k-1,k}), one chunk per rank (one GPU each):

1. local stage 1: every rank scans its own chunk (any of the library's
   schedules, one batched launch per level) -- its last element is the chunk
   total T_r;
2. global stage: an exclusive scan of the totals over the ranks by
   Kogge-Stone, ceil(log2 P) rounds; in round k rank r sends its partial
   S_r = T_{r-2^{k+1}+1} (.) ... (.) T_r to rank r + 2^k and combines what it
   receives from rank r - 2^k on the left (one displacement field per round
   and direction, received into local memory first);
3. local stage 2: every rank r > 0 combines its exclusive prefix
   E_r = T_0 (.) ... (.) T_{r-1} on the left of each of its scanned elements.

The operator (.) is function B; its left operand of the form phi_{0,j} needs
frame f_0 and a combination of partials phi_{a,b} (.) phi_{b,c} needs frames
f_a and f_c, so every rank holds the frames of the whole series (the paper's
workers read every image from shared storage) and registers only its chunk.

This module is host logic only: the combinations run in libreg's kernels
(reg_apply_operator_batch) and the exchange is torch.distributed send/recv
(NCCL on GPUs, gloo in the CPU tests).  ``global_exclusive_scan`` and
``chunk_bounds`` are independent of the element type, so the tests drive them
with an exactly associative stand-in operator.
"""
from __future__ import annotations

import numpy as np


def chunk_bounds(n_elems: int, world: int, rank: int):
    """Elements [a, b) of rank `rank`: contiguous chunks whose sizes differ by
    at most one, the larger ones first."""
    q, r = divmod(n_elems, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def global_exclusive_scan(total, rank: int, world: int, combine, send, recv):
    """Exclusive scan of the ranks' totals by Kogge-Stone over the ranks.

    total: this rank's chunk total (None for an empty chunk: the identity).
    combine(a, b) -> a (.) b (a on the left, the earlier elements).
    send(obj, dst), recv(src) -> obj: point-to-point transport; None travels
    as the identity.  Returns E_rank = T_0 (.) ... (.) T_{rank-1} (None on
    rank 0).  Rounds: ceil(log2 world); in each every rank sends at most one
    object and receives at most one."""
    part = total      # S_r: the inclusive partial of this rank
    excl = None       # E_r: the exclusive partial
    d = 1
    while d < world:
        # send before receive on even-odd ordered pairs would also work; the
        # transports used here (NCCL, gloo) buffer or pair the calls
        if rank + d < world:
            send(part, rank + d)
        if rank - d >= 0:
            left = recv(rank - d)
            if left is not None:
                excl = left if excl is None else combine(left, excl)
                part = left if part is None else combine(left, part)
        d *= 2
    return excl


def serial_fold(elems, combine):
    """Inclusive prefixes of elems by the serial fold (the reference order)."""
    out, acc = [], None
    for x in elems:
        acc = x if acc is None else combine(acc, x)
        out.append(acc)
    return out


def distributed_scan(local_elems, rank: int, world: int, combine, send, recv, local_scan=serial_fold):
    """The general strategy on one rank: local stage 1 (local_scan of this
    rank's chunk), the global exclusive scan of the totals, local stage 2.
    Returns this rank's inclusive prefixes."""
    y = local_scan(local_elems, combine) if local_elems else []
    total = y[-1] if y else None
    excl = global_exclusive_scan(total, rank, world, combine, send, recv)
    if excl is None:
        return y
    return [combine(excl, v) for v in y]


# ---------------------------------------------------------------------------
# The registration operator across ranks (one GPU per rank)
# ---------------------------------------------------------------------------
class SeriesChunk:
    """One rank's share of a series registration by the general strategy.

    series: a ``Series`` handle holding all frames of the series (every rank
    uploads them); this rank registers the elements [a, b) of
    chunk_bounds(n_frames - 1, world, rank).  Slots: data slot e holds x_{e+1}
    = phi_{e,e+1} and, after the scan, phi_{0,e+1} for e in [a, b); two
    auxiliary slots receive the neighbour's partial and hold this rank's
    partial and exclusive prefix.  Fields travel as CUDA tensors
    (2 x (side+1) x (side+1) float32, pixels) with torch.distributed."""

    def __init__(self, series, rank, world, kind=1, chunks=1, series_index=0, device="cuda"):
        self.s = series
        self.device = device  # where the exchanged fields live ("cpu" with gloo in the tests)
        self.rank, self.world = rank, world
        self.kind, self.chunks = kind, chunks
        self.k = series_index
        self.side = series.sides[series_index]
        self.n = series.counts[series_index] - 1
        self.a, self.b = chunk_bounds(self.n, world, rank)
        nslots = series.n_slots(series_index)
        if nslots < self.n + 3:
            raise ValueError("series needs three auxiliary slots")
        self.s_part, self.s_excl, self.s_recv = self.n, self.n + 1, self.n + 2

    # elements are (start, end, slot) with the field resident in that slot
    def _combine_into(self, left, right, dst):
        """dst <- left (.) right = B(left, right) on this rank's GPU."""
        (i, j, sa), (j2, k, sb) = left, right
        assert j == j2, "chain mismatch"
        self.s.apply_operator_batch([(self.k, sa, sb, dst, i, k)])
        return (i, k, dst)

    def _send(self, obj, dst):
        import torch
        import torch.distributed as dist
        hdr = torch.tensor([-1, -1] if obj is None else [obj[0], obj[1]], dtype=torch.int64, device=self.device)
        dist.send(hdr, dst)
        if obj is not None:
            f = self.s.get_slot_device(obj[2], series=self.k)
            dist.send(f, dst)

    def _recv(self, src):
        import torch
        import torch.distributed as dist
        hdr = torch.empty(2, dtype=torch.int64, device=self.device)
        dist.recv(hdr, src)
        i, j = (int(v) for v in hdr.tolist())
        if i < 0:
            return None
        f = torch.empty((2, self.side + 1, self.side + 1), dtype=torch.float32, device=self.device)
        dist.recv(f, src)
        self.s.set_slot_device(self.s_recv, f, i, j, series=self.k)
        return (i, j, self.s_recv)

    def run(self, local_ops_scan):
        """Stage 1 with the handle's batched operators (local_ops_scan(a, b)
        registers the chunk's neighbour pairs and scans them in place, leaving
        phi_{a,e+1} in slot e), then the global Kogge-Stone stage and stage 2.
        Leaves phi_{0,e+1} in slot e for e in [a, b)."""
        a, b = self.a, self.b
        if b > a:
            local_ops_scan(a, b)
            total = (a, b, b - 1)
        else:
            total = None
        # global stage: partial and exclusive prefix kept in their own slots
        state = {"part": total, "excl": None}

        def combine(left, right):
            # a received partial combines on the left of this rank's partial or
            # exclusive prefix; the result goes to the slot that one occupies
            dst = self.s_excl if right is state["excl"] else self.s_part
            return self._combine_into(left, right, dst)

        d = 1
        while d < self.world:
            if self.rank + d < self.world:
                self._send(state["part"], self.rank + d)
            if self.rank - d >= 0:
                left = self._recv(self.rank - d)
                if left is not None:
                    if state["excl"] is None:
                        self.s.copy_slot(left[2], self.s_excl, left[0], left[1], series=self.k)
                        state["excl"] = (left[0], left[1], self.s_excl)
                    else:
                        state["excl"] = combine(left, state["excl"])
                    if state["part"] is None:
                        self.s.copy_slot(left[2], self.s_part, left[0], left[1], series=self.k)
                        state["part"] = (left[0], left[1], self.s_part)
                    else:
                        state["part"] = combine(left, state["part"])
            d *= 2
        excl = state["excl"]
        if excl is not None and b > a:
            # stage 2: every local prefix gets the exclusive prefix on its left,
            # all in one batch
            ops = [(self.k, self.s_excl, e, e, 0, e + 1) for e in range(a, b)]
            self.s.apply_operator_batch(ops)
        return a, b


def local_ops_scan_fn(series, kind, chunks=1, series_index=0):
    """Stage 1 of the general strategy on one rank: all neighbour pairs of the
    chunk [a, b) in one batch (function A), then the chunk's inclusive scan
    with the library's schedule over its elements, each level one batch."""
    def run(a, b):
        k = series_index
        series.apply_operator_batch([(k, -1, -1, e, e, e + 1) for e in range(a, b)])
        levels, _aux = series.schedule_ops(kind, b - a, chunks)
        meta = {e: (e, e + 1) for e in range(a, b)}
        for lev in levels:
            batch = []
            writes = {}
            for o in lev:
                if o[0] != "op":
                    raise ValueError("stage 1 takes the schedules without copies or identities")
                _, dst, x, y = o
                (i, j), (j2, kk) = meta[a + x], meta[a + y]
                batch.append((k, a + x, a + y, a + dst, i, kk))
                writes[a + dst] = (i, kk)
            if batch:
                series.apply_operator_batch(batch)
            meta.update(writes)
        for e in range(a, b):
            assert meta[e] == (a, e + 1), "stage 1 did not produce the chunk's prefixes"
    return run


def flatten_check(elems):
    """Tests: the (start, end) chain of a list of elements."""
    return np.array([(x[0], x[1]) for x in elems])
