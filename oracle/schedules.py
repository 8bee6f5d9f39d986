"""Scan schedules of the oracle (test infrastructure only).

Each schedule turns N data slots holding x_0..x_{N-1} into the inclusive
prefix sums data[e] = x_0 (.) ... (.) x_e (Definition "Prefix sum"), for an
operator (.) that is only approximately associative, so the bracketing matters
and is part of the result.

A schedule is a list of levels.  All ops of a level read the values held
before the level and write afterwards (level-synchronous semantics; this is
the double buffering the paper prescribes for Kogge-Stone).  Op forms:
    ("op", dst, a, b)   data[dst] = data[a] (.) data[b]
    ("copy", dst, src)  data[dst] = data[src]
    ("id", dst)         data[dst] = identity I
Slots >= N are auxiliary (identity padding, chunk totals, a saved reduction).

Written from the algorithms of Chapter "Prefix sum" and Chapter "Distributed
prefix sum"; readings of garbled loop bounds are noted per function.
"""
from __future__ import annotations

SERIAL, SKLANSKY, KOGGE_STONE, BRENT_KUNG, BLELLOCH, CHUNKED, CHUNKED_ALT, HAN_CARLSON, LADNER_FISCHER = range(9)
NAMES = {SERIAL: "serial", SKLANSKY: "sklansky", KOGGE_STONE: "kogge_stone",
         BRENT_KUNG: "brent_kung", BLELLOCH: "blelloch", CHUNKED: "chunked",
         CHUNKED_ALT: "chunked_alt", HAN_CARLSON: "han_carlson", LADNER_FISCHER: "ladner_fischer"}


def _clog2(n: int) -> int:
    k = 0
    while (1 << k) < n:
        k += 1
    return k


def serial(n, base=0):
    """Algorithm "serial prefix sum": data[i] = data[i-1] (.) data[i], i = 1..N-1."""
    return [[("op", base + i, base + i - 1, base + i)] for i in range(1, n)]


def kogge_stone(n, base=0):
    """Algorithm "Kogge-Stone": in step i every j >= 2^i combines with j - 2^i
    (reading: the garbled lower bound is 2^i), double-buffered."""
    levels = []
    for i in range(_clog2(n)):
        s = 1 << i
        levels.append([("op", base + j, base + j - s, base + j) for j in range(s, n)])
    return levels


def sklansky(n, base=0):
    """Algorithm "Sklansky": in step i the source j = 2^i - 1 + m 2^{i+1} feeds the
    next 2^i slots (reading: inner loop k = 0 .. 2^i - 1).  Slots >= N dropped."""
    levels = []
    for i in range(_clog2(n)):
        s = 1 << i
        lv = []
        for j in range(s - 1, n, 2 * s):
            for k in range(s):
                if j + k + 1 < n:
                    lv.append(("op", base + j + k + 1, base + j, base + j + k + 1))
        levels.append(lv)
    return levels


def _upsweep(n, base):
    levels = []
    for i in range(_clog2(n)):
        s = 1 << i
        lv = [("op", base + j, base + j - s, base + j) for j in range(2 * s - 1, n, 2 * s)]
        if lv:
            levels.append(lv)
    return levels


def brent_kung(n, base=0):
    """Algorithm "Brent-Kung": Blelloch's up-sweep (reading: j = 2^{i+1}-1 step
    2^{i+1}, data[j] = data[j-2^i] (.) data[j]), then the breadth-first down-sweep
    data[j+2^i-1] = data[j-1] (.) data[j+2^i-1], j = 2^{i+1}, 2*2^{i+1}, ...
    Ops touching slots >= N are dropped."""
    levels = _upsweep(n, base)
    for i in range(_clog2(n) - 2, -1, -1):
        s = 1 << i
        lv = []
        j = 2 * s
        while j + s - 1 < n:
            lv.append(("op", base + j + s - 1, base + j - 1, base + j + s - 1))
            j += 2 * s
        if lv:
            levels.append(lv)
    return levels


def blelloch_exclusive(n, base, aux):
    """Algorithm "Blelloch": up-sweep, root <- identity, down-sweep in which the
    left child receives the parent's value and the right child becomes
    parent (.) left (reading: the prefix goes on the left of the operator, as a
    non-commutative operator needs).  N is padded to a power of two with
    identity elements in slots aux .. aux+P-N-1.  The root's reduction is saved
    into slot aux+P-N before it is replaced by the identity.
    Returns (levels, slot_of(e) for the exclusive result at e = 0..P-1, total_slot)."""
    p = 1 << _clog2(n)
    slot = [base + e if e < n else aux + (e - n) for e in range(p)]
    total = aux + (p - n)
    levels = []
    if p > n:
        levels.append([("id", slot[e]) for e in range(n, p)])
    for i in range(_clog2(p)):
        s = 1 << i
        lv = [("op", slot[j], slot[j - s], slot[j]) for j in range(2 * s - 1, p, 2 * s)]
        levels.append(lv)
    levels.append([("copy", total, slot[p - 1]), ("id", slot[p - 1])])
    for i in range(_clog2(p) - 1, -1, -1):
        s = 1 << i
        lv = []
        for j in range(0, p, 2 * s):
            left, right = slot[j + s - 1], slot[j + 2 * s - 1]
            lv.append(("copy", left, right))
            lv.append(("op", right, right, left))
        levels.append(lv)
    return levels, slot, total


def blelloch(n, base=0, aux=None):
    """Inclusive result from Blelloch's exclusive scan: y_e = excl_{e+1} for
    e < N-1 and y_{N-1} = the saved reduction (the 'receive from the successor'
    form of Section "Blelloch scan")."""
    if aux is None:
        aux = base + n
    levels, slot, total = blelloch_exclusive(n, base, aux)
    shift = [("copy", base + e, slot[e + 1]) for e in range(n - 1)]
    shift.append(("copy", base + n - 1, total))
    levels.append(shift)
    return levels


def han_carlson(n, k=1, base=0):
    """Han-Carlson hybrid of Brent-Kung and Kogge-Stone (Section "Other work";
    span log2 N + k).  Blocks of B = 2^k elements: the tree's first k levels
    leave each block's reduction in its last element; Kogge-Stone over those
    last elements of the complete blocks turns them into prefixes; the tree's
    down-sweep, levels k-1 .. 0, then gives every other element its prefix
    (those of an incomplete last block included).  k is clamped to [1, log2 N]."""
    L = _clog2(n)
    k = max(1, min(k, L))
    levels = []
    for i in range(k):
        st = 1 << i
        levels.append([("op", base + j, base + j - st, base + j) for j in range(2 * st - 1, n, 2 * st)])
    B = 1 << k
    ends = [base + (t + 1) * B - 1 for t in range(n // B)]
    for i in range(_clog2(len(ends))):
        st = 1 << i
        levels.append([("op", ends[t], ends[t - st], ends[t]) for t in range(st, len(ends))])
    for i in reversed(range(k)):
        st = 1 << i
        levels.append([("op", base + j + st - 1, base + j - 1, base + j + st - 1)
                       for j in range(2 * st, n - st + 1, 2 * st)])
    return [lv for lv in levels if lv]


def ladner_fischer(n, k=0, base=0):
    """Ladner-Fischer(k), Sklansky and Brent-Kung combined (Section "Other
    work"): as Han-Carlson, with Sklansky's tree instead of Kogge-Stone over
    the last elements of the complete blocks of 2^k elements; span
    log2 N + k; k = 0 is Sklansky.  k is clamped to [0, log2 N]."""
    L = _clog2(n)
    k = max(0, min(k, L))
    B = 1 << k
    up = [[("op", base + j, base + j - (1 << i), base + j) for j in range((2 << i) - 1, n, 2 << i)]
          for i in range(k)]
    ends = [base + (t + 1) * B - 1 for t in range(n // B)]
    middle = []
    for i in range(_clog2(len(ends))):
        st = 1 << i
        lv = []
        for src in range(st - 1, len(ends), 2 * st):
            lv += [("op", ends[t], ends[src], ends[t]) for t in range(src + 1, min(src + st, len(ends) - 1) + 1)]
        middle.append(lv)
    down = [[("op", base + j + (1 << i) - 1, base + j - 1, base + j + (1 << i) - 1)
             for j in range(2 << i, n - (1 << i) + 1, 2 << i)] for i in reversed(range(k))]
    return [lv for lv in up + middle + down if lv]


def aux_slots(kind, n, chunks=0, global_kind=KOGGE_STONE):
    """Number of auxiliary slots a schedule uses beyond the N data slots."""
    if kind == BLELLOCH:
        return (1 << _clog2(n)) - n + 1
    if kind in (CHUNKED, CHUNKED_ALT):
        p = max(1, min(chunks, n))
        extra = aux_slots(global_kind, p) if global_kind != BLELLOCH else (1 << _clog2(p)) - p + 1
        return p + extra
    return 0


def _chunks(n, p):
    """Chunk I gets K = floor(N/P)+1 elements for I < N mod P, else floor(N/P)
    (Section "General strategy")."""
    k, rem = divmod(n, p)
    bounds, l = [], 0
    for i in range(p):
        sz = k + (1 if i < rem else 0)
        bounds.append((l, l + sz - 1))
        l += sz
    return bounds


def _global(kind, p, gbase, gaux):
    if kind == SERIAL:
        return serial(p, gbase)
    if kind == SKLANSKY:
        return sklansky(p, gbase)
    if kind == KOGGE_STONE:
        return kogge_stone(p, gbase)
    if kind == BRENT_KUNG:
        return brent_kung(p, gbase)
    raise ValueError(kind)


def chunked(n, chunks, global_kind=KOGGE_STONE, base=0):
    """General strategy (Algorithm "Distributed parallel prefix sum"): local
    serial scans of P chunks, a global scan of the chunk totals, then every
    element of chunk I >= 1 is combined with the exclusive global value.  With
    an inclusive global algorithm the exclusive value of chunk I is the
    inclusive value of chunk I-1 and the last element of chunk I takes the
    inclusive value directly (Algorithm "general strategy with an inclusive
    scan"); with Blelloch the exclusive value is used as is."""
    p = max(1, min(chunks, n))
    bounds = _chunks(n, p)
    gbase = base + n
    gaux = gbase + p
    levels = []
    kmax = max(r - l + 1 for l, r in bounds)
    for t in range(1, kmax):
        levels.append([("op", base + l + t, base + l + t - 1, base + l + t)
                       for l, r in bounds if l + t <= r])
    if p == 1:
        return levels
    levels.append([("copy", gbase + i, base + r) for i, (l, r) in enumerate(bounds)])
    stage2 = []
    if global_kind == BLELLOCH:
        glev, gslot, _tot = blelloch_exclusive(p, gbase, gaux)
        levels += glev
        for i in range(1, p):
            l, r = bounds[i]
            for e in range(l, r + 1):
                stage2.append(("op", base + e, gslot[i], base + e))
    else:
        levels += _global(global_kind, p, gbase, gaux)
        for i in range(1, p):
            l, r = bounds[i]
            for e in range(l, r):
                stage2.append(("op", base + e, gbase + i - 1, base + e))
            stage2.append(("copy", base + r, gbase + i))
    levels.append(stage2)
    return levels


def chunked_alt(n, chunks, global_kind=KOGGE_STONE, base=0):
    """Alternative strategy (Algorithm "alternative distributed parallel prefix
    sum", reduce-then-scan): each chunk only reduces its elements into a total,
    the totals are scanned (exclusive), then each chunk combines the exclusive
    value with its first element and rescans serially."""
    p = max(1, min(chunks, n))
    bounds = _chunks(n, p)
    gbase = base + n
    gaux = gbase + p
    if p == 1:
        return serial(n, base)
    levels = [[("copy", gbase + i, base + l) for i, (l, r) in enumerate(bounds)]]
    kmax = max(r - l + 1 for l, r in bounds)
    for t in range(1, kmax):
        levels.append([("op", gbase + i, gbase + i, base + l + t)
                       for i, (l, r) in enumerate(bounds) if l + t <= r])
    if global_kind == BLELLOCH:
        glev, gslot, _tot = blelloch_exclusive(p, gbase, gaux)
        levels += glev
        excl = [gslot[i] for i in range(p)]
    else:
        levels += _global(global_kind, p, gbase, gaux)
        excl = [None] + [gbase + i - 1 for i in range(1, p)]
    levels.append([("op", base + bounds[i][0], excl[i], base + bounds[i][0]) for i in range(1, p)])
    for t in range(1, kmax):
        levels.append([("op", base + l + t, base + l + t - 1, base + l + t)
                       for l, r in bounds if l + t <= r])
    return levels


def schedule(kind, n, chunks=0, global_kind=KOGGE_STONE, base=0):
    if n <= 1:
        return []
    if kind == SERIAL:
        return serial(n, base)
    if kind == SKLANSKY:
        return sklansky(n, base)
    if kind == KOGGE_STONE:
        return kogge_stone(n, base)
    if kind == BRENT_KUNG:
        return brent_kung(n, base)
    if kind == BLELLOCH:
        return blelloch(n, base, base + n)
    if kind == CHUNKED:
        return chunked(n, chunks, global_kind, base)
    if kind == CHUNKED_ALT:
        return chunked_alt(n, chunks, global_kind, base)
    if kind == HAN_CARLSON:
        return han_carlson(n, chunks if chunks else 1, base)
    if kind == LADNER_FISCHER:
        return ladner_fischer(n, chunks, base)
    raise ValueError(kind)


def counts(levels):
    """(operator applications, steps) where a step is a level holding at least
    one operator application, as in the paper's figures."""
    ops = sum(1 for lv in levels for o in lv if o[0] == "op")
    steps = sum(1 for lv in levels if any(o[0] == "op" for o in lv))
    return ops, steps


def run(levels, data, op, identity=None):
    """Execute a schedule on a list of values with operator ``op``; the identity
    is represented by ``identity`` (default None) and short-circuits."""
    data = list(data)
    for lv in levels:
        new = {}
        for o in lv:
            if o[0] == "op":
                a, b = data[o[2]], data[o[3]]
                if a is identity:
                    new[o[1]] = b
                elif b is identity:
                    new[o[1]] = a
                else:
                    new[o[1]] = op(a, b)
            elif o[0] == "copy":
                new[o[1]] = data[o[2]]
            else:
                new[o[1]] = identity
        for k, v in new.items():
            data[k] = v
    return data
