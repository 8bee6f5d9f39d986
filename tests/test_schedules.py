"""Pins for the scan schedules (Chapters "Prefix sum" and "Distributed prefix
sum"): brute force with an exactly associative, non-commutative stand-in
operator, the paper's operation/step counts for 8 elements, and the closed
forms of the span/work table."""
import json
import math
import os

import numpy as np
import pytest

from oracle import schedules as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KINDS = [S.SERIAL, S.SKLANSKY, S.KOGGE_STONE, S.BRENT_KUNG, S.BLELLOCH]


def _mat(i):
    # distinct, non-commuting integer 2x2 matrices
    return (i, i + 1, ((1, i % 3 + 1), (i % 2, 1)))


def _op(a, b):
    # interval concatenation + matrix product: associative, not commutative
    assert a[1] == b[0], "operands are not adjacent"
    (p, q), (r, s) = a[2]
    (e, f), (g, h) = b[2]
    return (a[0], b[1], ((p * e + q * g, p * f + q * h), (r * e + s * g, r * f + s * h)))


def _fold(n):
    out, acc = [], None
    for i in range(n):
        acc = _mat(i) if acc is None else _op(acc, _mat(i))
        out.append(acc)
    return out


@pytest.mark.parametrize("kind", KINDS)
def test_schedule_equals_serial_fold(kind):
    for n in range(1, 65):
        lv = S.schedule(kind, n)
        data = [_mat(i) for i in range(n)] + [None] * S.aux_slots(kind, n)
        out = S.run(lv, data, _op)
        assert out[:n] == _fold(n), (S.NAMES[kind], n)


@pytest.mark.parametrize("kind", [S.CHUNKED, S.CHUNKED_ALT])
@pytest.mark.parametrize("gkind", KINDS)
def test_chunked_strategies_equal_serial_fold(kind, gkind):
    for n in list(range(1, 40)) + [64, 100]:
        for p in (1, 2, 3, 4, 7, 8, 16):
            lv = S.schedule(kind, n, p, gkind)
            data = [_mat(i) for i in range(n)] + [None] * S.aux_slots(kind, n, p, gkind)
            out = S.run(lv, data, _op)
            assert out[:n] == _fold(n), (S.NAMES[kind], S.NAMES[gkind], n, p)


def test_counts_for_eight_elements_match_paper():
    g = json.load(open(os.path.join(GOLDEN, "scan_counts_n8.json")))
    by_name = {S.NAMES[k]: k for k in KINDS}
    for name, c in g["counts"].items():
        ops, steps = S.counts(S.schedule(by_name[name], g["N"]))
        assert (ops, steps) == (c["ops"], c["steps"]), name


def test_span_and_work_closed_forms():
    """Table "Comparison of major strategies for parallel prefix sum"."""
    for k in range(1, 11):
        n = 1 << k
        lg = k
        assert S.counts(S.serial(n)) == (n - 1, n - 1)
        assert S.counts(S.blelloch(n)) == (2 * (n - 1), 2 * lg)
        assert S.counts(S.brent_kung(n)) == (2 * n - lg - 2, max(2 * lg - 1, 1))
        assert S.counts(S.kogge_stone(n)) == (n * lg - n + 1, lg)
        assert S.counts(S.sklansky(n)) == (n // 2 * lg, lg)


def test_snir_bound_for_inclusive_circuits():
    for n in range(2, 200):
        for kind in (S.SERIAL, S.SKLANSKY, S.KOGGE_STONE, S.BRENT_KUNG):
            ops, steps = S.counts(S.schedule(kind, n))
            assert ops + steps >= 2 * n - 2


def test_general_strategy_work():
    """Section "General strategy": W = 2N - P - N/P + W_GS for an exclusive global
    scan (Blelloch); an inclusive global scan saves the last combine of every
    chunk I >= 1 (Algorithm "general strategy with an inclusive scan")."""
    for n, p in [(64, 8), (128, 16), (400, 16), (96, 4)]:
        k = n // p
        ops, _ = S.counts(S.chunked(n, p, S.BLELLOCH))
        assert ops == 2 * n - p - k + 2 * (p - 1)
        ops, _ = S.counts(S.chunked(n, p, S.KOGGE_STONE))
        w_ks = sum(p - (1 << i) for i in range(math.ceil(math.log2(p))))
        assert ops == 2 * n - p - k - (p - 1) + w_ks


def test_level_synchronous_semantics_needed_for_kogge_stone():
    # Running Kogge-Stone in place (each op sees earlier writes of its level)
    # breaks the bracketing; the level-synchronous runner matches the fold.
    n = 8
    lv = S.kogge_stone(n)
    data = [_mat(i) for i in range(n)]
    inplace = list(data)
    with pytest.raises(AssertionError):
        for level in lv:
            for o in level:
                inplace[o[1]] = _op(inplace[o[2]], inplace[o[3]])
    assert S.run(lv, data, _op) == _fold(n)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_han_carlson_equals_serial_fold(k):
    for n in range(1, 65):
        lv = S.schedule(S.HAN_CARLSON, n, k)
        assert S.aux_slots(S.HAN_CARLSON, n, k) == 0
        out = S.run(lv, [_mat(i) for i in range(n)], _op)
        assert out == _fold(n), (k, n)


def test_han_carlson_span_and_work_closed_forms():
    """For N = 2^L and 1 <= k <= L: span L + k (Section "Other work"); work =
    up-sweep (N - M) + Kogge-Stone over M = N / 2^k block ends (M (L-k) - M + 1)
    + down-sweep (N - M - k), i.e. 2N - 3M - k + M (L - k) + 1.  At k = L this
    is Brent-Kung's 2N - log2 N - 2, and the op lists coincide."""
    for L in range(1, 9):
        n = 1 << L
        for k in range(1, L + 1):
            ops, steps = S.counts(S.han_carlson(n, k))
            m = n >> k
            assert steps == L + k - (1 if k == L else 0), (n, k, steps)
            assert ops == 2 * n - 3 * m - k + m * (L - k) + 1, (n, k, ops)
        assert S.han_carlson(n, L) == S.brent_kung(n)
    # between Kogge-Stone's work and span and Brent-Kung's
    for L in range(3, 9):
        n = 1 << L
        ks_ops, ks_steps = S.counts(S.kogge_stone(n))
        bk_ops, bk_steps = S.counts(S.brent_kung(n))
        hc_ops, hc_steps = S.counts(S.han_carlson(n, 1))
        assert bk_ops < hc_ops < ks_ops and ks_steps < hc_steps < bk_steps


@pytest.mark.parametrize("k", [0, 1, 2, 3, 5])
def test_ladner_fischer_equals_serial_fold(k):
    for n in range(1, 65):
        lv = S.schedule(S.LADNER_FISCHER, n, k)
        assert S.aux_slots(S.LADNER_FISCHER, n, k) == 0
        assert S.run(lv, [_mat(i) for i in range(n)], _op) == _fold(n), (k, n)


def test_ladner_fischer_span_and_work_closed_forms():
    """For N = 2^L and 0 <= k <= L: span L + k (one less at k = L, whose top
    down-sweep level is empty); work = up-sweep (N - M) + Sklansky over the
    M = N / 2^k block ends ((M/2) log2 M) + down-sweep (N - M - k).  k = 0 is
    Sklansky and k = L Brent-Kung, op list for op list."""
    for L in range(1, 9):
        n = 1 << L
        for k in range(0, L + 1):
            ops, steps = S.counts(S.ladner_fischer(n, k))
            m = n >> k
            assert steps == L + k - (1 if k == L else 0), (n, k, steps)
            assert ops == 2 * n - 2 * m - k + (m // 2) * (L - k), (n, k, ops)
        assert S.ladner_fischer(n, 0) == S.sklansky(n)
        assert S.ladner_fischer(n, L) == S.brent_kung(n)
