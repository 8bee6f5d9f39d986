"""The oracle's series driver: preprocessing with A, then the scan of B
(Definition "Image series registration", Section "Prefix sum for
registration problem").  On a tiny series its output must equal the fold
evaluated by hand in the same bracketing, bit for bit."""
import numpy as np
import pytest

from oracle import schedules as S


@pytest.fixture(scope="module")
def tiny(orc, syn):
    fr = syn.series(11, 5, 32, noise=True, peak=20.0, spacing=8.0, sigma=2.0)
    p = orc.params(n_levels=2, iter_max=8, lam=10.0)
    g = [orc.embed(f) for f in fr]
    A = [orc.register(g[e], g[e + 1], p)[0] for e in range(4)]
    return fr, g, p, A


def _B(orc, g, p, i, j, k, uij, ujk):
    out, st, it, tr, en = orc.apply_batch([dict(R=g[i], T=g[k], left=uij, right=ujk)], p)
    return out[0]


def test_serial_scan_equals_left_fold(orc, tiny):
    fr, g, p, A = tiny
    res = orc.register_series([fr], p, kind=S.SERIAL)[0]
    acc = A[0]
    assert np.array_equal(res[1], acc * 32)
    for k in range(2, 5):
        acc = _B(orc, g, p, 0, k - 1, k, acc, A[k - 1])
        assert np.array_equal(res[k], acc * 32)


def test_kogge_stone_scan_equals_its_bracketing(orc, tiny):
    fr, g, p, A = tiny
    res = orc.register_series([fr], p, kind=S.KOGGE_STONE)[0]
    x01 = _B(orc, g, p, 0, 1, 2, A[0], A[1])
    x12 = _B(orc, g, p, 1, 2, 3, A[1], A[2])
    x23 = _B(orc, g, p, 2, 3, 4, A[2], A[3])
    y3 = _B(orc, g, p, 0, 1, 3, A[0], x12)   # step 2: (x0) (x1 x2)
    y4 = _B(orc, g, p, 0, 2, 4, x01, x23)    # step 2: (x0 x1)(x2 x3)
    assert np.array_equal(res[1], A[0] * 32)
    assert np.array_equal(res[2], x01 * 32)
    assert np.array_equal(res[3], y3 * 32)
    assert np.array_equal(res[4], y4 * 32)


def test_segmented_scan_is_per_series(orc, tiny, syn):
    fr, g, p, A = tiny
    other = syn.series(12, 3, 32, noise=True)
    both = orc.register_series([fr, other], p, kind=S.SKLANSKY)
    alone = orc.register_series([fr], p, kind=S.SKLANSKY)[0]
    assert np.array_equal(both[0], alone)
    assert np.array_equal(both[1], orc.register_series([other], p, kind=S.SKLANSKY)[0])
