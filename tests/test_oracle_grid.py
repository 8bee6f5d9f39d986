"""Pins for the oracle's grid transfer operators (Section "Multilevel")."""
import numpy as np


def _grid(n):
    x = np.linspace(0.0, 1.0, n)
    return np.meshgrid(x, x, indexing="xy")  # X varies along columns, Y along rows


def test_embed_replicates_last_row_and_column(orc):
    f = np.arange(16, dtype=np.float32).reshape(4, 4)
    g = orc.embed(f)
    assert g.shape == (5, 5)
    assert np.array_equal(g[:4, :4], f)
    assert np.array_equal(g[4, :4], f[3])
    assert np.array_equal(g[:4, 4], f[:, 3])
    assert g[4, 4] == f[3, 3]


def test_restrict_preserves_constants(orc):
    for n in (3, 5, 9, 33):
        c = orc.restrict(np.full((n, n), 2.5))
        assert c.shape == ((n + 1) // 2,) * 2
        assert np.allclose(c, 2.5, rtol=0, atol=1e-15)


def test_restrict_stencil_and_mirror_boundary(orc):
    # A unit value at interior fine node (2,2) of a 5x5 grid is the centre of the
    # stencil 1/16 [1 2 1; 2 4 2; 1 2 1]: coarse (1,1) gets 4/16, nothing else.
    f = np.zeros((5, 5))
    f[2, 2] = 1.0
    assert np.allclose(orc.restrict(f), [[0, 0, 0], [0, 0.25, 0], [0, 0, 0]], atol=1e-16)
    # A unit value at fine node (1,1) is seen by coarse (0,0) four times through
    # the mirror (indices -1 -> 1) with weight 1/16 each, and once by (0,1),
    # (1,0), (1,1) with weight 1/16.
    f = np.zeros((5, 5))
    f[1, 1] = 1.0
    assert np.allclose(orc.restrict(f), [[4 / 16, 2 / 16, 0], [2 / 16, 1 / 16, 0], [0, 0, 0]], atol=1e-16)
    # Edge node (0,1): coarse (0,0) sees it at b=+1 and (mirrored) b=-1 with
    # weight 1/4*1/2 each -> 1/4; coarse (0,1) at b=-1 -> 1/8.
    f = np.zeros((5, 5))
    f[0, 1] = 1.0
    c = orc.restrict(f)
    assert np.isclose(c[0, 0], 0.25) and np.isclose(c[0, 1], 0.125) and np.isclose(c[1, 0], 0.0)


def test_restrict_is_quarter_transpose_of_prolongation_in_interior(orc):
    # Full weighting: away from the boundary, restriction = 1/4 P^T (P = bilinear
    # prolongation), checked column by column through brute force.
    nc, nf = 5, 9
    rng = np.random.default_rng(3)
    v = rng.normal(size=(nf, nf))
    r = orc.restrict(v)
    for I in range(1, nc - 1):
        for J in range(1, nc - 1):
            e = np.zeros((nc, nc))
            e[I, J] = 1.0
            P_col = orc.prolong(e)
            assert np.isclose(r[I, J], 0.25 * np.sum(P_col * v), rtol=0, atol=1e-13)


def test_restrict_reproduces_linear_functions_in_interior(orc):
    X, Y = _grid(17)
    f = 0.3 + 2.0 * X - 1.5 * Y
    c = orc.restrict(f)
    Xc, Yc = _grid(9)
    assert np.allclose(c[1:-1, 1:-1], (0.3 + 2.0 * Xc - 1.5 * Yc)[1:-1, 1:-1], atol=1e-13)


def test_prolong_copies_coarse_nodes_and_is_exact_for_bilinear(orc):
    rng = np.random.default_rng(1)
    c = rng.normal(size=(9, 9))
    f = orc.prolong(c)
    assert f.shape == (17, 17)
    assert np.array_equal(f[::2, ::2], c)
    X, Y = _grid(9)
    Xf, Yf = _grid(17)
    bil = lambda X, Y: 0.7 - 1.1 * X + 0.4 * Y + 2.3 * X * Y
    assert np.allclose(orc.prolong(bil(X, Y)), bil(Xf, Yf), atol=1e-14)
