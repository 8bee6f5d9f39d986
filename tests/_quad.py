"""Independent numerical integration of bilinear finite-element functions.

2x2 Gauss-Legendre quadrature per cell, which is exact for products of two
bilinear functions and for squared gradients of one.  Used to pin the
oracle's matrix-based mass/stiffness operators to the integrals they stand for.
"""
import numpy as np

_G = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])


def _corners(v):
    return v[:-1, :-1], v[:-1, 1:], v[1:, :-1], v[1:, 1:]  # (r,c) (r,c+1) (r+1,c) (r+1,c+1)


def _eval(v, s, t):
    """value and gradient (Omega units) of the bilinear interpolant at local
    coordinates s (along columns) and t (along rows) in every cell."""
    n = v.shape[0]
    h = 1.0 / (n - 1)
    a, b, c, d = _corners(v)
    val = (1 - t) * ((1 - s) * a + s * b) + t * ((1 - s) * c + s * d)
    dx = ((1 - t) * (b - a) + t * (d - c)) / h
    dy = ((1 - s) * (c - a) + s * (d - b)) / h
    return val, dx, dy


def integrate_product(v, w):
    n = v.shape[0]
    h = 1.0 / (n - 1)
    tot = 0.0
    for s in _G:
        for t in _G:
            tot += np.sum(_eval(v, s, t)[0] * _eval(w, s, t)[0]) * h * h / 4.0
    return tot


def integrate(v):
    return integrate_product(v, np.ones_like(v))


def dirichlet(v):
    n = v.shape[0]
    h = 1.0 / (n - 1)
    tot = 0.0
    for s in _G:
        for t in _G:
            _, dx, dy = _eval(v, s, t)
            tot += np.sum(dx * dx + dy * dy) * h * h / 4.0
    return tot
