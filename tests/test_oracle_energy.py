"""Pins for the oracle's warp, NCC energy and gradient (Section "Image
registration for electron microscopy" and Section "Spatial discretization")."""
import json
import os

import numpy as np
import pytest

from _quad import dirichlet, integrate, integrate_product

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _smooth(n, seed, k=4):
    """Random smooth nodal field: a few low-frequency cosines."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.zeros((n, n))
    for _ in range(k):
        a, b = rng.uniform(0.5, 3.0, size=2)
        f += rng.normal() * np.cos(2 * np.pi * (a * X + b * Y) + rng.uniform(0, 6.28))
    return f + 3.0


def test_interp_nodes_bilinear_and_clamp(orc):
    n = 9
    h = 1.0 / (n - 1)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    bil = lambda x0, x1: 0.5 + 1.7 * x0 - 0.8 * x1 + 1.2 * x0 * x1
    T = bil(X, Y)
    rng = np.random.default_rng(0)
    for _ in range(50):
        x0, x1 = rng.uniform(0, 1, size=2)
        v, d0, d1 = orc.interp(T, x0, x1)
        assert np.isclose(v, bil(x0, x1), atol=1e-14)
        assert np.isclose(d0, 1.7 + 1.2 * x1, atol=1e-12)
        assert np.isclose(d1, -0.8 + 1.2 * x0, atol=1e-12)
    v, d0, d1 = orc.interp(T, 3 * h, 5 * h)
    assert np.isclose(v, T[5, 3])
    # outside Omega: the point is clamped and the clamped derivative vanishes
    v, d0, d1 = orc.interp(T, 1.3, 0.4)
    assert np.isclose(v, bil(1.0, 0.4)) and d0 == 0.0 and np.isclose(d1, -0.8 + 1.2)
    v, d0, d1 = orc.interp(T, 0.2, -0.1)
    assert np.isclose(v, bil(0.2, 0.0)) and d1 == 0.0 and np.isclose(d0, 1.7)


def test_warp_by_whole_nodes_is_a_shift(orc):
    n = 17
    h = 1.0 / (n - 1)
    T = _smooth(n, 1)
    u = np.zeros((2, n, n))
    u[0] = 2 * h   # x_0 + 2 nodes
    u[1] = -1 * h  # x_1 - 1 node
    Th, _ = orc.warp(T, u)
    assert np.allclose(Th[1:, :-2], T[:-1, 2:], atol=1e-13)


def test_rectangle_example_direction_convention(orc):
    """Paper's worked example: f1(phi_01(x)) = f0(x) with phi_01(x) = x + G."""
    g = json.load(open(os.path.join(GOLDEN, "rectangle_example.json")))
    n = 65
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")

    def rect(c0, c1):
        w0, w1 = g["rect_size"]
        return ((X >= c0) & (X <= c0 + w0) & (Y >= c1) & (Y <= c1 + w1)).astype(float)

    f0, f1 = rect(*g["corner_f0"]), rect(*g["corner_f1"])
    u = np.zeros((2, n, n))
    u[0], u[1] = g["G"]
    Th, _ = orc.warp(f1, u)
    inside = X + g["G"][0] <= 1.0
    assert np.array_equal(Th[inside], f0[inside])
    # the opposite sign does not register the pair
    Th2, _ = orc.warp(f1, -u)
    assert not np.array_equal(Th2[inside], f0[inside])


def test_ncc_bounds_and_perfect_match(orc):
    n = 33
    R = _smooth(n, 2)
    z = np.zeros((2, n, n))
    E, p = orc.energy(R, R, z, 1.0)
    assert np.isclose(p["ncc"], 1.0, rtol=0, atol=1e-14) and E == -p["ncc"]
    E, p = orc.energy(R, 2.5 * R + 7.0, z, 1.0)
    assert np.isclose(p["ncc"], 1.0, atol=1e-14)
    E, p = orc.energy(R, -0.5 * R + 1.0, z, 1.0)
    assert np.isclose(p["ncc"], -1.0, atol=1e-14)
    rng = np.random.default_rng(3)
    for s in range(5):
        T = rng.normal(size=(n, n))
        u = rng.normal(size=(2, n, n)) * 0.02
        E, p = orc.energy(R, T, u, 0.0)
        assert -1.0 <= p["ncc"] <= 1.0


def test_ncc_mean_sigma_equal_quadrature(orc):
    """Mean, sigma and NCC of the FE interpolants by independent quadrature."""
    n = 17
    R, T = _smooth(n, 4), _smooth(n, 5) + 0.3 * _smooth(n, 4)
    E, p = orc.energy(R, T, np.zeros((2, n, n)), 0.0)
    Rb, Tb = integrate(R), integrate(T)
    sR, sT = np.sqrt(integrate_product(R - Rb, R - Rb)), np.sqrt(integrate_product(T - Tb, T - Tb))
    ncc = integrate_product(R - Rb, T - Tb) / (sR * sT)
    assert np.isclose(p["Rbar"], Rb, rtol=1e-12) and np.isclose(p["Tbar"], Tb, rtol=1e-12)
    assert np.isclose(p["sigR"], sR, rtol=1e-12) and np.isclose(p["sigT"], sT, rtol=1e-12)
    assert np.isclose(p["ncc"], ncc, rtol=1e-12)
    assert np.isclose(E, -ncc, rtol=1e-12)


def test_regulariser_is_dirichlet_energy(orc):
    n = 17
    R = _smooth(n, 6)
    rng = np.random.default_rng(7)
    u = rng.normal(size=(2, n, n)) * 0.01
    lam = 3.0
    E, p = orc.energy(R, R, u, lam)
    assert np.isclose(p["reg"], 0.5 * lam * (dirichlet(u[0]) + dirichlet(u[1])), rtol=1e-12)
    # a translation costs nothing
    u[:] = 0.0
    u[0], u[1] = 0.013, -0.021
    E, p = orc.energy(R, R, u, lam)
    assert abs(p["reg"]) < 1e-14


def _generic_u(n, seed, scale=0.35):
    """Displacement whose sample points stay clear of cell lines and of the
    clamp, so that E is differentiable in every component."""
    h = 1.0 / (n - 1)
    rng = np.random.default_rng(seed)
    u = rng.uniform(-scale, scale, size=(2, n, n)) * h
    x = np.arange(n) * h
    pos = np.stack([x[None, :] + u[0], x[:, None] + u[1]])
    frac = pos / h - np.floor(pos / h)
    bad = (frac < 0.05) | (frac > 0.95)
    u[bad] += 0.1 * h
    return u


def test_gradient_matches_central_differences(orc):
    n = 17
    h = 1.0 / (n - 1)
    R, T = _smooth(n, 8), _smooth(n, 9)
    u = _generic_u(n, 10)
    lam = 2.0
    g = orc.gradient(R, T, u, lam)
    eps = 1e-6 * h
    fd = np.empty_like(u)
    for idx in np.ndindex(u.shape):
        up, um = u.copy(), u.copy()
        up[idx] += eps
        um[idx] -= eps
        fd[idx] = (orc.energy(R, T, up, lam)[0] - orc.energy(R, T, um, lam)[0]) / (2 * eps)
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(g))


def test_gradient_vanishes_for_identical_frames(orc):
    n = 33
    R = _smooth(n, 11)
    g = orc.gradient(R, R, np.zeros((2, n, n)), 5.0)
    assert np.max(np.abs(g)) < 1e-15


def test_gradient_regulariser_part(orc):
    # with T = R at u = translation by whole nodes the data term is stationary in
    # the interior; the regulariser gradient is lambda K u (zero for constants)
    n = 17
    rng = np.random.default_rng(12)
    R = _smooth(n, 12)
    u = rng.normal(size=(2, n, n)) * 0.01
    g1 = orc.gradient(R, R, u, 1.0)
    g0 = orc.gradient(R, R, u, 0.0)
    assert np.allclose(g1 - g0, np.stack([orc.stiff_apply(u[0]), orc.stiff_apply(u[1])]), atol=1e-13)
