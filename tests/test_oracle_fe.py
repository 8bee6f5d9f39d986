"""Pins for the oracle's FE operators (Section "Spatial discretization"):
the mass matrix and the Dirichlet stiffness must equal the integrals of the
bilinear interpolants they discretise."""
import numpy as np

from _quad import dirichlet, integrate, integrate_product


def test_lumped_weights_closed_form(orc):
    for n in (3, 9, 65):
        h = 1.0 / (n - 1)
        w = orc.lumped(n)
        expect = np.full((n, n), h * h)
        expect[0, :] *= 0.5
        expect[-1, :] *= 0.5
        expect[:, 0] *= 0.5
        expect[:, -1] *= 0.5
        assert np.allclose(w, expect, rtol=1e-14, atol=0)
        assert np.isclose(w.sum(), 1.0, rtol=1e-14)


def test_mass_matrix_equals_quadrature(orc):
    rng = np.random.default_rng(0)
    for n in (2, 3, 9, 17):
        v, w = rng.normal(size=(n, n)), rng.normal(size=(n, n))
        assert np.isclose(np.sum(w * orc.mass_apply(v)), integrate_product(v, w), rtol=1e-12, atol=1e-14)
        assert np.isclose(np.sum(v * orc.mass_apply(w)), np.sum(w * orc.mass_apply(v)), rtol=1e-13)
        assert np.isclose(np.sum(orc.mass_apply(np.ones((n, n)))), 1.0, rtol=1e-14)


def test_mass_interior_stencil(orc):
    n = 9
    h = 1.0 / (n - 1)
    e = np.zeros((n, n))
    e[4, 4] = 1.0
    m = orc.mass_apply(e)[3:6, 3:6] / (h * h)
    assert np.allclose(m, np.array([[1, 4, 1], [4, 16, 4], [1, 4, 1]]) / 36.0, atol=1e-14)


def test_stiffness_equals_dirichlet_quadrature(orc):
    rng = np.random.default_rng(1)
    for n in (2, 3, 9, 17):
        v = rng.normal(size=(n, n))
        assert np.isclose(np.sum(v * orc.stiff_apply(v)), dirichlet(v), rtol=1e-12)
    # bilinear function a + bx + cy + dxy: int |grad|^2 = b^2 + c^2 + (bd + cd) + d^2 * 2/3
    n = 33
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    b, c, d = 0.7, -1.3, 0.9
    v = 0.2 + b * X + c * Y + d * X * Y
    closed = b * b + c * c + b * d + c * d + 2.0 * d * d / 3.0
    assert np.isclose(np.sum(v * orc.stiff_apply(v)), closed, rtol=1e-12)


def test_stiffness_kernel_symmetry_and_stencil(orc):
    n = 9
    assert np.allclose(orc.stiff_apply(np.ones((n, n))), 0.0, atol=1e-12)
    e = np.zeros((n, n))
    e[4, 4] = 1.0
    k = orc.stiff_apply(e)[3:6, 3:6]
    assert np.allclose(k, np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]]) / 3.0, atol=1e-13)
    rng = np.random.default_rng(2)
    v, w = rng.normal(size=(n, n)), rng.normal(size=(n, n))
    assert np.isclose(np.sum(w * orc.stiff_apply(v)), np.sum(v * orc.stiff_apply(w)), rtol=1e-12)
    assert np.sum(v * orc.stiff_apply(v)) > 0


def test_mean_and_integral(orc):
    rng = np.random.default_rng(3)
    v = rng.normal(size=(17, 17))
    assert np.isclose(np.sum(orc.lumped(17) * v), integrate(v), rtol=1e-12)
