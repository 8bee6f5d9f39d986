"""Pins for the oracle's rigid variant (Definition "Rigid transformation":
phi(x) = R(alpha) x + t; Section "Gradient flow": no smoother for the rigid
case; Algorithm "Multilevel gradient flow": the three parameters are not
restricted or prolongated)."""
import numpy as np
import pytest


def _rot(a):
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])


def test_rigid_field_is_the_rotation_plus_translation(orc):
    n = 9
    th = np.array([0.3, 0.05, -0.02])
    u = orc.rigid_field(th, n)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    P = np.einsum("ij,jrc->irc", _rot(th[0]), np.stack([X, Y])) + th[1:, None, None]
    assert np.allclose(u, P - np.stack([X, Y]), atol=1e-15)
    assert np.allclose(orc.rigid_field([0.0, 0.1, 0.2], n), np.stack([np.full((n, n), 0.1), np.full((n, n), 0.2)]))


def test_regulariser_of_a_rigid_map_is_closed_form(orc, syn):
    """lambda/2 int |D(phi - id)|^2 = lambda/2 |R(alpha) - I|_F^2 = 2 lambda (1 - cos alpha)
    on Omega = [0,1]^2; the discrete stiffness form is exact on linear fields."""
    fr = syn.series(2, 2, 32)
    R, T = orc.embed(fr[0]), orc.embed(fr[1])
    for a in (0.0, 0.1, -0.4):
        u = orc.rigid_field([a, 0.03, -0.01], 33)
        _, parts = orc.energy(R, T, u, 7.0)
        assert abs(parts["reg"] - 2 * 7.0 * (1 - np.cos(a))) < 1e-12


def test_rigid_gradient_matches_finite_differences(orc, syn):
    fr = syn.series(3, 2, 64, peak=20.0, spacing=10.0, sigma=2.5)
    R, T = orc.embed(fr[0]), orc.embed(fr[1])
    lam = 10.0
    th = np.array([0.013, 0.011, -0.007])
    g = orc.rigid_gradient(R, T, th, lam)
    h = 1e-7
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (orc.rigid_energy(R, T, th + e, lam) - orc.rigid_energy(R, T, th - e, lam)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * np.abs(g).max(), (j, fd, g[j])


def _analytic(side, pts):
    """A smooth test image: Gaussian blobs (sigma 4 px) at pts, sampled at
    pixel positions (c, r) by the given map of pixel coordinates."""
    def img(X, Y):
        v = np.zeros_like(X)
        for (a, b, w) in pts:
            v += w * np.exp(-((X - a) ** 2 + (Y - b) ** 2) / (2 * 4.0 ** 2))
        return v
    return img


@pytest.mark.slow
def test_rigid_registration_recovers_rotation_and_translation(orc):
    """Frames sampled from one smooth image I: f_0(y) = I(y), f_1(y) =
    I(phi^-1(y)) with phi(x) = R(alpha) x + t (pixels, rotation about the
    origin), so that f_1 o phi = f_0; the rigid flow recovers alpha and t."""
    side = 128
    rng = np.random.default_rng(4)
    pts = [(rng.uniform(-20, side + 20), rng.uniform(-20, side + 20), rng.uniform(0.5, 1.5)) for _ in range(160)]
    img = _analytic(side, pts)
    alpha, t = 0.02, np.array([2.3, -1.7])
    c = np.arange(side, dtype=np.float64)
    Xc, Yc = np.meshgrid(c, c, indexing="xy")
    f0 = img(Xc, Yc)
    Q = np.einsum("ij,jrc->irc", _rot(-alpha), np.stack([Xc - t[0], Yc - t[1]]))
    f1 = img(Q[0], Q[1])
    R, T = orc.embed(f0.astype(np.float32)), orc.embed(f1.astype(np.float32))
    # lambda = 0: for a rigid map the regulariser is 2 lambda (1 - cos alpha)
    # (pinned above), a bias towards alpha = 0 that is not part of the data
    p = orc.params(n_levels=3, iter_max=2000, lam=0.0, epsilon=1e-13)
    th, status, st = orc.rigid_register(R, T, p)
    assert abs(th[0] - alpha) < 2e-4, th
    assert np.abs(th[1:] * side - t).max() < 0.02, th[1:] * side


def test_rigid_composition_matches_field_composition(orc):
    """phi_b o phi_a of the parameters equals the composition of the two
    displacement fields (orc_compose, bilinear, exact on linear fields) where
    phi_a(x) stays inside Omega."""
    n = 33
    a, b = np.array([0.05, 0.02, 0.03]), np.array([-0.02, 0.01, -0.015])
    c = orc.rigid_compose(a, b)
    want = orc.rigid_field(c, n)
    got = orc.compose(orc.rigid_field(a, n), orc.rigid_field(b, n))
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ua = orc.rigid_field(a, n)
    inside = (X + ua[0] >= 0) & (X + ua[0] <= 1) & (Y + ua[1] >= 0) & (Y + ua[1] <= 1)
    assert inside.sum() > n * n // 2
    assert np.abs((got - want)[:, inside]).max() < 1e-14
    assert np.allclose(orc.rigid_compose(a, np.zeros(3)), a) and np.allclose(orc.rigid_compose(np.zeros(3), b), b)
