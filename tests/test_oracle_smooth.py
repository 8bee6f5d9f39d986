"""Pins for the oracle's H1-type smoother (Section "Gradient flow": the
direction is -A^{-1} E'[phi], A selected to smooth; here A = M_s (x) M_s with
the 1D H1 Gram matrix M_s = M1 + (s^2/2) K1, s a number of grid spacings)."""
import numpy as np
import pytest


def _fe_1d(n):
    """1D P1 mass and stiffness matrices on [0, 1] with n nodes, written out."""
    h = 1.0 / (n - 1)
    M = np.zeros((n, n))
    K = np.zeros((n, n))
    for e in range(n - 1):  # element [x_e, x_e+1]
        M[e:e + 2, e:e + 2] += h / 6.0 * np.array([[2, 1], [1, 2]])
        K[e:e + 2, e:e + 2] += 1.0 / h * np.array([[1, -1], [-1, 1]])
    return M, K


@pytest.mark.parametrize("smooth", [0.0, 0.7, 3.0])
def test_smoother_is_the_inverse_of_the_kronecker_gram_matrix(orc, smooth):
    """Brute force on a 9 x 9 grid: the dense Kronecker matrix assembled here
    element by element, solved by numpy, against orc_smooth_apply."""
    n = 9
    h = 1.0 / (n - 1)
    M, K = _fe_1d(n)
    s = smooth * h
    Ms = M + 0.5 * s * s * K
    A = np.kron(Ms, Ms)  # index r * n + c: rows couple through the first factor
    rng = np.random.default_rng(2)
    g = rng.normal(size=(2, n, n))
    d = orc.smooth_apply(g, smooth)
    for ch in range(2):
        want = -np.linalg.solve(A, g[ch].ravel()).reshape(n, n)
        assert np.allclose(d[ch], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert np.allclose(orc.smooth_matvec(g[0], smooth), (A @ g[0].ravel()).reshape(n, n), atol=1e-13)


def test_smoother_without_width_is_the_consistent_mass(orc):
    rng = np.random.default_rng(3)
    v = rng.normal(size=(17, 17))
    assert np.allclose(orc.smooth_matvec(v, 0.0), orc.mass_apply(v), atol=1e-15)


def test_smoother_round_trip_on_a_larger_grid(orc):
    n = 65
    rng = np.random.default_rng(4)
    g = rng.normal(size=(2, n, n))
    d = orc.smooth_apply(g, 2.5)
    for ch in range(2):
        back = -orc.smooth_matvec(d[ch], 2.5)
        assert np.abs(back - g[ch]).max() <= 1e-11 * np.abs(g[ch]).max()


def test_smoother_spreads_an_impulse(orc):
    """A point gradient becomes a positive, symmetric bump that decays away
    from the point and widens with the smoother's width."""
    n = 33
    g = np.zeros((2, n, n))
    g[0, 16, 16] = -1.0
    w = []
    for sm in (1.0, 4.0):
        d = orc.smooth_apply(g, sm)[0]
        assert np.allclose(d, d.T) and np.allclose(d, d[::-1, ::-1])
        prof = d[16, 16:]
        assert prof[0] > 0 and np.all(np.diff(prof[:6]) < 0)
        w.append(np.sum(d > 0.1 * d.max()))
    assert w[1] > w[0]


@pytest.mark.slow
def test_smoothed_flow_recovers_a_translation(orc, syn):
    t = np.array([1.3, -0.7])
    side = 128
    f = syn.series(1, 2, side, noise=False, drift=[[0, 0], t], dist_amp=0, sigma=5.0, spacing=20.0)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    p = orc.params(n_levels=3, iter_max=1000, lam=10.0, epsilon=1e-12, smooth=2.0)
    u, status, st = orc.register(R, T, p)
    m = 16
    err = np.abs(u * side + t[:, None, None])[:, m:-m, m:-m]
    assert err.max() < 0.01, err.max()
