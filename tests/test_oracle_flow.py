"""Pins for the oracle's gradient flow, function A / B and composition
(Sections "Gradient flow", "Summary" (Algorithm "Multilevel gradient flow")
and "Registration for series of images")."""
import numpy as np
import pytest


def _smooth(n, seed, k=4):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.zeros((n, n))
    for _ in range(k):
        a, b = rng.uniform(0.5, 3.0, size=2)
        f += rng.normal() * np.cos(2 * np.pi * (a * X + b * Y) + rng.uniform(0, 6.28))
    return f


def test_identical_frames_give_exactly_zero_displacement(orc, syn):
    f = syn.series(5, 1, 64, noise=True)[0]
    R = orc.embed(f)
    p = orc.params(n_levels=3, iter_max=20, lam=10.0)
    u, status, st = orc.register(R, R, p)
    # exactly zero in exact arithmetic (NCC = 1, g = 0); in double precision
    # NCC rounds a few ulp below 1 and leaves a gradient at rounding level
    assert np.max(np.abs(u)) * 64 < 1e-6
    assert all(abs(s.E + 1.0) < 1e-14 for s in st)


def test_level_solve_decreases_energy_monotonically(orc, syn):
    f = syn.series(2, 2, 32, noise=True, drift=[[0, 0], [0.6, -0.4]], dist_amp=0)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    n = R.shape[0]
    p = orc.params(n_levels=1, iter_max=1, lam=10.0)
    u = np.zeros((2, n, n))
    E_prev = orc.energy(R, T, u, 10.0)[0]
    for k in range(15):
        u, st = orc.solve_level(R, T, u, p)
        E = orc.energy(R, T, u, 10.0)[0]
        assert np.isclose(st.E, E, rtol=0, atol=1e-14)
        assert E <= E_prev
        E_prev = E


def test_armijo_condition_holds_for_accepted_step(orc, syn):
    f = syn.series(2, 2, 32, noise=True, drift=[[0, 0], [0.6, -0.4]], dist_amp=0)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    n = R.shape[0]
    lam = 10.0
    u0 = np.zeros((2, n, n))
    p = orc.params(n_levels=1, iter_max=1, lam=lam, tau_init=1.0)
    u1, st = orc.solve_level(R, T, u0, p)
    g = orc.gradient(R, T, u0, lam)
    w = orc.lumped(n)
    d = -g / w
    tau = st.tau
    assert np.allclose(u1, u0 + tau * d, rtol=0, atol=1e-18)
    E0, E1 = orc.energy(R, T, u0, lam)[0], orc.energy(R, T, u1, lam)[0]
    slope = np.sum(g * d)
    assert E1 - E0 <= 0.5 * tau * slope
    # the step came from halving 1.0; twice the step fails the test (widening
    # is not tried after a reduction, so 2 tau was the last rejected trial)
    assert np.log2(tau) == np.round(np.log2(tau))
    E2 = orc.energy(R, T, u0 + 2 * tau * d, lam)[0]
    assert not (E2 - E0 <= 0.5 * 2 * tau * slope)


def test_widening_doubles_step_while_accepted(orc, syn):
    f = syn.series(2, 2, 32, noise=True, drift=[[0, 0], [0.6, -0.4]], dist_amp=0)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    n = R.shape[0]
    lam = 10.0
    u0 = np.zeros((2, n, n))
    g = orc.gradient(R, T, u0, lam)
    d = -g / orc.lumped(n)
    slope = np.sum(g * d)
    tau0 = 2.0 ** -30  # tiny: accepted, then widened
    p = orc.params(n_levels=1, iter_max=1, lam=lam, tau_init=tau0)
    u1, st = orc.solve_level(R, T, u0, p)
    tau = st.tau
    assert tau > tau0
    E0 = orc.energy(R, T, u0, lam)[0]
    for t in [tau0 * 2 ** k for k in range(int(np.log2(tau / tau0)) + 1)]:
        assert orc.energy(R, T, u0 + t * d, lam)[0] - E0 <= 0.5 * t * slope
    assert not (orc.energy(R, T, u0 + 2 * tau * d, lam)[0] - E0 <= 0.5 * 2 * tau * slope)
    assert st.trials == int(np.log2(tau / tau0)) + 2


@pytest.mark.slow
def test_translation_recovery_below_one_hundredth_pixel(orc, syn):
    """A noise-free pair related by a known translation t: f_1(y) shows the
    specimen at y + t, so phi_01(x) = x - t; recovered to < 0.01 px inside."""
    t = np.array([1.3, -0.7])
    side = 128
    f = syn.series(1, 2, side, noise=False, drift=[[0, 0], t], dist_amp=0, sigma=5.0, spacing=20.0)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    p = orc.params(n_levels=3, iter_max=3000, lam=10.0, epsilon=1e-10)
    u, status, st = orc.register(R, T, p)
    upx = u * side
    m = 16
    err = np.abs(upx[:, m:-m, m:-m] + t[:, None, None])
    assert err.max() < 0.01


def test_compose_translations_and_identity(orc):
    n = 33
    h = 1.0 / (n - 1)
    a = np.zeros((2, n, n))
    a[0], a[1] = 1.5 * h, -0.25 * h
    b = np.zeros((2, n, n))
    b[0], b[1] = -0.5 * h, 2.0 * h
    c = orc.compose(a, b)
    # where x + a stays inside Omega the composition of translations adds them
    inside = np.ones((n, n), bool)
    inside[:, -2:] = False
    inside[:1, :] = False
    assert np.allclose(c[0][inside], 1.0 * h) and np.allclose(c[1][inside], 1.75 * h)
    rng = np.random.default_rng(0)
    u = rng.normal(size=(2, n, n)) * 0.3 * h
    z = np.zeros_like(u)
    assert np.allclose(orc.compose(z, u), u, atol=1e-16)
    assert np.allclose(orc.compose(u, z), u, atol=1e-16)


def test_compose_matches_pointwise_definition(orc):
    n = 17
    h = 1.0 / (n - 1)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    # u_jk bilinear in x -> its interpolant is exact anywhere inside Omega
    ujk = np.stack([0.01 + 0.02 * X - 0.03 * Y + 0.01 * X * Y, -0.02 + 0.01 * X + 0.02 * X * Y])
    uij = np.stack([0.05 * np.sin(3 * Y) * X * (1 - X), 0.04 * np.cos(2 * X) * Y * (1 - Y)])
    c = orc.compose(uij, ujk)
    P0, P1 = X + uij[0], Y + uij[1]
    expect = uij + np.stack([0.01 + 0.02 * P0 - 0.03 * P1 + 0.01 * P0 * P1,
                             -0.02 + 0.01 * P0 + 0.02 * P0 * P1])
    assert np.allclose(c, expect, atol=1e-15)


def test_function_b_is_a_with_composed_initial_guess(orc, syn):
    fr = syn.series(4, 3, 32, noise=True)
    g = [orc.embed(f) for f in fr]
    p = orc.params(n_levels=2, iter_max=10, lam=10.0)
    u01, _, _ = orc.register(g[0], g[1], p)
    u12, _, _ = orc.register(g[1], g[2], p)
    outs, st, it, tr, en = orc.apply_batch([dict(R=g[0], T=g[2], left=u01, right=u12)], p)
    direct, s, _ = orc.register(g[0], g[2], p, u_init=orc.compose(u01, u12))
    assert np.array_equal(outs[0], direct)


def test_exact_start_stays_put_on_the_finest_level(orc, syn):
    """Started from the exact solution of a noise-free translated pair (a
    constant field: the regulariser vanishes and the data term is stationary
    there up to boundary effects), function A on the finest level alone -- the
    learned form that skips every coarse level -- moves it by < 0.01 px
    inside.  (Coarse levels have their own, slightly different optimum, which
    is why a start that keeps them is not expected to stay put.)"""
    t = np.array([1.3, -0.7])
    side = 128
    f = syn.series(1, 2, side, noise=False, drift=[[0, 0], t], dist_amp=0, sigma=5.0, spacing=20.0)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    u0 = np.empty((2, side + 1, side + 1))
    u0[0], u0[1] = -t[0] / side, -t[1] / side
    p = orc.params(n_levels=1, iter_max=200, lam=10.0, epsilon=1e-10)
    u, status, st = orc.register(R, T, p, u_init=u0)
    assert len(st) == 1
    m = 16
    err = np.abs(u * side + t[:, None, None])[:, m:-m, m:-m]
    assert err.max() < 0.01, err.max()


def _field(n, seed):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return np.stack([0.02 * np.sin(2 * np.pi * (X + 0.3 * Y) + rng.uniform(0, 6)) + 0.004 * rng.normal(size=(n, n)),
                     0.03 * np.cos(2 * np.pi * (0.7 * X - Y) + rng.uniform(0, 6)) + 0.004 * rng.normal(size=(n, n))])


@pytest.mark.parametrize("n_levels", [2, 3, 4])
def test_multilevel_start_is_restricted_then_prolongated(orc, syn, n_levels):
    """Function A with a non-identity start on several levels (Algorithm
    "Multilevel gradient flow"): the start is restricted level by level down to
    m0 (in Omega units, not rescaled), and the result of each level is
    prolongated to the next.  With no gradient steps (iter_max 0) the result is
    therefore prolong^k(restrict^k(u0)), k = n_levels - 1, built here from the
    separately pinned grid-transfer operators.  A start dropped on the coarse
    levels, or rescaled between levels (pixels instead of Omega units), fails."""
    side = 64
    fr = syn.series(8, 2, side, noise=True)
    R, T = orc.embed(fr[0]), orc.embed(fr[1])
    u0 = _field(side + 1, n_levels)
    p = orc.params(n_levels=n_levels, iter_max=0, lam=10.0)
    u, status, st = orc.register(R, T, p, u_init=u0)
    assert [s.iters for s in st] == [0] * n_levels
    want = []
    for ch in range(2):
        v = u0[ch]
        for _ in range(n_levels - 1):
            v = orc.restrict(v)
        for _ in range(n_levels - 1):
            v = orc.prolong(v)
        want.append(v)
    assert np.array_equal(u, np.stack(want))


@pytest.mark.parametrize("n_levels", [2, 3, 4])
def test_multilevel_start_keeps_an_affine_field(orc, syn, n_levels):
    """Closed form: the full-weighting restriction reproduces an affine field
    a + B x at every coarse node whose stencil stays inside the grid, and
    bilinear prolongation is exact on it, so with iter_max 0 function A
    returns an affine start unchanged except within one coarsest cell of the
    border (where the mirrored restriction stencil bends it)."""
    side = 64
    n = side + 1
    fr = syn.series(8, 2, side, noise=True)
    R, T = orc.embed(fr[0]), orc.embed(fr[1])
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    u0 = np.stack([0.013 + 0.021 * X - 0.017 * Y, -0.008 + 0.011 * X + 0.019 * Y])
    p = orc.params(n_levels=n_levels, iter_max=0, lam=10.0)
    u, _, _ = orc.register(R, T, p, u_init=u0)
    m = 2 ** (n_levels - 1)  # fine nodes in one coarsest cell
    inner = (slice(None), slice(m, n - m), slice(m, n - m))
    assert np.max(np.abs(u[inner] - u0[inner])) < 1e-15
    if n_levels > 1:
        assert np.max(np.abs(u - u0)) > 1e-6  # the border really is bent


def test_multilevel_start_at_exact_translation_keeps_it(orc, syn):
    """A noise-free translated pair started from the exact translation on three
    levels: the coarse levels see the restricted start (the same constant in
    Omega units) and the result stays within 0.01 px of the translation inside."""
    t = np.array([1.3, -0.7])
    side = 128
    f = syn.series(1, 2, side, noise=False, drift=[[0, 0], t], dist_amp=0, sigma=5.0, spacing=20.0)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    u0 = np.empty((2, side + 1, side + 1))
    u0[0], u0[1] = -t[0] / side, -t[1] / side
    p = orc.params(n_levels=3, iter_max=500, lam=10.0, epsilon=1e-12)
    u, status, st = orc.register(R, T, p, u_init=u0)
    m = 16
    err = np.abs(u * side + t[:, None, None])[:, m:-m, m:-m]
    assert err.max() < 0.01, err.max()


@pytest.mark.slow
def test_smooth_displacement_recovery(orc, syn):
    """A noise-free pair related by the generator's drift plus its smooth
    sinusoidal distortion (1 px amplitude): the registered field follows the
    exact deformation (solved by the generator per pixel) far more closely than
    the identity does.  Measured with lambda = 1, 3 levels, run to convergence:
    mean error 0.016 px and max 0.047 px inside a 16 px margin.  The < 0.01 px
    of a pure translation is not reached for a spatially varying displacement
    at any lambda tried (0.01 to 10): the discrete optimum of the point-sampled
    bilinear energy lies a few hundredths of a pixel from the continuous one
    (the sweep is recorded with the design notes).  A dropped term, a wrong sign
    or swapped components in the energy or gradient leave errors of the order
    of the displacement itself."""
    side = 128
    f, gt, _ = syn.series(3, 2, side, noise=False, drift=[[0, 0], [0.8, -0.5]], dist_amp=1.0, sigma=5.0,
                          spacing=20.0, ground_truth=True)
    R, T = orc.embed(f[0]), orc.embed(f[1])
    p = orc.params(n_levels=3, iter_max=3000, lam=1.0, epsilon=1e-12)
    u, status, st = orc.register(R, T, p)
    m = 16
    err = np.abs((u * side)[:, :side, :side] - gt[1])[:, m:-m, m:-m]
    ident = np.abs(gt[1])[:, m:-m, m:-m]
    assert err.mean() < 0.025 and err.max() < 0.08, (err.mean(), err.max())
    assert err.mean() < 0.05 * ident.mean()
