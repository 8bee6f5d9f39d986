"""Pins for the oracle's series averaging (Section "Introduction": the aligned
frames f_i o phi_{0,i} of a series are averaged into one frame; Section
"Registration for series of images": the series averaging procedure repeats
the registration against the average)."""
import numpy as np
import pytest


def test_average_of_identical_frames_is_the_frame(orc, syn):
    f = syn.series(3, 1, 32)[0]
    g = orc.embed(f)
    avg = orc.average([g, g, g], [None, None, None])
    assert np.array_equal(avg, g)


def test_average_undoes_whole_pixel_translations(orc, syn):
    """Frames shifted by whole pixels, each warped back by its exact
    displacement, sample the first frame's node values exactly (bilinear
    interpolation at nodes), so their average equals the first frame wherever
    no shifted sample was clamped at the border."""
    side = 64
    t = np.array([[0, 0], [2, -1], [-3, 1], [1, 3]], dtype=np.float64)
    fr = syn.series(4, len(t), side, noise=False, drift=t, dist_amp=0.0)
    grids = [orc.embed(f) for f in fr]
    n = side + 1
    fields = []
    for k in range(len(t)):
        u = np.empty((2, n, n))
        u[0], u[1] = -t[k, 0] / side, -t[k, 1] / side
        fields.append(u)
    avg = orc.average(grids, fields)
    m = 4
    inner = (slice(m, side - m), slice(m, side - m))
    assert np.max(np.abs(avg[inner] - grids[0][inner])) < 1e-12
    # a wrong sign of the displacement (warping further away) does not
    assert np.max(np.abs(orc.average(grids, [-u for u in fields])[inner] - grids[0][inner])) > 0.1


def test_average_is_the_mean_of_the_warped_frames(orc, syn):
    """Brute force on a tiny grid: the average equals the mean of the frames
    warped one by one (the warp itself is pinned in test_oracle_energy.py)."""
    fr = syn.series(5, 3, 16)
    grids = [orc.embed(f) for f in fr]
    rng = np.random.default_rng(1)
    fields = [None] + [rng.uniform(-0.05, 0.05, size=(2, 17, 17)) for _ in range(2)]
    want = grids[0].copy()
    for g, u in zip(grids[1:], fields[1:]):
        want += orc.warp(g, u)[0]
    assert np.allclose(orc.average(grids, fields), want / 3, rtol=0, atol=1e-13)


@pytest.mark.slow
def test_averaging_procedure_iteration_keeps_a_stable_series(orc, syn):
    """On a noise-free series the registration is already consistent: one
    iteration of the averaging procedure (every frame registered to the
    average) changes the average by little and keeps the frames aligned: the
    refined deformations of frames 1.. stay within 0.2 px of phi_{0,k} minus
    the refined deformation of frame 0 (all now relative to the average)."""
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(noise=False, **cfg)
    p = orc.params(n_levels=nl, iter_max=50, lam=10.0)
    avg0, f0 = orc.average_series(fr, p, iterations=0)
    avg1, f1 = orc.average_series(fr, p, iterations=1)
    g0 = orc.embed(fr[0])
    rel = lambda a: np.abs(a - g0)[8:-8, 8:-8].mean() / np.abs(g0).mean()
    assert rel(avg0) < 0.1 and rel(avg1) < 0.1
    assert np.abs(avg1 - avg0)[8:-8, 8:-8].mean() < 0.05 * np.abs(g0).mean()
