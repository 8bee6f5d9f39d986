"""The synthetic series generator is deterministic, order independent and
consistent with its own ground truth."""
import numpy as np


def test_deterministic_and_order_independent(syn):
    a = syn.series(7, 4, 64)
    b = syn.series(7, 4, 64)
    assert np.array_equal(a, b)
    c = syn.series(7, 2, 64)
    assert np.array_equal(a[:2], c)
    d = syn.series(8, 4, 64)
    assert not np.array_equal(a, d)


def test_counts_are_integers_and_noise_free_mode(syn):
    a = syn.series(7, 2, 64, noise=True)
    assert np.all(a == np.round(a)) and a.min() >= 0
    b = syn.series(7, 2, 64, noise=False)
    assert not np.all(b == np.round(b))
    assert abs(a.mean() - b.mean()) < 0.05 * b.mean()


def test_ground_truth_of_pure_translation(syn):
    t = np.array([[0.0, 0.0], [1.25, -0.5], [-2.0, 3.0]])
    f, gt, tr = syn.series(3, 3, 32, drift=t, dist_amp=0.0, ground_truth=True)
    assert np.array_equal(tr, t)
    assert np.allclose(gt[0], 0.0)
    for k in range(3):
        assert np.allclose(gt[k, 0], -t[k, 0]) and np.allclose(gt[k, 1], -t[k, 1])


def test_integer_translation_moves_pixels(syn):
    f = syn.series(3, 2, 64, noise=False, drift=[[0, 0], [3, -2]], dist_amp=0.0)
    # frame 1 at pixel y shows the specimen at y + t: f1(y) = f0(y + t)
    assert np.array_equal(f[1][2:64, 0:61], f[0][0:62, 3:64])
