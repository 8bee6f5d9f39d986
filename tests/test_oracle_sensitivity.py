"""How sensitive the method itself is (the FP64 oracle, no GPU involved).

The energy is non-smooth (bilinear interpolation has kinks at cell lines)
and the Armijo rule takes discrete decisions, so that the iterates of a
gradient flow on noisy frames may depend on rounding: the paper observes that
computed deformations vary among implementations of the same algorithm
(Section "A note on the associativity").  These tests fix, on the oracle
alone, which inputs are stable under perturbations at the level of float
rounding (1e-7 relative) and which are not; the CUDA parity tests hold the
GPU to a strict node-wise bound on the stable input and to decision-by-
decision agreement on the others."""
import numpy as np
import pytest

from oracle import schedules as S


def _sensitivity(orc, fr, p, eps=1e-7, reps=2):
    base = orc.register_series([fr], p, kind=S.SKLANSKY)[0]
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(reps):
        fp = (fr.astype(np.float64) * (1 + eps * rng.standard_normal(fr.shape))).astype(np.float32)
        fp[0] = fr[0]
        u = orc.register_series([fp], p, kind=S.SKLANSKY)[0]
        worst = max(worst, float(np.abs(u - base).max()))
    return worst


@pytest.mark.slow
def test_noise_free_config1_series_is_stable(orc, syn):
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(noise=False, **cfg)
    assert _sensitivity(orc, fr, orc.params(n_levels=nl, iter_max=50, lam=10.0)) < 1e-5


@pytest.mark.slow
def test_noisy_config1_series_is_sensitive(orc, syn):
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(**cfg)
    assert _sensitivity(orc, fr, orc.params(n_levels=nl, iter_max=50, lam=10.0)) > 1e-2
