"""Config 5 at full size: one segmented scan over four series of 256^2, 512^2,
1024^2 and 2048^2 frames (16, 64, 400 and 32 frames) in shared launches, in
FP32 and in BF16 pyramid storage.  Properties checked at this size: every
operator ends with finite energies; batching with the larger series leaves the
smallest one's result bit-identical to scanning it alone (each operator's sums
are reduced over its own tiles in a fixed order); the BF16 form's deviation
from the FP32 form is stated per series and stays below a pixel."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIDES = (256, 512, 1024, 2048)
FRAMES = (16, 64, 400, 32)
GEN = dict(spacing=16.0, sigma=2.0, peak=5.0, drift_sd=1.0, dist_amp=2.0)


@pytest.fixture(scope="module")
def reg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1712_02533_gb300 import _build
    _build.build()
    import paper_1712_02533_gb300 as r
    return r


def test_config5_full_size_mixed_scan(reg, syn):
    series = [syn.series(6 + i, nf, side, **GEN) for i, (side, nf) in enumerate(zip(SIDES, FRAMES))]
    out, reps = {}, {}
    for storage in (reg.STORAGE_F32, reg.STORAGE_BF16):
        p = reg.default_params(n_levels=5, iter_max=50, lam=10.0, storage=storage)
        with reg.Series(series, p) as s:
            reps[storage] = s.prefix_scan(reg.SKLANSKY)
            out[storage] = [s.get_deformations(series=k) for k in range(len(series))]
    for storage, rep in reps.items():
        assert rep["preprocessing_ops"] == sum(f - 1 for f in FRAMES)
        assert rep["status"]["nonfinite"] == 0, rep
        print("storage", storage, "series time", rep["ms"], "ms,", rep["ops"], "operator applications")
    p = reg.default_params(n_levels=5, iter_max=50, lam=10.0)
    with reg.Series([series[0]], p) as s:
        s.prefix_scan(reg.SKLANSKY)
        alone = s.get_deformations()
    assert np.array_equal(out[reg.STORAGE_F32][0], alone)
    for k, side in enumerate(SIDES):
        err = np.abs(out[reg.STORAGE_BF16][k] - out[reg.STORAGE_F32][k])
        print(f"BF16 vs FP32 storage, {side}^2 x {FRAMES[k]}: mean {err.mean():.4f} px, "
              f"max {err.max():.3f} px, 99th percentile {np.quantile(err, 0.99):.4f} px")
        assert np.isfinite(err).all()
        assert err.mean() < 1.0, (side, float(err.mean()))
