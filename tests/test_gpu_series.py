"""Segmented scans over series of mixed sizes, and the BF16 storage form, on the
GPU through the C-ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1712_02533_gb300 import _build
    _build.build()
    import paper_1712_02533_gb300 as r
    return r


def _mixed(syn):
    # three series of different sides and lengths (config 5's shape at small sizes)
    return [syn.series(11, 6, 64, spacing=8.0, sigma=1.5, peak=20.0, drift_sd=0.5, dist_amp=1.0),
            syn.series(12, 5, 128, spacing=10.0, sigma=2.0, peak=10.0, drift_sd=0.5, dist_amp=1.0),
            syn.series(13, 4, 256, spacing=12.0, sigma=2.0, peak=10.0, drift_sd=0.5, dist_amp=1.0)]


@pytest.mark.parametrize("kind_name", ["sklansky", "blelloch"])
def test_mixed_sizes_in_one_segmented_scan_equal_separate_scans(reg, syn, kind_name):
    """Each operator's sums are reduced in a fixed order over its own tiles, so
    batching the scan levels of several series (of different sizes) together
    must not change any result: bit-identical to scanning each series alone."""
    kind = {v: k for k, v in reg.SCAN_NAMES.items()}[kind_name]
    series = _mixed(syn)
    p = reg.default_params(n_levels=3, iter_max=50, lam=10.0)
    with reg.Series(series, p) as s:
        rep = s.prefix_scan(kind)
        together = [s.get_deformations(series=k) for k in range(len(series))]
    assert rep["preprocessing_ops"] == sum(len(f) - 1 for f in series)
    for k, f in enumerate(series):
        with reg.Series(f, p) as s:
            s.prefix_scan(kind)
            alone = s.get_deformations()
        assert np.array_equal(together[k], alone), (k, float(np.abs(together[k] - alone).max()))


def test_bf16_storage_error_against_fp32(reg, syn):
    """BF16 pyramid storage (FP32 arithmetic): its deviation from the FP32 form
    is a property of the series, not bounded a priori; it must stay a fraction of
    a pixel on the config-1 series, and the run must converge like the FP32 one."""
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(**cfg)
    out = {}
    for storage in (reg.STORAGE_F32, reg.STORAGE_BF16):
        p = reg.default_params(n_levels=nl, iter_max=50, lam=10.0, storage=storage)
        with reg.Series(fr, p) as s:
            s.prefix_scan(reg.SKLANSKY)
            out[storage] = s.get_deformations()
    err = np.abs(out[reg.STORAGE_BF16] - out[reg.STORAGE_F32])
    assert np.isfinite(err).all()
    assert err.max() < 0.5, float(err.max())


def test_host_transfers_match_device_transfers(reg, syn):
    """Frames from host memory go up in chunks through two staging buffers
    (copies overlapping the pyramid kernels), and deformations come down the
    same way; both must give exactly what the device-resident path gives.
    20 frames of 1024^2 span two upload chunks (16 frames of 4 MB fill a 64 MB
    staging buffer) and three download chunks (8 frames of 8 MB, the last one
    ragged)."""
    import torch
    frames = syn.series(21, 20, 1024, spacing=16.0, sigma=2.0, peak=10.0, drift_sd=0.5, dist_amp=1.0)
    p = reg.default_params(n_levels=5, iter_max=3, lam=10.0)
    with reg.Series([frames], p) as s:
        s.prefix_scan(reg.SKLANSKY)
        u_host = s.get_deformations()
        u_dev = torch.empty((20, 2, 1024, 1024), dtype=torch.float32, device="cuda")
        s.get_deformations(out=u_dev)
    with reg.Series([torch.from_numpy(frames).cuda()], p) as s:
        s.prefix_scan(reg.SKLANSKY)
        u_ref = torch.empty((20, 2, 1024, 1024), dtype=torch.float32, device="cuda")
        s.get_deformations(out=u_ref)
    assert np.array_equal(u_host, u_dev.cpu().numpy())
    assert np.array_equal(u_host, u_ref.cpu().numpy())
    assert np.abs(u_host[1:]).max() > 0.1  # the frames did move


def test_host_upload_of_mixed_series_matches_device_upload(reg, syn):
    """Several series of different sizes in one handle from host memory: the
    staging buffers alternate over the chunks of all series, and each copy
    waits for the kernels that read its buffer last, so every series gives
    exactly what it gives alone from device memory (each operator's sums are
    its own, so batching series together changes no result), checked through
    the deformations of a short scan, which read every level of every frame."""
    import torch
    series = [syn.series(31, 18, 256, spacing=8.0, sigma=1.5, peak=20.0, drift_sd=0.5, dist_amp=1.0),
              syn.series(32, 20, 1024, spacing=16.0, sigma=2.0, peak=10.0, drift_sd=0.5, dist_amp=1.0),
              syn.series(33, 3, 512, spacing=12.0, sigma=2.0, peak=10.0, drift_sd=0.5, dist_amp=1.0)]
    p = reg.default_params(n_levels=4, iter_max=2, lam=10.0)
    with reg.Series(series, p) as s:
        s.prefix_scan(reg.SKLANSKY)
        mixed = [s.get_deformations(k) for k in range(len(series))]
    for f, got in zip(series, mixed):
        with reg.Series([torch.from_numpy(f).cuda()], p) as s:
            s.prefix_scan(reg.SKLANSKY)
            assert np.array_equal(got, s.get_deformations())
