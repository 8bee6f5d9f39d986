"""Tile shapes of the step kernels and the tile autotuner, through the C-ABI:
the strip rows of the gradient and trial tiles change only the order of the
FP32 partial sums, so per-node results are unchanged, sums agree to rounding,
and a series registered under other rows (or the autotuner's choice) still
matches the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROWS = (4, 8, 16, 32, 64)


@pytest.fixture(scope="module")
def reg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1712_02533_gb300 import _build
    _build.build()
    import paper_1712_02533_gb300 as r
    return r


def _rand_u(n, seed, amp):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.stack([amp * np.sin(2 * np.pi * (X + 0.3 * Y) + 0.4), amp * np.cos(2 * np.pi * (0.7 * X - Y))])
    return (u + rng.uniform(-0.2, 0.2, size=u.shape)).astype(np.float32)


def test_rows_are_validated_and_kept(reg, syn):
    fr = syn.series(5, 2, 256)
    with reg.Series(fr, reg.default_params(n_levels=3)) as s:
        assert s.get_tile_rows(8) == (16, 16) and s.get_tile_rows(6) == (8, 8)
        s.set_tile_rows(8, 4, 64)
        assert s.get_tile_rows(8) == (4, 64)
        for bad in ((3, 16), (16, 128), (0, 16)):
            with pytest.raises(reg.RegError):
                s.set_tile_rows(8, *bad)


@pytest.mark.parametrize("side", [256, 512])
def test_rows_change_sums_only_at_rounding(reg, syn, side):
    """Energies at a random displacement and the gradient-flow direction under
    every row choice: the direction is a per-node result (bit-identical), the
    energy and slope are FP64 sums of FP32 tile sums (1e-6 relative)."""
    fr = syn.series(3, 2, side, peak=10.0, spacing=10.0, sigma=2.0)
    L = int(np.log2(side))
    u = _rand_u(side + 1, 1, 1.3)
    res = {}
    with reg.Series(fr, reg.default_params(n_levels=2, lam=10.0)) as s:
        for rows in ROWS:
            s.set_tile_rows(L, rows, rows)
            e = s.eval_energy(0, 1, L, u)
            d, slope = s.eval_direction(0, 1, L, u)
            res[rows] = (e["E"], e["ncc"], d, slope)
    E0, n0, d0, s0 = res[16]
    for rows, (E, ncc, d, slope) in res.items():
        assert abs(ncc - n0) <= 1e-6 * abs(n0), rows
        assert abs(E - E0) <= 1e-6 * (abs(n0) + abs(E0 - (-n0))), rows
        assert np.array_equal(d, d0), rows
        assert abs(slope - s0) <= 1e-6 * abs(s0), rows


@pytest.mark.parametrize("kind", [1, 4])
def test_other_rows_keep_series_parity(reg, orc, syn, kind):
    """The stable config-1 input (no shot noise), registered with other strip
    rows at every level, still matches the oracle to 1e-3 px."""
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(noise=False, **cfg)
    with reg.Series(fr, reg.default_params(n_levels=nl, iter_max=50, lam=10.0)) as s:
        for lvl in (4, 5, 6):
            s.set_tile_rows(lvl, 4, 64)
        s.prefix_scan(kind)
        got = s.get_deformations()
    want = orc.register_series([fr], orc.params(n_levels=nl, iter_max=50, lam=10.0), kind=kind)[0][:, :, :64, :64]
    assert np.abs(got - want).max() <= 1e-3


def test_autotune_picks_valid_tiles_and_keeps_results(reg, syn):
    """The autotuner's table holds allowed rows for every level and a step-size
    count of 2, 3, 4 or 8; a series registered with it agrees with the default
    tiles to within the sub-pixel threshold (0.05 px) under which two results
    of the method count as the same."""
    fr = syn.series(12, 12, 256, spacing=12.0, sigma=2.0, peak=10.0, noise=False)
    p = reg.default_params(n_levels=3, iter_max=50, lam=10.0)
    with reg.Series(fr, p) as s:
        s.prefix_scan(reg.SKLANSKY)
        base = s.get_deformations()
    with reg.Series(fr, p) as s:
        rep = s.autotune(n_pairs=8, repeats=1)
        assert [lv["n"] for lv in rep["levels"]] == [65, 129, 257]
        for lv in rep["levels"]:
            assert lv["grad_rows"] in ROWS and lv["trial_rows"] in ROWS
            assert s.get_tile_rows(lv["level"]) == (lv["grad_rows"], lv["trial_rows"])
        assert rep["trials_per_pass"] in (2, 3, 4, 8)
        assert rep["runs"] > 8 and rep["ms_after"] > 0
        assert s.get_slot(0)[1] == (-1, -1)  # the sample's slots are marked empty
        s.prefix_scan(reg.SKLANSKY)
        got = s.get_deformations()
    assert np.abs(got - base).max() <= 0.05
