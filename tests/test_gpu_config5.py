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


def test_config5_sampled_operators_against_the_oracle(reg, orc, syn):
    """Config 5's four series (256^2, 512^2, 1024^2, 2048^2; c3's generator, 5
    levels) in one batch: operator A(1,2) of every series from the FP32 and the
    BF16 storage form against the FP64 oracle.  FP32: the parity criteria of
    the plain form, free running and in lockstep with the oracle's steps.
    BF16: max, 99th percentile and mean |du| and the final-energy difference
    are stated (the precision policy bounds them by nothing a priori)."""
    import _parity as P
    from concurrent.futures import ThreadPoolExecutor
    series = [syn.series(6 + i, 3, side, **GEN) for i, side in enumerate(SIDES)]
    lam, nl = 10.0, 5
    op = orc.params(n_levels=nl, iter_max=50, lam=lam)
    g = [(orc.embed(f[1]), orc.embed(f[2])) for f in series]

    def solve(k):
        with orc.trace() as t:
            u, _, _ = orc.register(g[k][0], g[k][1], op)
        return u, t.rows

    with ThreadPoolExecutor(max_workers=len(SIDES)) as ex:
        res = list(ex.map(solve, range(len(SIDES))))
    ops = [(k, -1, -1, 1, 1, 2) for k in range(len(SIDES))]
    for storage in (reg.STORAGE_F32, reg.STORAGE_BF16):
        p = reg.default_params(n_levels=nl, iter_max=50, lam=lam, storage=storage)
        with reg.Series(series, p) as s:
            s.set_trace(1 << 23)
            s.apply_operator_batch(ops)
            tr = s.get_trace()
            got = [s.get_slot(1, series=k)[0] for k in range(len(SIDES))]
            for k, side in enumerate(SIDES):
                u, rows = res[k]
                what = f"c5 {side}^2 A(1,2) {'bf16' if storage else 'fp32'}"
                if storage == reg.STORAGE_F32:
                    # lockstep one series at a time: the other series' ops take no steps
                    L = int(np.log2(side))
                    level_ns = [(1 << (L - nl + 1 + j)) + 1 for j in range(nl)]
                    counts, taus, _ = P.lock_sequence(rows, level_ns)
                    allc = [[0] * nl for _ in SIDES]
                    allc[k] = counts
                    s.set_lockstep(allc, taus)
                    s.set_trace(1 << 22)
                    try:
                        s.apply_operator_batch([(j, -1, -1, 0, 1, 2) for j in range(len(SIDES))])
                        ltr = s.get_trace()
                    finally:
                        s.set_lockstep(None)
                    lgot = s.get_slot(0, series=k)[0]
                    rec = dict(what=what, mode="lockstep", steps=len(taus), **P.field_stats(lgot, u * side))
                    gpu_e = P.gpu_energy_fn(s, 1, 2, L, k)
                    rec["E_rel"] = P.energy_rel(gpu_e, lgot, orc, g[k][0], g[k][1], u * side, lam)[0]
                    P.report("c5", rec)
                    assert rec["max_px"] <= P.TOL_PX or P._agreeing_fields_ok(rec), rec
                    P.report("c5", P.free_running_parity(orc, got[k], u * side, tr[tr[:, 0] == k][:, 1:], rows,
                                                         what, g[k][0], g[k][1], op, lam, gpu_e))
                else:
                    rec = dict(what=what, mode="free", **P.field_stats(got[k], u * side))
                    rec["E_rel"] = P.energy_rel(P.gpu_energy_fn(s, 1, 2, int(np.log2(side)), k), got[k], orc,
                                                g[k][0], g[k][1], u * side, lam)[0]
                    P.report("c5", rec)
                    assert np.isfinite(rec["max_px"])
