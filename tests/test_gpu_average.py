"""Series averaging on the GPU (reg_average_series) against the FP64 oracle
(Section "Introduction": the aligned frames f_i o phi_{0,i} are averaged;
Section "Registration for series of images": the series averaging procedure)."""
import numpy as np
import pytest

import _parity as P

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


def _fields(n_frames, n, seed):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    out = []
    for k in range(1, n_frames):
        a, b = rng.uniform(-3, 3, size=2)
        out.append(np.stack([a + 1.5 * np.sin(2 * np.pi * (X + 0.2 * k)),
                             b + 1.2 * np.cos(2 * np.pi * (Y - 0.1 * k))]).astype(np.float32))
    return out


@pytest.mark.parametrize("side,storage", [(64, 0), (256, 0), (256, 1)])
def test_average_of_given_deformations_matches_oracle(reg, orc, syn, side, storage):
    """The average of the frames deformed by given fields (set into the slots
    as the deformations phi_{0,k}), against the oracle's average of the same
    frames and fields: FP32 storage to 1e-5 of the intensity range, BF16 storage
    to the storage's rounding (1e-2 of the range)."""
    nf = 6
    fr = syn.series(41, nf, side, peak=20.0, spacing=10.0, sigma=2.0) + np.float32(50.0)
    n = side + 1
    fields = _fields(nf, n, 3)
    p = reg.default_params(n_levels=2, lam=10.0, storage=storage)
    with reg.Series(fr, p) as s:
        for k in range(1, nf):
            s.set_slot(k - 1, fields[k - 1], 0, k)
        got = s.average(iterations=0)
    grids = [orc.embed(f) for f in fr]
    want = orc.average(grids, [None] + [f.astype(np.float64) / side for f in fields])[:side, :side]
    rng_ = float(want.max() - want.min())
    tol = 1e-5 if storage == 0 else 1e-2
    err = float(np.abs(got - want).max())
    P.report("average", dict(side=side, storage=storage, max_abs=err, range=rng_))
    assert err <= tol * rng_, (err, rng_)


def test_averaging_procedure_matches_oracle_on_a_stable_series(reg, orc, syn):
    """The whole procedure on the config-1 series without shot noise (the
    oracle's result is stable there): registration, average, one iteration of
    registering every frame to the average, average again.  Deformations to
    1e-3 px at every node, averages to 1e-5 of the intensity range."""
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(noise=False, **cfg)
    p = reg.default_params(n_levels=nl, iter_max=50, lam=10.0)
    with reg.Series(fr, p) as s:
        s.prefix_scan(reg.SKLANSKY)
        avg0 = s.average(iterations=0)
        avg1 = s.average(iterations=1)
        d1 = s.get_deformations()
    op = orc.params(n_levels=nl, iter_max=50, lam=10.0)
    w0, _ = orc.average_series(fr, op, iterations=0)
    w1, f1 = orc.average_series(fr, op, iterations=1)
    rng_ = float(w0.max() - w0.min())
    e0 = float(np.abs(avg0 - w0[:64, :64]).max())
    e1 = float(np.abs(avg1 - w1[:64, :64]).max())
    ef = float(np.abs(d1 - f1[:, :, :64, :64]).max())
    P.report("average-procedure", dict(avg0_max=e0, avg1_max=e1, fields_max_px=ef, range=rng_))
    assert e0 <= 1e-5 * rng_ and e1 <= 1e-4 * rng_, (e0, e1, rng_)
    assert ef <= P.TOL_PX, ef
