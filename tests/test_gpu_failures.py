"""Failure detection on the GPU without faulting it: the failures are made on
the host.  A device step budget that runs out ends the batch with
REG_ETIMEOUT and leaves the handle usable; a frame with a non-finite pixel
makes the operators that read it report NONFINITE while every other operator
of the same batch is bit-identical to a run without it."""
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


def test_step_budget_times_out_and_handle_recovers(reg, syn):
    fr = syn.series(21, 4, 64)
    fr[3] = fr[2]  # an identical pair: done within a few steps
    p = reg.default_params(n_levels=1, iter_max=50, lam=10.0, max_steps=8)
    with reg.Series(fr, p) as s:
        with pytest.raises(reg.RegError) as e:
            s.apply_operator_batch([(0, -1, -1, 0, 0, 1)])  # needs far more than 8 device steps
        assert e.value.code == reg.ETIMEOUT
        st, it = s.apply_operator_batch([(0, -1, -1, 2, 2, 3)])
        # identical frames: NCC rounds a few ulp below 1, so the search either
        # finds no decrease (stalled) or sees a zero slope
        assert int(st[0]) in (reg.OP_ZERO_GRADIENT, reg.OP_CONVERGED, reg.OP_LS_STALLED), st
        u, se = s.get_slot(2)
        assert se == (2, 3) and np.abs(u).max() < 1e-6
    # the same operator with the default budget finishes normally
    with reg.Series(fr, reg.default_params(n_levels=1, iter_max=50, lam=10.0)) as s:
        st, it = s.apply_operator_batch([(0, -1, -1, 0, 0, 1)])
        assert int(it[0]) > 1


def test_nonfinite_frame_is_reported_per_operator(reg, syn):
    fr = syn.series(22, 5, 64)
    bad = fr.copy()
    bad[2, 17, 40] = np.nan
    p = reg.default_params(n_levels=2, iter_max=30, lam=10.0)
    ops = [(0, -1, -1, e, e, e + 1) for e in range(4)]
    out = {}
    for name, frames in (("clean", fr), ("nan", bad)):
        with reg.Series(frames, p) as s:
            st, it = s.apply_operator_batch(ops)
            out[name] = (st, it, [s.get_slot(e)[0] for e in range(4)])
    st, it, u = out["nan"]
    st0, it0, u0 = out["clean"]
    assert int(st[1]) == reg.OP_NONFINITE and int(st[2]) == reg.OP_NONFINITE, st  # A(1,2), A(2,3) read frame 2
    for e in (0, 3):
        assert int(st[e]) == int(st0[e]) and int(it[e]) == int(it0[e])
        assert np.array_equal(u[e], u0[e])
