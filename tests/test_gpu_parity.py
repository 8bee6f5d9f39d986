"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Tolerances (FP32 kernels against the FP64 oracle): single energy evaluations
to 1e-5 relative, gradient-flow directions to 1e-4 of their maximum, and
registered displacements to 1e-3 px with final energies to 1e-5 relative.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3
TOL_E = 1e-5


def orc_energy(R, T, u, lam):
    import oracle
    return oracle.energy(R, T, u, lam)


@pytest.fixture(scope="module")
def reg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1712_02533_gb300 import _build
    _build.build()
    import paper_1712_02533_gb300 as r
    return r


def _pyramid(orc, frame, nl):
    g = [orc.embed(frame)]
    for _ in range(nl - 1):
        g.append(orc.restrict(g[-1]))
    return g[::-1]  # coarsest first


def _rand_u(n, seed, amp):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.stack([amp * np.sin(2 * np.pi * (X + 0.3 * Y) + 0.4), amp * np.cos(2 * np.pi * (0.7 * X - Y))])
    return u + rng.uniform(-0.2, 0.2, size=u.shape)


@pytest.mark.parametrize("side,nl", [(64, 3), (128, 3), (256, 2), (512, 2)])
def test_energy_matches_oracle(reg, orc, syn, side, nl):
    fr = syn.series(3, 2, side, peak=10.0, spacing=10.0, sigma=2.0)
    lam = 10.0
    p = reg.default_params(n_levels=nl, lam=lam)
    Rp, Tp = _pyramid(orc, fr[0], nl), _pyramid(orc, fr[1], nl)
    L = int(np.log2(side))
    with reg.Series(fr, p) as s:
        for k in range(nl):
            n = Rp[k].shape[0]
            level = L - nl + 1 + k
            for seed, amp in [(0, 0.0), (1, 1.3), (2, 4.0)]:
                ug = _rand_u(n, seed, amp).astype(np.float32)
                got = s.eval_energy(0, 1, level, ug)
                E, parts = orc.energy(Rp[k], Tp[k], ug.astype(np.float64) / (n - 1), lam)
                # relative to the size of the two terms: E itself can cancel to ~0
                scale = abs(parts["ncc"]) + abs(parts["reg"])
                assert abs(got["E"] - E) <= TOL_E * scale, (level, seed, got, E)
                assert abs(got["ncc"] - parts["ncc"]) <= TOL_E * abs(parts["ncc"])
                assert abs(got["reg"] - parts["reg"]) <= 1e-5 * max(abs(parts["reg"]), 1e-6)


@pytest.mark.parametrize("side,nl", [(64, 3), (128, 2), (512, 2)])
def test_direction_matches_oracle(reg, orc, syn, side, nl):
    fr = syn.series(4, 2, side, peak=10.0, spacing=10.0, sigma=2.0)
    lam = 10.0
    p = reg.default_params(n_levels=nl, lam=lam)
    Rp, Tp = _pyramid(orc, fr[0], nl), _pyramid(orc, fr[1], nl)
    L = int(np.log2(side))
    with reg.Series(fr, p) as s:
        for k in range(nl):
            n = Rp[k].shape[0]
            h = 1.0 / (n - 1)
            level = L - nl + 1 + k
            for seed, amp in [(0, 0.5), (3, 2.5)]:
                ug = _rand_u(n, seed, amp).astype(np.float32)
                d, slope = s.eval_direction(0, 1, level, ug)
                uo = ug.astype(np.float64) * h
                g = orc.gradient(Rp[k], Tp[k], uo, lam)
                w = orc.lumped(n)
                dd = -g / w
                want = dd / h
                assert np.max(np.abs(d - want)) <= 1e-4 * np.max(np.abs(want)), (level, seed)
                want_slope = float(np.sum(g * dd))
                assert abs(slope - want_slope) <= 1e-5 * abs(want_slope), (slope, want_slope)


@pytest.mark.parametrize("side,nl", [(128, 2), (512, 2)])
def test_trial_pass_matches_oracle(reg, orc, syn, side, nl):
    """One trial pass of the Armijo search: the energy changes E(u + tau d) - E(u)
    for step sizes whose largest move spans 1e-6 to 3 grid units (moves inside a
    cell, across cell lines, past the grid border, beyond one cell), against the
    oracle's FP64 energies at the same u and d."""
    fr = syn.series(6, 2, side, peak=10.0, spacing=10.0, sigma=2.0)
    lam = 10.0
    p = reg.default_params(n_levels=nl, lam=lam, trials_per_pass=8)
    Rp, Tp = _pyramid(orc, fr[0], nl), _pyramid(orc, fr[1], nl)
    L = int(np.log2(side))
    moves = np.array([1e-6, 1e-4, 1e-2, 0.3, 0.7, 1.5, 3.0])
    with reg.Series(fr, p) as s:
        for k in range(nl):
            n = Rp[k].shape[0]
            h = 1.0 / (n - 1)
            level = L - nl + 1 + k
            for seed, amp in [(0, 0.5), (3, 2.5)]:
                ug = _rand_u(n, seed, amp).astype(np.float32)
                d0, _ = s.eval_direction(0, 1, level, ug)
                taus = moves / float(np.abs(d0).max())
                d, dE = s.eval_trials(0, 1, level, ug, taus)
                assert np.array_equal(d, d0)
                uo = ug.astype(np.float64) * h
                E0, _ = orc.energy(Rp[k], Tp[k], uo, lam)
                for j, t in enumerate(taus):
                    E1, _ = orc.energy(Rp[k], Tp[k], uo + t * d.astype(np.float64) * h, lam)
                    want = E1 - E0
                    assert abs(dE[j] - want) <= 1e-4 * abs(want) + 1e-9 * abs(E0), (level, seed, moves[j], dE[j], want)


def test_function_a_matches_oracle(reg, orc, syn):
    side, nl = 64, 3
    fr = syn.series(5, 2, side, peak=20.0, spacing=8.0, sigma=1.5, drift_sd=0.7)
    p = reg.default_params(n_levels=nl, iter_max=30, lam=10.0)
    with reg.Series(fr, p) as s:
        st, it = s.apply_operator_batch([(0, -1, -1, 0, 0, 1)])
        got, se = s.get_slot(0)
        assert se == (0, 1)
        eg = s.eval_energy(0, 1, int(np.log2(side)), got)
    op = orc.params(n_levels=nl, iter_max=30, lam=10.0)
    u, status, stl = orc.register(orc.embed(fr[0]), orc.embed(fr[1]), op)
    want = u * side
    assert int(st[0]) == status
    assert int(it[0]) == sum(x.iters for x in stl)
    assert np.max(np.abs(got - want)) <= TOL_PX
    assert abs(eg["E"] - stl[-1].E) <= TOL_E * abs(stl[-1].E)


def _assert_op_parity(gpu_u_px, orc_u_px, gtr, otr, what, R, T, lam=10.0):
    """Parity of one full operator application.  Either the displacement fields
    agree to TOL_PX everywhere, or the two Armijo decision sequences agree up to
    a decision that the oracle itself takes with a margin below 1e-3 (relative):
    from such a decision on, rounding at the 1e-7 level legitimately sends the
    iteration elsewhere (the same happens to the oracle under 1e-7 input
    perturbations, see test_oracle_sensitivity.py).  When every decision
    agrees, the fields may still differ at the few nodes that the iteration
    drives onto a cell line of the bilinear interpolant: the template's
    derivative jumps there, so which side such a node ends on is decided at the
    rounding level (in FP32 on the GPU, FP64 in the oracle).  Those nodes must
    stay rare (99.5% of the nodes within TOL_PX), and the GPU's field must be no
    worse a minimiser: the oracle's FP64 energy at it may exceed the energy at
    the oracle's own field by at most 1e-6 (relative)."""
    err = float(np.abs(gpu_u_px - orc_u_px).max())
    if err <= TOL_PX:
        return err
    m = min(len(gtr), len(otr))
    for k in range(m):
        a, b = gtr[k], otr[k]
        assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2], (what, "trial sequence differs before any decision", k)
        if a[5] != b[5]:
            # the oracle's own margin must lie within the disagreement of the two
            # energy changes at that point (plus 1e-3): the flip is explained by
            # the states having separated, not by a different decision rule
            margin = abs(b[3] - b[4]) / abs(b[4])
            spread = (abs(a[3] - b[3]) + abs(a[4] - b[4])) / abs(b[4])
            assert margin < spread + 1e-3, (what, "decision differs at a non-marginal test", k, a, b, err)
            return err
    side = gpu_u_px.shape[-1] - 1
    frac = float(np.mean(np.abs(gpu_u_px - orc_u_px) <= TOL_PX))
    e_gpu, _ = orc_energy(R, T, gpu_u_px.astype(np.float64) / side, lam)
    e_orc, _ = orc_energy(R, T, np.asarray(orc_u_px, np.float64) / side, lam)
    assert frac >= 0.995 and e_gpu - e_orc <= 1e-6 * abs(e_orc), (
        what, "fields differ although every decision agrees", err, frac, e_gpu, e_orc)
    return err


def _gpu_traces_by_op(tr, n_ops):
    return [tr[tr[:, 0] == o][:, 1:] for o in range(n_ops)]


def test_config1_operators_match_oracle(reg, orc, syn):
    """Config-1 series (8 x 64^2, Poisson noise): every preprocessing operator
    (function A) matches the oracle field by field or decision by decision."""
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(**cfg)
    g = [orc.embed(f) for f in fr]
    p = reg.default_params(n_levels=nl, iter_max=50, lam=10.0)
    op = orc.params(n_levels=nl, iter_max=50, lam=10.0)
    n = len(fr) - 1
    with reg.Series(fr, p) as s:
        s.set_trace(1 << 20)
        st, it = s.apply_operator_batch([(0, -1, -1, e, e, e + 1) for e in range(n)])
        gtr = _gpu_traces_by_op(s.get_trace(), n)
        got = [s.get_slot(e)[0] for e in range(n)]
    n_exact = 0
    for e in range(n):
        with orc.trace() as t:
            u, status, stl = orc.register(g[e], g[e + 1], op)
        err = _assert_op_parity(got[e], u * 64, gtr[e], t.rows, f"A({e},{e + 1})", g[e], g[e + 1])
        n_exact += err <= TOL_PX
    assert n_exact >= n - 1


def test_config1_scan_operators_match_oracle(reg, orc, syn):
    """Function B along the serial scan of config 1, each given the operands the
    GPU produced (so that both sides start from the same fields)."""
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(**cfg)
    g = [orc.embed(f) for f in fr]
    p = reg.default_params(n_levels=nl, iter_max=50, lam=10.0)
    op = orc.params(n_levels=nl, iter_max=50, lam=10.0)
    with reg.Series(fr, p) as s:
        s.apply_operator_batch([(0, -1, -1, e, e, e + 1) for e in range(7)])
        A = [s.get_slot(e)[0].astype(np.float64) / 64 for e in range(7)]
        acc = A[0]
        for k in range(1, 7):
            s.set_trace(1 << 20)
            s.apply_operator_batch([(0, k - 1, k, k, 0, k + 1)])
            got = s.get_slot(k)[0]
            gtr = s.get_trace()[:, 1:]
            with orc.trace() as t:
                out, _, _, _, _ = orc.apply_batch([dict(R=g[0], T=g[k + 1], left=acc, right=A[k])], op)
            _assert_op_parity(got, out[0] * 64, gtr, t.rows, f"B(0,{k},{k + 1})", g[0], g[k + 1])
            acc = got.astype(np.float64) / 64


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 7, 8])
def test_series_stable_input_matches_oracle(reg, orc, syn, kind):
    """Whole-series registration, every schedule, on the config-1 series
    without shot noise (expected counts), where the oracle's result is stable
    under 1e-7 input perturbations (test_oracle_sensitivity.py): the GPU
    deformations phi_{0,k} must match to TOL_PX at every node."""
    cfg = dict(syn.CONFIGS["c1_8x64"])
    nl = cfg.pop("n_levels")
    fr = syn.series(noise=False, **cfg)
    p = reg.default_params(n_levels=nl, iter_max=50, lam=10.0)
    hc_k = 1  # k of Han-Carlson and Ladner-Fischer (unused by the other kinds here)
    with reg.Series(fr, p) as s:
        rep = s.prefix_scan(kind, chunks=hc_k)
        got = s.get_deformations()
    op = orc.params(n_levels=nl, iter_max=50, lam=10.0)
    want, info = orc.register_series([fr], op, kind=kind, chunks=hc_k, return_info=True)
    want = want[0][:, :, :64, :64]
    assert rep["ops"] == info["ops"]
    err = np.abs(got - want)
    assert err.max() <= TOL_PX, (err.max(), [float(err[k].max()) for k in range(len(err))])


def test_config2_sampled_operators_match_oracle(reg, orc, syn):
    """Config-2 sizes (512^2, 4 levels): sampled A and B operators of the
    128-frame series, against the oracle computed one by one."""
    cfg = dict(syn.CONFIGS["c2_128x512"])
    nl = cfg.pop("n_levels")
    fr = syn.series(**cfg)
    p = reg.default_params(n_levels=nl, iter_max=50, lam=10.0)
    op = orc.params(n_levels=nl, iter_max=50, lam=10.0)
    side = 512
    with reg.Series(fr, p) as s:
        s.set_trace(1 << 22)
        n = len(fr) - 1
        s.apply_operator_batch([(0, -1, -1, e, e, e + 1) for e in range(n)])
        gtr = _gpu_traces_by_op(s.get_trace(), n)
        for e in (0, 77):
            got = s.get_slot(e)[0]
            R, T = orc.embed(fr[e]), orc.embed(fr[e + 1])
            with orc.trace() as t:
                u, _, _ = orc.register(R, T, op)
            _assert_op_parity(got, u * side, gtr[e], t.rows, f"A({e},{e + 1}) 512^2", R, T)
        left = s.get_slot(0)[0].astype(np.float64) / side
        right = s.get_slot(1)[0].astype(np.float64) / side
        s.set_trace(1 << 22)
        s.apply_operator_batch([(0, 0, 1, 1, 0, 2)])
        got = s.get_slot(1)[0]
        gtr2 = s.get_trace()[:, 1:]
    # B given the GPU's operands on both sides
    with orc.trace() as t:
        out, _, _, _, _ = orc.apply_batch([dict(R=orc.embed(fr[0]), T=orc.embed(fr[2]), left=left, right=right)], op)
    _assert_op_parity(got, out[0] * side, gtr2, t.rows, "B(0,1,2) 512^2", orc.embed(fr[0]), orc.embed(fr[2]))


def test_identical_frames_give_zero_displacement(reg, syn):
    f = syn.series(9, 1, 64)
    fr = np.concatenate([f, f, f])
    with reg.Series(fr, reg.default_params(n_levels=3, lam=10.0)) as s:
        s.prefix_scan(reg.SERIAL)
        d = s.get_deformations()
    assert np.abs(d).max() < 1e-6


def test_invalid_arguments_are_rejected(reg, syn):
    fr = syn.series(9, 3, 64)
    with reg.Series(fr, reg.default_params(n_levels=3)) as s:
        with pytest.raises(reg.RegError) as e:
            s.apply_operator_batch([(0, 0, -1, 1, 0, 1)])  # slot 0 holds nothing yet
        assert e.value.code == reg.EINVAL
        s.apply_operator_batch([(0, -1, -1, 0, 0, 1), (0, -1, -1, 1, 1, 2)])
        with pytest.raises(reg.RegError):
            s.apply_operator_batch([(0, 1, 0, 2, 0, 2)])  # chain mismatch: phi_12 then phi_01
        with pytest.raises(reg.RegError):
            s.apply_operator_batch([(0, -1, -1, 99, 0, 1)])
    with pytest.raises(reg.RegError):
        reg.Series(syn.series(9, 3, 48), reg.default_params(n_levels=2))  # not a power of two


def test_full_size_sampled_operators_match_oracle(reg, orc, syn):
    """The 400 x 1024^2 workload (5 levels) in the launch configuration the
    benchmark times (all 399 neighbour pairs in one batch): sampled operators
    against the oracle computed one by one, under the same criterion as the
    smaller configurations."""
    cfg = dict(syn.CONFIGS["c3_400x1024"])
    nl = cfg.pop("n_levels")
    fr = syn.series(**cfg)
    p = reg.default_params(n_levels=nl, iter_max=50, lam=10.0)
    op = orc.params(n_levels=nl, iter_max=50, lam=10.0)
    side = 1024
    n = len(fr) - 1
    with reg.Series(fr, p) as s:
        s.set_trace(1 << 23)
        s.apply_operator_batch([(0, -1, -1, e, e, e + 1) for e in range(n)])
        gtr = _gpu_traces_by_op(s.get_trace(), n)
        got = {e: s.get_slot(e)[0] for e in (0, 250)}
    for e, u_gpu in got.items():
        R, T = orc.embed(fr[e]), orc.embed(fr[e + 1])
        with orc.trace() as t:
            u, _, _ = orc.register(R, T, op)
        _assert_op_parity(u_gpu, u * side, gtr[e], t.rows, f"A({e},{e + 1}) 1024^2", R, T)
