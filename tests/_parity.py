"""Helpers shared by the GPU parity tests (CUDA path against the FP64 oracle).

Two ways of comparing one operator application (function A or B):

* Free running.  Both sides search their own Armijo steps (Section "Gradient
  flow").  On noisy frames the iteration is chaotic: a decision whose margin is
  at the rounding level sends two correct implementations to different, equally
  good fields (Section "A note on the associativity" notes that results differ
  among implementations).  ``free_running_parity`` therefore accepts one of
    1. max |du| <= TOL_PX at every node;
    2. every Armijo decision agrees, >= 99.5% of the nodes within TOL_PX, the
       others -- nodes around a cell line of the bilinear interpolant, where
       the template's derivative jumps, so that the side a node driven there
       lands on is decided at the rounding level -- within AGREE_CAP_PX, and
       the GPU's final energy no higher than the oracle's by more than TOL_E;
    3. the decisions agree up to one whose oracle margin is smaller than the
       disagreement of the two sides' energy changes at that point (no slack),
       that disagreement is itself within the energy tolerance (SPREAD_MAX =
       TOL_E relative to the energy), and afterwards max |du| and the final
       energy difference stay within FLIP_SPREAD_FACTOR times the oracle's own
       spread -- how far the oracle's field and final energy move when the
       template frame is perturbed by 1e-7 relative (two draws) -- plus TOL_PX
       and TOL_E.
* Lockstep.  The GPU replays the oracle's accepted step sizes
  (reg_set_lockstep); no decision is taken, so the fields must agree to
  TOL_PX and the final energies to TOL_E, for every operator -- except at the
  few nodes (< 0.5%) around nodes that the flow drives onto a cell line of the
  bilinear interpolant, where the template's derivative jumps and the side a
  node takes is decided at the rounding level even along the same steps;
  those stay within AGREE_CAP_PX, and the GPU's energy may then be lower.

Every comparison returns a record (max, 99th percentile and mean |du| in px,
relative final-energy difference) that the tests print on one line each.
"""
from __future__ import annotations

import json
from concurrent.futures import ThreadPoolExecutor

import numpy as np

TOL_PX = 1e-3        # spec tolerance on displacements, FP32 plain form
TOL_E = 1e-5         # spec tolerance on the final energy, relative
AGREE_CAP_PX = 0.5   # same steps taken: bound on the few nodes around cell lines (measured up to 0.32 px)
SPREAD_MAX = TOL_E   # a flip is excused only if the two energy changes agree to this (relative to |E|)
FLIP_SPREAD_FACTOR = 4.0
PERTURB_REL = 1e-7


def report(tag, rec):
    """One machine-readable line per compared operator (pytest -s shows it)."""
    print("PARITY " + tag + " " + json.dumps(rec, sort_keys=True))


def field_stats(gpu_px, orc_px):
    d = np.abs(np.asarray(gpu_px, np.float64) - np.asarray(orc_px, np.float64))
    return dict(max_px=float(d.max()), p99_px=float(np.quantile(d, 0.99)), mean_px=float(d.mean()),
                frac_within=float(np.mean(d <= TOL_PX)), n_beyond=int(np.sum(d > TOL_PX)))


def kink_excess(gpu_px, orc_px):
    """Nodes beyond TOL_PX must come from a kink of the energy: the bilinear
    interpolant's derivative jumps where a node's position x + u crosses a
    cell line (an integer number of pixels on the finest grid), the flow
    drives nodes onto such lines, and the side such a node ends on is decided
    at the rounding level; the mass and stiffness stencils then carry a
    decaying difference to the nodes around it (over the iterations, a few
    nodes far).  So every cluster of differing nodes (nodes at most six apart
    joined) must contain a node that lies on a cell line:
    within its own difference of one (in the oracle's or the GPU's position).
    Returns, over the clusters, the largest of the smallest excess of that
    distance over the node's difference (<= 0 when every cluster is explained
    so)."""
    from scipy import ndimage
    g = np.asarray(gpu_px, np.float64)
    o = np.asarray(orc_px, np.float64)
    d = np.abs(g - o).max(axis=0)  # per node, the larger component difference
    m = d > TOL_PX
    if not m.any():
        return 0.0
    dist = np.minimum(np.abs(o - np.round(o)), np.abs(g - np.round(g))).min(axis=0)
    joined = ndimage.binary_dilation(m, structure=np.ones((3, 3)), iterations=3)
    lab, n = ndimage.label(joined, structure=np.ones((3, 3)))
    worst = -np.inf
    for k in range(1, n + 1):
        sel = (lab == k) & m
        worst = max(worst, float(np.min(dist[sel] - d[sel])))
    return worst


def beyond_detail(gpu_px, orc_px, limit=16):
    """The nodes beyond TOL_PX: (row, col, |du| px, oracle and GPU distance of
    the node's position to the nearest cell line, per component)."""
    g = np.asarray(gpu_px, np.float64)
    o = np.asarray(orc_px, np.float64)
    d = np.abs(g - o).max(axis=0)
    idx = np.argwhere(d > TOL_PX)[:limit]
    out = []
    for r, c in idx:
        out.append([int(r), int(c), round(float(d[r, c]), 5),
                    [round(float(abs(o[k, r, c] - np.round(o[k, r, c]))), 5) for k in range(2)],
                    [round(float(abs(g[k, r, c] - np.round(g[k, r, c]))), 5) for k in range(2)]])
    return out


def _agreeing_fields_ok(rec):
    """Fields of two runs that took the same steps: all but a few nodes (at
    most 0.5%) within TOL_PX, those few within AGREE_CAP_PX, and the GPU's
    field no worse a minimiser of the oracle's FP64 energy (by at most TOL_E;
    lower is allowed).  The few are nodes around kinks of the energy
    (kink_excess_px records how well the finest grid's cell lines explain
    them; kinks met on a coarser level have moved on since, so it is not
    asserted)."""
    return (rec["frac_within"] >= 0.995 and rec["p99_px"] <= TOL_PX and rec["max_px"] <= AGREE_CAP_PX
            and rec["E_rel"] <= TOL_E)


def gpu_energy_fn(series, frame_i, frame_k, level, series_index=0):
    """The GPU's own energy of a field of its (reg_eval_energy, itself held to
    the oracle's energy to 1e-5 of |NCC| + |reg| and measured at ~1e-8)."""
    return lambda u: float(series.eval_energy(frame_i, frame_k, level, np.asarray(u, np.float32),
                                              series=series_index)["E"])


def energy_rel(gpu_energy, gpu_px, orc, R, T, orc_px, lam):
    """(E of the GPU's field, by the GPU - E of the oracle's field, by the
    oracle) / |E of the oracle's field|: every oracle input is the oracle's."""
    side = np.asarray(orc_px).shape[-1] - 1
    eg = gpu_energy(gpu_px)
    eo, _ = orc.energy(R, T, np.asarray(orc_px, np.float64) / side, lam)
    return (eg - eo) / abs(eo), eo


def lock_sequence(rows, level_ns):
    """Accepted step sizes of one oracle operator from its trace rows
    (n, iteration, tau, dE, sigma tau slope, accepted), per level in the order
    of level_ns (coarsest first): the last accepted trial of each iteration is
    the step taken; an iteration without one stalled and ended the level.
    Returns (counts per level, step sizes, the oracle's dE of each step)."""
    counts, taus, dEs = [], [], []
    for n in level_ns:
        r = rows[rows[:, 0] == n]
        cnt = 0
        for it in range(int(r[:, 1].max()) + 1 if len(r) else 0):
            ri = r[r[:, 1] == it]
            acc = ri[ri[:, 5] == 1]
            if len(ri) == 0 or len(acc) == 0:
                break
            taus.append(float(acc[-1, 2]))
            dEs.append(float(acc[-1, 3]))
            cnt += 1
        counts.append(cnt)
    return counts, np.array(taus), np.array(dEs)


def first_flip(gtr, otr):
    """Index of the first Armijo trial whose decision differs (None if none
    within the common prefix); asserts that the trial sequences agree before."""
    m = min(len(gtr), len(otr))
    for k in range(m):
        a, b = gtr[k], otr[k]
        assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2], ("trial sequence differs before any decision", k, a, b)
        if a[5] != b[5]:
            return k
    return None


def perturbed_spread(orc, R, T, p, u_init_omega, orc_px, lam, n=2, seed=0):
    """The oracle's own spread: max |du| (px) between its field and its fields
    for the template perturbed by 1e-7 relative (n draws, solved in parallel
    threads), and the largest relative change of the final energy (the
    unperturbed energy at those fields)."""
    side = R.shape[0] - 1
    rng = np.random.default_rng(seed)
    Ts = [T * (1.0 + PERTURB_REL * rng.standard_normal(T.shape)) for _ in range(n)]

    eo, _ = orc.energy(R, T, np.asarray(orc_px, np.float64) / side, lam)

    def one(Tp):
        u, _, _ = orc.register(R, Tp, p, u_init=u_init_omega)
        ep, _ = orc.energy(R, T, u, lam)
        return float(np.abs(u * side - orc_px).max()), abs(ep - eo) / abs(eo)

    with ThreadPoolExecutor(max_workers=n) as ex:
        res = list(ex.map(one, Ts))
    return max(r[0] for r in res), max(r[1] for r in res)


def free_running_parity(orc, gpu_px, orc_px, gtr, otr, what, R, T, p, lam, gpu_energy, u_init_omega=None):
    """Free-running comparison of one operator (see the module docstring);
    gpu_energy: the GPU's energy of a field (gpu_energy_fn).  Returns the
    record of what was compared."""
    rec = dict(what=what, mode="free", **field_stats(gpu_px, orc_px))
    e_rel, e0 = energy_rel(gpu_energy, gpu_px, orc, R, T, orc_px, lam)
    rec["E_rel"] = e_rel
    if rec["max_px"] <= TOL_PX:
        rec["criterion"] = "fields"
        assert abs(e_rel) <= TOL_E, rec
        return rec
    k = first_flip(gtr, otr)
    if k is None:
        rec["criterion"] = "decisions agree"
        rec["kink_excess_px"] = kink_excess(gpu_px, orc_px)
        rec["beyond"] = beyond_detail(gpu_px, orc_px)
        assert _agreeing_fields_ok(rec), rec
        return rec
    a, b = gtr[k], otr[k]
    margin = abs(b[3] - b[4])
    spread = abs(a[3] - b[3]) + abs(a[4] - b[4])
    rec.update(criterion="flip", flip_index=int(k), flip_margin=margin / abs(e0), flip_spread=spread / abs(e0))
    assert margin < spread, ("decision differs at a non-marginal test", rec, list(a), list(b))
    assert spread <= SPREAD_MAX * abs(e0), ("energy changes disagree beyond rounding", rec)
    sp, sp_e = perturbed_spread(orc, R, T, p, u_init_omega, orc_px, lam)
    rec["oracle_spread_px"] = sp
    rec["oracle_spread_E_rel"] = sp_e
    assert abs(e_rel) <= FLIP_SPREAD_FACTOR * sp_e + TOL_E, ("final energies differ beyond the oracle's own spread", rec)
    assert rec["max_px"] <= FLIP_SPREAD_FACTOR * sp + TOL_PX, ("fields differ beyond the oracle's own spread", rec)
    return rec


def lockstep_parity(orc, series, op, dst, n_levels, otr, orc_px, what, R, T, lam, slot_series=0):
    """Replay the oracle's accepted steps on the GPU for one operator (a
    reg_op_desc tuple writing slot dst) and compare fields, final energies and
    the energy change of every step."""
    side = orc_px.shape[-1] - 1
    L = int(round(np.log2(side)))
    level_ns = [(1 << (L - n_levels + 1 + k)) + 1 for k in range(n_levels)]
    counts, taus, dEs = lock_sequence(otr, level_ns)
    series.set_lockstep([counts], taus)
    series.set_trace(max(16, 2 * len(taus) + 16))
    try:
        series.apply_operator_batch([op])
        gtr = series.get_trace()
    finally:
        series.set_lockstep(None)
    got, _ = series.get_slot(dst, series=slot_series)
    rec = dict(what=what, mode="lockstep", steps=int(len(taus)), **field_stats(got, orc_px))
    e_rel, e0 = energy_rel(gpu_energy_fn(series, op[4], op[5], L, op[0]), got, orc, R, T, orc_px, lam)
    rec["E_rel"] = e_rel
    assert len(gtr) == len(taus), (rec, len(gtr))
    assert np.array_equal(gtr[:, 3], taus), rec
    if len(taus):
        dev = np.abs(gtr[:, 4] - dEs) / (np.abs(dEs) + 1e-9 * abs(e0))
        rec["dE_rel_max"] = float(dev.max())
        rec["dE_rel_median"] = float(np.median(dev))
    rec["kink_excess_px"] = kink_excess(got, orc_px)
    rec["beyond"] = beyond_detail(got, orc_px)
    if rec["max_px"] <= TOL_PX:
        assert abs(e_rel) <= TOL_E, rec
    else:
        assert _agreeing_fields_ok(rec), rec
    return rec
