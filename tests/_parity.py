"""Helpers shared by the GPU parity tests (CUDA path against the FP64 oracle).

Two ways of comparing one operator application (function A or B):

* Free running.  Both sides search their own Armijo steps (Section "Gradient
  flow").  On noisy frames the iteration is chaotic: a decision whose margin is
  at the rounding level sends two correct implementations to different, equally
  good fields (Section "A note on the associativity" notes that results differ
  among implementations).  ``free_running_parity`` therefore accepts one of
    1. max |du| <= TOL_PX at every node;
    2. every Armijo decision agrees, >= 99.5% of the nodes within TOL_PX, the
       others on a cell line of the bilinear interpolant (where the template's
       derivative jumps, so that the side a node driven there lands on is
       decided at the rounding level) and within AGREE_CAP_PX, and the final
       energies within TOL_E;
    3. the decisions agree up to one whose oracle margin is smaller than the
       disagreement of the two sides' energy changes at that point (no slack),
       that disagreement is itself at the rounding level (SPREAD_MAX relative to
       the energy), and afterwards the final energies agree within FLIP_E_REL
       and max |du| stays within FLIP_SPREAD_FACTOR times the oracle's own
       spread under 1e-7 relative perturbations of the template frame (plus
       TOL_PX).
* Lockstep.  The GPU replays the oracle's accepted step sizes
  (reg_set_lockstep); no decision is taken, so the fields must agree to
  TOL_PX and the final energies to TOL_E, for every operator -- except at the
  few nodes (< 0.5%) that the flow drives onto a cell line of the bilinear
  interpolant, where the template's derivative jumps and the side a node
  takes is decided at the rounding level even along the same steps; each such
  node must lie within its own difference of a cell line, and within
  AGREE_CAP_PX.

Every comparison returns a record (max, 99th percentile and mean |du| in px,
relative final-energy difference) that the tests print on one line each.
"""
from __future__ import annotations

import json
from concurrent.futures import ThreadPoolExecutor

import numpy as np

TOL_PX = 1e-3        # spec tolerance on displacements, FP32 plain form
TOL_E = 1e-5         # spec tolerance on the final energy, relative
AGREE_CAP_PX = 0.05  # all decisions agree: bound on the few cell-line nodes
SPREAD_MAX = 1e-6    # a flip is excused only if the two energy changes agree to this (relative to |E|)
FLIP_E_REL = 1e-5    # after an excused flip: final energies (oracle FP64 at both fields)
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
    decaying difference to the nodes around it (over the iterations, to
    neighbours of neighbours too).  So every cluster of differing nodes (nodes
    at most two apart joined) must peak at a node that lies on a cell line:
    within its own difference of one (in the oracle's or the GPU's position).
    Returns the largest excess of that distance over the peak's difference
    (<= 0 when every cluster is explained so)."""
    from scipy import ndimage
    g = np.asarray(gpu_px, np.float64)
    o = np.asarray(orc_px, np.float64)
    d = np.abs(g - o).max(axis=0)  # per node, the larger component difference
    m = d > TOL_PX
    if not m.any():
        return 0.0
    dist = np.minimum(np.abs(o - np.round(o)), np.abs(g - np.round(g))).min(axis=0)
    joined = ndimage.binary_dilation(m, structure=np.ones((3, 3)))
    lab, n = ndimage.label(joined, structure=np.ones((3, 3)))
    worst = -np.inf
    for k in range(1, n + 1):
        sel = (lab == k) & m
        idx = np.argwhere(sel)
        r, c = idx[np.argmax(d[sel])]
        worst = max(worst, float(dist[r, c] - d[r, c]))
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
    """Fields of two runs that took the same steps: all but a few nodes within
    TOL_PX, those few on cell lines and within AGREE_CAP_PX, and the GPU's
    field as good a minimiser of the oracle's energy (TOL_E)."""
    return (rec["frac_within"] >= 0.995 and rec["p99_px"] <= TOL_PX and rec["max_px"] <= AGREE_CAP_PX
            and rec["kink_excess_px"] <= 0.0 and abs(rec["E_rel"]) <= TOL_E)


def energy_rel(orc, R, T, gpu_px, orc_px, lam):
    """Oracle FP64 energy at both fields: (E at the GPU field - E at the oracle
    field) / |E at the oracle field|."""
    side = gpu_px.shape[-1] - 1
    eg, _ = orc.energy(R, T, np.asarray(gpu_px, np.float64) / side, lam)
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


def perturbed_spread(orc, R, T, p, u_init_omega, orc_px, n=2, seed=0):
    """Max |du| (px) between the oracle's field and the oracle's fields for the
    template perturbed by 1e-7 relative (n draws, solved in parallel threads)."""
    side = R.shape[0] - 1
    rng = np.random.default_rng(seed)
    Ts = [T * (1.0 + PERTURB_REL * rng.standard_normal(T.shape)) for _ in range(n)]

    def one(Tp):
        u, _, _ = orc.register(R, Tp, p, u_init=u_init_omega)
        return float(np.abs(u * side - orc_px).max())

    with ThreadPoolExecutor(max_workers=n) as ex:
        return max(ex.map(one, Ts))


def free_running_parity(orc, gpu_px, orc_px, gtr, otr, what, R, T, p, lam, u_init_omega=None):
    """Free-running comparison of one operator (see the module docstring).
    Returns the record of what was compared."""
    rec = dict(what=what, mode="free", **field_stats(gpu_px, orc_px))
    e_rel, e0 = energy_rel(orc, R, T, gpu_px, orc_px, lam)
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
    sp = perturbed_spread(orc, R, T, p, u_init_omega, orc_px)
    rec["oracle_spread_px"] = sp
    assert abs(e_rel) <= FLIP_E_REL, ("final energies differ after a marginal flip", rec)
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
    e_rel, e0 = energy_rel(orc, R, T, got, orc_px, lam)
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
