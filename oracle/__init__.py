"""FP64 CPU oracle for the registration prefix scan (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the arithmetic lives in ``oracle.c`` (plain double precision C written from the
paper's definitions) and the scan bracketing in ``schedules.py``.

Units: the C code works in Omega = [0,1]^2 units on vertex grids; this wrapper
takes frames in pixels and returns displacements in pixels (u_px = u * 2^L),
channel 0 = column (x_0), channel 1 = row (x_1), per node of the (2^L+1)^2 grid.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import schedules

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CONVERGED, MAXITER, LS_STALLED, NONFINITE, ZERO_GRADIENT = range(5)


class Params(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("iter_max", ctypes.c_int32),
                ("epsilon", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("armijo_sigma", ctypes.c_double), ("tau_init", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("tau_min", ctypes.c_double), ("smooth", ctypes.c_double)]


class LevelStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("E_start", ctypes.c_double), ("E", ctypes.c_double), ("tau", ctypes.c_double)]


def params(n_levels=3, iter_max=50, epsilon=1e-7, lam=0.01, armijo_sigma=0.5,
           tau_init=1.0, tau_max=1e4, tau_min=1e-12, smooth=0.0) -> Params:
    """Method parameters: pyramid depth, iteration cap and epsilon (Algorithm
    "Multilevel gradient flow" stopping criteria), regulariser weight lambda,
    Armijo sigma = 0.5 and the step-size bounds (Section "Gradient flow");
    smooth > 0 selects the H1-type smoother of that width (grid spacings)."""
    return Params(n_levels, iter_max, epsilon, lam, armijo_sigma, tau_init, tau_max, tau_min, smooth)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, OpenMP over independent ops)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    vp, i = ctypes.c_void_p, ctypes.c_int
    sig = {
        "orc_embed": ([vp, i, vp], None),
        "orc_restrict": ([vp, i, vp], None),
        "orc_prolong": ([vp, i, vp], None),
        "orc_mass_apply": ([vp, i, vp], None),
        "orc_stiff_apply": ([vp, i, vp], None),
        "orc_lumped": ([i, vp], None),
        "orc_interp": ([vp, i, ctypes.c_double, ctypes.c_double, vp, vp], ctypes.c_double),
        "orc_warp": ([vp, i, vp, vp, vp], None),
        "orc_energy": ([vp, vp, i, vp, ctypes.c_double, vp], ctypes.c_double),
        "orc_gradient": ([vp, vp, i, vp, ctypes.c_double, vp], None),
        "orc_solve_level": ([vp, vp, i, vp, ctypes.POINTER(Params), ctypes.POINTER(LevelStats)], i),
        "orc_register": ([vp, vp, i, vp, ctypes.POINTER(Params), vp, ctypes.POINTER(LevelStats)], i),
        "orc_compose": ([vp, vp, i, vp], None),
        "orc_apply_batch": ([i, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp, vp, vp], None),
        "orc_set_trace": ([vp, ctypes.c_long], None),
        "orc_average": ([i, vp, vp, i, vp], None),
        "orc_smooth_apply": ([i, ctypes.c_double, vp, vp], None),
        "orc_smooth_matvec": ([i, ctypes.c_double, vp, vp], None),
        "orc_rigid_field": ([vp, i, vp], None),
        "orc_rigid_energy": ([vp, vp, i, vp, ctypes.c_double], ctypes.c_double),
        "orc_rigid_gradient": ([vp, vp, i, vp, ctypes.c_double, vp], None),
        "orc_rigid_register": ([vp, vp, i, vp, ctypes.POINTER(Params), vp, ctypes.POINTER(LevelStats)], i),
        "orc_rigid_compose": ([vp, vp, vp], None),
        "orc_trace_len": ([], ctypes.c_long),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data if a is not None else None


# ---------------------------------------------------------------- primitives
def embed(frame):
    frame = np.ascontiguousarray(frame, dtype=np.float32)
    side = frame.shape[0]
    out = np.empty((side + 1, side + 1))
    _load().orc_embed(frame.ctypes.data, side, out.ctypes.data)
    return out


def restrict(fine):
    fine = _c(fine)
    nf = fine.shape[0]
    out = np.empty(((nf + 1) // 2, (nf + 1) // 2))
    _load().orc_restrict(fine.ctypes.data, nf, out.ctypes.data)
    return out


def prolong(coarse):
    coarse = _c(coarse)
    nc = coarse.shape[0]
    out = np.empty((2 * nc - 1, 2 * nc - 1))
    _load().orc_prolong(coarse.ctypes.data, nc, out.ctypes.data)
    return out


def mass_apply(v):
    v = _c(v)
    out = np.empty_like(v)
    _load().orc_mass_apply(v.ctypes.data, v.shape[0], out.ctypes.data)
    return out


def stiff_apply(v):
    v = _c(v)
    out = np.empty_like(v)
    _load().orc_stiff_apply(v.ctypes.data, v.shape[0], out.ctypes.data)
    return out


def lumped(n):
    out = np.empty((n, n))
    _load().orc_lumped(n, out.ctypes.data)
    return out


def interp(T, x0, x1):
    T = _c(T)
    d0, d1 = ctypes.c_double(), ctypes.c_double()
    v = _load().orc_interp(T.ctypes.data, T.shape[0], x0, x1, ctypes.addressof(d0), ctypes.addressof(d1))
    return v, d0.value, d1.value


def warp(T, u):
    """u: (2, n, n) Omega units -> (That (n, n), dT (2, n, n))."""
    T, u = _c(T), _c(u)
    n = T.shape[0]
    Th, dT = np.empty((n, n)), np.empty((2, n, n))
    _load().orc_warp(T.ctypes.data, n, u.ctypes.data, Th.ctypes.data, dT.ctypes.data)
    return Th, dT


def energy(R, T, u, lam):
    """Returns (E, dict of parts) for displacement u (2, n, n) in Omega units."""
    R, T, u = _c(R), _c(T), _c(u)
    parts = np.empty(6)
    E = _load().orc_energy(R.ctypes.data, T.ctypes.data, R.shape[0], u.ctypes.data, lam, parts.ctypes.data)
    keys = ("ncc", "reg", "Rbar", "sigR", "Tbar", "sigT")
    return E, dict(zip(keys, parts.tolist()))


def gradient(R, T, u, lam):
    R, T, u = _c(R), _c(T), _c(u)
    g = np.empty_like(u)
    _load().orc_gradient(R.ctypes.data, T.ctypes.data, R.shape[0], u.ctypes.data, lam, g.ctypes.data)
    return g


def smooth_apply(g, smooth):
    """d = -(M_s (x) M_s)^{-1} g for a nodal gradient g (2, n, n)."""
    g = _c(g)
    d = np.empty_like(g)
    _load().orc_smooth_apply(g.shape[1], smooth, g.ctypes.data, d.ctypes.data)
    return d


def smooth_matvec(v, smooth):
    """(M_s (x) M_s) v for one plane v (n, n)."""
    v = _c(v)
    out = np.empty_like(v)
    _load().orc_smooth_matvec(v.shape[0], smooth, v.ctypes.data, out.ctypes.data)
    return out


def solve_level(R, T, u, p: Params):
    R, T = _c(R), _c(T)
    u = _c(u).copy()
    st = LevelStats()
    _load().orc_solve_level(R.ctypes.data, T.ctypes.data, R.shape[0], u.ctypes.data,
                            ctypes.byref(p), ctypes.byref(st))
    return u, st


def register(R, T, p: Params, u_init=None):
    """Function A on level-L grids R, T ((2^L+1)^2); u in Omega units."""
    R, T = _c(R), _c(T)
    n = R.shape[0]
    L = int(round(np.log2(n - 1)))
    out = np.empty((2, n, n))
    st = (LevelStats * p.n_levels)()
    ui = _c(u_init) if u_init is not None else None
    s = _load().orc_register(R.ctypes.data, T.ctypes.data, L, _ptr(ui), ctypes.byref(p),
                             out.ctypes.data, st)
    return out, s, [st[i] for i in range(p.n_levels)]


class trace:
    """Context manager recording every Armijo trial of the level solves that
    the calling thread runs inside it (the trace is per host thread, so several
    threads may each trace their own operator): rows (n, iteration, tau, dE,
    sigma tau slope, accepted)."""

    def __init__(self, cap=1 << 20):
        self.buf = np.zeros((cap, 6))

    def __enter__(self):
        _load().orc_set_trace(self.buf.ctypes.data, self.buf.shape[0])
        return self

    def __exit__(self, *a):
        lib = _load()
        self.rows = self.buf[:lib.orc_trace_len()].copy()
        lib.orc_set_trace(None, 0)


def compose(u_ij, u_jk):
    u_ij, u_jk = _c(u_ij), _c(u_jk)
    out = np.empty_like(u_ij)
    _load().orc_compose(u_ij.ctypes.data, u_jk.ctypes.data, u_ij.shape[1], out.ctypes.data)
    return out


def apply_batch(ops, p: Params):
    """ops: list of dicts with R, T (level-L nodal grids), and optional left,
    right (Omega-unit fields).  Returns (outputs, status, iters, trials, energy)."""
    lib = _load()
    n = len(ops)
    keep = []
    arrs = {k: (ctypes.c_void_p * n)() for k in ("R", "T", "left", "right", "out")}
    L = np.empty(n, dtype=np.int32)
    outs = []
    for i, o in enumerate(ops):
        R, T = _c(o["R"]), _c(o["T"])
        nn = R.shape[0]
        L[i] = int(round(np.log2(nn - 1)))
        out = np.empty((2, nn, nn))
        outs.append(out)
        keep += [R, T]
        arrs["R"][i], arrs["T"][i], arrs["out"][i] = R.ctypes.data, T.ctypes.data, out.ctypes.data
        for k in ("left", "right"):
            v = o.get(k)
            if v is not None:
                v = _c(v)
                keep.append(v)
                arrs[k][i] = v.ctypes.data
            else:
                arrs[k][i] = None
    status = np.empty(n, dtype=np.int32)
    iters = np.empty(n, dtype=np.int32)
    trials = np.empty(n, dtype=np.int32)
    en = np.empty(n)
    lib.orc_apply_batch(n, arrs["R"], arrs["T"], L.ctypes.data, arrs["left"], arrs["right"],
                        arrs["out"], ctypes.byref(p), status.ctypes.data, iters.ctypes.data,
                        trials.ctypes.data, en.ctypes.data)
    return outs, status, iters, trials, en


# ------------------------------------------------------------- series driver
def register_series(series_frames, p: Params, kind=schedules.SERIAL, chunks=8,
                    global_kind=schedules.KOGGE_STONE, return_info=False):
    """Image series registration (Definition "Image series registration"):
    preprocessing x_e = A(f_e, f_{e+1}, I), then the prefix scan of B over
    x_0..x_{N-1} with the chosen schedule; several series form one segmented
    scan (levels of the per-series schedules run together, never across series).

    series_frames: list of arrays (n_frames, side, side).  Returns a list of
    (n_frames, 2, side+1, side+1) displacement fields in pixels, entry 0 the
    identity, entry k = phi_{0,k} - id."""
    grids, Ls = [], []
    for fr in series_frames:
        grids.append([embed(f) for f in fr])
        Ls.append(int(round(np.log2(fr.shape[1]))))
    # slot: (start_frame, end_frame, field or None for the identity)
    slots = []
    pre = []
    for s, g in enumerate(grids):
        N = len(g) - 1
        na = schedules.aux_slots(kind, N, chunks, global_kind)
        slots.append([None] * (N + na))
        for e in range(N):
            pre.append((s, e, dict(R=g[e], T=g[e + 1])))
    outs, st, it, tr, en = apply_batch([o for _, _, o in pre], p)
    info = dict(ops=len(pre), levels=0, status=list(st), iters=list(it), trials=list(tr))
    for (s, e, _), u in zip(pre, outs):
        slots[s][e] = (e, e + 1, u)
    scheds = [schedules.schedule(kind, len(g) - 1, chunks, global_kind) for g in grids]
    for t in range(max((len(x) for x in scheds), default=0)):
        batch, where, writes = [], [], []
        for s, sc in enumerate(scheds):
            if t >= len(sc):
                continue
            cur = slots[s]
            for o in sc[t]:
                if o[0] == "id":
                    writes.append((s, o[1], "id"))
                elif o[0] == "copy":
                    writes.append((s, o[1], cur[o[2]]))
                else:
                    a, b = cur[o[2]], cur[o[3]]
                    if a == "id":
                        writes.append((s, o[1], b))
                    elif b == "id":
                        writes.append((s, o[1], a))
                    else:
                        if a[1] != b[0]:
                            raise RuntimeError("chain mismatch in schedule")
                        g = grids[s]
                        batch.append(dict(R=g[a[0]], T=g[b[1]], left=a[2], right=b[2]))
                        where.append((s, o[1], a[0], b[1]))
        if batch:
            outs, st, it, tr, en = apply_batch(batch, p)
            info["ops"] += len(batch)
            info["levels"] += 1
            info["status"] += list(st)
            info["iters"] += list(it)
            info["trials"] += list(tr)
            for (s, dst, i0, k1), u in zip(where, outs):
                writes.append((s, dst, (i0, k1, u)))
        for s, dst, v in writes:
            slots[s][dst] = v
    results = []
    for s, g in enumerate(grids):
        N = len(g) - 1
        side = series_frames[s].shape[1]
        n = side + 1
        res = np.zeros((N + 1, 2, n, n))
        for e in range(N):
            v = slots[s][e]
            assert v != "id" and v[0] == 0 and v[1] == e + 1, "scan did not produce phi_{0,k}"
            res[e + 1] = v[2] * side
        results.append(res)
    if return_info:
        return results, info
    return results


# ------------------------------------------------------------ series averaging
def average(grids, fields):
    """Average of the deformed frames: grids are embedded frames (n x n nodal
    values), fields their displacements (2, n, n) in Omega units or None for
    the identity; returns the n x n nodal average of F_k o (id + u_k)."""
    m = len(grids)
    n = grids[0].shape[0]
    keep = [_c(g) for g in grids]
    ks = [None if f is None else _c(f) for f in fields]
    Fp = (ctypes.c_void_p * m)(*[g.ctypes.data for g in keep])
    Up = (ctypes.c_void_p * m)(*[None if f is None else f.ctypes.data for f in ks])
    out = np.empty((n, n))
    _load().orc_average(m, Fp, Up, n, out.ctypes.data)
    return out


def average_series(frames, p: Params, iterations=1, kind=schedules.SKLANSKY):
    """The series averaging procedure: register the series (preprocessing and
    prefix scan), average the deformed frames f_k o phi_{0,k} (phi_{0,0} the
    identity), then `iterations` times register every frame to the current
    average with function A, started from its current deformation, and average
    again.  frames: (m, side, side).  Returns (average n x n nodal, fields
    (m, 2, n, n) in pixels: the deformations from the last average's frame to
    each frame, or phi_{0,k} when iterations = 0)."""
    side = frames.shape[1]
    grids = [embed(f) for f in frames]
    phi = register_series([frames], p, kind=kind)[0] / side  # (m, 2, n, n) Omega units
    fields = [None] + [phi[k] for k in range(1, len(grids))]
    avg = average(grids, fields)
    for _ in range(iterations):
        ops = [dict(R=avg, T=grids[k], left=(np.zeros_like(phi[0]) if fields[k] is None else fields[k]))
               for k in range(len(grids))]
        outs, _, _, _, _ = apply_batch(ops, p)
        fields = outs
        avg = average(grids, fields)
    return avg, np.stack([np.zeros_like(phi[0]) if f is None else f for f in fields]) * side


# ------------------------------------------------------------- rigid variant
def rigid_field(theta, n):
    """u(x) = R(alpha) x + t - x at the n x n nodes, Omega units; theta =
    (alpha, t0, t1) with t in Omega units."""
    th = _c(theta)
    out = np.empty((2, n, n))
    _load().orc_rigid_field(th.ctypes.data, n, out.ctypes.data)
    return out


def rigid_energy(R, T, theta, lam):
    R, T, th = _c(R), _c(T), _c(theta)
    return _load().orc_rigid_energy(R.ctypes.data, T.ctypes.data, R.shape[0], th.ctypes.data, lam)


def rigid_gradient(R, T, theta, lam):
    R, T, th = _c(R), _c(T), _c(theta)
    g = np.empty(3)
    _load().orc_rigid_gradient(R.ctypes.data, T.ctypes.data, R.shape[0], th.ctypes.data, lam, g.ctypes.data)
    return g


def rigid_register(R, T, p: Params, theta_init=None):
    """Rigid function A on level-L grids: returns (theta, status, level stats)."""
    R, T = _c(R), _c(T)
    n = R.shape[0]
    L = int(round(np.log2(n - 1)))
    out = np.empty(3)
    st = (LevelStats * p.n_levels)()
    ti = _c(theta_init) if theta_init is not None else None
    s = _load().orc_rigid_register(R.ctypes.data, T.ctypes.data, L, _ptr(ti), ctypes.byref(p), out.ctypes.data, st)
    return out, s, [st[i] for i in range(p.n_levels)]


def rigid_compose(a, b):
    """phi_b o phi_a (a applied first) of rigid parameters."""
    a, b = _c(a), _c(b)
    out = np.empty(3)
    _load().orc_rigid_compose(a.ctypes.data, b.ctypes.data, out.ctypes.data)
    return out


def rigid_register_series(frames, p: Params, kind=schedules.SERIAL, chunks=8, global_kind=schedules.KOGGE_STONE):
    """Image series registration with the rigid operator: preprocessing
    x_e = A(f_e, f_{e+1}, I), then the prefix scan of
    B(a, b) = A(f_i, f_k, b o a) with the chosen schedule.  Returns
    (n_frames, 3) parameters of phi_{0,k} (row 0 the identity)."""
    grids = [embed(f) for f in frames]
    N = len(grids) - 1
    na = schedules.aux_slots(kind, N, chunks, global_kind)
    slots = [None] * (N + na)
    for e in range(N):
        th, _, _ = rigid_register(grids[e], grids[e + 1], p)
        slots[e] = (e, e + 1, th)
    for lev in schedules.schedule(kind, N, chunks, global_kind):
        writes = []
        for o in lev:
            if o[0] == "id":
                writes.append((o[1], "id"))
            elif o[0] == "copy":
                writes.append((o[1], slots[o[2]]))
            else:
                a, b = slots[o[2]], slots[o[3]]
                if a == "id":
                    writes.append((o[1], b))
                elif b == "id":
                    writes.append((o[1], a))
                else:
                    th, _, _ = rigid_register(grids[a[0]], grids[b[1]], p, rigid_compose(a[2], b[2]))
                    writes.append((o[1], (a[0], b[1], th)))
        for dst, v in writes:
            slots[dst] = v
    out = np.zeros((N + 1, 3))
    for e in range(N):
        assert slots[e][0] == 0 and slots[e][1] == e + 1
        out[e + 1] = slots[e][2]
    return out
