"""Python binding of libreg (GB300 registration prefix scan).

Argument marshalling only: every step of the registration runs in libreg's
CUDA kernels.  PyTorch provides the CUDA stream and device memory (its caching
allocator is handed to the library).  The functions mirror the C-ABI declared
in ``include/reg.h``; ``Series`` wraps a handle.

The library must be built (``__graft_entry__.build()`` or
``python -m paper_1712_02533_gb300._build``); importing this package on a
machine without ``libreg.so`` raises ImportError instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libreg.so")

# reg_status
OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, EKERNEL = range(7)
# reg_op_status
OP_CONVERGED, OP_MAXITER, OP_LS_STALLED, OP_NONFINITE, OP_ZERO_GRADIENT = range(5)
# reg_scan_kind
SERIAL, SKLANSKY, KOGGE_STONE, BRENT_KUNG, BLELLOCH, CHUNKED, CHUNKED_ALT, HAN_CARLSON, LADNER_FISCHER = range(9)
SCAN_NAMES = {SERIAL: "serial", SKLANSKY: "sklansky", KOGGE_STONE: "kogge_stone", BRENT_KUNG: "brent_kung",
              BLELLOCH: "blelloch", CHUNKED: "chunked", CHUNKED_ALT: "chunked_alt", HAN_CARLSON: "han_carlson",
              LADNER_FISCHER: "ladner_fischer"}
STORAGE_F32, STORAGE_BF16 = 0, 1
FLAG_PROFILE = 1
FLAG_RIGID = 2

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("iter_max", ctypes.c_int32), ("epsilon", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("armijo_sigma", ctypes.c_double), ("tau_init", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("tau_min", ctypes.c_double), ("storage", ctypes.c_int32),
                ("trials_per_pass", ctypes.c_int32), ("max_steps", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("init_levels", ctypes.c_int32), ("learned_fallback_px", ctypes.c_double),
                ("allocator", Allocator), ("smooth", ctypes.c_double)]


class OpDesc(ctypes.Structure):
    _fields_ = [("series", ctypes.c_int32), ("left_slot", ctypes.c_int32), ("right_slot", ctypes.c_int32),
                ("dst_slot", ctypes.c_int32), ("frame_i", ctypes.c_int32), ("frame_k", ctypes.c_int32)]


class ScheduleOp(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("kind", ctypes.c_int32), ("dst", ctypes.c_int32),
                ("a", ctypes.c_int32), ("b", ctypes.c_int32)]


class KernelStats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("items", ctypes.c_int64)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libreg.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "reg_default_params": ([P(Params)], None),
        "reg_create_series": ([vp, i32, vp, vp, i64, i32, P(Params), vp, P(vp)], ctypes.c_int),
        "reg_apply_operator_batch": ([vp, i32, vp, vp, vp], ctypes.c_int),
        "reg_prefix_scan": ([vp, ctypes.c_int, i32, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "reg_set_tile_rows": ([vp, i32, i32, i32], ctypes.c_int),
        "reg_get_tile_rows": ([vp, i32, P(i32), P(i32)], ctypes.c_int),
        "reg_autotune": ([vp, i32, i32, i32, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "reg_get_deformations": ([vp, i32, i32, i32, vp, i32], ctypes.c_int),
        "reg_get_slot": ([vp, i32, i32, vp, i32, vp], ctypes.c_int),
        "reg_set_slot": ([vp, i32, i32, vp, i32, i32, i32], ctypes.c_int),
        "reg_num_slots": ([vp, i32, P(i32)], ctypes.c_int),
        "reg_eval_energy": ([vp, i32, i32, i32, i32, vp, vp], ctypes.c_int),
        "reg_eval_direction": ([vp, i32, i32, i32, i32, vp, vp, P(d)], ctypes.c_int),
        "reg_eval_trials": ([vp, i32, i32, i32, i32, vp, i32, vp, vp, vp], ctypes.c_int),
        "reg_schedule": ([ctypes.c_int, i32, i32, ctypes.c_int, vp, i64, P(i64), P(i32)], ctypes.c_int),
        "reg_get_kernel_stats": ([vp, vp, i32, P(i32)], ctypes.c_int),
        "reg_reset_kernel_stats": ([vp], ctypes.c_int),
        "reg_set_trace": ([vp, i64], ctypes.c_int),
        "reg_get_trace": ([vp, vp, i64, P(i64)], ctypes.c_int),
        "reg_set_lockstep": ([vp, i32, i32, vp, vp], ctypes.c_int),
        "reg_set_flags": ([vp, i32], ctypes.c_int),
        "reg_average_series": ([vp, i32, i32, vp, i32], ctypes.c_int),
        "reg_get_rigid": ([vp, i32, i32, vp, vp], ctypes.c_int),
        "reg_set_rigid": ([vp, i32, i32, vp, i32, i32], ctypes.c_int),
        "reg_eval_energy_noalloc": ([vp, vp, i32, i32, vp, d, vp, i32, vp], ctypes.c_int),
        "reg_destroy_series": ([vp], ctypes.c_int),
        "reg_cnn_num_params": ([], i64),
        "reg_cnn_create": ([i32, i32, vp, P(vp)], ctypes.c_int),
        "reg_cnn_set_params": ([vp, vp, i32], ctypes.c_int),
        "reg_cnn_get_params": ([vp, vp, i32], ctypes.c_int),
        "reg_cnn_forward": ([vp, vp, i32, vp, i32], ctypes.c_int),
        "reg_cnn_loss_grad": ([vp, vp, vp, i32, P(d), vp], ctypes.c_int),
        "reg_cnn_adam_step": ([vp, d, d, d, d], ctypes.c_int),
        "reg_cnn_loss_grad_tc": ([vp, vp, vp, i32, P(d), vp], ctypes.c_int),
        "reg_cnn_destroy": ([vp], ctypes.c_int),
        "reg_cnn_pairs": ([vp, i32, i32, i32, vp], ctypes.c_int),
        "reg_cnn_init_series": ([vp, i32, vp, i32], ctypes.c_int),
        "reg_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "reg_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def build(force: bool = False) -> str:
    return _build.build(force=force)


class RegError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _check(code):
    if code != OK:
        lib = _load()
        raise RegError(code, f"{lib.reg_status_string(code).decode()}: {lib.reg_last_error().decode()}")


def default_params(**kw) -> Params:
    p = Params()
    _load().reg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


# --- torch plumbing: stream and caching allocator --------------------------------
def _torch():
    import torch
    return torch


_keep = []


def _torch_allocator(device):
    torch = _torch()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a = Allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)
    _keep.append(a)
    return a


def _stream_ptr(stream):
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(st.cuda_stream)


def _ptr(x):
    """(pointer, on_device) of a contiguous numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data, 0
    return x.data_ptr(), int(x.is_cuda)


# --- C-ABI mirrors ----------------------------------------------------------------
def create_series(frames, frames_per_series, side_px, params: Params | None = None, stream=None,
                  use_torch_allocator=True):
    """frames: float32 (total_frames, side, side) numpy array (host) or torch
    tensor (host or CUDA), all series back to back with a common row pitch."""
    lib = _load()
    torch = _torch()
    p = params if params is not None else default_params()
    if stream is None:
        stream = torch.cuda.current_stream()
    if use_torch_allocator and not p.allocator.alloc:
        p.allocator = _torch_allocator(torch.cuda.current_device())
    if isinstance(frames, np.ndarray):
        frames = np.ascontiguousarray(frames, dtype=np.float32)
    else:
        frames = frames.contiguous()
        assert frames.dtype == torch.float32
    pitch = frames.shape[-1]
    fps = (ctypes.c_int32 * len(frames_per_series))(*frames_per_series)
    sides = (ctypes.c_int32 * len(side_px))(*side_px)
    ptr, on_dev = _ptr(frames)
    h = ctypes.c_void_p()
    _check(lib.reg_create_series(ptr, len(frames_per_series), fps, sides, pitch, on_dev, ctypes.byref(p),
                                 ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
    return h, p


def apply_operator_batch(h, ops):
    lib = _load()
    n = len(ops)
    arr = (OpDesc * n)(*[OpDesc(*o) for o in ops])
    st = np.empty(n, np.int32)
    it = np.empty(n, np.int32)
    _check(lib.reg_apply_operator_batch(h, n, arr, st.ctypes.data, it.ctypes.data))
    return st, it


def prefix_scan(h, kind=SERIAL, chunks=None, global_kind=KOGGE_STONE):
    """chunks: chunk count of the chunked kinds (default 16), k of Han-Carlson
    and Ladner-Fischer (default 1)."""
    if chunks is None:
        chunks = 1 if kind in (HAN_CARLSON, LADNER_FISCHER) else 16
    buf = ctypes.create_string_buffer(4096)
    _check(_load().reg_prefix_scan(h, kind, chunks, global_kind, buf, len(buf)))
    return json.loads(buf.value.decode())


def get_deformations(h, series, first, count, side, out=None):
    if out is None:
        out = np.empty((count, 2, side, side), np.float32)
    ptr, on_dev = _ptr(out)
    _check(_load().reg_get_deformations(h, series, first, count, ptr, on_dev))
    return out


def get_slot(h, series, slot, side):
    out = np.empty((2, side + 1, side + 1), np.float32)
    se = np.empty(2, np.int32)
    _check(_load().reg_get_slot(h, series, slot, out.ctypes.data, 0, se.ctypes.data))
    return out, (int(se[0]), int(se[1]))


def set_slot(h, series, slot, field, start, end):
    f = None if field is None else np.ascontiguousarray(field, np.float32)
    _check(_load().reg_set_slot(h, series, slot, None if f is None else f.ctypes.data, 0, start, end))


def num_slots(h, series=0):
    n = ctypes.c_int32()
    _check(_load().reg_num_slots(h, series, ctypes.byref(n)))
    return n.value


def eval_energy(h, series, frame_i, frame_k, level, u_grid):
    u = np.ascontiguousarray(u_grid, np.float32)
    parts = np.empty(5)
    _check(_load().reg_eval_energy(h, series, frame_i, frame_k, level, u.ctypes.data, parts.ctypes.data))
    return dict(E=parts[0], ncc=parts[1], reg=parts[2], Tbar=parts[3], sigT=parts[4])


def eval_direction(h, series, frame_i, frame_k, level, u_grid):
    u = np.ascontiguousarray(u_grid, np.float32)
    d = np.empty_like(u)
    sl = ctypes.c_double()
    _check(_load().reg_eval_direction(h, series, frame_i, frame_k, level, u.ctypes.data, d.ctypes.data,
                                      ctypes.byref(sl)))
    return d, sl.value


def eval_trials(h, series, frame_i, frame_k, level, u_grid, taus):
    """One gradient pass and one trial pass at u: returns (d, dE) with dE[j] the
    energy change for step size taus[j] as the Armijo search forms it."""
    u = np.ascontiguousarray(u_grid, np.float32)
    t = np.ascontiguousarray(taus, np.float64)
    d = np.empty_like(u)
    dE = np.empty(len(t))
    _check(_load().reg_eval_trials(h, series, frame_i, frame_k, level, u.ctypes.data, len(t), t.ctypes.data,
                                   d.ctypes.data, dE.ctypes.data))
    return d, dE


def schedule(kind, n, chunks=0, global_kind=KOGGE_STONE):
    """Op list of a scan schedule: list of levels of (kind, dst, a, b); kind
    'op' | 'copy' | 'id' as in the oracle's schedules module."""
    lib = _load()
    cnt = ctypes.c_int64()
    aux = ctypes.c_int32()
    _check(lib.reg_schedule(kind, n, chunks, global_kind, None, 0, ctypes.byref(cnt), ctypes.byref(aux)))
    buf = (ScheduleOp * max(1, cnt.value))()
    _check(lib.reg_schedule(kind, n, chunks, global_kind, buf, cnt.value, ctypes.byref(cnt), ctypes.byref(aux)))
    levels = []
    names = {0: "op", 1: "copy", 2: "id"}
    for k in range(cnt.value):
        o = buf[k]
        while len(levels) <= o.level:
            levels.append([])
        t = names[o.kind]
        levels[o.level].append((t, o.dst, o.a, o.b) if t == "op" else ((t, o.dst, o.a) if t == "copy" else (t, o.dst)))
    return levels, aux.value


def get_kernel_stats(h):
    buf = (KernelStats * 16)()
    n = ctypes.c_int32()
    _check(_load().reg_get_kernel_stats(h, buf, 16, ctypes.byref(n)))
    return {buf[k].name.decode(): dict(launches=buf[k].launches, ms=buf[k].ms, bytes=buf[k].bytes,
                                       items=buf[k].items) for k in range(n.value)}


def reset_kernel_stats(h):
    _check(_load().reg_reset_kernel_stats(h))


def set_trace(h, capacity):
    _check(_load().reg_set_trace(h, capacity))


def get_trace(h):
    """Armijo trial records: rows (op, n, iteration, tau, dE, sigma tau slope, accepted)."""
    n = ctypes.c_int64()
    _check(_load().reg_get_trace(h, None, 0, ctypes.byref(n)))
    out = np.empty((max(1, n.value), 7))
    _check(_load().reg_get_trace(h, out.ctypes.data, n.value, ctypes.byref(n)))
    return out[:n.value]


def set_lockstep(h, counts, taus):
    """Lockstep replay for the next batches: counts (n_ops, n_levels) accepted
    steps per op and level (coarsest first), taus the step sizes in op, level,
    iteration order.  counts=None switches it off."""
    if counts is None:
        _check(_load().reg_set_lockstep(h, 0, 0, None, None))
        return
    c = np.ascontiguousarray(counts, np.int32)
    t = np.ascontiguousarray(taus, np.float64)
    assert c.ndim == 2 and t.size == int(c.sum())
    _check(_load().reg_set_lockstep(h, c.shape[0], c.shape[1], c.ctypes.data, t.ctypes.data if t.size else None))


def eval_energy_noalloc(R, T, u_grid, lam, stream=None):
    """Energy of one pair at one level through the allocation-free entry point.
    R, T: CUDA float32 tensors (n, n) of the level's raw images; u_grid: CUDA
    float32 tensor (2, n, n) in grid units.  Returns the same dict as
    eval_energy.  The caller owns every buffer; the library allocates none."""
    torch = _torch()
    n = int(R.shape[-1])
    assert R.is_cuda and T.is_cuda and u_grid.is_cuda
    # the kernels read n x n nodes of R and T and 2 x n x n of u: smaller buffers
    # would be read past their end on the device
    assert tuple(R.shape) == (n, n) and tuple(T.shape) == (n, n) and tuple(u_grid.shape) == (2, n, n)
    assert R.dtype == T.dtype == u_grid.dtype == torch.float32
    R, T, u = R.contiguous(), T.contiguous(), u_grid.contiguous()
    parts = np.empty(5)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(_load().reg_eval_energy_noalloc(R.data_ptr(), T.data_ptr(), n, n, u.data_ptr(), lam,
                                           parts.ctypes.data, 0, ctypes.c_void_p(st.cuda_stream)))
    return dict(E=parts[0], ncc=parts[1], reg=parts[2], Tbar=parts[3], sigT=parts[4])


def destroy_series(h):
    _check(_load().reg_destroy_series(h))


class Cnn:
    """The learned initialiser (C-ABI reg_cnn_*): a network for side x side input
    pairs (side a multiple of 4) and batches of up to max_batch pairs.  Device
    tensors in and out (torch CUDA tensors, float32, contiguous)."""

    def __init__(self, params=None, side=256, max_batch=64, stream=None):
        lib = _load()
        h = ctypes.c_void_p()
        _check(lib.reg_cnn_create(side, max_batch, _stream_ptr(stream), ctypes.byref(h)))
        self.h, self.side, self.max_batch = h, side, max_batch
        if params is not None:
            self.set_params(params)

    @staticmethod
    def num_params():
        return int(_load().reg_cnn_num_params())

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, np.float32)
        assert theta.size == self.num_params()
        _check(_load().reg_cnn_set_params(self.h, theta.ctypes.data, 0))

    def get_params(self):
        out = np.empty(self.num_params(), np.float32)
        _check(_load().reg_cnn_get_params(self.h, out.ctypes.data, 0))
        return out

    def forward(self, x, y=None, tensor_cores=False):
        torch = _torch()
        b = int(x.shape[0])
        if y is None:
            y = torch.empty((b, 2, self.side // 4, self.side // 4), dtype=torch.float32, device=x.device)
        _check(_load().reg_cnn_forward(self.h, x.data_ptr(), b, y.data_ptr(), int(bool(tensor_cores))))
        return y

    def loss_grad(self, x, target, want_grad=False, tensor_cores=False):
        loss = ctypes.c_double()
        g = np.empty(self.num_params(), np.float32) if want_grad else None
        fn = _load().reg_cnn_loss_grad_tc if tensor_cores else _load().reg_cnn_loss_grad
        _check(fn(self.h, x.data_ptr(), target.data_ptr(), int(x.shape[0]), ctypes.byref(loss),
                  g.ctypes.data if want_grad else None))
        return (loss.value, g) if want_grad else loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(_load().reg_cnn_adam_step(self.h, lr, beta1, beta2, eps))

    def close(self):
        if self.h:
            _load().reg_cnn_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Series:
    """A handle over one or several frame series (one segmented scan)."""

    def __init__(self, series_frames, params: Params | None = None, stream=None, use_torch_allocator=True):
        if not isinstance(series_frames, (list, tuple)):
            series_frames = [series_frames]
        self.sides = [int(f.shape[-1]) for f in series_frames]
        self.counts = [int(f.shape[0]) for f in series_frames]
        pitch = max(self.sides)
        if isinstance(series_frames[0], np.ndarray):
            if len(set(self.sides)) == 1:
                frames = np.ascontiguousarray(np.concatenate(series_frames), dtype=np.float32)
            else:
                frames = np.zeros((sum(self.counts), pitch, pitch), np.float32)
                o = 0
                for f in series_frames:
                    n, s = f.shape[0], f.shape[-1]
                    # series s occupies rows of side s with the common pitch
                    flat = np.zeros((n * s, pitch), np.float32)
                    flat[:, :s] = f.reshape(n * s, s)
                    frames.reshape(-1, pitch)[o:o + n * s] = flat
                    o += n * s
        else:
            torch = _torch()
            if len(set(self.sides)) != 1:
                raise ValueError("mixed sides need host frames")
            # one tensor passes through as a view (a pinned host tensor stays
            # pinned, so the upload is a direct DMA); several are concatenated
            flat = [f.reshape(-1, f.shape[-1]) for f in series_frames]
            frames = flat[0] if len(flat) == 1 else torch.cat(flat)
        self.h, self.params = create_series(frames, self.counts, self.sides, params, stream, use_torch_allocator)

    def apply_operator_batch(self, ops):
        return apply_operator_batch(self.h, ops)

    def prefix_scan(self, kind=SERIAL, chunks=None, global_kind=KOGGE_STONE):
        return prefix_scan(self.h, kind, chunks, global_kind)

    def get_deformations(self, series=0, first=0, count=None, out=None):
        if count is None:
            count = self.counts[series] - first
        return get_deformations(self.h, series, first, count, self.sides[series], out)

    def average(self, iterations=0, series=0, out=None):
        """Series averaging after prefix_scan: the average of the deformed
        frames (side x side float32), after `iterations` rounds of registering
        every frame to the average (C-ABI reg_average_series)."""
        side = self.sides[series]
        if out is None:
            out = np.empty((side, side), np.float32)
        ptr, on_dev = _ptr(out)
        _check(_load().reg_average_series(self.h, series, iterations, ptr, on_dev))
        return out

    def n_slots(self, series=0):
        return num_slots(self.h, series)

    def get_slot_device(self, slot, series=0):
        """A slot's field as a CUDA tensor (2, side+1, side+1), pixels."""
        torch = _torch()
        side = self.sides[series]
        out = torch.empty((2, side + 1, side + 1), dtype=torch.float32, device="cuda")
        se = np.empty(2, np.int32)
        _check(_load().reg_get_slot(self.h, series, slot, out.data_ptr(), 1, se.ctypes.data))
        return out

    def set_slot_device(self, slot, field, start, end, series=0):
        """Set a slot from a CUDA tensor (2, side+1, side+1), pixels."""
        f = field.contiguous()
        _check(_load().reg_set_slot(self.h, series, slot, f.data_ptr(), 1, start, end))

    def copy_slot(self, src, dst, start, end, series=0):
        self.set_slot_device(dst, self.get_slot_device(src, series), start, end, series)

    def schedule_ops(self, kind, n, chunks=1, global_kind=KOGGE_STONE):
        return schedule(kind, n, chunks, global_kind)

    def get_rigid(self, slot, series=0):
        """Rigid handles: (theta (alpha, t0, t1 in Omega units), (start, end)) of a slot."""
        th = np.empty(3)
        se = np.empty(2, np.int32)
        _check(_load().reg_get_rigid(self.h, series, slot, th.ctypes.data, se.ctypes.data))
        return th, (int(se[0]), int(se[1]))

    def set_rigid(self, slot, theta, start, end, series=0):
        th = np.ascontiguousarray(theta, np.float64)
        _check(_load().reg_set_rigid(self.h, series, slot, th.ctypes.data, start, end))

    def rigid_params(self, series=0):
        """Rigid handles after prefix_scan: (n_frames, 3) parameters of phi_{0,k}
        (row 0 the identity)."""
        out = np.zeros((self.counts[series], 3))
        for k in range(1, self.counts[series]):
            th, se = self.get_rigid(k - 1, series)
            assert se == (0, k), se
            out[k] = th
        return out

    def get_slot(self, slot, series=0):
        return get_slot(self.h, series, slot, self.sides[series])

    def set_slot(self, slot, field, start, end, series=0):
        return set_slot(self.h, series, slot, field, start, end)

    def eval_energy(self, frame_i, frame_k, level, u_grid, series=0):
        return eval_energy(self.h, series, frame_i, frame_k, level, u_grid)

    def eval_direction(self, frame_i, frame_k, level, u_grid, series=0):
        return eval_direction(self.h, series, frame_i, frame_k, level, u_grid)

    def eval_trials(self, frame_i, frame_k, level, u_grid, taus, series=0):
        return eval_trials(self.h, series, frame_i, frame_k, level, u_grid, taus)

    def cnn_pairs(self, first, count, out, series=0):
        """Network inputs of neighbour pairs first..first+count-1 into the CUDA
        tensor out (count x 2 x 256 x 256)."""
        _check(_load().reg_cnn_pairs(self.h, series, first, count, out.data_ptr()))
        return out

    def set_tile_rows(self, level, grad_rows, trial_rows):
        _check(_load().reg_set_tile_rows(self.h, level, grad_rows, trial_rows))

    def get_tile_rows(self, level):
        g, t = ctypes.c_int32(), ctypes.c_int32()
        _check(_load().reg_get_tile_rows(self.h, level, ctypes.byref(g), ctypes.byref(t)))
        return g.value, t.value

    def autotune(self, n_pairs=16, repeats=1, series=0):
        """Tile rows per level and step sizes per pass picked by timing a sample
        batch (overwrites data slots 0..n_pairs-1); returns the report."""
        buf = ctypes.create_string_buffer(4096)
        _check(_load().reg_autotune(self.h, series, n_pairs, repeats, buf, len(buf)))
        return json.loads(buf.value.decode())

    def cnn_init(self, cnn, series=0, tensor_cores=False):
        """Initial displacements of all neighbour pairs from the network; the next
        prefix_scan starts its preprocessing operators from them."""
        _check(_load().reg_cnn_init_series(self.h, series, cnn.h, int(bool(tensor_cores))))

    def set_trace(self, capacity):
        set_trace(self.h, capacity)

    def get_trace(self):
        return get_trace(self.h)

    def set_lockstep(self, counts, taus=None):
        set_lockstep(self.h, counts, taus)

    def kernel_stats(self):
        return get_kernel_stats(self.h)

    def set_flags(self, flags):
        """Replace the handle's flags (FLAG_PROFILE: per-kernel CUDA-event timing)."""
        _check(_load().reg_set_flags(self.h, int(flags)))

    def reset_kernel_stats(self):
        reset_kernel_stats(self.h)

    def close(self):
        if self.h:
            destroy_series(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
