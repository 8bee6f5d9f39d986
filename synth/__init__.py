"""Seeded synthetic micrograph series (input producer shared by the oracle tests,
the CUDA path's tests and the benchmark).

The paper's aluminium-oxidation frames (Section "Electron microscopy data") are
not available; these series stand in for them with the shapes of its workloads.
The module holds no registration arithmetic: see ``synth.c`` for the model.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_frames", ctypes.c_int32),
        ("side", ctypes.c_int32),
        ("spacing", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("peak", ctypes.c_double),
        ("background", ctypes.c_double),
        ("blob_amp", ctypes.c_double),
        ("n_blobs", ctypes.c_int32),
        ("noise", ctypes.c_int32),
        ("drift_sd", ctypes.c_double),
        ("dist_amp", ctypes.c_double),
        ("dist_period", ctypes.c_double * 2),
        ("dist_freq", ctypes.c_double * 2),
        ("drift_override", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (portable flags only: builds on x86-64 and aarch64)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_series.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_series.restype = ctypes.c_int
        _lib = lib
    return _lib


# Workload recipes (frame counts, sizes, lattice, noise, drift, distortion,
# pyramid depth) shaped like the paper's experiments.
CONFIGS = {
    "c1_8x64": dict(seed=1, n_frames=8, side=64, spacing=8.0, sigma=1.5, peak=20.0,
                    drift_sd=0.5, dist_amp=1.0, n_levels=3),
    "c2_128x512": dict(seed=2, n_frames=128, side=512, spacing=12.0, sigma=2.0, peak=10.0,
                       drift_sd=0.5, dist_amp=1.0, n_levels=4),
    "c3_400x1024": dict(seed=3, n_frames=400, side=1024, spacing=16.0, sigma=2.0, peak=5.0,
                        drift_sd=1.0, dist_amp=2.0, n_levels=5),
}


def series(seed: int, n_frames: int, side: int, spacing: float = 8.0, sigma: float = 1.5,
           peak: float = 20.0, background: float = 0.15, blob_amp: float = 0.6, n_blobs: int = 6,
           noise: bool = True, drift_sd: float = 0.5, dist_amp: float = 1.0,
           dist_period=(37.0, 91.0), dist_freq=(1.0, 2.0), drift=None,
           ground_truth: bool = False, **_ignored):
    """Generate ``n_frames`` frames of ``side`` x ``side`` float32 pixels.

    Returns ``frames`` (n, side, side) float32, and when ``ground_truth`` is set
    also ``gt`` (n, 2, side, side) float64 with phi_{0,k}(x) - x in pixels
    (channel 0 = column, channel 1 = row) and the per-frame translations.
    ``drift`` overrides the random walk with explicit (n, 2) translations.
    """
    lib = _load()
    p = _Params()
    p.seed = seed
    p.n_frames = n_frames
    p.side = side
    p.spacing = spacing
    p.sigma = sigma
    p.peak = peak
    p.background = background
    p.blob_amp = blob_amp
    p.n_blobs = n_blobs
    p.noise = 1 if noise else 0
    p.drift_sd = drift_sd
    p.dist_amp = dist_amp
    p.dist_period[0], p.dist_period[1] = dist_period
    p.dist_freq[0], p.dist_freq[1] = dist_freq
    keep = None
    if drift is not None:
        keep = np.ascontiguousarray(np.asarray(drift, dtype=np.float64).reshape(n_frames, 2))
        p.drift_override = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    frames = np.empty((n_frames, side, side), dtype=np.float32)
    gt = np.empty((n_frames, 2, side, side), dtype=np.float64) if ground_truth else None
    tr = np.empty((n_frames, 2), dtype=np.float64)
    rc = lib.synth_series(ctypes.byref(p), frames.ctypes.data,
                          gt.ctypes.data if gt is not None else None, tr.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"synth_series failed ({rc})")
    if ground_truth:
        return frames, gt, tr
    return frames


# Layer shapes (in channels, out channels) of the learned initialiser's six 3x3
# convolutions, for drawing its initial parameters.
CNN_SHAPES = [(2, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 2)]


def cnn_params(seed: int) -> np.ndarray:
    """Initial parameters of the learned initialiser as one flat float32 vector
    (layer by layer: W as out x in x 3 x 3, then b): He-normal weights with
    variance 2 / (9 in), zero biases, drawn from numpy's PCG64 with `seed`."""
    rng = np.random.default_rng(seed)
    parts = []
    for c, o in CNN_SHAPES:
        parts.append(rng.standard_normal(o * c * 9) * np.sqrt(2.0 / (9 * c)))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)
