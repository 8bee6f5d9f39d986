"""Training the learned initialiser on displacements the plain method computes.

The training pairs are neighbour pairs of seeded generator series of 256^2
pixels; the plain GPU method (identity start) registers every pair, and the
target is its displacement at the network's output positions (pixels (4i, 4j),
i, j < 64).  The network trains on the GPU with the library's own forward,
backward and Adam kernels; this module only moves data and loops.
"""
from __future__ import annotations

import numpy as np

from . import Cnn, Series, default_params, _torch

# Generator parameters of the training series (256^2 pixels): a well-sampled
# lattice (12 px, atoms of sigma 2 px) under large frame-to-frame motion (a
# random-walk drift of 3 px steps and 2 px distortions), where the starting
# guess matters to the gradient flow.
TRAIN_SERIES = dict(spacing=12.0, sigma=2.0, peak=10.0, drift_sd=3.0, dist_amp=2.0)


def training_set(n_pairs, seed=100, frames_per_series=64, n_levels=3, iter_max=50, lam=10.0, device="cuda"):
    """Inputs x (n_pairs x 2 x 256 x 256) and targets t (n_pairs x 2 x 64 x 64),
    CUDA float32 tensors; pairs of consecutive series are interleaved so that a
    contiguous slice mixes series."""
    import synth
    torch = _torch()
    n_series = -(-n_pairs // (frames_per_series - 1))
    xs, ts = [], []
    p = default_params(n_levels=n_levels, iter_max=iter_max, lam=lam)
    for k in range(n_series):
        fr = synth.series(seed + k, frames_per_series, 256, **TRAIN_SERIES)
        n = frames_per_series - 1
        x = torch.empty((n, 2, 256, 256), dtype=torch.float32, device=device)
        with Series(fr, p) as s:
            s.apply_operator_batch([(0, -1, -1, e, e, e + 1) for e in range(n)])
            s.cnn_pairs(0, n, x)
            t = np.stack([s.get_slot(e)[0][:, 0:256:4, 0:256:4] for e in range(n)])
        xs.append(x)
        ts.append(torch.from_numpy(np.ascontiguousarray(t)).to(device))
    # interleave: pair j of series k at position j * n_series + k
    x = torch.stack(xs, 1).reshape(-1, 2, 256, 256)[:n_pairs].contiguous()
    t = torch.stack(ts, 1).reshape(-1, 2, 64, 64)[:n_pairs].contiguous()
    return x, t


def train(cnn: Cnn, x, t, epochs=4, batch=64, lr=1e-3, log=None):
    """Adam on contiguous minibatches; returns the mean loss of each epoch."""
    n = int(x.shape[0])
    hist = []
    for ep in range(epochs):
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            loss = cnn.loss_grad(x[i:i + batch], t[i:i + batch])
            cnn.adam_step(lr)
            tot += loss
            cnt += 1
        hist.append(tot / max(1, cnt))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f} px^2")
    return hist
