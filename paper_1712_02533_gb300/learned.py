"""Training the learned initialiser on displacements the plain method computes,
and comparing the learned form with the plain one.

- training_set(): neighbour pairs of seeded generator series (256^2 frames by
  default, or larger frames seen through their 257^2 pyramid level); the plain
  GPU method (identity start) registers every pair, and the target is its
  displacement at the network's output positions (every side/64-th frame
  pixel), in pixels of the 256^2 input.
- train(): Adam on minibatches with the library's own forward, backward and
  update kernels; this module only moves data and loops.
- compare(): series time and accuracy of the plain form against the learned
  form (network start on the finest init_levels levels).
- forward_rate(): forward throughput on the CUDA cores and the tensor cores.
- main(): ``python -m paper_1712_02533_gb300.learned`` trains on pairs shaped
  like the 400 x 1024^2 workload and compares on a fresh series (one JSON
  object); ``--forward-rate B`` only times the forward pass.
"""
from __future__ import annotations

import numpy as np

from . import Cnn, Series, default_params, _torch

# Generator parameters of the training series (256^2 pixels): a well-sampled
# lattice (12 px, atoms of sigma 2 px) under large frame-to-frame motion (a
# random-walk drift of 3 px steps and 2 px distortions), where the starting
# guess matters to the gradient flow.
TRAIN_SERIES = dict(spacing=12.0, sigma=2.0, peak=10.0, drift_sd=3.0, dist_amp=2.0)


def training_set(n_pairs, seed=100, frames_per_series=64, n_levels=3, iter_max=50, lam=10.0, device="cuda",
                 side=256, series_kw=None):
    """Inputs x (n_pairs x 2 x 256 x 256) and targets t (n_pairs x 2 x 64 x 64),
    CUDA float32 tensors, from generator series of side^2 pixels (series_kw:
    generator parameters, default TRAIN_SERIES; the pyramid of n_levels must
    hold the 257^2 level); pairs of consecutive series are interleaved so that a
    contiguous slice mixes series.  Targets are the plain method's displacement
    at frame pixels (side/64) (i, j), in pixels of the 256^2 input."""
    import synth
    torch = _torch()
    kw = TRAIN_SERIES if series_kw is None else series_kw
    step, scale = side // 64, side / 256.0
    n_series = -(-n_pairs // (frames_per_series - 1))
    xs, ts = [], []
    p = default_params(n_levels=n_levels, iter_max=iter_max, lam=lam)
    for k in range(n_series):
        fr = synth.series(seed + k, frames_per_series, side, **kw)
        n = frames_per_series - 1
        x = torch.empty((n, 2, 256, 256), dtype=torch.float32, device=device)
        with Series(fr, p) as s:
            s.apply_operator_batch([(0, -1, -1, e, e, e + 1) for e in range(n)])
            s.cnn_pairs(0, n, x)
            t = np.stack([s.get_slot(e)[0][:, 0:side:step, 0:side:step] / scale for e in range(n)])
        xs.append(x)
        ts.append(torch.from_numpy(np.ascontiguousarray(t)).to(device))
    # interleave: pair j of series k at position j * n_series + k
    x = torch.stack(xs, 1).reshape(-1, 2, 256, 256)[:n_pairs].contiguous()
    t = torch.stack(ts, 1).reshape(-1, 2, 64, 64)[:n_pairs].contiguous()
    return x, t


def train(cnn: Cnn, x, t, epochs=4, batch=64, lr=1e-3, log=None, lr_final=None, tensor_cores=False):
    """Adam on contiguous minibatches, the rate decaying geometrically from lr
    to lr_final (if given) over the epochs; returns the mean loss of each
    epoch.  tensor_cores: the loss and gradients of the 32-channel layers on
    the tensor cores (BF16 operands, FP32 accumulation)."""
    n = int(x.shape[0])
    hist = []
    for ep in range(epochs):
        rate = lr if lr_final is None or epochs < 2 else lr * (lr_final / lr) ** (ep / (epochs - 1))
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            loss = cnn.loss_grad(x[i:i + batch], t[i:i + batch], tensor_cores=tensor_cores)
            cnn.adam_step(rate)
            tot += loss
            cnt += 1
        hist.append(tot / max(1, cnt))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f} px^2")
    return hist


# Multiply-adds of the network per pair of 256^2 inputs, layer by layer
# (output pixels x output channels x input channels x 9), and the share of the
# four 32 -> 32 layers that the tensor-core path runs.
_SHAPES = [(2, 32, 128), (32, 32, 64), (32, 32, 64), (32, 32, 64), (32, 32, 64), (32, 2, 64)]  # C, O, output side
FLOP_PER_PAIR = sum(2 * q * q * o * c * 9 for c, o, q in _SHAPES)
TC_FLOP_PER_PAIR = sum(2 * q * q * o * c * 9 for c, o, q in _SHAPES[1:5])


def training_rate(cnn: Cnn, batch=64, reps=10, tensor_cores=True, seed=0):
    """Loss-and-gradient passes (forward + backward) of `batch` random pairs
    and targets, timed with CUDA events on the current stream after two
    warm-up passes: (ms per pass, TFLOP/s counting 3x the forward's FLOPs:
    forward, data and weight gradients)."""
    torch = _torch()
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((batch, 2, 256, 256), generator=g, device="cuda")
    t = torch.randn((batch, 2, 64, 64), generator=g, device="cuda")
    for _ in range(2):
        cnn.loss_grad(x, t, tensor_cores=tensor_cores)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        cnn.loss_grad(x, t, tensor_cores=tensor_cores)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return ms, 3 * FLOP_PER_PAIR * batch / (ms * 1e-3) / 1e12


def forward_rate(cnn: Cnn, batch=64, reps=20, tensor_cores=True, seed=0):
    """Forward passes of `batch` random pairs, timed with CUDA events on the
    current stream after two warm-up passes: (ms per pass, whole-network
    TFLOP/s)."""
    torch = _torch()
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((batch, 2, 256, 256), device="cuda", generator=g)
    y = torch.empty((batch, 2, 64, 64), device="cuda")
    for _ in range(2):
        cnn.forward(x, y, tensor_cores=tensor_cores)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        cnn.forward(x, y, tensor_cores=tensor_cores)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return ms, FLOP_PER_PAIR * batch / (ms * 1e-3) / 1e12


def compare(cnn: Cnn, frames, gt, n_levels=5, iter_max=50, lam=10.0, kind=None, init_levels=(5, 4, 3, 1),
            tensor_cores=True, margin=32):
    """Series registration of `frames` by the plain method (identity start of
    the preprocessing operators) and by the learned form (network start on the
    finest init_levels levels), each timed from frames resident on the device
    (pyramid built) to all deformations phi_{0,k} on the device, network
    inference included.  Accuracy: mean interior error against the generator's
    ground truth `gt` (n x 2 x side x side px, `margin` px border left out) and
    the distance to the plain result."""
    import time
    torch = _torch()
    from . import SKLANSKY
    kind = SKLANSKY if kind is None else kind
    rows, plain = [], None
    for il in (None,) + tuple(init_levels):
        p = default_params(n_levels=n_levels, iter_max=iter_max, lam=lam, init_levels=il or 0)
        with Series(frames, p) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if il is not None:
                s.cnn_init(cnn, tensor_cores=tensor_cores)
            t1 = time.perf_counter()
            rep = s.prefix_scan(kind)
            t2 = time.perf_counter()
            d = s.get_deformations()
        err = np.abs(d[1:] - gt[1:])[:, :, margin:-margin, margin:-margin]
        row = dict(form="plain" if il is None else "learned", init_levels=n_levels if il is None else il,
                   series_s=t2 - t0, cnn_ms=1e3 * (t1 - t0), preprocessing_ms=rep["preprocessing_ms"],
                   iters=rep["iters"], status=rep["status"], judged=rep.get("learned"), gt_err_px=float(err.mean()))
        if plain is None:
            plain = d
        else:
            dev = np.abs(d[1:] - plain[1:])[:, :, margin:-margin, margin:-margin]
            row.update(dev_from_plain_mean_px=float(dev.mean()), dev_from_plain_max_px=float(dev.max()),
                       frac_within_005px=float(np.mean(dev <= 0.05)))
        rows.append(row)
    return rows


def main(argv=None):
    """Train the network on neighbour pairs of generator series shaped like the
    1024^2 workload (plain-method targets), then compare the plain and learned
    forms on a fresh series; prints one JSON object."""
    import argparse
    import json
    import time
    import synth
    torch = _torch()
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--train-seed", type=int, default=4000)
    ap.add_argument("--eval-seed", type=int, default=5)
    ap.add_argument("--frames", type=int, default=400)
    ap.add_argument("--side", type=int, default=1024)
    ap.add_argument("--init-levels", default="5,4,3,1")
    ap.add_argument("--iter-max", type=int, default=50, help="gradient steps per level of the compared forms")
    ap.add_argument("--weights-out", default=None, help="save the trained parameters (.npy)")
    ap.add_argument("--weights-in", default=None, help="skip training, load parameters (.npy)")
    ap.add_argument("--forward-rate", type=int, default=0, metavar="BATCH",
                    help="only time the forward pass (FP32 and tensor cores) on BATCH random pairs")
    ap.add_argument("--training-rate", type=int, default=0, metavar="BATCH",
                    help="only time loss-and-gradient passes (FP32 and tensor cores) on BATCH random pairs")
    ap.add_argument("--tc-train", action="store_true", help="train with the tensor-core loss and gradients")
    a = ap.parse_args(argv)
    if a.training_rate:
        with Cnn(synth.cnn_params(1), side=256, max_batch=a.training_rate) as net:
            res = {}
            for tc in (False, True):
                ms, tf = training_rate(net, batch=a.training_rate, tensor_cores=tc)
                res["tensor_cores" if tc else "fp32"] = dict(ms_per_pass=ms, tflops_network=tf,
                                                             pairs_per_s=a.training_rate / ms * 1e3)
        print(json.dumps(dict(batch=a.training_rate, flop_per_pair=3 * FLOP_PER_PAIR, **res)))
        return
    if a.forward_rate:
        with Cnn(synth.cnn_params(1), side=256, max_batch=a.forward_rate) as net:
            res = {}
            for tc in (False, True):
                ms, tf = forward_rate(net, batch=a.forward_rate, tensor_cores=tc)
                res["tensor_cores" if tc else "fp32"] = dict(ms_per_forward=ms, tflops_network=tf,
                                                             pairs_per_s=a.forward_rate / ms * 1e3)
        print(json.dumps(dict(batch=a.forward_rate, flop_per_pair=FLOP_PER_PAIR,
                              tc_flop_per_pair=TC_FLOP_PER_PAIR, **res)))
        return
    gen = {k: v for k, v in synth.CONFIGS["c3_400x1024"].items() if k not in ("seed", "n_frames", "side", "n_levels")}
    out = dict(workload=f"{a.frames}x{a.side}^2", generator=gen)
    net = Cnn(synth.cnn_params(1), side=256, max_batch=64)
    if a.weights_in:
        net.set_params(np.load(a.weights_in))
    else:
        t0 = time.perf_counter()
        x, t = training_set(a.pairs, seed=a.train_seed, frames_per_series=64, n_levels=5, side=a.side,
                            series_kw=gen)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hist = train(net, x, t, epochs=a.epochs, batch=a.batch, lr=a.lr, lr_final=a.lr_final,
                     tensor_cores=a.tc_train)
        torch.cuda.synchronize()
        out.update(pairs=a.pairs, epochs=a.epochs, data_s=t1 - t0, train_s=time.perf_counter() - t1,
                   target_ms_px2=float(t.pow(2).mean()), loss_first=hist[0], loss_last=hist[-1])
        del x, t
        if a.weights_out:
            np.save(a.weights_out, net.get_params())
    frames, gt, _ = synth.series(a.eval_seed, a.frames, a.side, ground_truth=True, **gen)
    out["iter_max"] = a.iter_max
    out["rows"] = compare(net, frames, gt, iter_max=a.iter_max, init_levels=tuple(int(v) for v in a.init_levels.split(",")))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
