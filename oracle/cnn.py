"""FP64 CPU oracle of the learned initialiser (TEST INFRASTRUCTURE ONLY: only
``tests/`` and the CPU legs of ``bench.py`` may use it; it shares no code with
the CUDA path).

The network predicts a coarse initial displacement for a frame pair:
- input: 2 x S x S (channel 0 the reference frame, channel 1 the template,
  both normalised), S a multiple of 4;
- six 3x3 convolutions with zero padding 1: 2 -> 32 stride 2, 32 -> 32 stride
  2, three 32 -> 32 stride 1, 32 -> 2 stride 1, a ReLU after every layer but
  the last;
- output: 2 x S/4 x S/4, the displacement (pixels of the input resolution,
  channel 0 along columns, channel 1 along rows) at input pixels (4i, 4j).

A convolution of stride s computes, for output channel o at (y, x),
    out[o, y, x] = b[o] + sum_{c, dy, dx} W[o, c, dy, dx] in_pad[c, s y + dy, s x + dx]
with in_pad the input with one ring of zeros.  The tensor-core form of the
forward rounds the operands of the 32 -> 32 layers (their input activations and
weights, not the biases) to BF16 (8 significant bits, round to nearest, ties to
even) and contracts them exactly; ``forward(..., bf16_layers=(0, ..., 5))``
models the tensor-core forward, all six layers of which take BF16 operands.  The loss is the mean of the
squared differences to a target displacement.  Parameters are one flat vector:
layer by layer, W (O x C x 3 x 3, row-major) then b (O).
"""
from __future__ import annotations

import numpy as np

LAYERS = [(2, 32, 2), (32, 32, 2), (32, 32, 1), (32, 32, 1), (32, 32, 1), (32, 2, 1)]  # (C, O, stride)


def n_params():
    return sum(o * c * 9 + o for c, o, _ in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W, b), ...]."""
    theta = np.asarray(theta, np.float64)
    out, k = [], 0
    for c, o, _ in LAYERS:
        W = theta[k:k + o * c * 9].reshape(o, c, 3, 3)
        k += o * c * 9
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    assert k == theta.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def _out_size(h, stride):
    return (h + 2 - 3) // stride + 1


def conv_forward(x, W, b, stride):
    """x: (B, C, H, W) -> (B, O, Ho, Wo), the definition above (one 3x3 offset at a
    time, each a channel contraction)."""
    B, C, H, Wd = x.shape
    Ho, Wo = _out_size(H, stride), _out_size(Wd, stride)
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.empty((B, W.shape[0], Ho, Wo))
    out[...] = b[None, :, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + stride * (Ho - 1) + 1:stride, dx:dx + stride * (Wo - 1) + 1:stride]
            out += np.einsum("oc,bchw->bohw", W[:, :, dy, dx], patch)
    return out


def conv_backward(x, W, stride, gout):
    """Gradients of sum(gout * conv_forward(x, W, b, stride)) with respect to x, W
    and b."""
    B, C, H, Wd = x.shape
    Ho, Wo = gout.shape[2], gout.shape[3]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(3):
        for dx in range(3):
            sl = (slice(None), slice(None), slice(dy, dy + stride * (Ho - 1) + 1, stride),
                  slice(dx, dx + stride * (Wo - 1) + 1, stride))
            gW[:, :, dy, dx] = np.einsum("bohw,bchw->oc", gout, xp[sl])
            gxp[sl] += np.einsum("oc,bohw->bchw", W[:, :, dy, dx], gout)
    return gxp[:, :, 1:-1, 1:-1], gW, gout.sum(axis=(0, 2, 3))


def round_bf16(v):
    """v rounded to the nearest BF16 value (the float32 value's top 16 bits after
    rounding to nearest, ties to even), returned in float64; v is first rounded
    to float32."""
    f = np.ascontiguousarray(np.asarray(v, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, keep=False, bf16_layers=()):
    """Network output for inputs x (B, 2, S, S); with keep, also the layer inputs
    and pre-activations for backward(); layers listed in bf16_layers take BF16
    operands."""
    layers = unpack(theta)
    a, cache = np.asarray(x, np.float64), []
    for k, ((W, b), (_, _, s)) in enumerate(zip(layers, LAYERS)):
        if k in bf16_layers:
            z = conv_forward(round_bf16(a), round_bf16(W), b, s)
        else:
            z = conv_forward(a, W, b, s)
        cache.append((a, z))
        a = z if k == len(LAYERS) - 1 else np.maximum(z, 0.0)
    return (a, cache) if keep else a


def loss(theta, x, target):
    y = forward(theta, x)
    return float(np.mean((y - target) ** 2))


def loss_and_grad(theta, x, target, bf16_layers=(), bf16_data=(), bf16_weights=(), bf16_stored=()):
    """Mean squared error and its gradient with respect to the flat parameters.

    The tensor-core form of training takes BF16 operands in three places,
    modelled here by rounding those operands (the contraction itself exact):
    the forward of the layers in bf16_layers (their input and weights), the
    data gradient of the layers in bf16_data (the output gradient and the
    weights), and the weight gradient of the layers in bf16_weights (the
    output gradient and the layer's input).  A layer in bf16_stored keeps its
    input activation in BF16, so its weight gradient (on the CUDA cores, the
    output gradient unrounded) takes the rounded input.  Bias gradients sum
    the unrounded output gradient."""
    layers = unpack(theta)
    y, cache = forward(theta, x, keep=True, bf16_layers=bf16_layers)
    g = 2.0 * (y - target) / y.size
    grads = [None] * len(LAYERS)
    for k in range(len(LAYERS) - 1, -1, -1):
        a, z = cache[k]
        if k < len(LAYERS) - 1:
            g = g * (z > 0.0)  # ReLU
        W, s = layers[k][0], LAYERS[k][2]
        ga, gW, gb = conv_backward(a, W, s, g)
        if k in bf16_data:
            ga = conv_backward(a, round_bf16(W), s, round_bf16(g))[0]
        if k in bf16_weights:
            gW = conv_backward(round_bf16(a), W, s, round_bf16(g))[1]
        elif k in bf16_stored:
            gW = conv_backward(round_bf16(a), W, s, g)[1]
        grads[k] = (gW, gb)
        g = ga
    return float(np.mean((y - target) ** 2)), pack(grads)


def upsample(out, side):
    """The network output (2, S/4, S/4) in input pixels, for an input of S = 256
    pixels downsampled from frames of `side` pixels, as a displacement in frame
    pixels on the frame's (side+1)^2 vertex grid: bilinear in the output grid
    (spacing 4 S-pixels = 4 side/S frame pixels), clamped at its border, scaled
    by side/S."""
    q = out.shape[-1]
    k = side / (4.0 * q)  # frame pixels per input pixel
    r = np.arange(side + 1) / (4.0 * k)
    i0 = np.clip(np.floor(r).astype(int), 0, q - 2)
    f = np.clip(r - i0, 0.0, 1.0)
    res = np.empty((2, side + 1, side + 1))
    for ch in range(2):
        rows = out[ch][i0] * (1 - f)[:, None] + out[ch][i0 + 1] * f[:, None]
        res[ch] = rows[:, i0] * (1 - f)[None, :] + rows[:, i0 + 1] * f[None, :]
    return res * k
