"""Pins of the learned initialiser's FP64 oracle (oracle/cnn.py): the convolution
against scipy's correlation and against its own stride-1 form, every gradient
against central finite differences, and the output upsampling against exact
cases."""
import numpy as np
import pytest

from oracle import cnn


def test_layer_shapes_and_parameter_count_match_the_generator():
    import synth
    assert [(c, o) for c, o, _ in cnn.LAYERS] == synth.CNN_SHAPES
    assert cnn.n_params() == 608 + 4 * 9248 + 578
    assert synth.cnn_params(0).size == cnn.n_params()


def test_single_channel_convolution_is_scipy_correlation():
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 1, 9, 7))
    W = rng.standard_normal((1, 1, 3, 3))
    want = sig.correlate2d(np.pad(x[0, 0], 1), W[0, 0], mode="valid") + 0.25
    got = cnn.conv_forward(x, W, np.array([0.25]), 1)[0, 0]
    assert np.allclose(got, want, atol=1e-13)


def test_multichannel_convolution_sums_channels():
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 6, 6))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = cnn.conv_forward(x, W, b, 1)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(sig.correlate2d(np.pad(x[n, c], 1), W[o, c], mode="valid") for c in range(3))
            assert np.allclose(got[n, o], want, atol=1e-12)


def test_stride_two_is_stride_one_at_even_positions():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 12, 12))
    W = rng.standard_normal((5, 3, 3, 3))
    b = rng.standard_normal(5)
    full = cnn.conv_forward(x, W, b, 1)
    half = cnn.conv_forward(x, W, b, 2)
    assert half.shape == (2, 5, 6, 6)
    assert np.allclose(half, full[:, :, ::2, ::2], atol=1e-13)


@pytest.mark.parametrize("stride", [1, 2])
def test_convolution_gradients_are_finite_differences(stride):
    rng = np.random.default_rng(4 + stride)
    x = rng.standard_normal((2, 2, 6, 6))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    G = rng.standard_normal(cnn.conv_forward(x, W, b, stride).shape)
    f = lambda x_, W_, b_: float(np.sum(G * cnn.conv_forward(x_, W_, b_, stride)))
    gx, gW, gb = cnn.conv_backward(x, W, stride, G)
    eps = 1e-6
    for arr, g, name in ((x, gx, "x"), (W, gW, "W"), (b, gb, "b")):
        for idx in list(np.ndindex(arr.shape))[::5]:
            d = np.zeros_like(arr)
            d[idx] = eps
            args_p = [x, W, b]
            args_m = [x, W, b]
            k = {"x": 0, "W": 1, "b": 2}[name]
            args_p[k] = arr + d
            args_m[k] = arr - d
            fd = (f(*args_p) - f(*args_m)) / (2 * eps)
            assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[idx])


def test_network_gradient_is_finite_differences():
    import synth
    rng = np.random.default_rng(6)
    theta = synth.cnn_params(7).astype(np.float64)
    theta += 0.01 * rng.standard_normal(theta.size)  # nonzero biases too
    x = rng.standard_normal((2, 2, 16, 16))
    t = rng.standard_normal((2, 2, 4, 4))
    L, g = cnn.loss_and_grad(theta, x, t)
    assert L == pytest.approx(cnn.loss(theta, x, t), rel=1e-14)
    eps = 1e-6
    picks = rng.choice(theta.size, 60, replace=False)
    for i in picks:
        d = np.zeros_like(theta)
        d[i] = eps
        fd = (cnn.loss(theta + d, x, t) - cnn.loss(theta - d, x, t)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (i, fd, g[i])


def test_relu_blocks_the_gradient_of_a_dead_layer():
    # a first layer whose pre-activations are all negative passes no gradient
    import synth
    theta = synth.cnn_params(8).astype(np.float64)
    layers = cnn.unpack(theta)
    layers[0] = (np.zeros_like(layers[0][0]), np.full_like(layers[0][1], -1.0))
    theta = cnn.pack(layers)
    rng = np.random.default_rng(9)
    _, g = cnn.loss_and_grad(theta, rng.standard_normal((1, 2, 8, 8)), rng.standard_normal((1, 2, 2, 2)))
    assert np.all(cnn.unpack(g)[0][0] == 0.0) and np.all(cnn.unpack(g)[0][1] == 0.0)


def test_upsampling_reproduces_constant_and_linear_fields():
    q, side = 8, 128  # input 32 px, frames of 128 px: 4 frame px per input px
    out = np.ones((2, q, q)) * np.array([1.5, -0.5])[:, None, None]
    up = cnn.upsample(out, side)
    assert up.shape == (2, side + 1, side + 1)
    assert np.allclose(up[0], 1.5 * 4) and np.allclose(up[1], -0.5 * 4)
    # a field linear in the output grid is reproduced exactly inside it
    i = np.arange(q, dtype=np.float64)
    lin = np.stack([np.add.outer(0 * i, i), np.add.outer(i, 0 * i)])
    up = cnn.upsample(lin, side)
    r = np.arange(side + 1) / 16.0
    inside = r <= q - 1
    assert np.allclose(up[0][:, inside], 4 * r[inside][None, :])
    assert np.allclose(up[1][inside, :], 4 * r[inside][:, None])


def test_bf16_rounding_exact_cases():
    """BF16 keeps 8 significant bits: 1 + 2^-7 is representable, 1 + 2^-8 lies
    halfway between 1 and 1 + 2^-7 and rounds to the even neighbour 1, 1 + 3 2^-8
    rounds up to 1 + 2^-6, and sign, zero and powers of two pass unchanged."""
    v = np.array([1 + 2.0 ** -7, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -12,
                  -(1 + 2.0 ** -8 + 2.0 ** -12), 0.0, 2.0 ** -40, -1024.0])
    want = [1 + 2.0 ** -7, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -(1 + 2.0 ** -7), 0.0, 2.0 ** -40, -1024.0]
    assert cnn.round_bf16(v).tolist() == want


def test_bf16_rounding_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    v = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.round_bf16(v), want)


def test_bf16_forward_error_is_within_the_operand_rounding_bound():
    """Rounding to 8 significant bits moves each operand by at most 2^-8 of its
    size, so each product by at most (1 + 2^-8)^2 - 1 = 2^-7 + 2^-16 of its size
    and a layer output by at most that times the sum of its absolute products;
    the untouched layers give identical results."""
    import synth
    rng = np.random.default_rng(10)
    theta = synth.cnn_params(5).astype(np.float64)
    x = rng.standard_normal((1, 2, 16, 16))
    assert np.array_equal(cnn.forward(theta, x), cnn.forward(theta, x, bf16_layers=()))
    layers = cnn.unpack(theta)
    a = cnn.forward(theta, x, keep=True)[1][1][0]  # input of layer 1
    W, b = layers[1]
    exact = cnn.conv_forward(a, W, b, 2)
    rounded = cnn.conv_forward(cnn.round_bf16(a), cnn.round_bf16(W), b, 2)
    bound = cnn.conv_forward(np.abs(a), np.abs(W), 0 * b, 2) * (2.0 ** -7 + 2.0 ** -16)
    assert np.all(np.abs(rounded - exact) <= bound)
    assert np.abs(rounded - exact).max() > 0


def test_bf16_operand_gradients_reduce_to_the_exact_ones_on_bf16_values():
    """With every operand already a BF16 value (parameters, inputs and a target
    that keep the intermediate values exact is not possible, so instead: the
    rounding hooks change nothing when the listed sets are empty, and with all
    sets listed the result differs from the exact gradient by about the BF16
    operand error (2^-8 relative), not more."""
    from oracle import cnn as ocnn
    import synth
    rng = np.random.default_rng(5)
    theta = synth.cnn_params(2).astype(np.float64)
    x = rng.standard_normal((1, 2, 32, 32))
    t = rng.standard_normal((1, 2, 8, 8))
    l0, g0 = ocnn.loss_and_grad(theta, x, t)
    l1, g1 = ocnn.loss_and_grad(theta, x, t, (), (), ())
    assert l0 == l1 and np.array_equal(g0, g1)
    l2, g2 = ocnn.loss_and_grad(theta, x, t, bf16_layers=(1, 2, 3, 4), bf16_data=(2, 3, 4), bf16_weights=(1, 2, 3, 4))
    rel = np.abs(g2 - g0).max() / np.abs(g0).max()
    assert 1e-5 < rel < 0.1, rel
    assert abs(l2 - l0) < 0.05 * l0


def test_bf16_stored_input_changes_only_that_layers_weight_gradient():
    """A layer whose input is stored in BF16 (bf16_stored) differs from the
    exact gradient only in its own weight gradient, and there by no more than
    the input's rounding allows: each product moves by at most 2^-8 of its
    size, so gW by at most 2^-8 sum |g| |a|."""
    from oracle import cnn as ocnn
    import synth
    rng = np.random.default_rng(6)
    theta = synth.cnn_params(3).astype(np.float64)
    x = rng.standard_normal((2, 2, 32, 32))
    t = rng.standard_normal((2, 2, 8, 8))
    l0, g0 = ocnn.loss_and_grad(theta, x, t)
    l1, g1 = ocnn.loss_and_grad(theta, x, t, bf16_stored=(5,))
    assert l0 == l1
    parts0, parts1 = ocnn.unpack(g0), ocnn.unpack(g1)
    for k in range(5):
        assert np.array_equal(parts0[k][0], parts1[k][0]) and np.array_equal(parts0[k][1], parts1[k][1]), k
    assert np.array_equal(parts0[5][1], parts1[5][1])  # bias gradient: the unrounded output gradient
    y, cache = ocnn.forward(theta, x, keep=True)
    a = cache[5][0]
    g = 2.0 * (y - t) / y.size
    bound = ocnn.conv_backward(np.abs(a), np.abs(ocnn.unpack(theta)[5][0]), 1, np.abs(g))[1] * 2.0 ** -8
    d = np.abs(parts1[5][0] - parts0[5][0])
    assert np.all(d <= bound * (1 + 1e-12)) and d.max() > 0
