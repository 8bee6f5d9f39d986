"""The learned initialiser on the GPU through the C-ABI: forward pass, loss and
gradients against the FP64 oracle (oracle/cnn.py), the Adam step against its
definition, the network inputs against the normalised frames, and what the
trained network gains over the identity start."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the tensor-core forward takes BF16 operands in all six layers; its training
# pass also in the data and weight gradients of the 32-channel layers, and the
# last layer's weight gradient takes its BF16-stored input
TC_LAYERS = (0, 1, 2, 3, 4, 5)
TC_TRAIN = dict(bf16_layers=TC_LAYERS, bf16_data=(1, 2, 3, 4), bf16_weights=(1, 2, 3, 4), bf16_stored=(5,))


@pytest.fixture(scope="module")
def reg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1712_02533_gb300 import _build
    _build.build()
    import paper_1712_02533_gb300 as r
    return r


def test_forward_loss_and_gradients_match_the_oracle(reg):
    import torch
    import synth
    from oracle import cnn as ocnn
    rng = np.random.default_rng(0)
    theta = (synth.cnn_params(3) + 0.01 * rng.standard_normal(ocnn.n_params())).astype(np.float32)
    x = rng.standard_normal((2, 2, 64, 64)).astype(np.float32)
    t = rng.standard_normal((2, 2, 16, 16)).astype(np.float32)
    with reg.Cnn(theta, side=64, max_batch=4) as net:
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        y = net.forward(xd).cpu().numpy()
        loss, g = net.loss_grad(xd, td, want_grad=True)
    th, x64, t64 = theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64)
    yo = ocnn.forward(th, x64)
    lo, go = ocnn.loss_and_grad(th, x64, t64)
    assert np.abs(y - yo).max() <= 1e-5 * np.abs(yo).max()
    assert abs(loss - lo) <= 1e-6 * lo
    for k, ((gw, gb), (ow, ob)) in enumerate(zip(ocnn.unpack(g.astype(np.float64)), ocnn.unpack(go))):
        assert np.abs(gw - ow).max() <= 1e-5 * np.abs(ow).max(), k
        assert np.abs(gb - ob).max() <= 1e-5 * np.abs(ob).max(), k


@pytest.mark.parametrize("side,batch", [(64, 2), (36, 3), (88, 3)])
def test_tensor_core_forward_matches_the_bf16_operand_oracle(reg, side, batch):
    """The 32 -> 32 layers on the tensor cores take BF16 operands and accumulate
    in FP32: against the oracle with the same operand rounding the output agrees
    to FP32 accumulation plus the rare operand that rounds the other way (its
    FP32 input differs from the FP64 one in the last bits); against the exact
    oracle it differs by the BF16 operand error.  Side 36 leaves 81 pixels per
    pair in the 32-channel layers, a ragged last tile; side 88 gives the
    stride-1 layers 22 x 22 pixels, several tiles of 16 x 8 with ragged rows
    and columns."""
    import torch
    import synth
    from oracle import cnn as ocnn
    rng = np.random.default_rng(side)
    theta = synth.cnn_params(6)
    x = rng.standard_normal((batch, 2, side, side)).astype(np.float32)
    with reg.Cnn(theta, side=side, max_batch=batch) as net:
        xd = torch.from_numpy(x).cuda()
        y_tc = net.forward(xd, tensor_cores=True).cpu().numpy().astype(np.float64)
        y_f32 = net.forward(xd).cpu().numpy().astype(np.float64)
    th, x64 = theta.astype(np.float64), x.astype(np.float64)
    y_exact = ocnn.forward(th, x64)
    y_bf16 = ocnn.forward(th, x64, bf16_layers=TC_LAYERS)
    scale = np.abs(y_exact).max()
    assert np.abs(y_tc - y_bf16).max() <= 2e-3 * scale
    assert np.median(np.abs(y_tc - y_bf16)) <= 1e-5 * scale
    assert np.abs(y_tc - y_exact).max() <= 5e-2 * scale
    # the FP32 path is the exact one; the tensor-core path is not the same code
    assert np.abs(y_f32 - y_exact).max() <= 1e-5 * scale
    assert np.abs(y_tc - y_f32).max() > 1e-4 * scale


def test_adam_step_follows_its_definition(reg):
    import torch
    import synth
    rng = np.random.default_rng(1)
    theta = synth.cnn_params(4)
    x = torch.from_numpy(rng.standard_normal((2, 2, 32, 32)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((2, 2, 8, 8)).astype(np.float32)).cuda()
    with reg.Cnn(theta, side=32, max_batch=2) as net:
        _, g = net.loss_grad(x, t, want_grad=True)
        net.adam_step(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
        got = net.get_params()
    g = g.astype(np.float64)
    m, v = 0.1 * g, 0.001 * g * g
    want = theta - 1e-2 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    assert np.abs(got - want).max() <= 1e-6 * max(1.0, np.abs(want).max())


def test_network_inputs_are_the_normalised_257_level(reg, orc, syn):
    import torch
    fr = syn.series(21, 3, 256, spacing=12.0, sigma=2.0, peak=10.0)
    x = torch.empty((2, 2, 256, 256), dtype=torch.float32, device="cuda")
    with reg.Series(fr, reg.default_params(n_levels=3)) as s:
        s.cnn_pairs(0, 2, x)
    x = x.cpu().numpy()
    for e in range(2):
        for ch in range(2):
            F = orc.embed(fr[e + ch])
            w = orc.lumped(F.shape[0])
            Fc = F - float(np.sum(w * F))
            want = Fc / np.sqrt(float(np.sum(Fc * orc.mass_apply(Fc))))
            assert np.abs(x[e, ch] - want[:256, :256]).max() <= 1e-5 * np.abs(want).max()


def _oracle_inputs(orc, fr):
    """Network inputs of the pair (fr[0], fr[1]) of 256^2 frames, from the
    oracle: each frame's grid function centred and scaled to unit FE norm, its
    first 256 rows and columns."""
    x = []
    for f in fr[:2]:
        F = orc.embed(f)
        Fc = F - float(np.sum(orc.lumped(F.shape[0]) * F))
        x.append((Fc / np.sqrt(float(np.sum(Fc * orc.mass_apply(Fc)))))[:256, :256])
    return np.stack(x)[None]


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_learned_start_matches_the_oracle(reg, orc, syn, tensor_cores):
    """The learned start of a preprocessing operator is the network's output
    upsampled onto the finest grid (oracle: FP64 network, BF16 operands in the
    32-channel layers on the tensor-core path); the operator then runs function
    A from it on the finest init_levels levels, which the oracle's A with that
    many levels and that start reproduces (decision by decision)."""
    import synth
    from oracle import cnn as ocnn
    from paper_1712_02533_gb300 import learned
    import _parity as P
    from test_gpu_parity import _gpu_traces_by_op
    fr = syn.series(31, 2, 256, **learned.TRAIN_SERIES)
    theta = synth.cnn_params(7)
    y = ocnn.forward(theta.astype(np.float64), _oracle_inputs(orc, fr),
                     bf16_layers=TC_LAYERS if tensor_cores else ())
    u0 = ocnn.upsample(y[0], 256)
    p = reg.default_params(n_levels=3, init_levels=2, iter_max=50, lam=10.0, learned_fallback_px=0.0)
    g0, g1 = orc.embed(fr[0]), orc.embed(fr[1])
    op = orc.params(n_levels=2, iter_max=50, lam=10.0)
    with orc.trace() as t:
        u, _, stl = orc.register(g0, g1, op, u_init=u0 / 256)
    assert len(stl) == 2
    with reg.Cnn(theta, side=256, max_batch=4) as net, reg.Series(fr, p) as s:
        s.cnn_init(net, tensor_cores=tensor_cores)
        init, se = s.get_slot(0)
        assert tuple(se) == (0, 1)
        s.set_trace(1 << 20)
        s.prefix_scan(reg.SERIAL)
        gtr = _gpu_traces_by_op(s.get_trace(), 1)[0]
        d, se = s.get_slot(0)  # phi_{0,1} on the vertex grid
        assert tuple(se) == (0, 1)
        tol = 2e-3 if tensor_cores else 2e-5
        assert np.abs(init - u0).max() <= tol * np.abs(u0).max()
        if not tensor_cores:  # the start differs by the BF16 rounding flips; the FP32 case pins the operator
            P.report("learned", P.free_running_parity(orc, d, u * 256, gtr, t.rows, "A(0,1) from the learned start",
                                                       g0, g1, op, 10.0, P.gpu_energy_fn(s, 0, 1, 8),
                                                       u_init_omega=u0 / 256))


def test_plain_method_judges_the_learned_start_and_falls_back(reg, syn):
    """The plain method judges each learned start by how far it has to move it.
    A network whose predictions are far off (its weights scaled up) makes every
    operator exceed the threshold; each is then run again from the identity on
    every level, so the series equals the plain scan bit for bit.  With the
    threshold at 0 the judgement is reported but nothing falls back."""
    import synth
    from paper_1712_02533_gb300 import learned
    fr = syn.series(41, 6, 256, **learned.TRAIN_SERIES)
    theta = synth.cnn_params(8)
    theta[-2 - 32 * 9 * 2:] *= 200.0  # last layer: predictions of tens of pixels
    p = reg.default_params(n_levels=3, init_levels=1, iter_max=50, lam=10.0)
    with reg.Series(fr, p) as s:
        s.prefix_scan(reg.SKLANSKY)
        plain = s.get_deformations()
    with reg.Cnn(theta, side=256, max_batch=8) as net:
        with reg.Series(fr, p) as s:
            s.cnn_init(net)
            rep = s.prefix_scan(reg.SKLANSKY)
            got = s.get_deformations()
        assert rep["learned"]["ops"] == 5 and rep["learned"]["fallbacks"] == 5, rep["learned"]
        assert rep["learned"]["mean_correction_px"] > 2.0
        assert np.array_equal(got, plain)
        p0 = reg.default_params(n_levels=3, init_levels=1, iter_max=50, lam=10.0, learned_fallback_px=0.0)
        with reg.Series(fr, p0) as s:
            s.cnn_init(net)
            rep0 = s.prefix_scan(reg.SKLANSKY)
        assert rep0["learned"]["ops"] == 5 and rep0["learned"]["fallbacks"] == 0
        assert rep0["learned"]["max_correction_px"] > 2.0


def test_trained_network_gains_over_the_identity_start(reg, syn):
    """Trained on 512 pairs of large-motion series (plain-method targets), the
    network's initial displacements bring the registered series of a held-out
    series closer to the generator's ground truth than the identity start."""
    import torch
    from paper_1712_02533_gb300 import learned
    X, T = learned.training_set(512, seed=100)
    with reg.Cnn(syn.cnn_params(1), side=256, max_batch=64) as net:
        hist = learned.train(net, X, T, epochs=12, batch=32, lr=1e-3)
        assert hist[-1] < 0.5 * hist[0]
        fr, gt, _ = syn.series(999, 24, 256, ground_truth=True, **learned.TRAIN_SERIES)
        p = reg.default_params(n_levels=3, iter_max=50, lam=10.0)
        err = {}
        for name in ("identity", "learned", "learned_tc"):
            with reg.Series(fr, p) as s:
                if name != "identity":
                    s.cnn_init(net, tensor_cores=name == "learned_tc")
                s.prefix_scan(reg.SKLANSKY)
                d = s.get_deformations()
            err[name] = float(np.abs(d[1:] - gt[1:])[:, :, 16:-16, 16:-16].mean())
    assert err["learned"] < 0.8 * err["identity"], err
    assert err["learned_tc"] < 0.8 * err["identity"], err


@pytest.mark.parametrize("side,batch", [(64, 2), (36, 3), (88, 3)])
def test_tensor_core_training_gradients_match_the_bf16_operand_oracle(reg, side, batch):
    """Training on the tensor cores (reg_cnn_loss_grad_tc): the 32-channel
    layers' forward and weight gradients and the stride-1 layers' data
    gradients take BF16 operands.  Against the oracle with the same operand
    rounding the loss and every parameter gradient agree to FP32 accumulation
    plus the rare operand that rounds the other way; against the exact oracle
    they differ by the BF16 operand error.  Sides 36 and 88 give ragged tiles.

    An operand that rounds the other way moves the pre-activations of its
    cone by about a BF16 unit, which can turn a ReLU mask near zero; a turned
    mask passes a full gradient term.  The oracle shows the same sensitivity:
    its own gradients move that much when its input moves by one FP32 unit.
    The bound per layer is therefore the larger of a fixed floor and four
    times that spread (elementwise maximum over two perturbations)."""
    import torch
    import synth
    from oracle import cnn as ocnn
    rng = np.random.default_rng(side + 1)
    theta = (synth.cnn_params(9) + 0.01 * rng.standard_normal(ocnn.n_params())).astype(np.float32)
    x = rng.standard_normal((batch, 2, side, side)).astype(np.float32)
    q = side // 4
    t = rng.standard_normal((batch, 2, q, q)).astype(np.float32)
    with reg.Cnn(theta, side=side, max_batch=batch) as net:
        loss, g = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), want_grad=True,
                                tensor_cores=True)
    th, x64, t64 = theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64)
    lb, gb = ocnn.loss_and_grad(th, x64, t64, **TC_TRAIN)
    le, ge = ocnn.loss_and_grad(th, x64, t64)
    spread = np.zeros_like(gb)
    for seed in (7, 8):
        xp = x64 * (1.0 + 2.0 ** -24 * np.random.default_rng(seed).standard_normal(x.shape))
        spread = np.maximum(spread, np.abs(ocnn.loss_and_grad(th, xp, t64, **TC_TRAIN)[1] - gb))
    assert abs(loss - lb) <= 1e-4 * lb, (loss, lb, le)
    worst_b, worst_e = 0.0, 0.0
    for k, ((gw, gbias), (bw, bb), (ew, eb), (sw, _)) in enumerate(zip(ocnn.unpack(g.astype(np.float64)),
                                                                       ocnn.unpack(gb), ocnn.unpack(ge),
                                                                       ocnn.unpack(spread))):
        sc = np.abs(bw).max()
        err = np.abs(gw - bw)
        tol_max = max(2e-2 * sc, 4.0 * sw.max())
        tol_med = max(2e-4 * sc, 4.0 * np.median(sw))
        print(f"layer {k}: max {err.max() / sc:.2e} (bound {tol_max / sc:.2e}), median {np.median(err) / sc:.2e} "
              f"(bound {tol_med / sc:.2e}) of the largest gradient")
        assert err.max() <= tol_max and np.median(err) <= tol_med, (k, err.max() / sc, np.median(err) / sc)
        assert np.abs(gbias - bb).max() <= 2e-2 * np.abs(bb).max(), k
        worst_b = max(worst_b, float(err.max() / sc))
        worst_e = max(worst_e, float(np.abs(gw - ew).max() / np.abs(ew).max()))
    print(f"TC training gradients: max rel. error {worst_b:.2e} against the BF16-operand oracle, "
          f"{worst_e:.2e} against the exact oracle")
    assert worst_e <= 0.2


def test_tensor_core_training_learns(reg, syn):
    """A network trained with the tensor-core loss and gradients (512
    large-motion pairs, plain-method targets) lowers its loss like the FP32
    training does, and its training passes are faster."""
    from paper_1712_02533_gb300 import learned
    X, T = learned.training_set(512, seed=100)
    hist = {}
    for tc in (False, True):
        with reg.Cnn(syn.cnn_params(1), side=256, max_batch=64) as net:
            hist[tc] = learned.train(net, X, T, epochs=6, batch=32, lr=1e-3, tensor_cores=tc)
            ms, tf = learned.training_rate(net, batch=32, tensor_cores=tc)
            print(f"training {'tensor cores' if tc else 'CUDA cores'}: losses {[round(h, 5) for h in hist[tc]]}, "
                  f"{ms:.3f} ms per 32-pair pass, {tf:.1f} TFLOP/s")
    assert hist[True][-1] < 0.6 * hist[True][0]
    assert hist[True][-1] < 1.2 * hist[False][-1]
