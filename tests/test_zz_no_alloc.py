"""The allocation-free energy entry point (reg_eval_energy_noalloc).

Callers that must not allocate device memory (a plug-in inside an
acquisition pipeline whose host application reserved the device memory up
front, or a per-frame loop that cannot afford the synchronisation cudaMalloc
implies) get one entry point that works from buffers they pass in and a
fixed-size scratch array inside the library.  These tests check it through the
C-ABI against the handle-based reg_eval_energy on two calls in a row, and that
it refuses sizes its scratch array cannot hold.  This file is named so that
pytest collects it last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1712_02533_gb300 import _build
    _build.build()
    import paper_1712_02533_gb300 as r
    return r


def _field(n, seed, amp):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.stack([amp * np.sin(2 * np.pi * (X + 0.3 * Y) + 0.4), amp * np.cos(2 * np.pi * (0.7 * X - Y))])
    return (u + rng.uniform(-0.2, 0.2, size=u.shape)).astype(np.float32)


def test_noalloc_energy_matches_handle_entry_point_twice(reg, syn):
    import torch
    side, lam = 256, 10.0
    n, level = side + 1, 8
    fr = syn.series(3, 2, side, peak=10.0, spacing=10.0, sigma=2.0)
    # the finest level as the library embeds a frame: last row and column repeated
    R = torch.from_numpy(np.pad(fr[0], ((0, 1), (0, 1)), mode="edge")).cuda()
    T = torch.from_numpy(np.pad(fr[1], ((0, 1), (0, 1)), mode="edge")).cuda()
    with reg.Series(fr, reg.default_params(n_levels=2, lam=lam)) as s:
        for seed, amp in [(0, 1.3), (1, 3.0)]:  # two calls in a row share the scratch array
            u = _field(n, seed, amp)
            want = s.eval_energy(0, 1, level, u)
            got = reg.eval_energy_noalloc(R, T, torch.from_numpy(u).cuda(), lam)
            scale = abs(want["ncc"]) + abs(want["reg"])
            for k in ("E", "ncc", "reg"):
                assert abs(got[k] - want[k]) <= 1e-5 * scale, (seed, k, got, want)


def test_noalloc_rejects_sizes_beyond_its_scratch(reg):
    import torch
    lib = reg._load()
    t = torch.zeros(16, device="cuda")
    parts = np.zeros(5)
    too_big = 2049 + 1  # REG_NOALLOC_MAX_NODES + 1
    rc = lib.reg_eval_energy_noalloc(t.data_ptr(), t.data_ptr(), too_big, too_big, t.data_ptr(), 1.0,
                                     parts.ctypes.data, 0, None)
    assert rc == reg.EINVAL
    rc = lib.reg_eval_energy_noalloc(None, t.data_ptr(), 17, 17, t.data_ptr(), 1.0, parts.ctypes.data, 0, None)
    assert rc == reg.EINVAL


@pytest.mark.parametrize("side,offset", [(256, 0.0), (256, 1000.0), (2048, 0.0)])
def test_noalloc_energy_matches_oracle(reg, orc, syn, side, offset):
    """Against the FP64 oracle directly: raw embedded frames (a constant
    offset of 1000 counts makes the mean large against the spread, where a
    one-pass variance would cancel), and the largest size the scratch array
    holds (frames of 2048^2, REG_NOALLOC_MAX_NODES nodes per side)."""
    import torch
    lam = 10.0
    n = side + 1
    fr = syn.series(5, 2, side, peak=10.0, spacing=12.0, sigma=2.0) + np.float32(offset)
    R, T = orc.embed(fr[0]), orc.embed(fr[1])
    Rt = torch.from_numpy(R.astype(np.float32)).cuda()
    Tt = torch.from_numpy(T.astype(np.float32)).cuda()
    for seed, amp in [(2, 0.7), (3, 2.5)]:
        u = _field(n, seed, amp)
        got = reg.eval_energy_noalloc(Rt, Tt, torch.from_numpy(u).cuda(), lam)
        E, parts = orc.energy(R, T, u.astype(np.float64) / side, lam)
        scale = abs(parts["ncc"]) + abs(parts["reg"])
        assert abs(got["E"] - E) <= 1e-5 * scale, (side, offset, seed, got, E)
        assert abs(got["ncc"] - parts["ncc"]) <= 1e-5 * abs(parts["ncc"])
        assert abs(got["reg"] - parts["reg"]) <= 1e-5 * abs(parts["reg"])
        assert abs(got["Tbar"] - parts["Tbar"]) <= 1e-5 * abs(parts["Tbar"])
        assert abs(got["sigT"] - parts["sigT"]) <= 1e-5 * parts["sigT"]
