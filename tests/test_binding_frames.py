"""Host-side marshalling of the Series binding (no GPU): what the creation call
receives for torch frames.  A single tensor reaches reg_create_series as the
caller's own memory (a view: no host copy, and a pinned tensor stays pinned
for a direct DMA upload); several tensors of one side are concatenated in
order; several sides need host frames (numpy), as reg.h's common-pitch layout
asks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def captured(monkeypatch):
    import paper_1712_02533_gb300 as reg
    seen = {}

    def fake_create(frames, counts, sides, params, stream, use_torch_allocator):
        seen["frames"], seen["counts"], seen["sides"] = frames, list(counts), list(sides)
        return None, params

    monkeypatch.setattr(reg, "create_series", fake_create)
    return reg, seen


def test_single_tensor_is_passed_as_a_view(captured):
    reg, seen = captured
    f = torch.arange(3 * 8 * 8, dtype=torch.float32).reshape(3, 8, 8)
    s = reg.Series([f])
    s.h = None  # nothing was created
    assert seen["frames"].data_ptr() == f.data_ptr()
    assert tuple(seen["frames"].shape) == (24, 8)
    assert seen["counts"] == [3] and seen["sides"] == [8]


def test_several_tensors_of_one_side_are_concatenated_in_order(captured):
    reg, seen = captured
    a = torch.zeros(2, 4, 4)
    b = torch.ones(3, 4, 4)
    s = reg.Series([a, b])
    s.h = None
    fr = seen["frames"]
    assert tuple(fr.shape) == (20, 4)
    assert float(fr[:8].sum()) == 0.0 and float(fr[8:].sum()) == 12 * 4.0
    assert seen["counts"] == [2, 3] and seen["sides"] == [4, 4]


def test_mixed_sides_need_host_frames(captured):
    reg, _ = captured
    with pytest.raises(ValueError):
        reg.Series([torch.zeros(2, 4, 4), torch.zeros(2, 8, 8)])
    # host frames of mixed sides are laid out with the common pitch instead
    reg.Series([np.zeros((2, 4, 4), np.float32), np.ones((1, 8, 8), np.float32)]).h = None
