"""Host-side layout helpers of the Python binding: padded-row fields for the
batched z-march and the pitch the binding derives from a field's strides."""
import pytest
import torch

from paper_2211_15634_gb300 import api


@pytest.mark.parametrize("dtype,per", [(torch.float64, 2), (torch.float32, 4)])
@pytest.mark.parametrize("nx", [3, 4, 5, 33, 64, 161])
def test_pitched_rows_start_on_16_byte_boundaries(dtype, per, nx):
    t = api.pitched_empty((5, 7, nx), dtype, device="cpu")
    assert t.shape == (5, 7, nx)
    pitch = api._pitch(t, "T")
    assert pitch >= nx and pitch - nx < per and pitch * t.element_size() % 16 == 0
    assert t.stride() == (7 * pitch, pitch, 1)
    assert (pitch == nx) == t.is_contiguous()


def test_pitched_copy_keeps_values():
    a = torch.arange(3 * 4 * 5, dtype=torch.float64).reshape(3, 4, 5)
    b = api.pitched_copy(a)
    assert torch.equal(a, b) and api._pitch(b, "T") == 6


def test_pitch_rejects_other_layouts():
    a = torch.zeros((4, 6, 8), dtype=torch.float64)
    with pytest.raises(ValueError):
        api._pitch(a[:, :, ::2], "T")  # strided along x
    with pytest.raises(ValueError):
        api._pitch(a[:, :3, :], "T")  # rows cut, planes not rows*ny apart
    with pytest.raises(ValueError):
        api._pitch(a[0], "T")  # not 3-D
    assert api._pitch(a, "T") == 8


def test_solve_pipeline_rejects_mismatched_host_tensors():
    ok = torch.zeros((4, 5, 6), dtype=torch.float64)
    api.SolvePipeline.check_host((4, 5, 6), torch.float64, T0_host=ok, Ci_host=ok, out_host=ok)
    with pytest.raises(ValueError):  # would broadcast
        api.SolvePipeline.check_host((4, 5, 6), torch.float64, T0_host=torch.zeros((1, 5, 6), dtype=torch.float64))
    with pytest.raises(ValueError):  # would convert
        api.SolvePipeline.check_host((4, 5, 6), torch.float64, Ci_host=ok.float())
    with pytest.raises(ValueError):
        api.SolvePipeline.check_host((4, 5, 6), torch.float64, out_host=torch.zeros((4, 5, 6, 1), dtype=torch.float64))


def test_run_states_refuses_a_block_of_another_dtype_or_shape():
    """The state block goes to the library as a base pointer and a stride in T0's
    elements: a block of another dtype or grid shape is refused before any call."""
    T0 = torch.zeros((5, 6, 8), dtype=torch.float64)
    Ci = torch.ones_like(T0)
    for blk in (api.StateBlock(T0.float(), 4, boundary=False),
                api.StateBlock(torch.zeros((5, 6, 12), dtype=torch.float64), 4, boundary=False)):
        with pytest.raises(ValueError, match="state block"):
            api.run_states(T0, blk, 1, Ci, 1.0, 1e-3, (7.0, 5.0, 4.0), 4)
