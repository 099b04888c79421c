"""The overlapped end-to-end solver: every submitted problem's result equals a
plain end-to-end solve of it, whatever the order of buffer-set reuse."""
import numpy as np
import pytest
import torch

from paper_2211_15634_gb300 import api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("dtype,shape,inv", [
    (torch.float64, (24, 20, 64), None),              # equal spacings: pre-scaled coefficient
    (torch.float64, (17, 19, 33), (30.0, 18.0, 16.0)),  # unequal spacings, odd nx
    (torch.float32, (16, 16, 64), None),
])
def test_pipeline_results_equal_plain_solves(dtype, shape, inv):
    nz, ny, nx = shape
    if inv is None:
        d = 1.0 / (max(shape) - 1)
        inv = (1.0 / d,) * 3
    lengths = tuple((n - 1) / i for n, i in zip((nx, ny, nz), inv))
    nt = 7
    probs = []
    for q in range(5):
        T0 = 1.7 + inputs.random_field(shape, 40 + q, 0.0, 1.0)
        Ci = inputs.ci_random(nx, ny, nz, seed=60 + q)
        if dtype == torch.float32:
            T0 = T0 - 1.7
        probs.append((torch.from_numpy(T0).to(dtype).pin_memory(),
                      torch.from_numpy(Ci).to(dtype).pin_memory()))
    ref = [api.solve(T0, Ci, 1.0, None, inv, nt, lengths=lengths).clone() for T0, Ci in probs]
    pipe = api.SolvePipeline(shape, dtype, 1.0, inv, nt, lengths=lengths)
    outs = [torch.empty(shape, dtype=dtype).pin_memory() for _ in probs]
    events = [pipe.submit(T0, Ci, o) for (T0, Ci), o in zip(probs, outs)]
    pipe.finish()
    assert all(e.query() for e in events)
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    assert api.device_error() == 0
    api.clear_graph_cache()


def test_pipeline_reuses_one_output_buffer_in_order():
    """The same pinned output buffer for every problem holds the last problem's result
    (copies out run in submission order)."""
    shape = (12, 12, 32)
    inv = (31.0,) * 3
    pipe = api.SolvePipeline(shape, torch.float64, 1.0, inv, 4)
    out = torch.empty(shape, dtype=torch.float64).pin_memory()
    last = None
    for q in range(4):
        T0 = torch.from_numpy(1.7 + inputs.random_field(shape, 80 + q, 0.0, 1.0)).pin_memory()
        Ci = torch.from_numpy(inputs.ci_random(32, 12, 12, seed=90 + q)).pin_memory()
        pipe.submit(T0, Ci, out)
        last = (T0, Ci)
    pipe.finish()
    assert torch.equal(out, api.solve(last[0], last[1], 1.0, None, inv, 4))
    api.clear_graph_cache()
