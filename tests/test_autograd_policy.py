"""Checkpoint-interval policy of the differentiable time loop (host logic): every
state is kept when the nt states and the sweep's working fields fit in the free
device memory with a margin, else a checkpoint every ceil(sqrt(nt)) steps."""
import torch

from paper_2211_15634_gb300 import autograd as ag

GIB = 1 << 30


def test_sqrt_interval():
    assert [ag.default_every(n) for n in (1, 2, 4, 5, 200, 1000)] == [1, 2, 2, 3, 15, 32]


def test_all_states_when_they_fit():
    field = 128 * 1024 * 1024  # 256^3 FP64
    # 200 states + working fields = 208 x 128 MiB = 26 GiB
    assert ag.choose_every(200, field, 270 * GIB) == 1
    assert ag.choose_every(200, field, 33 * GIB) == 1  # 26 GiB <= 0.8 * 33 GiB
    assert ag.choose_every(200, field, 32 * GIB) == 15  # 26 GiB > 0.8 * 32 GiB
    assert ag.choose_every(200, field, 0) == 15


def test_margin_boundary_is_inclusive():
    field = 1000
    need = (50 + ag.WORK_FIELDS) * field
    assert ag.choose_every(50, field, need / 0.8) == 1
    assert ag.choose_every(50, field, need / 0.8 - 1) == ag.default_every(50)


def test_host_tensors_take_the_sqrt_interval():
    assert ag.auto_every(torch.zeros(4, 4, 4, dtype=torch.float64), 200) == 15
