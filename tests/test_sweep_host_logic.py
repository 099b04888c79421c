"""Host logic of the checkpointed reverse sweep (autograd.forward_checkpointed /
backward_checkpointed) on CPU: the library calls are replaced by the oracle's step and
transposed step on host tensors, so what is checked is the bookkeeping - which states
the forward keeps (the checkpoints and the last two segments), which segment is
recomputed into which block, and which state each transposed step reads.  The gradient
must equal the oracle's own gradient bit for bit (same steps, same order) for every
checkpoint interval, including segments that do not divide nt."""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_15634_gb300 import autograd as ag
from paper_2211_15634_gb300 import inputs


class FakeBlock:
    """``count`` host grids with T0's boundary (the library's StateBlock on the device)."""

    def __init__(self, T0, count, boundary=True):
        self.grids = [T0.clone() for _ in range(max(count, 1))]
        self.count = count


class FakeApi:
    """The calls the sweep makes, on host tensors through the oracle."""

    StateBlock = FakeBlock

    def __init__(self):
        self.writes = []  # (block id, grid index) of every state the loops write

    def run_states(self, T0, block, every, Ci, lam, dt, inv, nt, *, ci_scaled=False, graph=False,
                   temporal2=False):
        assert not ci_scaled
        nslots = nt // every
        need = nslots + (2 if every > 1 and nt > 0 else 0)
        assert len(block.grids) >= need, (len(block.grids), need)
        cur, cur_slot, work_next = T0, -3, 0
        for t in range(1, nt + 1):
            if t % every == 0:
                slot = t // every - 1
            else:  # a work grid, never the one this step reads
                if cur_slot == -1 - work_next:
                    work_next ^= 1
                slot = -1 - work_next
                work_next ^= 1
            dst = block.grids[slot] if slot >= 0 else block.grids[nslots + (-1 - slot)]
            assert dst.data_ptr() != cur.data_ptr()
            out = cur.numpy().copy()  # the boundary stays T's (fixed)
            oracle.step(out, cur.numpy(), Ci.numpy(), lam, dt, *inv)
            dst.copy_(torch.from_numpy(out))
            self.writes.append((id(block), slot))
            cur, cur_slot = dst, slot
        return cur

    def adjoint(self, tbar, cibar, ybar, T, Ci, lam, dt, inv, *, ci_scaled=False):
        assert not ci_scaled
        cib = cibar.numpy()
        tbar.copy_(torch.from_numpy(oracle.adjoint_step(ybar.numpy(), T.numpy(), Ci.numpy(), cib, lam, dt,
                                                         *inv)))

    @staticmethod
    def adjoint2_supported(_):
        return False


def problem(nx=9, ny=8, nz=7, nt=13):
    T0 = inputs.t0_gaussian(nx, ny, nz)
    Ci = inputs.ci_random(nx, ny, nz)
    inv = inputs.inverse_spacing(nx, ny, nz)  # unequal spacings: no pre-scaled coefficient
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / Ci.max() / 6.1
    Tobs = oracle.run(T0, Ci * 1.1, 1.0, dt, *inv, nt)
    return T0, Ci, Tobs, dt, inv


@pytest.mark.parametrize("nt,every", [(13, 1), (13, 2), (13, 3), (13, 4), (13, 5), (13, 13), (13, 20),
                                      (12, 4), (1, 3), (2, 3), (7, 3)])
def test_sweep_bookkeeping_gives_the_oracle_gradient(monkeypatch, nt, every):
    fake = FakeApi()
    monkeypatch.setattr(ag, "api", fake)
    T0, Ci, Tobs, dt, inv = problem(nt=nt)
    T0t, Cit = torch.from_numpy(T0.copy()), torch.from_numpy(Ci.copy())
    coef = ag.coefficient(Cit, 1.0, dt, inv)
    assert coef[1] is False
    out, ckpts, kept = ag.forward_checkpointed(T0t, Cit, 1.0, dt, inv, nt, every, coef, graph=False)
    nseg = (nt - 1) // every + 1 if every > 1 else nt
    assert len(ckpts) == nseg
    if every > 1:
        assert sorted(kept) == list(range(max(0, nseg - 2), nseg))
    resid = out - torch.from_numpy(Tobs)
    dT0, dCi = ag.backward_checkpointed(resid, Cit, 1.0, dt, inv, nt, every, ckpts, coef, kept=kept,
                                        graph=False)
    L_ref, dT0_ref, dCi_ref = oracle.gradient(T0, Ci, Tobs, 1.0, dt, *inv, nt)
    assert np.array_equal(out.numpy(), oracle.run(T0, Ci, 1.0, dt, *inv, nt))
    assert np.array_equal(dT0.numpy(), dT0_ref)
    assert np.array_equal(dCi.numpy(), dCi_ref)
    # the states computed: nt in the forward, plus the recomputed segments (all but the
    # last two) in the sweep
    recomputed = sum(max(0, min(s * every + every, nt) - s * every - 1) for s in range(max(0, nseg - 2)))
    assert len(fake.writes) == nt + (recomputed if every > 1 else 0)
