"""sim_read_state_noalloc: the state read for callers that cannot allocate device memory
(a control loop that must not block on the allocator, or a framework that owns all device
memory under a fixed budget).  It stages through the library's fixed 1 MiB device array
instead of a buffer of the simulation, so its output must equal sim_read_state's, call
after call.  This file is collected last on purpose."""
import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu


def _pinned(n):
    import torch
    return torch.full((n,), float("nan"), dtype=torch.float64).pin_memory()


def test_noalloc_read_matches_read_state_on_two_calls_in_a_row():
    from paper_2302_14344_gb300 import subadmm as sa
    p = sg.robots(5, n_robots=8)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    nb = sim.sizes()["bodies"]
    for _ in range(2):
        sim.step(3)
        ref, got = _pinned(13 * nb), _pinned(13 * nb)
        sa.sim_read_state(sim.h, ref.data_ptr())
        sa.sim_read_state_noalloc(sim.h, got.data_ptr())
        # the same bytes copied through another staging buffer: equal exactly, which is
        # within any tolerance the other tests use
        assert np.array_equal(ref.numpy(), got.numpy())
        assert np.isfinite(got.numpy()).all()
    sim.close()


def test_noalloc_read_rejects_unlaid_and_oversized_simulations():
    from paper_2302_14344_gb300 import subadmm as sa
    fresh = sa.Simulation(sg.robots(1, n_robots=1))
    buf = _pinned(13 * 13)
    with pytest.raises(sa.SimError) as ei:
        sa.sim_read_state_noalloc(fresh.h, buf.data_ptr())   # not laid out: it would allocate
    assert ei.value.code == sa.SIM_EINVAL
    fresh.close()
    big = sa.Simulation(sg.robots(2, n_robots=800))              # 10400 bodies > 10082
    assert big.sizes()["bodies"] == 10400
    buf = _pinned(13 * 10400)
    with pytest.raises(sa.SimError) as ei:
        sa.sim_read_state_noalloc(big.h, buf.data_ptr())
    assert ei.value.code == sa.SIM_EINVAL
    big.close()
