"""Parity at the benchmark's full sizes and launch configurations, and checks of the
library's graph, device and measurement services.

* FEM slabs of the full beam's size (10 x 10 nodes per plane: n = 1200 and 900 DOF) on the
  grid kernel with a launch small enough that every warp stages many D rows through its two
  shared-memory buffers: FP64 against the oracle (1e-9) and bit-equal to direct reads.
* The 64-robot batch after landing, stepped 200 steps in the benchmark's launch structure
  (graph replay, autotuned variants, 50 steps per launch): sampled scenes are loaded into the
  oracle (bodies and warm-start duals) and the next step of both is compared (FP64 to 1e-9;
  the mixed form's error against the FP64 oracle is stated)."""
import numpy as np
import pytest

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu

TOL = 1e-9


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if a.size == 0 and b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-12))


@pytest.fixture(scope="module")
def sa():
    from paper_2302_14344_gb300 import subadmm
    subadmm.load()
    return subadmm


def _state(sim, n):
    return (np.concatenate([sim.scene_vhat(k) for k in range(n)]),
            np.concatenate([sim.scene_lam(k) for k in range(n)]),
            np.concatenate([sim.scene_nodes(k).ravel() for k in range(n)]),
            np.concatenate([sim.scene_bodies(k).ravel() for k in range(n)]))


def test_full_size_slabs_fp64_staged_rows_reused_against_oracle(sa):
    """Three slabs of 10 x 10 nodes (n = 1200, 900, 900) joined by node-node equality, with
    ground contacts, on a grid launch of 8 blocks (64 warps): each warp stages over 20 D
    rows per iteration through its two buffers.  FP64 at a fixed iteration count against the
    oracle over two steps, and bit-equal to the same launch reading D rows directly."""
    p = sg.fem_beam(0, ny=10, nz=10, planes=8, slabs=3, length=0.03, with_gripper=False,
                    tol_primal=-1, max_iters=8)
    assert sorted(s.n for s in p.scenes[0].subs) == [900, 900, 1200]
    a = sa.Simulation(p, grid_side_rows=1)
    b = sa.Simulation(p, grid_side_rows=1)
    for s in (a, b):
        s.grid_blocks(8)
    b.grid_staging(False)
    assert a.sizes()["side_rows"] > 3 * 64            # at least three rows per warp
    o = oracle.OracleScene(p.scenes[0], p.options)
    for _ in range(2):
        a.step(1)
        b.step(1)
        o.step()
        for x, y in zip(_state(a, 1), _state(b, 1)):
            assert np.array_equal(x, y)
        assert rel(a.scene_vhat(0), o.vhat_all()) < TOL
        assert rel(a.scene_nodes(0), o.nodes_all()) < TOL
    (ca,), (cb,) = a.launch_classes(), b.launch_classes()
    assert ca["cached"] == 2 and ca["split"] == 32 and ca["smem_bytes"] > 0
    assert cb["smem_bytes"] == 0


def _load_oracle(sim, p, k):
    """An oracle scene in the state sim's scene k has reached: bodies, and each constraint's
    warm-start lambda and z."""
    sc = p.scenes[k]
    o = oracle.OracleScene(sc, p.options)
    recs = sim.scene_bodies(k)
    r = 0
    for i, sub in enumerate(sc.subs):
        for b in range(len(sub.bodies)):
            o.set_body(i, b, recs[r])
            r += 1
    for j, iid in enumerate(sim.if_ids[k]):
        o.set_warm(j, sim.lam(iid), sim.z(iid))
    return o


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_robot_batch_after_landing_sampled(sa, precision, capsys):
    """The 64-robot workload in the benchmark's launch configuration, 200 steps (drops of
    0.3-0.5 m land between steps 125 and 160); then scenes 0, 31 and 63 continue on the
    oracle from the device's state and the next step of both is compared: FP64 to 1e-9 with
    iteration counts within one; the mixed form's v-hat error against the FP64 oracle is
    stated and bounded."""
    prec = sa.SIM_FP64 if precision == "fp64" else sa.SIM_MIXED
    p = sg.robots(0, n_robots=64, tol_primal=1e-6, max_iters=1000)
    sim = sa.Simulation(p, precision=prec)
    sim.step(1)
    sim.autotune(steps=3)
    sim.use_graph(True)
    for n in (50, 50, 50, 49):
        sim.step(n)
    orcs = {k: _load_oracle(sim, p, k) for k in (0, 31, 63)}
    sim.step(1)
    worst = 0.0
    for k, o in orcs.items():
        o.step()
        r, ro = sim.residuals(k), o.residuals()
        err = rel(sim.scene_vhat(k), o.vhat_all())
        worst = max(worst, err)
        if precision == "fp64":
            assert r["converged"] == ro["converged"]
            assert abs(r["iters"] - ro["iters"]) <= 1
            assert err < TOL
            assert rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) < TOL
        else:
            assert r["r_p"] <= 1e-6 or not r["converged"]
            assert err < 1e-3
    # the contact phase: every sampled robot carries its weight through its feet
    assert min(np.max(np.abs(o.lam_all())) for o in orcs.values()) > 0.5
    with capsys.disabled():
        print(f"\n[64 robots after landing, {precision}] next step from the device state: "
              f"v-hat rel err against the FP64 oracle {worst:.3e}")


def test_keep_factors_switch_takes_effect_under_graph_replay(sa):
    """Switching sim_keep_factors between steps with graph replay on gives the same bits as
    the same sequence launched directly (a graph captured with the old flag is dropped)."""
    p = sg.batched(3, n_scenes=4, tol_primal=-1, max_iters=30)
    a = sa.Simulation(p, precision=sa.SIM_MIXED)
    b = sa.Simulation(p, precision=sa.SIM_MIXED)
    b.use_graph(True)
    for flag in (True, True, False, False, True):
        a.keep_factors(flag)
        b.keep_factors(flag)
        a.step(1)
        b.step(1)
        for x, y in zip(_state(a, 4), _state(b, 4)):
            assert np.array_equal(x, y)


def test_library_calls_keep_the_callers_device(sa):
    import torch
    torch.cuda.set_device(0)
    p = sg.chain(0, max_iters=20, tol_primal=-1, rho=1e3)
    sim = sa.Simulation(p, device=0)
    sim.step(2)
    sim.residuals(0)
    assert torch.cuda.current_device() == 0
    sim.close()


def test_barrier_floor(sa):
    f = sa.sim_barrier_floor(0, 5000)
    assert 5.0 < f["cycles"] < 5000.0 and f["ns"] > 0.0
