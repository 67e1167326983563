"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides get the same seeded scene descriptions.  Tolerance: FP64 results agree to 1e-9
relative: max-norm of the difference over the max-norm of the oracle's value.  The two sides
reassociate the same arithmetic (the device evaluates the v-step through the per-step map
x = c + D w, multiplies by 1/beta and 1/s, and uses u = -lambda), so they differ by rounding.

For lambda the denominator is the magnitude of the operands lambda is computed from: each
row's multiplier is -(q + e)/s with q = sum_i y_ij / beta_i (Eq. surrogate), a difference of
terms of size (|q| + |e|)/s; when a constraint carries almost no force (free fall) lambda is
far below those operands and its rounding floor is eps (|q| + |e|)/s, not eps |lambda|."""
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


def lam_scale(o, problem_scene, h):
    """max over rows of the operand magnitude of the z-step (see the module docstring)."""
    out = 0.0
    for j, itf in enumerate(problem_scene.ifs):
        subs = o.sides(j)
        beta = np.array([o.beta(i) for i in subs])
        s = np.sum(1.0 / beta)
        y = o.side(j, "y")
        e, _ = o.con_rows(j)
        q = np.abs(y / beta[:, None]).sum(0)
        kind = getattr(itf, "type", None)
        if kind is None:
            kind = {1: 0, 2: 0, 3: 2, 4: 3}[itf.kind]
        if kind == 2:
            k = getattr(itf, "k", 0.0) or itf.kp
            al = getattr(itf, "alpha", 0.0) if hasattr(itf, "J") else itf.kd / itf.kp + 0.5 * h
            out = max(out, float(np.max(k * (np.abs(e) + al * q) / (1 + s * al * k))))
        else:
            out = max(out, float(np.max((q + np.abs(e)) / s)))
    return out


def rel_lam(sim, o, k, problem):
    a, b = sim.scene_lam(k), o.lam_all()
    if a.size == 0:
        return 0.0
    scale = lam_scale(o, problem.scenes[k], problem.options.h)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), scale, 1e-12))


def _compare(sim, orcs, problem, what=("vhat", "lam", "bodies"), tol=TOL):
    for k, o in enumerate(orcs):
        if "vhat" in what:
            assert rel(sim.scene_vhat(k), o.vhat_all()) < tol, ("vhat", k)
        if "lam" in what:
            assert rel_lam(sim, o, k, problem) < tol, ("lambda", k)
        if "bodies" in what and any(hasattr(s, "bodies") for s in problem.scenes[k].subs):
            gb, ob = sim.scene_bodies(k), o.bodies_all()
            assert rel(gb[:, 4:], ob[:, 4:]) < tol, ("bodies", k)


@pytest.mark.parametrize("seed", range(5))
def test_generic_fixed_iterations(sa, seed):
    p = sg.generic(seed, n_scenes=6, max_iters=40, tol_primal=-1, n_sub=2 + seed,
                   max_sides=3)
    orcs = oracle.run(p)
    sim = sa.Simulation(p)
    sim.step(1)
    _compare(sim, orcs, p, what=("vhat", "lam"))
    for k, o in enumerate(orcs):
        r, ro = sim.residuals(k), o.residuals()
        assert r["iters"] == ro["iters"] == 40
        assert abs(r["theta"] - ro["theta"]) <= 1e-9 * max(ro["theta"], 1e-300) + 1e-30
        for j, iid in enumerate(sim.if_ids[k]):
            assert rel(sim.z(iid), o.side(j, "z")) < TOL
        for i, sid in enumerate(sim.sub_ids[k]):
            assert abs(sim.beta(sid) - o.beta(i)) <= 1e-13 * o.beta(i)


@pytest.mark.parametrize("seed", range(3))
def test_generic_converged_and_warm(sa, seed):
    p = sg.generic(10 + seed, n_scenes=5, max_iters=20000, tol_primal=1e-9, warm="prev",
                   n_range=(6, 12), types=(sg.EQUALITY, sg.SOFT, sg.HARD, sg.CONTACT))
    orcs = oracle.run(p, steps=2)
    sim = sa.Simulation(p)
    sim.step(2)
    for k, o in enumerate(orcs):
        r, ro = sim.residuals(k), o.residuals()
        assert r["converged"] == ro["converged"]
        assert abs(r["iters"] - ro["iters"]) <= 1
        assert rel(sim.scene_vhat(k), o.vhat_all()) < 1e-6


def test_chain_fixed_iterations_several_steps(sa):
    p = sg.chain(0, max_iters=100, tol_primal=-1, rho=1e3)
    o = oracle.OracleScene(p.scenes[0], p.options)
    sim = sa.Simulation(p)
    for _ in range(5):
        o.step()
        sim.step(1)
        _compare(sim, [o], p)


def test_chain_in_one_launch_equals_stepwise(sa):
    p = sg.chain(1, max_iters=100, tol_primal=-1, rho=1e3)
    a = sa.Simulation(p)
    b = sa.Simulation(p)
    a.step(6)
    for _ in range(6):
        b.step(1)
    assert np.array_equal(a.scene_bodies(0), b.scene_bodies(0))


def test_robots_fixed_iterations(sa):
    p = sg.robots(3, n_robots=4, max_iters=60, tol_primal=-1)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    for _ in range(4):
        for o in orcs:
            o.step()
        sim.step(1)
        _compare(sim, orcs, p)


def test_standing_robots_fixed_iterations_lambda_plain_relative(sa):
    """Robots whose feet start on the plane carry their weight through joints and contacts,
    so lambda is large and the plain relative measure applies to it too."""
    p = sg.robots(8, n_robots=3, max_iters=80, tol_primal=-1, drop=(0.0, 0.0))
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    for _ in range(6):
        for o in orcs:
            o.step()
        sim.step(1)
    for k, o in enumerate(orcs):
        lam_o = o.lam_all()
        assert np.max(np.abs(lam_o)) > 1.0
        assert rel(sim.scene_lam(k), lam_o) < TOL
        assert rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) < TOL


def test_robots_converged_iteration_counts(sa):
    p = sg.robots(4, n_robots=3, tol_primal=1e-6, max_iters=1000)
    orcs = oracle.run(p, steps=3)
    sim = sa.Simulation(p)
    sim.step(3)
    for k, o in enumerate(orcs):
        r, ro = sim.residuals(k), o.residuals()
        assert r["converged"] and ro["converged"]
        assert abs(r["iters"] - ro["iters"]) <= 1
        assert rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) < 1e-7


def test_full_size_robot_batch_sampled(sa):
    """The 64-robot workload in the benchmark's launch configuration (all scenes in one
    launch, several steps per launch); scenes 0, 31 and 63 checked against the oracle."""
    p = sg.robots(0, n_robots=64, tol_primal=1e-6, max_iters=1000)
    sim = sa.Simulation(p)
    sim.step(5)
    for k in (0, 31, 63):
        o = oracle.OracleScene(p.scenes[k], p.options)
        for _ in range(5):
            o.step()
        assert sim.residuals(k)["converged"]
        assert abs(sim.residuals(k)["iters"] - o.residuals()["iters"]) <= 1
        assert rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) < 1e-7


def test_edge_cases(sa):
    rng = np.random.default_rng(0)
    subs = []
    for n in (1, 2, 64):
        G = rng.standard_normal((n, n))
        subs.append(sg.GenericSub(G @ G.T + n * np.eye(n), rng.standard_normal(n)))
    ifs = [
        sg.RowsIf(sg.EQUALITY, [0, 1, 2], [rng.standard_normal((1, 1)),
                                           rng.standard_normal((1, 2)),
                                           rng.standard_normal((1, 64))], rng.standard_normal(1)),
        sg.RowsIf(sg.HARD, [2], [rng.standard_normal((8, 64))], rng.standard_normal(8)),
        sg.RowsIf(sg.CONTACT, [1, 2], [rng.standard_normal((3, 2)), rng.standard_normal((3, 64))],
                  np.array([0.1, 0.0, 0.0]), mu=0.4),
        sg.RowsIf(sg.SOFT, [0], [rng.standard_normal((2, 1))], rng.standard_normal(2), k=5.0,
                  alpha=0.1),
    ]
    lone = sg.GenericSub(np.diag([2.0, 3.0]), np.array([1.0, -1.0]))   # no constraints
    scenes = [sg.Scene(subs, ifs), sg.Scene([lone], [])]
    p = sg.Problem(scenes, sg.Options(gravity=(0, 0, 0), warm="cold", tol_primal=-1,
                                      max_iters=25))
    orcs = oracle.run(p)
    sim = sa.Simulation(p)
    sim.step(1)
    _compare(sim, orcs, p, what=("vhat", "lam"))
    assert np.allclose(sim.scene_vhat(1), [0.5, -1.0 / 3.0], rtol=1e-15)


def test_many_ragged_scenes_in_one_launch(sa):
    """More scenes than SMs, of uneven sizes (tail scenes share blocks)."""
    p = sg.generic(21, n_scenes=400, max_iters=12, tol_primal=-1, n_sub=3, n_range=(1, 9))
    sim = sa.Simulation(p)
    sim.step(1)
    for k in (0, 151, 152, 399):
        o = oracle.OracleScene(p.scenes[k], p.options)
        o.step()
        assert rel(sim.scene_vhat(k), o.vhat_all()) < TOL
        assert rel_lam(sim, o, k, p) < TOL


@pytest.mark.parametrize("seed", range(2))
def test_large_blocks_in_global_workspace_fp64(sa, seed):
    """Subsystems of 100-240 DOF do not fit a block's shared memory: their factors, maps
    and D live in the global workspace.  FP64, fixed iterations, against the oracle."""
    p = sg.generic(30 + seed, n_scenes=3, max_iters=25, tol_primal=-1, n_sub=3,
                   n_range=(100, 240), max_sides=2, extra=2)
    sim = sa.Simulation(p)
    assert any(sa.sim_scene_info(sim.h, k)["global_workspace"] for k in range(3))
    sim.step(1)
    orcs = oracle.run(p)
    _compare(sim, orcs, p, what=("vhat", "lam"))


def test_large_blocks_mixed_close_to_oracle(sa, capsys):
    p = sg.generic(40, n_scenes=2, max_iters=400, tol_primal=1e-8, n_sub=3,
                   n_range=(100, 240), max_sides=2, extra=1, warm="cold",
                   types=(sg.EQUALITY, sg.SOFT, sg.HARD))
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    assert all(sa.sim_scene_info(sim.h, k)["global_workspace"] for k in range(2))
    sim.step(1)
    orcs = oracle.run(p)
    errs = [rel(sim.scene_vhat(k), o.vhat_all()) for k, o in enumerate(orcs)]
    with capsys.disabled():
        print(f"\n[mixed vs FP64 oracle, 100-240 DOF blocks] v-hat rel err max {max(errs):.3e}")
    assert max(errs) < 1e-5


def test_linear_blocks_with_contacts_and_a_body_fp64(sa):
    """Spring blocks (linear kind), node contacts, node-world pins, a node-body ball joint:
    several steps at a fixed iteration count, FP64, against the oracle."""
    rng = np.random.default_rng(3)
    scenes = [sg.hanging_scene(rng, n_blocks=2 + k % 2) for k in range(3)]
    p = sg.Problem(scenes, sg.Options(h=1e-3, warm="prev", tol_primal=-1, max_iters=60))
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    for _ in range(4):
        for o in orcs:
            o.step()
        sim.step(1)
        _compare(sim, orcs, p)
        for k, o in enumerate(orcs):
            assert rel(sim.scene_nodes(k), o.nodes_all()) < TOL


def test_linear_blocks_converged_mixed(sa, capsys):
    """Spring blocks, mixed form to r_p <= 1e-6 over 10 steps (the factor of each block is
    kept after the first step).  The FP64 oracle's own answer at that tolerance is ~4e-4
    (relative) from the exact trajectory, so both are compared with the oracle converged to
    1e-11: the mixed form must be as close as the oracle at the same tolerance."""
    def problem(tol):
        rng = np.random.default_rng(4)
        scenes = [sg.hanging_scene(rng, n_blocks=2) for _ in range(3)]
        return sg.Problem(scenes, sg.Options(h=1e-3, warm="prev", tol_primal=tol,
                                             max_iters=400000))
    p = problem(1e-6)
    same = oracle.run(p, steps=10)
    tight = oracle.run(problem(1e-11), steps=10)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    sim.step(10)
    errs = [rel(sim.scene_nodes(k), o.nodes_all()) for k, o in enumerate(tight)]
    spreads = [rel(a.nodes_all(), o.nodes_all()) for a, o in zip(same, tight)]
    with capsys.disabled():
        print(f"\n[mixed vs FP64 oracle, spring blocks 10 steps, r_p<=1e-6] node state rel err "
              f"to the exact trajectory max {max(errs):.3e}; oracle at the same tolerance "
              f"{max(spreads):.3e}")
    for k in range(3):
        assert sim.residuals(k)["converged"]
        assert errs[k] <= 3 * spreads[k] + 0.1 * max(spreads), (k, errs[k], spreads[k])
    assert max(errs) <= 2 * max(spreads)


def _compare_states(sim, orcs, tol):
    for k, o in enumerate(orcs):
        if o.bodies_all().size:
            assert rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) < tol, ("bodies", k)
        if o.nodes_all().size:
            assert rel(sim.scene_nodes(k), o.nodes_all()) < tol, ("nodes", k)


def test_batched_uneven_scenes_fp64_fixed_iterations(sa):
    """Scenes of the batched workload (2-32 subsystems of 6-240 DOF: rigid chains and
    spring blocks, tree + chord ball joints, plane contacts); scenes too large for shared
    memory run from the global workspace.  FP64, fixed iterations, two steps."""
    p = sg.batched(1, n_scenes=6, tol_primal=-1, max_iters=40)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    assert any(sa.sim_scene_info(sim.h, k)["global_workspace"] for k in range(6))
    classes = sim.launch_classes()
    assert sum(c["scenes"] for c in classes) == 6
    for _ in range(2):
        for o in orcs:
            o.step()
        sim.step(1)
        _compare(sim, orcs, p, what=("vhat", "lam"))
        _compare_states(sim, orcs, TOL)


@pytest.mark.parametrize("tol", [1e-6, 1e-8])
def test_batched_uneven_scenes_mixed_converged(sa, capsys, tol):
    """On these scenes (long floating chains, chords) v-hat is poorly determined by the stop
    rule: the FP64 oracle's own answer at r_p <= tol is ~1e4 tol (relative) away from the
    exact step.  The mixed form must land as close to the exact step (the oracle converged to
    1e-10) as the oracle itself does at the same tolerance."""
    steps = 2
    p = sg.batched(2, n_scenes=8, tol_primal=tol, max_iters=20000)
    same = oracle.run(p, steps=steps)
    tight = oracle.run(sg.batched(2, n_scenes=8, tol_primal=1e-10, max_iters=400000),
                       steps=steps)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    sim.step(steps)
    errs, spreads = [], []
    for k in range(8):
        r = sim.residuals(k)
        assert r["converged"] and r["r_p"] <= tol, (k, r)
        ref = tight[k].vhat_all()
        errs.append(rel(sim.scene_vhat(k), ref))
        spreads.append(rel(same[k].vhat_all(), ref))
    with capsys.disabled():
        print(f"\n[mixed vs FP64 oracle, batched scenes, r_p<={tol:g}] v-hat rel err to the "
              f"exact step max {max(errs):.3e}; oracle at the same tolerance {max(spreads):.3e}")
    # a converging iteration may stop anywhere in the tolerance ball, so a scene whose oracle
    # stop happened to land close to the exact step gets a floor from the batch's spread
    for k in range(8):
        assert errs[k] <= 3 * spreads[k] + 0.1 * max(spreads), (k, errs[k], spreads[k])
    assert max(errs) <= 2 * max(spreads)


def _batch_state(sim, n):
    return (np.concatenate([sim.scene_vhat(k) for k in range(n)]),
            np.concatenate([sim.scene_lam(k) for k in range(n)]),
            np.concatenate([sim.scene_nodes(k).ravel() for k in range(n)]),
            np.concatenate([sim.scene_bodies(k).ravel() for k in range(n)]))


def test_scenes_of_different_sizes_run_in_concurrent_launch_classes(sa):
    """Small scenes (the register-cached kernel) and large ones (the generic kernel) of one
    batch are separate launches on forked streams; results match the oracle per scene."""
    small = sg.robots(11, n_robots=3).scenes
    large = sg.batched(5, n_scenes=3, tol_primal=-1, max_iters=30).scenes
    p = sg.Problem(small + large, sg.Options(h=1e-3, warm="prev", tol_primal=-1, max_iters=30,
                                             beta_mode="trace"))
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    classes = sim.launch_classes()
    assert len(classes) >= 2 and sum(c["scenes"] for c in classes) == 6
    # kernel kinds: 0 / 3 generic (256 / 512 threads), 1 register-cached
    assert any(c["cached"] == 1 for c in classes)
    assert any(c["cached"] in (0, 3) for c in classes)
    for _ in range(2):
        for o in orcs:
            o.step()
        sim.step(1)
        _compare(sim, orcs, p, what=("vhat", "lam"))


def test_graph_replay_equals_direct_launches(sa):
    p = sg.batched(6, n_scenes=5, max_iters=200)
    a = sa.Simulation(p, precision=sa.SIM_MIXED)
    b = sa.Simulation(p, precision=sa.SIM_MIXED)
    b.use_graph(True)
    for n in (2, 2, 3):
        a.step(n)
        b.step(n)
    for x, y in zip(_batch_state(a, 5), _batch_state(b, 5)):
        assert np.array_equal(x, y)
    b.use_graph(False)
    b.step(1)
    a.step(1)
    for x, y in zip(_batch_state(a, 5), _batch_state(b, 5)):
        assert np.array_equal(x, y)


def test_autotune_leaves_no_trace_and_keeps_parity(sa):
    """Tuning times kernel variants on a snapshot and restores it: the state after tuning is
    the state before, bit for bit; stepping on with the tuned variants matches the oracle."""
    import torch
    p = sg.batched(7, n_scenes=6, tol_primal=-1, max_iters=25)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    for o in orcs:
        o.step()
    sim.step(1)
    sz = sim.sizes()
    before = torch.empty(13 * sz["bodies"] + 6 * sz["nodes"], dtype=torch.float64).pin_memory()
    after = torch.empty_like(before).pin_memory()
    sa.sim_read_state(sim.h, before.data_ptr())
    lam0 = np.concatenate([sim.scene_lam(k) for k in range(6)])
    rows = sim.autotune(steps=2)
    assert sum(r["scenes"] for r in rows) == 6 and all(r["ns_per_step"] > 0 for r in rows)
    sa.sim_read_state(sim.h, after.data_ptr())
    assert np.array_equal(before.numpy(), after.numpy())
    assert np.array_equal(lam0, np.concatenate([sim.scene_lam(k) for k in range(6)]))
    assert sim.iteration_stats()["scene_steps"] == 6          # only the real step counted
    for _ in range(2):
        for o in orcs:
            o.step()
        sim.step(1)
        _compare(sim, orcs, p, what=("vhat", "lam"))


# ---------------------------------------------------------------------------------------
# grid kernel: one scene over the whole GPU


def test_grid_barrier_time_limit_raises_the_error_flag(sa):
    """The grid barrier's bounded wait: with one arrival missing nothing completes the
    barrier, every wait runs out after 50 ms and the flag is raised; with all arrivals the
    barrier passes without it."""
    r = sa.sim_probe_barrier(0, 4, 5, 0.05)
    assert r["timed_out"] and r["passed"] == 4
    r = sa.sim_probe_barrier(0, 4, 4, 0.05)
    assert not r["timed_out"] and r["passed"] == 4


def _small_beam(**kw):
    base = dict(ny=3, nz=3, planes=8, slabs=3, length=0.03, width=0.01, height=0.01)
    base.update(kw)
    return sg.fem_beam(0, **base)


@pytest.mark.parametrize("grid", [False, True])
def test_small_fem_beam_fp64_fixed_iterations(sa, grid):
    """Tetrahedral slabs coupled by node-node equality, ground contacts on the bottom nodes
    and a 7-R arm holding one end: FP64 at a fixed iteration count, block kernel and grid
    kernel, against the oracle over three steps."""
    p = _small_beam(tol_primal=-1, max_iters=40)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p, grid_side_rows=1 if grid else None)
    kinds = {c["cached"] for c in sim.launch_classes()}
    assert kinds == ({2} if grid else kinds - {2})
    for _ in range(3):
        for o in orcs:
            o.step()
        sim.step(1)
        _compare(sim, orcs, p)
        _compare_states(sim, orcs, TOL)


@pytest.mark.parametrize("grid", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_refactoring_every_step_matches_the_kept_factors(sa, grid, precision):
    """Constant (linear) blocks keep their factor, W and D across steps by default; with
    sim_keep_factors(0) every step computes them again, as Algorithm 1 states it.  The
    matrix is the same; g = L^-1 b comes from the multi-column solve instead of the
    single-vector one, so the two agree to rounding.  FP64: both match the oracle (which
    refactors every step) to 1e-9; mixed: they agree with each other to FP32 rounding
    (1e-5 relative after 30 iterations a step)."""
    prec = sa.SIM_FP64 if precision == "fp64" else sa.SIM_MIXED
    p = _small_beam(tol_primal=-1, max_iters=30)
    a = sa.Simulation(p, precision=prec, grid_side_rows=1 if grid else None)
    b = sa.Simulation(p, precision=prec, grid_side_rows=1 if grid else None)
    b.keep_factors(False)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes] if precision == "fp64" else []
    for _ in range(3):
        a.step(1)
        b.step(1)
        for o in orcs:
            o.step()
        if orcs:
            _compare(a, orcs, p)
            _compare(b, orcs, p)
        else:
            for x, y in zip(_batch_state(a, 1), _batch_state(b, 1)):
                assert rel(y, x) < 1e-5


def _staged_and_direct(sa, p, prec):
    a = sa.Simulation(p, precision=prec, grid_side_rows=1)
    b = sa.Simulation(p, precision=prec, grid_side_rows=1)
    b.grid_staging(False)
    (ca,), (cb,) = a.launch_classes(), b.launch_classes()
    assert ca["cached"] == 2 and ca["split"] == 32 and cb["split"] == 32   # warp per side-row
    return a, b


def _assert_staged(a, b):
    (ca,), (cb,) = a.launch_classes(), b.launch_classes()
    assert ca["smem_bytes"] > 0 and cb["smem_bytes"] == 0      # staged / direct


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_staged_rows_equal_direct_rows(sa, precision):
    """The grid kernel's v-step with D rows staged in shared memory by bulk copies gives the
    same bits as the direct reads (same products, same order) over three steps of a beam of
    three slabs without the arm (warp per side-row), and matches the oracle (FP64)."""
    prec = sa.SIM_FP64 if precision == "fp64" else sa.SIM_MIXED
    p = _small_beam(ny=8, nz=8, with_gripper=False, tol_primal=-1, max_iters=40)
    a, b = _staged_and_direct(sa, p, prec)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes] if precision == "fp64" else []
    for _ in range(3):
        a.step(1)
        b.step(1)
        for x, y in zip(_batch_state(a, 1), _batch_state(b, 1)):
            assert np.array_equal(x, y)
        for o in orcs:
            o.step()
        if orcs:
            _compare(a, orcs, p)
    _assert_staged(a, b)


def test_grid_staged_rows_several_per_warp(sa):
    """Nine slabs of 10 x 10 nodes: more side-rows than warps in the grid, so a warp stages
    several rows per iteration through its two buffers (each reused, its barrier phase
    flipping every use); staged and direct reads give the same bits over two steps."""
    p = _small_beam(ny=10, nz=10, planes=21, slabs=9, with_gripper=False, tol_primal=-1,
                    max_iters=30)
    a, b = _staged_and_direct(sa, p, sa.SIM_MIXED)
    # more than two rows for some warps: 8 warps x 2 blocks x 152 SMs = 2432 warps
    assert a.sizes()["side_rows"] > 2 * 2432
    for _ in range(2):
        a.step(1)
        b.step(1)
        for x, y in zip(_batch_state(a, 1), _batch_state(b, 1)):
            assert np.array_equal(x, y)
    _assert_staged(a, b)


def test_grid_kernel_batched_scenes_fp64(sa):
    """Several uneven scenes, each run over the whole GPU in turn (the grid kernel forced
    for every scene), against the oracle; two steps in one call."""
    p = sg.batched(8, n_scenes=3, tol_primal=-1, max_iters=30)
    orcs = oracle.run(p, steps=2)
    sim = sa.Simulation(p, grid_side_rows=1)
    assert all(c["cached"] == 2 for c in sim.launch_classes())
    sim.step(2)
    _compare(sim, orcs, p, what=("vhat", "lam"))
    _compare_states(sim, orcs, TOL)


def test_grid_kernel_mixed_converged_small_beam(sa, capsys):
    def problem(tol):
        return _small_beam(tol_primal=tol, max_iters=200000)
    steps = 3
    same = oracle.run(problem(1e-6), steps=steps)
    tight = oracle.run(problem(1e-11), steps=steps)
    sim = sa.Simulation(problem(1e-6), precision=sa.SIM_MIXED, grid_side_rows=1)
    sim.step(steps)
    r = sim.residuals(0)
    assert r["converged"] and r["r_p"] <= 1e-6
    err = rel(sim.scene_vhat(0), tight[0].vhat_all())
    spread = rel(same[0].vhat_all(), tight[0].vhat_all())
    with capsys.disabled():
        print(f"\n[mixed grid kernel vs FP64 oracle, small FEM beam, r_p<=1e-6] v-hat rel err "
              f"to the exact step {err:.3e}; oracle at the same tolerance {spread:.3e}")
    assert err <= 3 * spread + 1e-6


def test_not_spd_is_reported_not_faulted(sa):
    A = -np.eye(3)
    p = sg.Problem([sg.Scene([sg.GenericSub(A, np.ones(3))], [])],
                   sg.Options(gravity=(0, 0, 0), max_iters=5))
    sim = sa.Simulation(p)
    sim.step(1)
    with pytest.raises(sa.SimError) as ei:
        sim.residuals(0)
    assert ei.value.code == sa.SIM_ENOTSPD


def test_non_finite_residual_is_reported_by_both_kernels(sa):
    """A NaN planted in one body's velocity (it enters b_i only, so K_i stays SPD) makes that
    scene's iterates non-finite: its step reports SIM_ENAN, in the register-cached kernel (a
    robot) and in the generic kernel (a large batched scene) alike, and the other scenes of
    the launch step on with finite residuals."""
    import torch
    small = sg.robots(11, n_robots=3).scenes
    large = sg.batched(5, n_scenes=3, tol_primal=-1, max_iters=30).scenes
    p = sg.Problem(small + large, sg.Options(h=1e-3, warm="prev", tol_primal=1e-6, max_iters=300,
                                             beta_mode="trace"))
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    classes = sim.launch_classes()
    # kernel kinds: 0 / 3 generic (256 / 512 threads), 1 register-cached
    assert any(c["cached"] == 1 for c in classes)
    assert any(c["cached"] in (0, 3) for c in classes)
    sim.step(1)
    nb = [len(sim.scene_bodies(k)) for k in range(6)]
    big = next(k for k in range(3, 6) if nb[k] > 0)
    sz = sim.sizes()
    st = torch.empty(13 * sz["bodies"] + 6 * sz["nodes"], dtype=torch.float64).pin_memory()
    sa.sim_read_state(sim.h, st.data_ptr())
    for k in (0, big):
        st[13 * sum(nb[:k]) + 7] = float("nan")          # v_x of the scene's first body
    sa.sim_write_state(sim.h, st.data_ptr())
    sim.step(1)
    for k in range(6):
        if k in (0, big):
            with pytest.raises(sa.SimError) as ei:
                sim.residuals(k)
            assert ei.value.code == sa.SIM_ENAN, k
        else:
            r = sim.residuals(k)
            assert np.isfinite(r["r_p"]) and r["status"] == 0, k


def test_invalid_topology_is_rejected(sa):
    p = sg.chain(0)
    sim = sa.Simulation(p)
    with pytest.raises(sa.SimError):
        sa.sim_add_interface(sim.h, 0, sa.SIM_IF_BALL, 0, 0, [0, 5, 1, 0], None, None,
                             np.zeros(23))
    with pytest.raises(sa.SimError):
        sa.sim_add_interface(sim.h, 0, sa.SIM_IF_EQUALITY, 9, 1, [0], np.zeros(9 * 12),
                             np.zeros(9), None)
    sim.step(1)
    with pytest.raises(sa.SimError):
        sa.sim_add_subsystem(sim.h, 0, sa.SIM_SUB_GENERIC, 1, np.ones(2))


def test_bitwise_deterministic(sa):
    p = sg.robots(7, n_robots=8, tol_primal=1e-6)
    a, b = sa.Simulation(p), sa.Simulation(p)
    a.step(3)
    b.step(3)
    for k in range(8):
        assert np.array_equal(a.scene_bodies(k), b.scene_bodies(k))
        assert np.array_equal(a.scene_lam(k), b.scene_lam(k))


def test_per_scene_iteration_counts_match_the_residuals(sa):
    p = sg.batched(4, n_scenes=5, max_iters=500)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    sim.step(1)
    st = sim.iteration_stats(per_scene=True)
    ps = st["per_scene"]
    assert ps.shape == (5, 5)
    assert ps[:, 0].sum() == st["total_iters"] and ps[:, 1].max() == st["max_iters"]
    assert (ps[:, 3] == 1).all() and (ps[:, 4] == 0).all()
    for k in range(5):
        r = sim.residuals(k)
        assert ps[k, 0] == ps[k, 1] == r["iters"]
        assert ps[k, 2] == (0 if r["converged"] else 1)
    assert sim.iteration_stats()["total_iters"] == 0       # cleared by the read


def test_state_roundtrip_through_host_buffers(sa):
    import torch
    p = sg.robots(1, n_robots=2)
    sim = sa.Simulation(p)
    nb = sim.sizes()["bodies"]
    buf = torch.empty(13 * nb, dtype=torch.float64).pin_memory()
    sa.sim_read_state(sim.h, buf.data_ptr())
    ref = np.concatenate([sim.scene_bodies(k)[:, 4:] for k in range(2)]).ravel()
    assert np.array_equal(buf.numpy(), ref)
    buf[2] += 1.0
    sa.sim_write_state(sim.h, buf.data_ptr())
    sim.sync()
    assert sim.scene_bodies(0)[0, 6] == ref[2] + 1.0


def test_state_roundtrip_with_nodes_of_linear_blocks(sa):
    """The packed state holds the bodies, then the nodes of the linear blocks."""
    import torch
    p = sg.batched(3, n_scenes=3)
    sim = sa.Simulation(p)
    sim.step(1)
    sz = sim.sizes()
    nb, nn = sz["bodies"], sz["nodes"]
    assert nb > 0 and nn > 0
    buf = torch.empty(13 * nb + 6 * nn, dtype=torch.float64).pin_memory()
    sa.sim_read_state(sim.h, buf.data_ptr())
    bodies = np.concatenate([sim.scene_bodies(k)[:, 4:] for k in range(3)
                             if sim.scene_bodies(k).size]).ravel()
    nodes = np.concatenate([sim.scene_nodes(k) for k in range(3)
                            if sim.scene_nodes(k).size]).ravel()
    assert np.array_equal(buf.numpy(), np.concatenate([bodies, nodes]))
    buf[13 * nb + 4] += 0.5        # v_y of the first node
    sa.sim_write_state(sim.h, buf.data_ptr())
    sim.sync()
    k0 = next(k for k in range(3) if sim.scene_nodes(k).size)
    assert sim.scene_nodes(k0).ravel()[4] == nodes[4] + 0.5


# ---------------------------------------------------------------------------------------
# mixed precision: FP64 setup and final residual check, FP32 iterations


def test_mixed_meets_the_primal_tolerance_in_fp64(sa):
    """The mixed form reports r_p from its FP64 check, so every converged scene-step has
    max|J v - z| <= tol evaluated in FP64."""
    p = sg.robots(2, n_robots=8, tol_primal=1e-6, max_iters=1000)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    for _ in range(20):
        sim.step(1)
        for k in range(8):
            r = sim.residuals(k)
            if r["converged"]:
                assert r["r_p"] <= 1e-6


def test_mixed_error_against_fp64_oracle(sa, capsys):
    """State the mixed form's error against the FP64 oracle as numbers: after 20 steps of
    the robots, both run to r_p <= 1e-6.  Each step's v-hat differs from the exact step
    solution by the stop tolerance times the condition of the step (about 1e-6 x 10 here),
    and the differences compound over the steps: the bound asserted is 1e-4 relative."""
    p = sg.robots(2, n_robots=4, tol_primal=1e-6, max_iters=1000)
    orcs = oracle.run(p, steps=20)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    sim.step(20)
    errs = [rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) for k, o in enumerate(orcs)]
    vh = [rel(sim.scene_vhat(k), o.vhat_all()) for k, o in enumerate(orcs)]
    with capsys.disabled():
        print(f"\n[mixed vs FP64 oracle, 20 steps] state rel err max {max(errs):.3e}, "
              f"v-hat rel err max {max(vh):.3e}")
    assert max(errs) < 1e-4
    assert max(vh) < 1e-3


def test_mixed_fixed_iterations_close_to_oracle(sa, capsys):
    p = sg.chain(0, max_iters=100, tol_primal=-1, rho=1e3)
    o = oracle.OracleScene(p.scenes[0], p.options)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    for _ in range(3):
        o.step()
        sim.step(1)
    e = rel(sim.scene_bodies(0)[:, 4:], o.bodies_all()[:, 4:])
    ev = rel(sim.scene_vhat(0), o.vhat_all())
    with capsys.disabled():
        print(f"\n[mixed vs FP64 oracle, chain 3 x 100 it] state rel err {e:.3e}, "
              f"v-hat rel err {ev:.3e}")
    assert e < 1e-6 and ev < 1e-4


def test_phase_trace_counts_match_iteration_stats(sa):
    p = sg.robots(3, n_robots=4, tol_primal=1e-6, max_iters=1000)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    sa.sim_phase_trace(sim.h, True)
    sim.iteration_stats()
    sim.step(3)
    tr = sa.sim_phase_trace(sim.h, False)
    st = sim.iteration_stats()
    assert tr["iterations"] == st["total_iters"] and tr["scene_steps"] == 12
    assert all(tr[k] > 0 for k in ("assemble", "factor", "v_step", "z_step", "exit", "recover"))


def test_wide_block_variant_fp64(sa):
    """Scenes that take a whole SM's shared memory launch 512-thread blocks (kernel kind 3):
    FP64 parity with the oracle, as for the 256-thread variant."""
    p = sg.batched(5, n_scenes=6, tol_primal=-1, max_iters=40, n_sub=(12, 24), n_range=(60, 240))
    sim = sa.Simulation(p)
    kinds = [c["cached"] for c in sim.launch_classes()]
    assert 3 in kinds, kinds
    orcs = oracle.run(p, steps=2)
    sim.step(2)
    for k, o in enumerate(orcs):
        assert rel(sim.scene_vhat(k), o.vhat_all()) < 1e-9
        assert rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) < 1e-9
