"""The learned warm start in the simulator: interface features and targets, the learned
start with a zero network (must reproduce the previous-step warm start), and what a
trained network gains over the previous-step warm start."""
import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2302_14344_gb300 import learned, subadmm, warmstart
    return subadmm, warmstart, learned


def _features(sa, sim, nif):
    import torch
    x = torch.empty((nif, 32), device="cuda")
    sa.sim_interface_features(sim.h, x.data_ptr())
    return x


def test_features_of_chain_joints_and_robot_feet(mods):
    sa, ws, lr = mods
    p = sg.chain(1)
    sim = sa.Simulation(p)
    x = _features(sa, sim, len(p.scenes[0].ifs)).cpu().numpy()
    for i, itf in enumerate(p.scenes[0].ifs):
        assert np.array_equal(x[i, :4], [1, 0, 0, 0])                 # equality rows
        assert np.abs(x[i, 4:7]).max() < 1e-6                       # anchors coincide at t = 0
        assert np.abs(x[i, 17:23]).max() == 0.0                     # no previous duals yet
        if itf.b is not None:
            qa = p.scenes[0].subs[itf.a[0]].bodies[itf.a[1]].q
            qb = p.scenes[0].subs[itf.b[0]].bodies[itf.b[1]].q
            w = qa[0] * qb[0] + np.dot(qa[1:], qb[1:])           # scalar part of conj(qa) qb
            assert abs(x[i, 7] - w) < 1e-6
    sim.close()
    r = sg.robots(2, n_robots=2)
    sim = sa.Simulation(r)
    nif = sum(len(sc.ifs) for sc in r.scenes)
    x = _features(sa, sim, nif).cpu().numpy()
    k = 0
    for sc in r.scenes:
        for itf in sc.ifs:
            if itf.kind == sg.PLANE_CONTACT:
                b = sc.subs[itf.a[0]].bodies[itf.a[1]]
                R = np.array(sg._quat_to_mat(b.q))
                foot = b.p + R @ itf.anchor_a
                assert np.array_equal(x[k, :4], [0, 0, 0, 1])
                assert abs(x[k, 28] - foot[2]) < 1e-5 and abs(x[k, 26] - itf.mu) < 1e-6
            k += 1
    sim.close()


def test_targets_are_the_dual_change_on_the_interface_rows(mods):
    import torch
    sa, ws, lr = mods
    p = sg.robots(3, n_robots=3)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    sim.step(20)
    nif = sum(len(sc.ifs) for sc in p.scenes)
    lam_prev = np.concatenate([sim.scene_lam(k) for k in range(3)])
    x = _features(sa, sim, nif)
    sim.step(1)
    t = torch.empty((nif, 7), device="cuda")
    m = torch.empty((nif, 7), device="cuda")
    sa.sim_interface_targets(sim.h, x.data_ptr(), t.data_ptr(), m.data_ptr())
    lam = np.concatenate([sim.scene_lam(k) for k in range(3)])
    t, m = t.cpu().numpy(), m.cpu().numpy()
    row = 0
    for i in range(nif):
        rows = sim.if_rows[i]
        # the dual rows, plus column 6 (log2 beta scale): target 0, the trace rule
        assert m[i, :6].sum() == min(rows, 6) and m[i, 6] == 1 and t[i, 6] == 0
        for r in range(min(rows, 6)):
            want = lam[row + r] - np.float32(lam_prev[row + r])
            assert abs(t[i, r] - want) <= 1e-6 * max(1.0, abs(lam[row + r]))
        row += rows
    sim.close()


@pytest.mark.parametrize("grid", [False, True])
def test_zero_network_reproduces_the_previous_step_warm_start(mods, grid):
    """With all parameters zero the network proposes no change: lambda^0 is the previous
    step's lambda, so the trajectory equals the plain warm start's bit for bit (a first
    fallback only costs iterations)."""
    sa, ws, lr = mods
    if grid:
        p = sg.fem_beam(0, ny=3, nz=3, planes=8, slabs=3, length=0.03, width=0.01, height=0.01)
    else:
        p = sg.robots(4, n_robots=4)
    kw = {"grid_side_rows": 1} if grid else {}
    a = sa.Simulation(p, precision=sa.SIM_MIXED, **kw)
    b = sa.Simulation(p, precision=sa.SIM_MIXED, **kw)
    net = ws.Network(lr.SIZES)
    for _ in range(4):
        a.step(1)
    b.step_learned(net, 4)
    n = len(p.scenes)
    for k in range(n):
        assert np.array_equal(a.scene_vhat(k), b.scene_vhat(k))
        assert np.array_equal(a.scene_lam(k), b.scene_lam(k))
    sa_ = a.iteration_stats()
    sb = b.iteration_stats()
    assert sb["fallbacks"] >= n                           # every scene's first learned step
    assert sb["total_iters"] >= sa_["total_iters"]


def test_learned_steps_by_graph_replay_equal_direct_ones(mods):
    sa, ws, lr = mods
    p = sg.robots(5, n_robots=6)
    net = lr.init_network(seed=2)              # an untrained network: nonzero corrections
    a = sa.Simulation(p, precision=sa.SIM_MIXED)
    b = sa.Simulation(p, precision=sa.SIM_MIXED)
    b.use_graph(True)
    for n in (2, 2, 2, 3, 3, 1):     # captures at each new count, replays the repeats
        a.step_learned(net, n)
        b.step_learned(net, n)
    for k in range(6):
        assert np.array_equal(a.scene_vhat(k), b.scene_vhat(k))
        assert np.array_equal(a.scene_lam(k), b.scene_lam(k))
    assert a.iteration_stats() == b.iteration_stats()


def test_trained_network_against_the_previous_step_warm_start(mods, capsys):
    """Train on robots from two seeds after landing (steps 200-400), evaluate on a third
    (steps 250-350): iterations per scene-step of the learned start against the
    previous-step warm start (the fallback bounds any loss by 10 iterations per
    scene-step)."""
    sa, ws, lr = mods
    parts = [lr.collect(sg.robots(s, n_robots=64), steps=200, warmup=200) for s in (11, 12)]
    import torch
    X = torch.cat([q[0] for q in parts]); T = torch.cat([q[1] for q in parts])
    M = torch.cat([q[2] for q in parts])
    net = lr.init_network(seed=1)
    losses = lr.train(net, X, T, M, epochs=8)
    res = lr.compare(sg.robots(13, n_robots=64), net, steps=100, warmup=250)
    with capsys.disabled():
        print(f"\n[learned warm start, 64 robots, {X.shape[0]} training samples] loss "
              f"{losses[0]:.3e} -> {losses[-1]:.3e}; iterations per scene-step: plain "
              f"{res['plain']['iters_per_scene_step']:.1f}, learned "
              f"{res['learned']['iters_per_scene_step']:.1f} ({res['learned']['fallbacks']} "
              f"fallbacks in {100 * 64} scene-steps); ms per step: plain "
              f"{res['plain']['ms_per_step']:.3f}, learned {res['learned']['ms_per_step']:.3f}")
    assert losses[-1] < losses[0]
    assert (res["learned"]["iters_per_scene_step"]
            <= res["plain"]["iters_per_scene_step"] + 10.0)


def test_learned_rho_on_uneven_batched_scenes(mods, capsys):
    """The learned beta scale where the trace rule of Sec. III-D is far from the best one:
    uneven batched scenes.  Training samples come from a rho search on 128 scenes (each scene
    in seven copies, beta scaled 2^-3 .. 2^3, the largest scale within 10% of the fewest
    iterations labelling the step);
    evaluation on 512 other scenes after 100 steps, 20 steps in one launch for both forms:
    the learned start needs at least 5% fewer iterations per scene-step and leaves fewer
    scene-steps at the iteration limit."""
    sa, ws, lr = mods
    X, T, M = lr.collect_rho(sg.batched(201, n_scenes=128), steps=20, warmup=100, slack=0.1)
    net = lr.init_network(seed=3)
    losses = lr.train(net, X, T, M, epochs=6)
    res = lr.compare(sg.batched(202, n_scenes=512), net, steps=20, warmup=100, per_launch=20)
    pl, le = res["plain"], res["learned"]
    with capsys.disabled():
        print(f"\n[learned rho, batched scenes, {X.shape[0]} samples] iterations per scene-step "
              f"{pl['iters_per_scene_step']:.1f} -> {le['iters_per_scene_step']:.1f}; at the "
              f"limit {pl['not_converged']} -> {le['not_converged']}; ms per step "
              f"{pl['ms_per_step']:.2f} -> {le['ms_per_step']:.2f}")
    assert losses[-1] < losses[0]
    assert le["iters_per_scene_step"] < 0.95 * pl["iters_per_scene_step"]
    assert le["not_converged"] < pl["not_converged"]
