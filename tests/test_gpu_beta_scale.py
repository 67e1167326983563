"""Per-subsystem beta scales (the input a learned rho sets): FP64 parity with the oracle given
the same scales, including a scale change on blocks whose factor is kept across steps (the
changed K_i = A_i + beta_i J^T J must be factorised again)."""
import numpy as np
import pytest

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-12))


@pytest.fixture(scope="module")
def sa():
    from paper_2302_14344_gb300 import subadmm
    subadmm.load()
    return subadmm


def _scales(p, seed):
    rng = np.random.default_rng(seed)
    return [[float(2.0 ** rng.integers(-3, 4)) for _ in sc.subs] for sc in p.scenes]


def _apply(sim, orcs, scales):
    flat = [s for sc in scales for s in sc]
    sim.set_beta_scale(flat)
    for o, sc in zip(orcs, scales):
        for i, s in enumerate(sc):
            o.set_beta_scale(i, s)


@pytest.mark.parametrize("maker", ["generic", "robots", "batched"])
def test_beta_scales_fp64_against_oracle(sa, maker):
    if maker == "generic":
        p = sg.generic(31, n_scenes=4, max_iters=40, tol_primal=-1, n_sub=4, max_sides=3)
    elif maker == "robots":
        p = sg.robots(5, n_robots=3, max_iters=50, tol_primal=-1, drop=(0.0, 0.0))
    else:
        p = sg.batched(9, n_scenes=3, max_iters=30, tol_primal=-1)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    for step in range(3):
        _apply(sim, orcs, _scales(p, 100 + step))
        sim.step(1)
        for o in orcs:
            o.step()
        for k, o in enumerate(orcs):
            assert rel(sim.scene_vhat(k), o.vhat_all()) < 1e-9, (maker, step, k)
            for i, sid in enumerate(sim.sub_ids[k]):
                assert abs(sim.beta(sid) - o.beta(i)) <= 1e-12 * o.beta(i)


@pytest.mark.parametrize("grid", [False, True])
def test_beta_scale_change_refactorises_kept_blocks(sa, grid):
    """Linear blocks keep their factor across steps; a new scale changes K_i, so the next step
    factorises it again: FP64 parity over scale 1, 1, 2, 2, 1/4 (block and grid kernel)."""
    p = sg.fem_beam(0, ny=3, nz=3, planes=8, slabs=3, length=0.03, width=0.01, height=0.01,
                    tol_primal=-1, max_iters=30)
    o = oracle.OracleScene(p.scenes[0], p.options)
    sim = sa.Simulation(p, grid_side_rows=1 if grid else None)
    n = len(p.scenes[0].subs)
    for s in (1.0, 1.0, 2.0, 2.0, 0.25):
        _apply(sim, [o], [[s] * n])
        sim.step(1)
        o.step()
        assert rel(sim.scene_vhat(0), o.vhat_all()) < 1e-9, s
        assert rel(sim.scene_nodes(0), o.nodes_all()) < 1e-9, s
