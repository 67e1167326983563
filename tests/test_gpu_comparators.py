"""The paper's comparison solver that this library runs itself: full-system ADMM (Sec. IV-B,
FADMM), i.e. the same iteration on each scene merged into one subsystem
(scenegen.merged).  FP64 parity with the oracle on the merged scenes, fixed iterations."""
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


def test_full_system_admm_robots_fp64(sa):
    p = sg.merged(sg.robots(3, n_robots=3, max_iters=60, tol_primal=-1, drop=(0.0, 0.0)))
    assert all(len(sc.subs) == 1 and sc.subs[0].n == 78 for sc in p.scenes)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p)
    for _ in range(4):
        sim.step(1)
        for o in orcs:
            o.step()
        for k, o in enumerate(orcs):
            assert rel(sim.scene_vhat(k), o.vhat_all()) < 1e-9
            assert rel(sim.scene_bodies(k)[:, 4:], o.bodies_all()[:, 4:]) < 1e-9


def test_full_system_admm_generic_converged(sa):
    p = sg.merged(sg.generic(21, n_scenes=4, tol_primal=1e-9, max_iters=20000, warm="prev",
                             n_range=(6, 12), types=(sg.EQUALITY, sg.SOFT, sg.HARD, sg.CONTACT)))
    orcs = oracle.run(p, steps=2)
    sim = sa.Simulation(p)
    sim.step(2)
    for k, o in enumerate(orcs):
        r, ro = sim.residuals(k), o.residuals()
        assert r["converged"] == ro["converged"]
        assert abs(r["iters"] - ro["iters"]) <= 1
        assert rel(sim.scene_vhat(k), o.vhat_all()) < 1e-6


@pytest.mark.parametrize("grid", [False, True])
def test_cable_fp64_fixed_iterations(sa, grid):
    """The cable scene (discrete rod: ball joints and PD bending / twist rows between
    segments, plane contacts, two arm stand-ins holding the ends), shortened to 24 segments in
    6 subsystems: FP64 at a fixed 60 iterations per step against the oracle, block and grid
    kernel."""
    p = sg.cable(0, segments=24, tol_primal=-1, max_iters=60)
    orcs = [oracle.OracleScene(sc, p.options) for sc in p.scenes]
    sim = sa.Simulation(p, grid_side_rows=1 if grid else None)
    for _ in range(3):
        sim.step(1)
        for o in orcs:
            o.step()
        assert rel(sim.scene_vhat(0), orcs[0].vhat_all()) < 1e-9
        assert rel(sim.scene_bodies(0)[:, 4:], orcs[0].bodies_all()[:, 4:]) < 1e-9
