"""Projected Jacobi on the device (sim_set_solver(SIM_SOLVER_PJ), the paper's PJ
comparison solver, Sec. IV-B) against the oracle's Projected Jacobi: FP64 at fixed
iteration counts to 1e-9 on random scenes with every row type (block and grid kernel), the
reduced and the full stir scene and the cable; the mixed form's distance printed and
bounded; the solver's argument checks."""
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


def _pj(p, omega):
    p.options.solver = "pj"
    p.options.pj_omega = omega
    return p


def _compare(sa, p, steps, grid=False, openmp=False):
    orcs = [oracle.OracleScene(sc, p.options, openmp=openmp) for sc in p.scenes]
    sim = sa.Simulation(p, grid_side_rows=1 if grid else None)
    worst = 0.0
    for _ in range(steps):
        sim.step(1)
        for o in orcs:
            o.step()
        for k, o in enumerate(orcs):
            worst = max(worst, rel(sim.scene_vhat(k), o.vhat_all()),
                        rel(sim.scene_lam(k), o.lam_all()))
            r, ro = sim.residuals(k), o.residuals()
            assert r["iters"] == ro["iters"] == p.options.max_iters and not r["converged"]
            # r_p travels as x - z of a side-row: |x| rounds it at ~1e-16 |x| absolute
            assert abs(r["r_p"] - ro["r_p"]) <= 1e-6 * ro["r_p"] + 1e-13 * max(1.0, np.max(
                np.abs(o.vhat_all())))
    return worst


@pytest.mark.parametrize("grid", [False, True])
def test_generic_scenes_fp64(sa, grid):
    p = _pj(sg.generic(5, n_scenes=4, tol_primal=-1, max_iters=30, warm="prev", n_range=(3, 12),
                       types=(sg.EQUALITY, sg.HARD, sg.SOFT, sg.CONTACT)), 0.5)
    assert _compare(sa, p, 4, grid) < 1e-9


def test_stir_small_fp64(sa):
    p = _pj(sg.stir(1, n_side=3, layers=3, tol_primal=-1, max_iters=30), 0.3)
    assert _compare(sa, p, 5) < 1e-9


def test_stir_full_fp64_grid(sa):
    p = _pj(sg.stir(0, tol_primal=-1, max_iters=30), 0.3)
    assert _compare(sa, p, 3, openmp=True) < 1e-9


def test_cable_fp64_grid(sa):
    p = _pj(sg.cable(0, segments=24, tol_primal=-1, max_iters=30), 0.3)
    assert _compare(sa, p, 4, grid=True) < 1e-9


def test_stir_full_mixed(sa, capsys):
    p = _pj(sg.stir(0, tol_primal=-1, max_iters=30), 0.3)
    o = oracle.OracleScene(p.scenes[0], p.options, openmp=True)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    errs = []
    for _ in range(3):
        sim.step(1)
        o.step()
        errs.append(rel(sim.scene_vhat(0), o.vhat_all()))
    with capsys.disabled():
        print(f"\n[Projected Jacobi, stir, 30 iterations, mixed form] v-hat rel err vs FP64 "
              f"oracle per step: {', '.join(f'{e:.1e}' for e in errs)}")
    assert max(errs) < 1e-2


def test_solver_argument_checks(sa):
    p = sg.chain(0)
    sim = sa.Simulation(p)
    with pytest.raises(sa.SimError):
        sa.sim_set_solver(sim.h, 7)
    with pytest.raises(sa.SimError):
        sa.sim_set_solver(sim.h, sa.SIM_SOLVER_PJ, 0.0)
    sim.step(1)
    with pytest.raises(sa.SimError):
        sa.sim_set_solver(sim.h, sa.SIM_SOLVER_PJ, 0.5)
