"""Co-rotational FEM slabs (the paper's beam model): each step assembles every element's
rotation, rotated stiffness and force, and refactorises the slabs (never kept).  FP64 parity
with the oracle (block and grid kernel); the mixed form refactorising every step on the
tensor-core map against the FP64 oracle."""
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


def _beam(**kw):
    base = dict(ny=3, nz=3, planes=8, slabs=3, length=0.03, width=0.01, height=0.01,
                corotational=True)
    base.update(kw)
    return sg.fem_beam(0, **base)


def _tilted(p, angle=0.6):
    """The beam rotated about x by `angle` (rest shape kept): large rotations, where the
    co-rotational force differs from the linear model's."""
    c, s_ = np.cos(angle), np.sin(angle)
    Q = np.array([[1, 0, 0], [0, c, -s_], [0, s_, c]])
    for sub in p.scenes[0].subs:
        if hasattr(sub, "Kv"):
            x = sub.x.reshape(-1, 3)
            sub.x = (x @ Q.T + np.array([0.0, 0.0, 0.02])).ravel()
    return p


@pytest.mark.parametrize("grid", [False, True])
def test_corotational_fp64_against_oracle(sa, grid):
    p = _tilted(_beam(tol_primal=-1, max_iters=30, with_gripper=False))
    o = oracle.OracleScene(p.scenes[0], p.options)
    sim = sa.Simulation(p, grid_side_rows=1 if grid else None)
    for _ in range(3):
        sim.step(1)
        o.step()
        assert rel(sim.scene_vhat(0), o.vhat_all()) < 1e-9
        assert rel(sim.scene_nodes(0), o.nodes_all()) < 1e-9


def test_corotational_mixed_tensor_core_map_against_oracle(sa, capsys):
    """Slabs of >= 128 DOF in the mixed form on the grid kernel: every step takes the
    tensor-core path (setup with the element pass, the blocked factorisation, tcgen05 Gram,
    iterations)."""
    p = _tilted(_beam(ny=8, nz=8, tol_primal=-1, max_iters=30, with_gripper=False))
    assert all(s.n >= 128 for s in p.scenes[0].subs)
    o = oracle.OracleScene(p.scenes[0], p.options)
    a = sa.Simulation(p, precision=sa.SIM_MIXED, grid_side_rows=1)
    b = sa.Simulation(p, precision=sa.SIM_MIXED, grid_side_rows=1)
    b.tensor_cores(False)
    errs = []
    for _ in range(3):
        a.step(1)
        b.step(1)
        o.step()
        da, db = rel(a.scene_vhat(0), o.vhat_all()), rel(b.scene_vhat(0), o.vhat_all())
        errs.append((da, db))
        assert a.residuals(0)["status"] == 0
        assert da <= 3 * db + 1e-6
    with capsys.disabled():
        print(f"\n[co-rotational slabs, mixed, 30 iterations] v-hat rel err vs FP64 oracle: "
              f"tensor-core map {', '.join(f'{x:.2e}' for x, _ in errs)}; CUDA-core map "
              f"{', '.join(f'{y:.2e}' for _, y in errs)}")


def test_corotational_full_beam_lays_out_and_steps(sa):
    """The full co-rotational beam (64 slabs of 900 / 1200 DOF, the arm) lays out and takes
    two converged mixed steps."""
    p = sg.fem_beam(0, corotational=True, tol_primal=1e-6, max_iters=1000)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    sim.step(2)
    r = sim.residuals(0)
    assert r["status"] == 0 and r["converged"]
    assert np.all(np.isfinite(sim.scene_nodes(0)))
