"""Blocked Cholesky with tensor-core Schur updates (Algorithm 1, factorise; grid kernel, mixed
form).

A refactorised block of >= 128 DOF that the mixed form factorises in FP32 is factorised by
panels of 128 columns: the diagonal tile and the rows below it on the CUDA cores, the trailing
tiles inside K_i's envelope by the tcgen05 Gram kernel (C -= P P^T, split-TF32).  With
sim_tc_factor(0) the setup launch factorises it with one warp (the envelope factorisation).

* Fixed iterations: both factorisations are FP32 approximations; the blocked one differs from
  the one-warp one by rounding (~1e-6 of v-hat, amplified by the iterations), and its distance
  from the FP64 oracle's step is within 3x the one-warp factor's.  The two are not bitwise
  equal: the blocked path ran.
* The slabs' sizes leave a ragged last panel (576 = 4.5 tiles, 1200 = 9.4, 900 = 7.03), and the
  beam's envelope makes each panel reach 3-4 tiles of rows, so the trailing update covers
  diagonal and off-diagonal tiles.
* Converged to r_p <= 1e-6: the answer is as close to the exact step as the FP64 oracle's own
  answer at the same tolerance."""
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


def _pair(sa, p):
    a = sa.Simulation(p, precision=sa.SIM_MIXED, grid_side_rows=1)
    b = sa.Simulation(p, precision=sa.SIM_MIXED, grid_side_rows=1)
    b.tc_factor(False)
    for s in (a, b):
        s.keep_factors(False)
    return a, b


@pytest.mark.parametrize("corot", [False, True])
def test_blocked_factor_matches_one_warp_factor(sa, corot, capsys):
    p = sg.fem_beam(0, ny=8, nz=8, planes=8, slabs=3, length=0.03, width=0.01, height=0.01,
                    tol_primal=-1, max_iters=30, corotational=corot)
    ns = [s.n for s in p.scenes[0].subs if hasattr(s, "Kv")]
    assert min(ns) >= 128 and any(n % 128 for n in ns)
    a, b = _pair(sa, p)
    o = oracle.OracleScene(p.scenes[0], p.options)
    out = []
    for _ in range(3):
        a.step(1)
        b.step(1)
        o.step()
        assert a.residuals(0)["status"] == 0 and b.residuals(0)["status"] == 0
        d_a = rel(a.scene_vhat(0), o.vhat_all())
        d_b = rel(b.scene_vhat(0), o.vhat_all())
        d_ab = rel(a.scene_vhat(0), b.scene_vhat(0))
        out.append((d_a, d_b, d_ab))
        assert 0.0 < d_ab < 1e-4
        assert d_a <= 3 * d_b + 1e-6
        assert rel(a.scene_nodes(0), o.nodes_all()) <= 3 * rel(b.scene_nodes(0), o.nodes_all()) + 1e-7
    with capsys.disabled():
        print(f"\n[blocked tensor-core factor vs one-warp factor, corotational={corot}, 30 "
              f"iterations] v-hat rel err vs FP64 oracle per step: blocked "
              f"{', '.join(f'{x[0]:.2e}' for x in out)}; one warp "
              f"{', '.join(f'{x[1]:.2e}' for x in out)}; between them "
              f"{', '.join(f'{x[2]:.2e}' for x in out)}")


def test_blocked_factor_full_size_slabs(sa, capsys):
    """Slabs of the full beam's size (n = 1200, 900, 900), refactorised every step."""
    p = sg.fem_beam(0, ny=10, nz=10, planes=8, slabs=3, length=0.03, with_gripper=False,
                    tol_primal=-1, max_iters=20)
    assert sorted(s.n for s in p.scenes[0].subs if hasattr(s, "Kv")) == [900, 900, 1200]
    a, b = _pair(sa, p)
    o = oracle.OracleScene(p.scenes[0], p.options)
    for _ in range(2):
        a.step(1)
        b.step(1)
        o.step()
    d_ab = rel(a.scene_vhat(0), b.scene_vhat(0))
    d_a = rel(a.scene_vhat(0), o.vhat_all())
    d_b = rel(b.scene_vhat(0), o.vhat_all())
    with capsys.disabled():
        print(f"\n[full-size slabs, blocked factor, 20 iterations] v-hat: blocked vs one-warp "
              f"factor {d_ab:.2e}; vs FP64 oracle {d_a:.2e} (one warp {d_b:.2e})")
    assert 0.0 < d_ab < 1e-4
    assert d_a < 3 * d_b + 1e-5


def test_blocked_factor_converged_against_fp64_oracle(sa, capsys):
    steps = 3
    kw = dict(ny=8, nz=8, planes=8, slabs=3, length=0.03, width=0.01, height=0.01,
              max_iters=200000)
    same = oracle.run(sg.fem_beam(0, tol_primal=1e-6, **kw), steps=steps)
    tight = oracle.run(sg.fem_beam(0, tol_primal=1e-11, **kw), steps=steps)
    a = sa.Simulation(sg.fem_beam(0, tol_primal=1e-6, **kw), precision=sa.SIM_MIXED,
                      grid_side_rows=1)
    a.keep_factors(False)
    a.tc_factor(True)
    a.step(steps)
    r = a.residuals(0)
    assert r["converged"] and r["r_p"] <= 1e-6
    err = rel(a.scene_vhat(0), tight[0].vhat_all())
    spread = rel(same[0].vhat_all(), tight[0].vhat_all())
    with capsys.disabled():
        print(f"\n[blocked tensor-core factor, refactorised every step, r_p<=1e-6] v-hat rel "
              f"err to the exact step {err:.3e}; FP64 oracle at the same tolerance {spread:.3e}")
    assert err <= 3 * spread + 1e-6


def test_blocked_factor_reports_not_spd(sa):
    """An indefinite block whose diagonal spread passes the stiffness test (so the blocked
    factorisation, not the FP64 one, meets the non-positive pivot): the step ends with
    SIM_ENOTSPD status, with the blocked factorisation and with the one-warp one alike."""
    rng = np.random.default_rng(3)
    n = 160
    A = np.eye(n)
    A[0, 1] = A[1, 0] = 2.0                 # eigenvalue -1: pivot 1 - 4 < 0
    ifs = []
    for k in range(6):                      # 18 side-rows on the block, away from DOF 0 and 1
        J = np.zeros((3, n))
        J[:, 10 + 20 * k: 10 + 20 * k + 8] = rng.standard_normal((3, 8))
        ifs.append(sg.RowsIf(sg.EQUALITY, [0], [J], np.zeros(3)))
    p = sg.Problem([sg.Scene([sg.GenericSub(A, np.ones(n))], ifs)],
                   sg.Options(gravity=(0, 0, 0), max_iters=5))
    for blocked in (True, False):
        sim = sa.Simulation(p, precision=sa.SIM_MIXED, grid_side_rows=1)
        sim.tc_factor(blocked)
        sim.step(1)
        with pytest.raises(sa.SimError) as ei:
            sim.residuals(0)
        assert ei.value.code == sa.SIM_ENOTSPD
        sim.close()
