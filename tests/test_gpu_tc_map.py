"""The per-step map of large blocks formed on the tensor cores (grid kernel, mixed form).

A step that factorises a block of >= 128 DOF anew runs as three launches: the grid kernel up
to W = L^-1 [J^T b] (columns solved in chunks over every warp), the tcgen05 Gram kernel
(D = W^T W, c = W^T g, split-TF32), and the grid kernel from the initial duals on (the
blocked factorisation's launches, on by default, come between the first two).  With
sim_tensor_cores(0) the grid kernel forms D and c on the CUDA cores instead.

* Fixed iteration counts: both maps are FP32 approximations of the FP64 oracle's step (the
  Gram kernel's D differs from the CUDA cores' by ~1e-5 of max|D|, amplified by the
  iterations); the tensor-core map's distance from the oracle is within 3x the CUDA-core
  map's.
* Converged to r_p <= 1e-6 (the mixed form's final check in FP64): the answer is as close to
  the exact step (the FP64 oracle converged to 1e-11) as the FP64 oracle's own answer at the
  same tolerance."""
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
    base = dict(ny=8, nz=8, planes=8, slabs=3, length=0.03, width=0.01, height=0.01)
    base.update(kw)
    return sg.fem_beam(0, **base)


def _pair(sa, p, keep=False):
    a = sa.Simulation(p, precision=sa.SIM_MIXED, grid_side_rows=1)
    b = sa.Simulation(p, precision=sa.SIM_MIXED, grid_side_rows=1)
    b.tensor_cores(False)
    for s in (a, b):
        s.keep_factors(keep)
    return a, b


@pytest.mark.parametrize("keep", [False, True])
def test_tensor_core_map_matches_cuda_core_map(sa, keep, capsys):
    p = _beam(tol_primal=-1, max_iters=30)
    assert all(s.n >= 128 for s in p.scenes[0].subs if hasattr(s, "Kv"))
    a, b = _pair(sa, p, keep)
    o = oracle.OracleScene(p.scenes[0], p.options)
    out = []
    for _ in range(3):
        a.step(1)
        b.step(1)
        o.step()
        assert a.residuals(0)["status"] == 0
        d_a = rel(a.scene_vhat(0), o.vhat_all())
        d_b = rel(b.scene_vhat(0), o.vhat_all())
        out.append((d_a, d_b, rel(a.scene_vhat(0), b.scene_vhat(0))))
        assert d_a <= 3 * d_b + 1e-6
        assert rel(a.scene_nodes(0), o.nodes_all()) <= 3 * rel(b.scene_nodes(0), o.nodes_all()) + 1e-7
    with capsys.disabled():
        print(f"\n[tensor-core vs CUDA-core map, keep_factors={keep}, 30 iterations] v-hat rel "
              f"err vs FP64 oracle per step: tensor cores "
              f"{', '.join(f'{x[0]:.2e}' for x in out)}; CUDA cores "
              f"{', '.join(f'{x[1]:.2e}' for x in out)}; between them "
              f"{', '.join(f'{x[2]:.2e}' for x in out)}")


def test_tensor_core_map_converged_against_fp64_oracle(sa, capsys):
    steps = 3
    same = oracle.run(_beam(tol_primal=1e-6, max_iters=200000), steps=steps)
    tight = oracle.run(_beam(tol_primal=1e-11, max_iters=200000), steps=steps)
    a = sa.Simulation(_beam(tol_primal=1e-6, max_iters=200000), precision=sa.SIM_MIXED,
                      grid_side_rows=1)
    a.keep_factors(False)
    a.step(steps)
    r = a.residuals(0)
    assert r["converged"] and r["r_p"] <= 1e-6
    err = rel(a.scene_vhat(0), tight[0].vhat_all())
    spread = rel(same[0].vhat_all(), tight[0].vhat_all())
    with capsys.disabled():
        print(f"\n[tensor-core map, refactorised every step, r_p<=1e-6] v-hat rel err to the "
              f"exact step {err:.3e}; FP64 oracle at the same tolerance {spread:.3e}")
    assert err <= 3 * spread + 1e-6


def test_tensor_core_map_full_size_slabs(sa, capsys):
    """Slabs of the full beam's size (n = 1200, 900, 900; m ~ 300-600): fixed iterations,
    tensor-core map against the CUDA-core map, and the FP64 oracle's step for scale."""
    p = sg.fem_beam(0, ny=10, nz=10, planes=8, slabs=3, length=0.03, with_gripper=False,
                    tol_primal=-1, max_iters=20)
    a, b = _pair(sa, p, keep=False)
    o = oracle.OracleScene(p.scenes[0], p.options)
    for _ in range(2):
        a.step(1)
        b.step(1)
        o.step()
    d_ab = rel(a.scene_vhat(0), b.scene_vhat(0))
    d_a = rel(a.scene_vhat(0), o.vhat_all())
    d_b = rel(b.scene_vhat(0), o.vhat_all())
    with capsys.disabled():
        print(f"\n[full-size slabs, 20 iterations] v-hat: tensor-core vs CUDA-core map "
              f"{d_ab:.2e}; vs FP64 oracle {d_a:.2e} (CUDA-core map {d_b:.2e})")
    assert d_ab < 1e-4
    assert d_a < 3 * d_b + 1e-5
