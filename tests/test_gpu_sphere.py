"""Sphere-sphere contacts and plane contacts with any normal and a radius (the granular
stirring scene's contact model, Sec. IV-A) on the device, against the FP64 oracle.

* Rows in isolation: a few spheres (and a node of a linear block) with sphere-sphere,
  world-sphere and tilted-plane contacts, random orientations, FP64 to 1e-9 over several
  steps, block and grid kernel.
* The stir scene (scenegen.stir: 216 spheres + the arm stand-in, 217 subsystems) at the
  paper's fixed iteration counts (Table I: 30 / 60 / 90): a reduced 27-sphere version on the
  block kernel and the full scene on the grid kernel, FP64 to 1e-9; the mixed form's
  distance from the oracle is printed and bounded."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

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


def _sphere(rng, m, r, p, v):
    I = 0.4 * m * r * r
    q = Rotation.random(random_state=int(rng.integers(1 << 30))).as_quat()[[3, 0, 1, 2]]
    return sg.Body(m, np.array([I, I, I]), np.array(p, float), q, np.array(v, float),
                   rng.standard_normal(3))


def _contact_scene(seed=0, tol=-1.0, iters=80):
    """Three spheres, each its own subsystem, and a 2x2x2-node linear block: sphere-sphere
    (with off-centre anchors), a sphere against a world sphere, a node as a sphere against a
    rigid sphere, and plane contacts with tilted normals and radii."""
    rng = np.random.default_rng(seed)
    r = [0.01, 0.013, 0.008]
    bodies = [_sphere(rng, 0.004, r[0], (0.0, 0.0, 0.021), (0.05, 0.0, -0.1)),
              _sphere(rng, 0.006, r[1], (0.0205, 0.004, 0.024), (-0.1, 0.02, 0.0)),
              _sphere(rng, 0.003, r[2], (-0.019, 0.002, 0.012), (0.0, 0.0, -0.05))]
    subs = [sg.RigidSub([b]) for b in bodies]
    blk = sg.lattice_block((2, 2, 2), spacing=0.01, origin=(-0.004, 0.03, 0.03), k=200.0)
    subs.append(blk)
    ifs = [
        sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=(1, 0), anchor_a=np.array([0.0005, 0, 0.0]),
                   anchor_b=np.array([0.0, -0.0005, 0.0]), radius_a=r[0], radius_b=r[1],
                   mu=0.4),
        sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=(2, 0), radius_a=r[0], radius_b=r[2], mu=0.6),
        sg.JointIf(sg.SPHERE_CONTACT, a=(2, 0), b=None, anchor_b=np.array([-0.04, 0.0, 0.01]),
                   radius_a=r[2], radius_b=0.013, mu=0.3),
        sg.JointIf(sg.SPHERE_CONTACT, a=(3, 0), b=(1, 0), radius_a=0.004, radius_b=r[1],
                   mu=0.5),
        sg.JointIf(sg.PLANE_CONTACT, a=(1, 0), radius_a=r[1], normal=np.array([0.1, -0.2, 1.0]),
                   plane_z=0.0, mu=0.5),
        sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), radius_a=r[0], normal=np.array([0.0, 0.0, 1.0]),
                   plane_z=0.0, mu=0.5),
        sg.JointIf(sg.PLANE_CONTACT, a=(2, 0), anchor_a=np.array([0.001, 0.0, -0.001]),
                   radius_a=r[2], normal=np.array([0.95, 0.0, 0.3]), plane_z=-0.03, mu=0.5),
        sg.JointIf(sg.PLANE_CONTACT, a=(3, 1), radius_a=0.002, normal=np.array([0.0, 0.3, 1.0]),
                   plane_z=0.02, mu=0.3),
    ]
    opts = sg.Options(h=1e-3, warm="prev", tol_primal=tol, max_iters=iters)
    return sg.Problem([sg.Scene(subs, ifs)], opts)


@pytest.mark.parametrize("grid", [False, True])
@pytest.mark.parametrize("per_launch", [1, 3])
def test_contact_rows_fp64(sa, grid, per_launch):
    """Several steps per launch exercise the factors kept across steps (a node in a sphere
    contact turns its rows, so its block's map must be formed anew every step)."""
    p = _contact_scene()
    o = oracle.OracleScene(p.scenes[0], p.options)
    sim = sa.Simulation(p, grid_side_rows=1 if grid else None)
    worst = 0.0
    for _ in range(6 // per_launch):
        sim.step(per_launch)
        for _ in range(per_launch):
            o.step()
        for a, b in ((sim.scene_vhat(0), o.vhat_all()), (sim.scene_lam(0), o.lam_all()),
                     (sim.scene_bodies(0)[:, 4:], o.bodies_all()[:, 4:]),
                     (sim.scene_nodes(0), o.nodes_all())):
            worst = max(worst, rel(a, b))
    assert worst < 1e-9
    assert np.max(np.abs(o.lam_all())) > 0.0      # some contacts are closed


def test_contact_rows_converged(sa):
    p = _contact_scene(tol=1e-9, iters=100000)
    orcs = oracle.run(p, steps=3)
    sim = sa.Simulation(p)
    sim.step(3)
    r, ro = sim.residuals(0), orcs[0].residuals()
    assert r["converged"] and ro["converged"]
    assert abs(r["iters"] - ro["iters"]) <= 1
    assert rel(sim.scene_vhat(0), orcs[0].vhat_all()) < 1e-7


@pytest.mark.parametrize("iters", [30, 90])
def test_stir_small_fp64_fixed_iterations(sa, iters):
    p = sg.stir(1, n_side=3, layers=3, tol_primal=-1, max_iters=iters)
    o = oracle.OracleScene(p.scenes[0], p.options)
    sim = sa.Simulation(p)
    for _ in range(5):
        sim.step(1)
        o.step()
        assert rel(sim.scene_vhat(0), o.vhat_all()) < 1e-9
        assert rel(sim.scene_bodies(0)[:, 4:], o.bodies_all()[:, 4:]) < 1e-9
        assert rel(sim.scene_lam(0), o.lam_all()) < 1e-9


def test_stir_full_fp64_grid(sa, capsys):
    """The full scene (9,558 side-rows: the grid kernel) at 30 iterations per step."""
    p = sg.stir(0, tol_primal=-1, max_iters=30)
    o = oracle.OracleScene(p.scenes[0], p.options, openmp=True)
    sim = sa.Simulation(p)
    assert [c["cached"] for c in sim.launch_classes()] == [2]     # 2: the grid kernel
    errs = []
    for _ in range(4):
        sim.step(1)
        o.step()
        errs.append(max(rel(sim.scene_vhat(0), o.vhat_all()),
                        rel(sim.scene_bodies(0)[:, 4:], o.bodies_all()[:, 4:]),
                        rel(sim.scene_lam(0), o.lam_all())))
    with capsys.disabled():
        print(f"\n[stir, 217 subsystems, 30 iterations, FP64 grid kernel] max rel err per "
              f"step: {', '.join(f'{e:.1e}' for e in errs)}")
    assert max(errs) < 1e-9


def test_stir_full_mixed_grid(sa, capsys):
    p = sg.stir(0, tol_primal=-1, max_iters=30)
    o = oracle.OracleScene(p.scenes[0], p.options, openmp=True)
    sim = sa.Simulation(p, precision=sa.SIM_MIXED)
    errs = []
    for _ in range(4):
        sim.step(1)
        o.step()
        errs.append(rel(sim.scene_vhat(0), o.vhat_all()))
    with capsys.disabled():
        print(f"\n[stir, 30 iterations, mixed form] v-hat rel err vs FP64 oracle per step: "
              f"{', '.join(f'{e:.1e}' for e in errs)}")
    assert max(errs) < 1e-3
