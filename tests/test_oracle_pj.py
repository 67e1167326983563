"""Pins of the oracle's Projected Jacobi step (the paper's PJ comparison solver, Sec. IV-B):

* one row: with omega = 1 a single iteration solves it exactly (J v-hat + e = 0 for an
  equality or active hard row, lambda = 0 for an inactive hard row); omega scales the step;
* Coulomb sliding of a point mass on the ground (orthonormal contact frame, a diagonal
  Delassus block): one iteration with omega = 1 gives the closed form, and it is a fixed
  point of further iterations;
* the converged ADMM step of a random scene with equality, hard, soft and contact rows is a
  fixed point of one PJ iteration (every projection's formula and sign against the other
  solver's);
* a bilateral chain: PJ iterated to convergence reaches the KKT solution of the step's
  assembled system (dense LU).
CPU only."""
import numpy as np
import pytest

import oracle
import scenegen as sg


def _pj(options, omega=1.0, iters=1):
    options.solver = "pj"
    options.pj_omega = omega
    options.max_iters = iters
    options.tol_primal = -1.0
    return options


def _one_row_problem(kind, e_val, omega, iters=1, seed=0):
    rng = np.random.default_rng(seed)
    n = 5
    G = rng.standard_normal((n, n))
    A = G @ G.T / n + np.diag(rng.uniform(0.5, 2.0, n))
    b = rng.standard_normal(n)
    J = rng.standard_normal((1, n))
    itf = sg.RowsIf(kind, [0], [J], np.array([e_val]))
    opts = _pj(sg.Options(warm="cold"), omega, iters)
    return sg.Problem([sg.Scene([sg.GenericSub(A, b)], [itf])], opts), A, b, J


@pytest.mark.parametrize("omega", [1.0, 0.5])
def test_single_equality_row(omega):
    p, A, b, J = _one_row_problem(sg.EQUALITY, 0.3, omega)
    o = oracle.run(p)[0]
    free = float((J @ np.linalg.solve(A, b))[0]) + 0.3
    delta = float((J @ np.linalg.solve(A, J.T))[0, 0])
    lam = -omega * free / delta
    assert np.allclose(o.lam(0), lam, rtol=1e-12)
    v = o.vhat(0)
    assert np.allclose(v, np.linalg.solve(A, b + J[0] * lam), rtol=1e-12)
    assert np.isclose(float((J @ v)[0]) + 0.3, (1.0 - omega) * free, rtol=1e-10, atol=1e-14)
    # the natural residual of the one iteration: |d lambda| delta / omega = |free|
    assert np.isclose(o.residuals()["r_p"], abs(free), rtol=1e-12)


@pytest.mark.parametrize("e_val", [-5.0, 5.0])
def test_single_hard_row(e_val):
    p, A, b, J = _one_row_problem(sg.HARD, e_val, 1.0)
    o = oracle.run(p)[0]
    free = float((J @ np.linalg.solve(A, b))[0]) + e_val
    if free < 0:                    # violated without the row: pushed onto J v + e = 0
        assert o.lam(0)[0] > 0 and abs(float((J @ o.vhat(0))[0]) + e_val) < 1e-12
    else:                           # satisfied: no impulse
        assert o.lam(0)[0] == 0.0
        assert np.allclose(o.vhat(0), np.linalg.solve(A, b), rtol=1e-13)


@pytest.mark.parametrize("vx0,mu", [(0.5, 0.4), (0.001, 0.4), (-0.3, 0.9)])
@pytest.mark.parametrize("iters", [1, 25])
def test_sliding_point_mass(vx0, mu, iters):
    m, h, g = 2.0, 1e-3, 9.81
    body = sg.Body(m, np.array([0.1, 0.2, 0.3]), np.zeros(3), np.array([1.0, 0, 0, 0]),
                   np.array([vx0, 0, 0]), np.zeros(3))
    c = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.zeros(3), plane_z=0.0, mu=mu)
    opts = _pj(sg.Options(h=h, warm="cold"), 1.0, iters)
    o = oracle.run(sg.Problem([sg.Scene([sg.RigidSub([body])], [c])], opts))[0]
    v, lam = o.vhat(0), o.lam(0)
    assert abs(v[2]) < 1e-12 and np.isclose(lam[0], m * g, rtol=1e-12)
    if abs(vx0) > mu * g * h / 2:
        assert np.isclose(v[0], vx0 - np.sign(vx0) * mu * g * h / 2, rtol=1e-12)
        assert np.isclose(lam[1], -np.sign(vx0) * mu * m * g, rtol=1e-12)
    else:
        assert abs(v[0]) < 1e-12
    assert abs(lam[2]) < 1e-12


@pytest.mark.parametrize("seed", [1, 3, 5, 11, 17, 22])
def test_converged_admm_is_a_fixed_point(seed):
    types = (sg.EQUALITY, sg.HARD, sg.SOFT, sg.CONTACT)
    rng = np.random.default_rng(seed)
    scene = sg.generic_scene(rng, n_sub=4, n_range=(3, 8), types=types)
    admm = sg.Problem([scene], sg.Options(warm="cold", tol_primal=1e-13, max_iters=400000))
    a = oracle.OracleScene(scene, admm.options)
    a.step()
    assert a.residuals()["converged"]
    opts = _pj(sg.Options(warm="prev"), 0.7, 1)
    b = oracle.OracleScene(scene, opts)
    for j in range(a.ncon):
        b.set_warm(j, a.lam(j), np.zeros((len(a.sides(j)), a.rows(j))))
    b.step()
    la, lb = a.lam_all(), b.lam_all()
    assert np.max(np.abs(lb - la)) <= 1e-8 * max(np.max(np.abs(la)), 1.0)
    assert np.max(np.abs(b.vhat_all() - a.vhat_all())) <= 1e-8 * np.max(np.abs(a.vhat_all()))
    assert np.max(np.abs(la)) > 0.0


def _full_system(o, scene):
    offs = np.cumsum([0] + [s.n for s in scene.subs])
    n = offs[-1]
    A = np.zeros((n, n))
    b = np.zeros(n)
    for i in range(len(scene.subs)):
        Ai, bi = o.Ab(i)
        A[offs[i]:offs[i + 1], offs[i]:offs[i + 1]] = Ai
        b[offs[i]:offs[i + 1]] = bi
    Js, es = [], []
    for j in range(o.ncon):
        e, Jl = o.con_rows(j)
        R = np.zeros((o.rows(j), n))
        for s, Jm in zip(o.sides(j), Jl):
            R[:, offs[s]:offs[s + 1]] += Jm
        Js.append(R)
        es.append(e)
    return A, b, np.vstack(Js), np.concatenate(es)


def test_chain_converges_to_the_kkt_solution():
    p = sg.chain(0, n_links=4, warm="cold")
    _pj(p.options, 0.3, 60000)
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.step()
    A, b, J, e = _full_system(o, p.scenes[0])
    m, n = J.shape
    KKT = np.block([[A, -J.T], [J, np.zeros((m, m))]])
    sol = np.linalg.solve(KKT, np.concatenate([b, -e]))
    v = o.vhat_all()
    assert np.max(np.abs(v - sol[:n])) / np.max(np.abs(sol[:n])) < 1e-8
    assert o.residuals()["r_p"] < 1e-9
