"""Pins of the oracle's linear elastic blocks (Eq. ddyn with the elastic force at the
midpoint of the step) and of node-sided constraints.  CPU only."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import scenegen as sg


def _opts(**kw):
    base = dict(h=1e-3, gravity=(0.0, 0.0, 0.0), warm="cold", tol_primal=1e-12,
                max_iters=200000)
    base.update(kw)
    return sg.Options(**base)


def _energy(blk: sg.LinearSub, nodes: np.ndarray) -> float:
    x = nodes[:, :3].ravel()
    v = nodes[:, 3:].ravel()
    K = blk.K_dense()
    m = np.repeat(blk.mass, 3)
    d = x - blk.X0
    return 0.5 * np.dot(m * v, v) + 0.5 * d @ K @ d


def test_midpoint_rule_conserves_spring_energy_exactly():
    """The implicit midpoint rule conserves quadratic invariants of a linear system, so an
    unconstrained spring block keeps E = v^T M v / 2 + (x - X0)^T K (x - X0) / 2 to rounding."""
    rng = np.random.default_rng(0)
    blk = sg.lattice_block(dims=(2, 2, 3), k=800.0)
    blk.x = blk.X0 + rng.standard_normal(blk.n) * 1e-3
    blk.v = rng.standard_normal(blk.n) * 0.1
    p = sg.Problem([sg.Scene([blk], [])], _opts(max_iters=1, tol_primal=-1))
    o = oracle.OracleScene(p.scenes[0], p.options)
    E0 = _energy(blk, o.nodes_all())
    for _ in range(200):
        o.step()
    E1 = _energy(blk, o.nodes_all())
    assert abs(E1 - E0) <= 1e-12 * E0
    assert np.abs(o.nodes_all()[:, :3].ravel() - blk.x).max() > 1e-5   # it did move


def test_rigid_translation_of_a_block_is_free_fall():
    blk = sg.lattice_block(dims=(2, 2, 2), v=(0.2, -0.1, 0.3))
    p = sg.Problem([sg.Scene([blk], [])], _opts(gravity=(0, 0, -9.81), max_iters=1,
                                                 tol_primal=-1))
    o = oracle.run(p)[0]
    v = o.vhat(0).reshape(-1, 3)
    assert np.allclose(v, [0.2, -0.1, 0.3 - 9.81e-3 / 2], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("vx0,mu", [(0.5, 0.4), (0.001, 0.4)])
def test_node_contact_coulomb_closed_form(vx0, mu):
    m, h, g = 0.3, 1e-3, 9.81
    blk = sg.LinearSub(np.array([m]), np.zeros(0, int), np.zeros(0, int), np.zeros(0),
                       np.zeros(3), np.zeros(3), np.zeros(3), np.array([vx0, 0.0, 0.0]))
    c = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), plane_z=0.0, mu=mu)
    p = sg.Problem([sg.Scene([blk], [c])], _opts(gravity=(0, 0, -g)))
    o = oracle.run(p)[0]
    v, lam = o.vhat(0), o.lam(0)
    assert abs(v[2]) < 1e-9 and np.isclose(lam[0], m * g, rtol=1e-9)
    if vx0 > mu * g * h / 2:
        assert np.isclose(v[0], vx0 - mu * g * h / 2, rtol=1e-8)
    else:
        assert abs(v[0]) < 1e-9


def _advance_body(rec, nu, eps):
    out = rec.copy()
    out[4:7] = rec[4:7] + eps * nu[:3]
    r = Rotation.from_quat([rec[8], rec[9], rec[10], rec[7]]) * Rotation.from_rotvec(eps * nu[3:])
    x, y, z, w = r.as_quat()
    out[7:11] = [w, x, y, z]
    return out


def test_node_body_ball_jacobian_matches_finite_differences():
    rng = np.random.default_rng(2)
    blk = sg.lattice_block(dims=(2, 2, 2), origin=(0.3, 0.0, 0.0))
    q = Rotation.from_rotvec(rng.standard_normal(3)).as_quat()
    body = sg.Body(0.5, np.array([1e-3, 2e-3, 3e-3]), np.array([0.1, 0.05, -0.02]),
                   np.array([q[3], q[0], q[1], q[2]]), np.zeros(3), np.zeros(3))
    anc = rng.standard_normal(3) * 0.05
    joint = sg.JointIf(sg.BALL, a=(0, 0), b=(1, 3), anchor_a=anc)
    p = sg.Problem([sg.Scene([sg.RigidSub([body]), blk], [joint])], _opts())
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.assemble()
    R = Rotation.from_quat(q).as_matrix()
    node = o.node(1, 3)
    phi_ref = body.p + R @ anc - node[:3]
    assert np.allclose(o.phi(0), phi_ref, atol=1e-14)
    nu_b = rng.standard_normal(6)
    nu_n = rng.standard_normal(blk.n)
    eps = 1e-6
    rec = o.body(0, 0)

    def phi_at(s):
        rb = _advance_body(rec, nu_b, s)
        Rb = Rotation.from_quat([rb[8], rb[9], rb[10], rb[7]]).as_matrix()
        xn = node[:3] + s * nu_n[9:12]
        return rb[4:7] + Rb @ anc - xn

    fd = (phi_at(eps) - phi_at(-eps)) / (2 * eps)
    _, Js = o.con_rows(0)
    Jnu = Js[0] @ nu_b + Js[1] @ nu_n
    assert np.allclose(Jnu, fd, atol=1e-7, rtol=1e-6)
    # the node side is a selector of the node's three velocity components
    assert np.array_equal(np.nonzero(Js[1].any(axis=0))[0], np.arange(9, 12))


def test_rigid_and_linear_bilateral_step_matches_full_kkt():
    """A rigid body hung from a pinned spring block by a ball joint: the converged step
    equals the KKT solution of the assembled system (dense LU)."""
    blk = sg.lattice_block(dims=(2, 2, 2), origin=(0.0, 0.0, 0.0), k=2000.0)
    body = sg.Body(0.2, np.array([1e-4, 1e-4, 1e-4]), np.array([0.01, 0.01, -0.05]),
                   np.array([1.0, 0, 0, 0]), np.zeros(3), np.zeros(3))
    ifs = [sg.JointIf(sg.BALL, a=(1, 0), b=None, anchor_b=blk.X0[0:3].copy()),
           sg.JointIf(sg.BALL, a=(1, 1), b=None, anchor_b=blk.X0[3:6].copy()),
           sg.JointIf(sg.BALL, a=(0, 0), b=(1, 0), anchor_a=np.array([-0.01, -0.01, 0.05]))]
    p = sg.Problem([sg.Scene([sg.RigidSub([body]), blk], ifs)],
                   _opts(gravity=(0, 0, -9.81), beta_mode="trace"))
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.step()
    assert o.residuals()["converged"]
    offs = np.cumsum([0, 6, blk.n])
    n = offs[-1]
    A = np.zeros((n, n)); b = np.zeros(n)
    for i in range(2):
        Ai, bi = o.Ab(i)
        A[offs[i]:offs[i + 1], offs[i]:offs[i + 1]] = Ai
        b[offs[i]:offs[i + 1]] = bi
    rows, es = [], []
    for j in range(o.ncon):
        e, Jl = o.con_rows(j)
        Rj = np.zeros((o.rows(j), n))
        for s_, Jm in zip(o.sides(j), Jl):
            Rj[:, offs[s_]:offs[s_ + 1]] += Jm
        rows.append(Rj); es.append(e)
    J = np.vstack(rows); e = np.concatenate(es)
    m = J.shape[0]
    sol = np.linalg.solve(np.block([[A, -J.T], [J, np.zeros((m, m))]]), np.concatenate([b, -e]))
    v = o.vhat_all()
    assert np.max(np.abs(v - sol[:n])) / np.max(np.abs(sol[:n])) < 1e-7
