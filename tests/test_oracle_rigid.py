"""Pins of the oracle's rigid-body model (Eq. ddyn, Sec. II-A constraint rows) and of the
time step on the chain and legged-robot scenes: Jacobians against finite differences of
independently computed position-level constraints, closed forms of free fall, spin and
Coulomb sliding, the full-system KKT solution, and momentum conservation.  CPU only."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import scenegen as sg


def _R(q):
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def _advance(rec, nu, eps):
    """Body record moved along generalized velocity nu = [v, w_body] for time eps."""
    out = rec.copy()
    out[4:7] = rec[4:7] + eps * nu[:3]
    r = Rotation.from_quat([rec[8], rec[9], rec[10], rec[7]]) * Rotation.from_rotvec(eps * nu[3:])
    x, y, z, w = r.as_quat()
    out[7:11] = [w, x, y, z]
    return out


def _phi_independent(scene_bodies, itf):
    """Position-level constraint value written from its definition (not the oracle's)."""
    A = scene_bodies[itf.a]
    Ra, pa = _R(A[7:11]), A[4:7]
    if itf.b is not None:
        B = scene_bodies[itf.b]
        Rb, pb = _R(B[7:11]), B[4:7]
    else:
        Rb, pb = np.eye(3), np.zeros(3)
    if itf.kind in (sg.BALL, sg.REVOLUTE):
        qa = pa + Ra @ itf.anchor_a
        qb = pb + Rb @ itf.anchor_b if itf.b is not None else itf.anchor_b
        out = list(qa - qb)
        if itf.kind == sg.REVOLUTE:
            ub = Rb @ itf.axis_b
            t1 = Ra @ itf.ref_a
            t2 = Ra @ np.cross(itf.axis_a, itf.ref_a)
            out += [t1 @ ub, t2 @ ub]
        return np.array(out)
    if itf.kind == sg.ANGLE_PD:
        u = Ra @ itf.axis_a
        na = Ra @ itf.ref_a
        nb = Rb @ itf.ref_b
        return np.array([np.arctan2(np.cross(na, nb) @ u, na @ nb)])
    if itf.kind == sg.PLANE_CONTACT:
        P = pa + Ra @ itf.anchor_a
        return np.array([P[2] - itf.plane_z, P[0], P[1]])
    raise AssertionError


def _bodies(o, scene):
    out = {}
    for i, sub in enumerate(scene.subs):
        for k in range(len(sub.bodies)):
            out[(i, k)] = o.body(i, k)
    return out


def _perturb_scene(o, scene, rng):
    """Give every body a random pose offset and velocity so Jacobians are generic."""
    for i, sub in enumerate(scene.subs):
        for k in range(len(sub.bodies)):
            rec = o.body(i, k)
            rec = _advance(rec, rng.standard_normal(6) * 0.3, 1.0)
            rec[11:17] = rng.standard_normal(6)
            o.set_body(i, k, rec)


@pytest.mark.parametrize("which", ["chain", "robot"])
def test_jacobians_match_finite_differences(which):
    rng = np.random.default_rng(1)
    if which == "chain":
        p = sg.chain(3)
    else:
        p = sg.robots(2, n_robots=1)
    sc = p.scenes[0]
    o = oracle.OracleScene(sc, p.options)
    if which == "chain":
        _perturb_scene(o, sc, rng)   # joints then no longer closed: phi != 0 generic
    o.assemble()
    base = _bodies(o, sc)
    nus = {key: rng.standard_normal(6) for key in base}
    eps = 1e-6
    for j, itf in enumerate(sc.ifs):
        # phi from the oracle equals phi written from its definition
        phi_o = o.phi(j)
        phi_i = _phi_independent(base, itf)
        if itf.kind == sg.PLANE_CONTACT:
            assert np.isclose(phi_o[0], phi_i[0], atol=1e-14)
        else:
            assert np.allclose(phi_o, phi_i, atol=1e-13)
        # J nu against central differences of the definition
        plus = {k: _advance(v, nus[k], eps) for k, v in base.items()}
        minus = {k: _advance(v, nus[k], -eps) for k, v in base.items()}
        fd = (_phi_independent(plus, itf) - _phi_independent(minus, itf)) / (2 * eps)
        _, Js = o.con_rows(j)
        subs = o.sides(j)
        Jnu = np.zeros(o.rows(j))
        for s, Jm in zip(subs, Js):
            nu_sub = np.concatenate([nus[(s, k)] for k in range(len(sc.subs[s].bodies))])
            Jnu += Jm @ nu_sub
        if itf.kind == sg.ANGLE_PD and which == "chain":
            continue
        assert np.allclose(Jnu, fd, atol=1e-7, rtol=1e-6), (itf.kind, Jnu, fd)


def _single_body_problem(m=2.0, I=(0.1, 0.2, 0.3), p=(0, 0, 1.0), v=(0, 0, 0), w=(0, 0, 0),
                         ifs=(), h=1e-3, g=(0, 0, -9.81), tol=1e-12, iters=100000):
    body = sg.Body(m, np.array(I, float), np.array(p, float), np.array([1.0, 0, 0, 0]),
                   np.array(v, float), np.array(w, float))
    opts = sg.Options(h=h, gravity=g, warm="cold", tol_primal=tol, max_iters=iters)
    return sg.Problem([sg.Scene([sg.RigidSub([body])], list(ifs))], opts)


def test_free_fall_and_gyroscopic_closed_forms():
    h = 1e-3
    # Eq. ddyn: (2/h) M (v-hat - v_k) = f - C v_k  ->  v-hat = v_k + (h/2) g
    p = _single_body_problem(v=(0.3, -0.2, 1.0), h=h)
    o = oracle.run(p)[0]
    assert np.allclose(o.vhat(0)[:3], [0.3, -0.2, 1.0 - 9.81 * h / 2], rtol=1e-14)
    # spin about a principal axis: w x I w = 0, angular velocity unchanged
    p = _single_body_problem(w=(0, 5.0, 0), g=(0, 0, 0))
    o = oracle.run(p)[0]
    assert np.allclose(o.vhat(0)[3:], [0, 5.0, 0], atol=1e-15)
    # general spin: I (w-hat - w) = -(h/2) w x I w
    w = np.array([1.0, 2.0, 3.0])
    I = np.array([0.1, 0.2, 0.3])
    p = _single_body_problem(w=tuple(w), I=tuple(I), g=(0, 0, 0), h=h)
    o = oracle.run(p)[0]
    ref = w - (h / 2) * np.cross(w, I * w) / I
    assert np.allclose(o.vhat(0)[3:], ref, rtol=1e-14)


@pytest.mark.parametrize("vx0,mu", [(0.5, 0.4), (0.001, 0.4), (-0.3, 0.9), (0.0, 0.5)])
def test_sliding_block_coulomb_closed_form(vx0, mu):
    """A point mass resting on the plane (gap 0) with horizontal speed vx0.

    Normal: v-hat_z = 0, lambda_n = m g.  Tangent (Eq. scc): it slides with
    lambda_t = -mu m g sign(vx0) and v-hat_x = vx0 - mu g h / 2 while that keeps the sign,
    otherwise it sticks: v-hat_x = 0, lambda_t = -(2m/h) vx0."""
    m, h, g = 2.0, 1e-3, 9.81
    c = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.zeros(3), plane_z=0.0, mu=mu)
    p = _single_body_problem(m=m, p=(0, 0, 0.0), v=(vx0, 0, 0), ifs=[c], h=h)
    o = oracle.run(p)[0]
    assert o.residuals()["converged"]
    v = o.vhat(0)
    lam = o.lam(0)
    assert abs(v[2]) < 1e-9 and np.isclose(lam[0], m * g, rtol=1e-9)
    if abs(vx0) > mu * g * h / 2:
        assert np.isclose(v[0], vx0 - np.sign(vx0) * mu * g * h / 2, rtol=1e-8, atol=1e-10)
        assert np.isclose(lam[1], -np.sign(vx0) * mu * m * g, rtol=1e-8)
    else:
        assert abs(v[0]) < 1e-9
        assert np.isclose(lam[1], -(2 * m / h) * vx0, rtol=1e-7, atol=1e-8)
    assert abs(v[1]) < 1e-9 and abs(lam[2]) < 1e-8


def test_open_contact_is_free_fall():
    c = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.zeros(3), plane_z=0.0, mu=0.5)
    p = _single_body_problem(p=(0, 0, 0.5), ifs=[c])
    o = oracle.run(p)[0]
    assert np.allclose(o.vhat(0)[:3], [0, 0, -9.81 * 1e-3 / 2], rtol=1e-12)
    assert np.all(o.lam(0) == 0.0)


def test_speculative_contact_lands_exactly():
    # falling at 2 m/s from 1 mm: gap/h = 1 m/s, so v-hat_z = -1 m/s exactly
    c = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.zeros(3), plane_z=0.0, mu=0.5)
    p = _single_body_problem(p=(0, 0, 1e-3), v=(0, 0, -2.0), ifs=[c])
    o = oracle.run(p)[0]
    assert np.isclose(o.vhat(0)[2], -1.0, rtol=1e-9)


def _assembled_full_system(o, scene):
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


@pytest.mark.parametrize("rho", [1e3, None])
def test_chain_step_matches_full_kkt(rho):
    """Bilateral-only chain: the converged step equals the KKT solution of the system the
    step assembled, [A -J^T; J 0][v; lambda] = [b; -e] (dense LU)."""
    p = sg.chain(0, rho=rho, tol_primal=1e-12, max_iters=200000, warm="cold")
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.step()
    assert o.residuals()["converged"]
    A, b, J, e = _assembled_full_system(o, p.scenes[0])
    m, n = J.shape
    KKT = np.block([[A, -J.T], [J, np.zeros((m, m))]])
    sol = np.linalg.solve(KKT, np.concatenate([b, -e]))
    v = o.vhat_all()
    # the stop rule bounds |x - z| and |dz| by 1e-12 in velocity units; the rotational
    # DOFs of the thin links (inertia ~3e-6 kg m^2) amplify that by cond(K) ~ 1e4
    assert np.max(np.abs(v - sol[:n])) / np.max(np.abs(sol[:n])) < 1e-7
    assert np.max(np.abs(J @ v + e)) < 5e-12
    lam = np.concatenate([o.lam(j) for j in range(o.ncon)])
    assert np.max(np.abs(lam - sol[n:])) / np.max(np.abs(sol[n:])) < 1e-7


def test_free_chain_conserves_linear_momentum():
    """No pin, no gravity: ball-joint rows carry equal and opposite identity blocks, so at
    the fixed point sum_b m_b v_b is unchanged by a step (Eq. ddyn)."""
    p = sg.chain(4, pinned=False, gravity=False, tol_primal=1e-12, max_iters=200000,
                 rho=None)
    rng = np.random.default_rng(0)
    sc = p.scenes[0]
    o = oracle.OracleScene(sc, p.options)
    for i, sub in enumerate(sc.subs):
        for k in range(len(sub.bodies)):
            rec = o.body(i, k)
            rec[11:17] = rng.standard_normal(6)
            o.set_body(i, k, rec)
    B = o.bodies_all()
    P0 = (B[:, :1] * B[:, 11:14]).sum(0)
    for _ in range(5):
        o.step()
        assert o.residuals()["converged"]
    B = o.bodies_all()
    P1 = (B[:, :1] * B[:, 11:14]).sum(0)
    assert np.allclose(P1, P0, atol=1e-9 * np.sum(B[:, 0]) * 10)


def test_constraint_violation_goes_to_zero_with_tolerance():
    viol = []
    for tol in (1e-4, 1e-7, 1e-10):
        p = sg.chain(0, rho=None, tol_primal=tol, max_iters=200000, warm="cold")
        o = oracle.OracleScene(p.scenes[0], p.options)
        o.step()
        A, b, J, e = _assembled_full_system(o, p.scenes[0])
        viol.append(np.max(np.abs(J @ o.vhat_all() + e)))
    assert viol[0] > viol[1] > viol[2] and viol[2] < 1e-9


def test_same_seed_is_bitwise_deterministic():
    a = oracle.run(sg.robots(5, n_robots=2), steps=3)
    b = oracle.run(sg.robots(5, n_robots=2), steps=3)
    for x, y in zip(a, b):
        assert np.array_equal(x.bodies_all(), y.bodies_all())
        assert np.array_equal(x.lam_all(), y.lam_all())


def test_state_and_warm_duals_determine_the_next_step():
    """Bodies plus each constraint's warm-start lambda and z are the whole state a step
    starts from: a fresh oracle scene given them (set_body, set_warm) takes the same next
    step, bit for bit, as the scene that reached them."""
    p = sg.robots(5, n_robots=1, tol_primal=1e-6, max_iters=1000)
    sc = p.scenes[0]
    a = oracle.OracleScene(sc, p.options)
    for _ in range(30):
        a.step()
    b = oracle.OracleScene(sc, p.options)
    for i, sub in enumerate(sc.subs):
        for k in range(len(sub.bodies)):
            b.set_body(i, k, a.body(i, k))
    for j in range(a.ncon):
        b.set_warm(j, a.lam(j), a.side(j, "z"))
    a.step()
    b.step()
    assert np.array_equal(a.bodies_all(), b.bodies_all())
    assert np.array_equal(a.lam_all(), b.lam_all())
    assert a.residuals()["iters"] == b.residuals()["iters"]
