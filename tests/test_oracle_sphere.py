"""Pins of the oracle's sphere-sphere contact and of plane contacts with any normal (the
contact model of the paper's granular stirring scene, Sec. IV-A; contact rows of
Sec. II-A, Signorini-Coulomb Eq. scc).

* Rows: the normal row is the time derivative of the gap |P_a - P_b| - r_a - r_b (central
  finite differences); all three rows equal the relative velocity of the two material
  points at the contact along (n, t1, t2), written here from rigid-body kinematics; the
  frame is orthonormal and right-handed, and n = +z gives the (z, x, y) rows of the
  ground contact.
* Closed forms: head-on collision of two spheres at contact (perfectly inelastic at v-hat,
  momentum kept); a sphere resting on a sphere fixed in the world (lambda_n = m g); a
  point on a tilted plane that sticks (mu >= tan theta: v-hat = 0, lambda balances
  gravity) or slides (v-hat along the slope = (h/2) g (sin theta - mu cos theta)); a solid
  sphere on a tilted plane that rolls (5/7 g sin theta, w = n x v / r) or slides.
CPU only."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import scenegen as sg


def _R(q):
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def _advance(rec, nu, eps):
    out = rec.copy()
    out[4:7] = rec[4:7] + eps * nu[:3]
    r = Rotation.from_quat([rec[8], rec[9], rec[10], rec[7]]) * Rotation.from_rotvec(eps * nu[3:])
    x, y, z, w = r.as_quat()
    out[7:11] = [w, x, y, z]
    return out


def _sphere(m, r, p, v=(0, 0, 0), w=(0, 0, 0), q=(1.0, 0, 0, 0)):
    I = 0.4 * m * r * r
    return sg.Body(m, np.array([I, I, I]), np.array(p, float), np.array(q, float),
                   np.array(v, float), np.array(w, float))


def _problem(bodies, ifs, g=(0, 0, -9.81), h=1e-3, tol=1e-12, iters=200000):
    subs = [sg.RigidSub([b]) for b in bodies]
    opts = sg.Options(h=h, gravity=g, warm="cold", tol_primal=tol, max_iters=iters)
    return sg.Problem([sg.Scene(subs, list(ifs))], opts)


def _center(rec, anchor):
    return rec[4:7] + _R(rec[7:11]) @ anchor


def _gap(recs, itf):
    Pa = _center(recs[itf.a[0]], itf.anchor_a)
    Pb = _center(recs[itf.b[0]], itf.anchor_b) if itf.b is not None else itf.anchor_b
    return np.linalg.norm(Pa - Pb) - itf.radius_a - itf.radius_b


def _point_velocity(rec, nu, point):
    """Velocity of the material point at world position `point` of a body moving with
    nu = [v, w_body]."""
    R = _R(rec[7:11])
    return nu[:3] + np.cross(R @ nu[3:], point - rec[4:7])


def _random_scene(rng):
    r = [0.01, 0.013, 0.008]
    bodies = [_sphere(0.004, r[0], (0.0, 0.0, 0.05)),
              _sphere(0.006, r[1], (0.015, 0.012, 0.062)),
              _sphere(0.003, r[2], (-0.02, 0.004, 0.04))]
    for b in bodies:
        b.q = Rotation.random(random_state=rng.integers(1 << 30)).as_quat()[[3, 0, 1, 2]]
    ifs = [
        sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=(1, 0), anchor_a=np.array([0.001, 0, 0.002]),
                   anchor_b=np.array([0.0, -0.002, 0.001]), radius_a=r[0], radius_b=r[1],
                   mu=0.4),
        sg.JointIf(sg.SPHERE_CONTACT, a=(2, 0), b=None, anchor_a=np.zeros(3),
                   anchor_b=np.array([-0.03, 0.0, 0.03]), radius_a=r[2], radius_b=0.005,
                   mu=0.3),
        sg.JointIf(sg.PLANE_CONTACT, a=(1, 0), anchor_a=np.zeros(3), radius_a=r[1],
                   normal=np.array([0.3, -0.2, 1.0]), plane_z=0.01, mu=0.5),
        sg.JointIf(sg.PLANE_CONTACT, a=(2, 0), anchor_a=np.array([0.001, -0.002, 0.0]),
                   radius_a=r[2], normal=np.array([1.0, 0.05, 0.0]), plane_z=-0.05, mu=0.5),
        sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.array([0.0, 0.0, -r[0]]),
                   normal=np.array([-0.1, 0.4, 1.0]), plane_z=0.0, mu=0.5),
    ]
    return _problem(bodies, ifs)


def test_rows_match_kinematics_and_finite_differences():
    rng = np.random.default_rng(3)
    p = _random_scene(rng)
    sc = p.scenes[0]
    o = oracle.OracleScene(sc, p.options)
    o.assemble()
    recs = {i: o.body(i, 0) for i in range(len(sc.subs))}
    nus = {i: rng.standard_normal(6) for i in recs}
    eps = 1e-7
    for j, itf in enumerate(sc.ifs):
        e, Js = o.con_rows(j)
        subs = o.sides(j)
        Jnu = sum(Jm @ nus[s] for s, Jm in zip(subs, Js))
        if itf.kind == sg.SPHERE_CONTACT:
            Pa = _center(recs[itf.a[0]], itf.anchor_a)
            Pb = _center(recs[itf.b[0]], itf.anchor_b) if itf.b is not None else itf.anchor_b
            n = (Pa - Pb) / np.linalg.norm(Pa - Pb)
            ca, cb = Pa - itf.radius_a * n, Pb + itf.radius_b * n
            phi = _gap(recs, itf)
            va = _point_velocity(recs[itf.a[0]], nus[itf.a[0]], ca)
            vb = (_point_velocity(recs[itf.b[0]], nus[itf.b[0]], cb) if itf.b is not None
                  else np.zeros(3))
            # normal row: d gap / dt by central differences
            plus = {k: _advance(v, nus[k], eps) for k, v in recs.items()}
            minus = {k: _advance(v, nus[k], -eps) for k, v in recs.items()}
            fd = (_gap(plus, itf) - _gap(minus, itf)) / (2 * eps)
            assert np.isclose(Jnu[0], fd, rtol=1e-6, atol=1e-9)
        else:
            n = itf.normal / np.linalg.norm(itf.normal)
            P = _center(recs[itf.a[0]], itf.anchor_a)
            phi = n @ P - itf.plane_z - itf.radius_a
            va = _point_velocity(recs[itf.a[0]], nus[itf.a[0]], P - itf.radius_a * n)
            vb = np.zeros(3)
        assert np.isclose(o.phi(j)[0], phi, rtol=1e-13, atol=1e-15)
        # the frame: rows' world directions from the translational columns of side a
        F = Js[0][:, :3]
        assert np.allclose(F @ F.T, np.eye(3), atol=1e-14)
        assert np.allclose(F[0], n, atol=1e-14)
        assert np.isclose(np.linalg.det(F), 1.0, atol=1e-13)
        assert np.allclose(Jnu, F @ (va - vb), rtol=1e-12, atol=1e-13)
        h = p.options.h
        want = phi / h if phi >= 0 else p.options.baumgarte * phi / h
        assert np.isclose(e[0], want, rtol=1e-12) and e[1] == 0.0 and e[2] == 0.0


def test_plus_z_normal_gives_the_ground_rows():
    body = _sphere(0.004, 0.01, (0.0, 0.0, 0.02))
    body.q = np.array([0.9, 0.1, -0.3, 0.2]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2])
    old = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.array([0.001, 0.002, -0.01]),
                     plane_z=0.005, mu=0.5)
    p = _problem([body], [old])
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.assemble()
    _, Js = o.con_rows(0)
    assert np.array_equal(Js[0][:, :3], np.array([[0, 0, 1.0], [1.0, 0, 0], [0, 1.0, 0]]))
    # a sphere contact against a huge world sphere far below is (to first order) the same
    # ground: n = +z exactly when the centres are vertically aligned
    big = 1e3
    s = sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=None, anchor_a=np.zeros(3),
                   anchor_b=np.array([0.0, 0.0, 0.02 - 0.01 - big - 0.003]), radius_a=0.01,
                   radius_b=big, mu=0.5)
    p = _problem([_sphere(0.004, 0.01, (0.0, 0.0, 0.02))], [s])
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.assemble()
    e, Js = o.con_rows(0)
    assert np.array_equal(Js[0][:, :3], np.array([[0, 0, 1.0], [1.0, 0, 0], [0, 1.0, 0]]))
    assert np.isclose(o.phi(0)[0], 0.003, rtol=1e-9)


@pytest.mark.parametrize("ma,mb", [(0.004, 0.004), (0.004, 0.012)])
def test_head_on_collision_is_inelastic_and_keeps_momentum(ma, mb):
    r, v = 0.01, 0.8
    a = _sphere(ma, r, (0.0, 0.0, 0.0), v=(v, 0, 0))
    b = _sphere(mb, r, (2 * r, 0.0, 0.0))
    c = sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=(1, 0), radius_a=r, radius_b=r, mu=0.5)
    p = _problem([a, b], [c], g=(0, 0, 0))
    o = oracle.run(p)[0]
    assert o.residuals()["converged"]
    common = ma * v / (ma + mb)
    assert np.allclose(o.vhat(0)[:3], [common, 0, 0], rtol=1e-9, atol=1e-12)
    assert np.allclose(o.vhat(1)[:3], [common, 0, 0], rtol=1e-9, atol=1e-12)
    assert np.allclose(o.vhat(0)[3:], 0, atol=1e-12) and np.allclose(o.vhat(1)[3:], 0, atol=1e-12)
    # normal along (P_a - P_b) = -x: lambda_n = (2/h) m_a (v - common)  (force units)
    h = p.options.h
    assert np.isclose(o.lam(0)[0], 2 * ma * (v - common) / h, rtol=1e-8)


def test_resting_on_a_world_sphere():
    m, r, R0 = 0.004, 0.01, 0.05
    s = sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=None, anchor_a=np.zeros(3),
                   anchor_b=np.array([0.0, 0.0, -R0]), radius_a=r, radius_b=R0, mu=0.5)
    p = _problem([_sphere(m, r, (0.0, 0.0, r))], [s])
    o = oracle.run(p)[0]
    assert o.residuals()["converged"]
    assert np.allclose(o.vhat(0), 0.0, atol=1e-10)
    assert np.isclose(o.lam(0)[0], m * 9.81, rtol=1e-9)
    assert np.allclose(o.lam(0)[1:], 0.0, atol=1e-9)


@pytest.mark.parametrize("theta,mu", [(0.3, 0.5), (0.3, 0.1), (0.6, 0.2)])
def test_tilted_plane_stick_and_slide(theta, mu):
    """A point mass (anchor at the centre, no rolling lever) at rest on the plane through the
    origin with normal (sin theta, 0, cos theta)."""
    m, h, g = 0.004, 1e-3, 9.81
    n = np.array([np.sin(theta), 0.0, np.cos(theta)])
    c = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.zeros(3), normal=n, plane_z=0.0,
                   mu=mu)
    p = _problem([_sphere(m, 0.01, (0.0, 0.0, 0.0))], [c], h=h)
    o = oracle.run(p)[0]
    assert o.residuals()["converged"]
    v = o.vhat(0)[:3]
    lam = o.lam(0)
    down = np.array([np.cos(theta), 0.0, -np.sin(theta)])     # down-slope direction
    assert abs(n @ v) < 1e-10
    assert np.isclose(lam[0], m * g * np.cos(theta), rtol=1e-9)
    if mu >= np.tan(theta):
        assert np.allclose(v, 0.0, atol=1e-10)
        assert np.isclose(np.linalg.norm(lam[1:]), m * g * np.sin(theta), rtol=1e-9)
    else:
        want = 0.5 * h * g * (np.sin(theta) - mu * np.cos(theta))
        assert np.isclose(v @ down, want, rtol=1e-8)
        assert np.isclose(np.linalg.norm(lam[1:]), mu * lam[0], rtol=1e-9)


@pytest.mark.parametrize("theta,mu", [(0.4, 0.5), (0.4, 0.05), (0.7, 0.1)])
def test_sphere_rolls_or_slides_down_a_tilted_plane(theta, mu):
    """A solid sphere (I = 2/5 m r^2) at rest touching the plane through the origin with
    normal n = (sin theta, 0, cos theta).  Rolling (mu >= 2/7 tan theta): acceleration
    5/7 g sin theta down the slope and w = n x v / r.  Sliding: g (sin theta - mu cos theta)
    and angular acceleration 5/2 mu g cos theta / r about n x down.  At v-hat: times h/2."""
    m, r, h, g = 0.004, 0.01, 1e-3, 9.81
    n = np.array([np.sin(theta), 0.0, np.cos(theta)])
    down = np.array([np.cos(theta), 0.0, -np.sin(theta)])
    c = sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), anchor_a=np.zeros(3), radius_a=r, normal=n,
                   plane_z=0.0, mu=mu)
    p = _problem([_sphere(m, r, tuple(r * n))], [c], h=h)
    o = oracle.run(p)[0]
    assert o.residuals()["converged"]
    v, w = o.vhat(0)[:3], o.vhat(0)[3:]
    if mu >= 2.0 / 7.0 * np.tan(theta):
        want_v = 0.5 * h * 5.0 / 7.0 * g * np.sin(theta) * down
        assert np.allclose(v, want_v, rtol=1e-8, atol=1e-12)
        assert np.allclose(w, np.cross(n, want_v) / r, rtol=1e-8, atol=1e-10)
    else:
        want_v = 0.5 * h * g * (np.sin(theta) - mu * np.cos(theta)) * down
        want_w = 0.5 * h * 2.5 * mu * g * np.cos(theta) / r * np.cross(n, down)
        assert np.allclose(v, want_v, rtol=1e-8, atol=1e-12)
        assert np.allclose(w, want_w, rtol=1e-8, atol=1e-10)
    assert np.isclose(o.lam(0)[0], m * g * np.cos(theta), rtol=1e-9)


def test_coincident_centres_take_plus_z():
    s = sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=(1, 0), radius_a=0.01, radius_b=0.01, mu=0.2)
    p = _problem([_sphere(0.004, 0.01, (0, 0, 0)), _sphere(0.004, 0.01, (0, 0, 0))], [s],
                 g=(0, 0, 0))
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.assemble()
    _, Js = o.con_rows(0)
    assert np.array_equal(Js[0][0, :3], [0, 0, 1.0])
    assert np.isclose(o.phi(0)[0], -0.02)


def test_rejects_bad_parameters():
    body = _sphere(0.004, 0.01, (0, 0, 0.1))
    for itf in (sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), normal=np.zeros(3), mu=0.5),
                sg.JointIf(sg.PLANE_CONTACT, a=(0, 0), radius_a=-0.01, mu=0.5),
                sg.JointIf(sg.SPHERE_CONTACT, a=(0, 0), b=None, radius_a=-0.01, mu=0.5)):
        p = _problem([body], [itf])
        with pytest.raises(ValueError):
            oracle.OracleScene(p.scenes[0], p.options)
