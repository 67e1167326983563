"""Pins of the tetrahedral FEM beam generator (the rigid-deformable workload): element
stiffness against continuum mechanics, the Kuhn split, and the sizes of the full beam.
CPU only."""
import numpy as np
import pytest

import scenegen as sg


def _unit_tets():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((4, 3))
    return X, np.array([[0, 1, 2, 3]])


def test_element_stiffness_has_exactly_the_six_rigid_modes_as_kernel():
    X, tets = _unit_tets()
    Ke, vol = sg.tet_stiffness(X, tets, 1e5, 0.3)
    K = Ke[0]
    assert np.allclose(K, K.T, atol=1e-9 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 6 and ev.min() > -1e-9 * ev.max()
    for t in np.eye(3):                                  # translations
        assert np.abs(K @ np.tile(t, 4)).max() < 1e-9 * np.abs(K).max()
    for w in np.eye(3):                                  # infinitesimal rotations w x X
        u = np.cross(w, X).ravel()
        assert np.abs(K @ u).max() < 1e-9 * np.abs(K).max() * np.abs(X).max()


def test_uniform_strain_energy_matches_the_compliance_route():
    """A linear displacement u = G X has constant strain eps = sym(G); the element energy
    u^T K u / 2 must equal V eps^T C eps / 2 with C the inverse of the isotropic compliance
    matrix (built here from E and nu directly, not from the Lame form)."""
    X, tets = _unit_tets()
    E, nu = 1e5, 0.45
    Ke, vol = sg.tet_stiffness(X, tets, E, nu)
    S = np.zeros((6, 6))
    S[:3, :3] = -nu / E
    S[np.arange(3), np.arange(3)] = 1.0 / E
    S[np.arange(3, 6), np.arange(3, 6)] = 2.0 * (1.0 + nu) / E
    C = np.linalg.inv(S)
    rng = np.random.default_rng(1)
    for _ in range(3):
        G = rng.standard_normal((3, 3)) * 1e-3
        u = (X @ G.T).ravel()
        e = 0.5 * (G + G.T)
        eps = np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[0, 2], 2 * e[0, 1]])
        assert np.isclose(0.5 * u @ Ke[0] @ u, 0.5 * vol[0] * eps @ C @ eps, rtol=1e-10)


def test_kuhn_split_fills_the_cell_and_conforms():
    corners = np.arange(8)[None, :]
    tets = sg.kuhn_tets(corners)
    assert tets.shape == (6, 4)
    X = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float) * [2, 3, 5]
    _, vol = sg.tet_stiffness(X, tets, 1.0, 0.3)
    assert np.isclose(vol.sum(), 30.0) and (vol > 0).all()
    # two cells side by side: every interior face is shared by exactly two tets
    two = np.array([[0, 1, 2, 3, 4, 5, 6, 7], [4, 5, 6, 7, 8, 9, 10, 11]])
    tt = sg.kuhn_tets(two)
    faces = {}
    for t in tt:
        for drop in range(4):
            f = tuple(sorted(np.delete(t, drop)))
            faces[f] = faces.get(f, 0) + 1
    assert all(c in (1, 2) for c in faces.values())
    # the common quad {4, 5, 6, 7} is cut the same way from both cells: its two triangles
    # are each shared by one tet of either cell
    on_quad = [f for f in faces if set(f) <= {4, 5, 6, 7}]
    assert len(on_quad) == 2 and all(faces[f] == 2 for f in on_quad)


def test_slab_stiffness_rigid_modes_and_mass():
    sub, nid, tets = sg.fem_slab(np.array([0.0, 0.01, 0.02]), 3, 4, 0.02, 0.03, 1e5, 0.45,
                                 1000.0)
    K = sub.K_dense()
    X = sub.X0.reshape(-1, 3)
    assert np.allclose(K, K.T, atol=1e-9 * np.abs(K).max())
    for t in np.eye(3):
        assert np.abs(K @ np.tile(t, sub.nodes)).max() < 1e-8 * np.abs(K).max()
    for w in np.eye(3):
        assert np.abs(K @ np.cross(w, X).ravel()).max() < 1e-8 * np.abs(K).max()
    assert np.isclose(sub.mass.sum(), 1000.0 * 0.02 * 0.02 * 0.03)
    assert tets.shape[0] == 6 * 2 * 2 * 3
    # plane-fastest numbering keeps the stiffness band narrow
    Ki, Kj = sub.Ki.astype(int), sub.Kj.astype(int)
    assert np.abs(Ki - Kj).max() <= 3 * ((4 + 1) * 3 + 1) + 2      # node offset, then xyz


def test_full_beam_has_the_sizes_of_the_workload():
    p = sg.fem_beam(0)
    sc = p.scenes[0]
    slabs = sc.subs[:64]
    assert sorted({s.n for s in slabs}) == [900, 1200]
    assert sum(s.nodes for s in slabs) == 20000
    assert np.isclose(sum(s.mass.sum() for s in slabs), 1000.0 * 0.5 * 0.05 * 0.05)
    balls = [f for f in sc.ifs if f.kind == sg.BALL and f.b is not None
             and f.a[0] < 64 and f.b[0] < 64]
    contacts = [f for f in sc.ifs if f.kind == sg.PLANE_CONTACT]
    assert 3 * len(balls) == 18900 and len(contacts) == 2000
    assert len(sc.subs[64].bodies) == 7                 # the 7-R arm stand-in


def test_tet_count_of_the_full_beam():
    total = 0
    ks = [4 if g % 8 == 0 else 3 for g in range(64)]
    for k in ks:
        total += 6 * 9 * 9 * (k - 1)
    assert total == 66096


def test_cable_scene_shape():
    """The cable workload: 640 segments in 160 subsystems of 4 plus two arms (162
    subsystems, 3,840 cable DOF), a ball joint and three PD rows between neighbouring
    segments, a plane contact per segment, and the straight rest shape (every PD target and
    every joint anchor pair coincide at t = 0)."""
    p = sg.cable(0)
    sc = p.scenes[0]
    assert len(sc.subs) == 162
    assert sum(s.n for s in sc.subs[:160]) == 3840
    kinds = [f.kind for f in sc.ifs]
    assert kinds.count(sg.PLANE_CONTACT) == 640
    assert kinds.count(sg.ANGLE_PD) >= 3 * 639
    for f in sc.ifs:
        if f.kind == sg.BALL and f.b is not None and f.a[0] < 160 and f.b[0] < 160:
            ba = sc.subs[f.a[0]].bodies[f.a[1]]
            bb = sc.subs[f.b[0]].bodies[f.b[1]]
            assert np.allclose(ba.p + f.anchor_a, bb.p + f.anchor_b, atol=1e-12)


def test_stir_scene_shape():
    """The stir workload: 216 spheres (r 1 cm, 4 g) and the arm stand-in (217 subsystems,
    1,296 sphere DOF), no two bodies overlapping at t = 0 (every sphere-sphere gap and every
    wall / floor gap non-negative), candidate pairs closer than 1.5 diameters, and tool
    contacts only with spheres of the two top layers."""
    from scipy.spatial.transform import Rotation
    p = sg.stir(0)
    sc = p.scenes[0]
    assert len(sc.subs) == 217 and sum(s.n for s in sc.subs[:216]) == 1296
    assert p.options.h == 1e-2
    centres = np.array([s.bodies[0].p for s in sc.subs[:216]])
    r = 0.01
    for s in sc.subs[:216]:
        b = s.bodies[0]
        assert np.isclose(b.m, 0.004) and np.allclose(b.I, 0.4 * b.m * r * r)
    ztop = centres[:, 2].max()
    arm = sc.subs[216]
    for f in sc.ifs:
        if f.kind == sg.SPHERE_CONTACT and f.a[0] < 216:
            pa, pb = centres[f.a[0]], centres[f.b[0]]
            d = np.linalg.norm(pa - pb)
            assert d - f.radius_a - f.radius_b >= 0.0 and d < 1.5 * 2 * r
        elif f.kind == sg.SPHERE_CONTACT:               # the tool
            b = arm.bodies[f.a[1]]
            R = Rotation.from_quat([b.q[1], b.q[2], b.q[3], b.q[0]]).as_matrix()
            tool = b.p + R @ f.anchor_a
            pb = centres[f.b[0]]
            assert pb[2] >= ztop - 2.1 * r
            assert np.linalg.norm(tool - pb) - f.radius_a - f.radius_b >= 0.0
        elif f.kind == sg.PLANE_CONTACT:
            n = f.normal / np.linalg.norm(f.normal)
            assert n @ centres[f.a[0]] - f.plane_z - f.radius_a >= 0.0
    kinds = [f.kind for f in sc.ifs]
    assert kinds.count(sg.PLANE_CONTACT) == 180
