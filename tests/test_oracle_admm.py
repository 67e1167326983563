"""Pins of the oracle's ADMM loop (Algorithm 1, Eqs. admm-1i / admm-2j / admm-3 /
residual) against plain definitions: dense LU solves of the full KKT system, brute-force
contact-mode enumeration, and the fixed-point proposition.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle
import scenegen as sg


def test_cholesky_solve_matches_lapack_lu():
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 18, 40):
        G = rng.standard_normal((n, n))
        K = G @ G.T + n * np.eye(n)
        r = rng.standard_normal(n)
        x = oracle.chol_solve(K, r)
        assert np.allclose(x, np.linalg.solve(K, r), rtol=1e-12, atol=1e-12)


def test_cholesky_rejects_indefinite():
    with pytest.raises(np.linalg.LinAlgError):
        oracle.chol_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))


def _one_scene(subs, ifs, **opt):
    o = sg.Options(gravity=(0.0, 0.0, 0.0), warm="cold", **opt)
    return sg.Problem([sg.Scene(subs, ifs)], o)


def _full_system(scene):
    """Dense A, b, J, e of the whole scene (block diagonal A; Eq. sdyn-total2)."""
    offs = np.cumsum([0] + [s.n for s in scene.subs])
    n = offs[-1]
    A = np.zeros((n, n))
    b = np.zeros(n)
    for i, s in enumerate(scene.subs):
        A[offs[i]:offs[i + 1], offs[i]:offs[i + 1]] = s.A
        b[offs[i]:offs[i + 1]] = s.b
    rows = []
    es = []
    for itf in scene.ifs:
        R = np.zeros((itf.rows, n))
        for s, Js in zip(itf.subs, itf.J):
            R[:, offs[s]:offs[s + 1]] += Js
        rows.append(R)
        es.append(itf.e)
    J = np.vstack(rows) if rows else np.zeros((0, n))
    e = np.concatenate(es) if es else np.zeros(0)
    return A, b, J, e


def test_unconstrained_block_is_plain_solve():
    rng = np.random.default_rng(1)
    G = rng.standard_normal((9, 9))
    A = G @ G.T + 9 * np.eye(9)
    b = rng.standard_normal(9)
    p = _one_scene([sg.GenericSub(A, b)], [], max_iters=3, tol_primal=-1)
    o = oracle.run(p)[0]
    assert np.allclose(o.vhat(0), np.linalg.solve(A, b), rtol=1e-12)


def test_trace_rule_for_beta():
    # Sec. III-D: beta_i = Tr(A_i) / Tr(J_ci^T J_ci); Tr(J^T J) = sum of squared entries
    rng = np.random.default_rng(2)
    A0 = np.diag([1.0, 2.0, 3.0])
    A1 = np.diag([4.0, 5.0])
    J0 = rng.standard_normal((2, 3))
    J1 = rng.standard_normal((2, 2))
    J0b = rng.standard_normal((1, 3))
    ifs = [sg.RowsIf(sg.EQUALITY, [0, 1], [J0, J1], np.zeros(2)),
           sg.RowsIf(sg.HARD, [0], [J0b], np.zeros(1))]
    p = _one_scene([sg.GenericSub(A0, np.zeros(3)), sg.GenericSub(A1, np.zeros(2))], ifs,
                   max_iters=1, tol_primal=-1)
    o = oracle.run(p)[0]
    assert np.isclose(o.beta(0), 6.0 / (np.sum(J0 ** 2) + np.sum(J0b ** 2)), rtol=1e-14)
    assert np.isclose(o.beta(1), 9.0 / np.sum(J1 ** 2), rtol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_bilateral_converges_to_full_kkt_solve(seed):
    """Equality-only systems: the ADMM fixed point is the KKT solution of the full system
    [A -J^T; J 0] [v; lambda] = [b; -e], solved with dense LU (LAPACK)."""
    rng = np.random.default_rng(seed)
    sc = sg.generic_scene(rng, n_sub=3 + seed % 3, n_range=(8, 12), types=(sg.EQUALITY,),
                          extra=2)
    A, b, J, e = _full_system(sc)
    assert np.linalg.matrix_rank(J) == J.shape[0]
    m, n = J.shape
    KKT = np.block([[A, -J.T], [J, np.zeros((m, m))]])
    sol = np.linalg.solve(KKT, np.concatenate([b, -e]))
    v_ref, lam_ref = sol[:n], sol[n:]
    p = sg.Problem([sc], sg.Options(gravity=(0, 0, 0), warm="cold", tol_primal=1e-13,
                                    max_iters=200000))
    o = oracle.run(p)[0]
    res = o.residuals()
    assert res["converged"], res
    v = o.vhat_all()
    assert np.max(np.abs(v - v_ref)) / np.max(np.abs(v_ref)) < 1e-9
    lam = o.lam_all()
    assert np.max(np.abs(lam - lam_ref)) / np.max(np.abs(lam_ref)) < 1e-7
    # the returned v-hat satisfies the constraints to the primal tolerance
    assert np.max(np.abs(J @ v + e)) < 1e-11


@pytest.mark.parametrize("seed", range(4))
def test_u_equals_minus_lambda_after_each_update(seed):
    # Eq. admm-3 with Eq. surrogate: u^{l+1} = y^{l+1} - beta z^{l+1} = -lambda^{l+1}
    p = sg.generic(seed, n_scenes=1, max_iters=1 + seed * 5, tol_primal=-1)
    o = oracle.run(p)[0]
    for j in range(o.ncon):
        u = o.side(j, "u")
        assert np.allclose(u, -o.lam(j)[None, :], atol=1e-12)


def test_fixed_point_proposition():
    """Sec. III-D proposition: at theta = 0 the iterate is a fixed point.  Generic blocks
    carry no state, so a second step warm-started from the converged (lambda, z) must
    start at the fixed point: one iteration, theta ~ 0, v-hat and lambda unchanged."""
    p = sg.generic(11, n_scenes=1, types=(sg.EQUALITY, sg.SOFT, sg.HARD), max_iters=100000,
                   tol_primal=1e-12, warm="prev", n_range=(8, 12))
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.step()
    assert o.residuals()["converged"]
    v1, l1 = o.vhat_all(), o.lam_all()
    o.step()
    res = o.residuals()
    assert res["iters"] == 1 and res["theta"] < 1e-20 and res["r_p"] <= 1e-12
    assert np.allclose(o.vhat_all(), v1, rtol=1e-10, atol=1e-12)
    assert np.allclose(o.lam_all(), l1, rtol=1e-10, atol=1e-12)


def test_theta_stop_rule_stops_after_v_step():
    p = sg.generic(3, n_scenes=1, max_iters=100000, tol_primal=-1, n_range=(8, 12))
    p.options.stop = "theta"
    p.options.theta_th = 1e-20
    o = oracle.run(p, trace_cap=100000)[0]
    res = o.residuals()
    assert res["converged"] and res["theta"] < 1e-20
    tr = o.trace_array()[: res["iters"]]
    assert np.all(tr[1:-1, 0] >= 1e-20)


# ---------------------------------------------------------------------------------------
# tiny planar contact systems against full-system mode enumeration (Eq. scc)


def _enumerate_planar(A, b, Jn, Jt, en, mu):
    """Every solution of the full-system Signorini-Coulomb problem with one tangent per
    contact: modes {open, stick, slip+, slip-} per contact, each a linear system."""
    n = A.shape[0]
    m = Jn.shape[0]
    sols = []
    for modes in itertools.product(range(4), repeat=m):
        # unknowns v (n), ln (m), lt (m)
        N = n + 2 * m
        M = np.zeros((N, N))
        r = np.zeros(N)
        M[:n, :n] = A
        M[:n, n:n + m] = -Jn.T
        M[:n, n + m:] = -Jt.T
        r[:n] = b
        for c, md in enumerate(modes):
            i1, i2 = n + c, n + m + c
            if md == 0:      # open
                M[i1, n + c] = 1.0
                M[i2, n + m + c] = 1.0
            elif md == 1:    # stick: c_n = 0, c_t = 0
                M[i1, :n] = Jn[c]; r[i1] = -en[c]
                M[i2, :n] = Jt[c]
            else:            # slip: c_n = 0, lt = -+ mu ln
                M[i1, :n] = Jn[c]; r[i1] = -en[c]
                sgn = 1.0 if md == 2 else -1.0
                M[i2, n + m + c] = 1.0
                M[i2, n + c] = sgn * mu[c]
        try:
            x = np.linalg.solve(M, r)
        except np.linalg.LinAlgError:
            continue
        v, ln, lt = x[:n], x[n:n + m], x[n + m:]
        cn = Jn @ v + en
        ct = Jt @ v
        ok = True
        tol = 1e-9
        for c, md in enumerate(modes):
            if md == 0:
                ok &= cn[c] >= -tol
            elif md == 1:
                ok &= ln[c] >= -tol and abs(lt[c]) <= mu[c] * ln[c] + tol
            elif md == 2:
                ok &= ln[c] >= -tol and ct[c] >= -tol
            else:
                ok &= ln[c] >= -tol and ct[c] <= tol
        if ok:
            sols.append(v)
    return sols


@pytest.mark.parametrize("seed", range(12))
def test_planar_contact_matches_enumeration(seed):
    rng = np.random.default_rng(500 + seed)
    n = 3
    m = 1 + seed % 2
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    b = rng.standard_normal(n) * 2
    Jn = rng.standard_normal((m, n))
    Jt = rng.standard_normal((m, n))
    en = rng.standard_normal(m) * 0.5
    mu = rng.uniform(0.2, 1.0, m)
    ifs = []
    for c in range(m):
        Jc = np.vstack([Jn[c], Jt[c], np.zeros(n)])
        ifs.append(sg.RowsIf(sg.CONTACT, [0], [Jc], np.array([en[c], 0.0, 0.0]), mu=mu[c]))
    p = _one_scene([sg.GenericSub(A, b)], ifs, tol_primal=1e-12, max_iters=200000)
    o = oracle.run(p)[0]
    assert o.residuals()["converged"]
    v = o.vhat(0)
    sols = _enumerate_planar(A, b, Jn, Jt, en, mu)
    assert sols, "the enumeration always has a solution here"
    err = min(np.max(np.abs(v - s)) / max(np.max(np.abs(s)), 1e-12) for s in sols)
    assert err < 1e-8, (v, sols)


@pytest.mark.parametrize("seed", range(3))
def test_full_system_admm_converges_to_the_same_kkt_solve(seed):
    """The full-system ADMM comparator (Sec. IV-B, FADMM) is the same iteration on the scene
    merged into one subsystem: its fixed point is the same KKT solution as the split
    scene's, and its one block is the block-diagonal A of the full system."""
    rng = np.random.default_rng(40 + seed)
    sc = sg.generic_scene(rng, n_sub=3 + seed, n_range=(6, 10), types=(sg.EQUALITY,), extra=2)
    A, b, J, e = _full_system(sc)
    m, n = J.shape
    KKT = np.block([[A, -J.T], [J, np.zeros((m, m))]])
    v_ref = np.linalg.solve(KKT, np.concatenate([b, -e]))[:n]
    p = sg.Problem([sc], sg.Options(gravity=(0, 0, 0), warm="cold", tol_primal=1e-13,
                                    max_iters=200000))
    q = sg.merged(p)
    assert len(q.scenes[0].subs) == 1 and np.array_equal(q.scenes[0].subs[0].A, A)
    o = oracle.run(q)[0]
    assert o.residuals()["converged"]
    assert np.max(np.abs(o.vhat_all() - v_ref)) / np.max(np.abs(v_ref)) < 1e-9


def test_merged_rigid_chain_matches_the_split_chain():
    """A bilateral rigid chain merged into one subsystem steps to the same state as the
    chain split into four (both converged tightly: the same KKT solution per step)."""
    p = sg.chain(0, tol_primal=1e-12, max_iters=200000, rho=1e3)
    a = oracle.run(p, steps=3)[0]
    b = oracle.run(sg.merged(p), steps=3)[0]
    assert len(sg.merged(p).scenes[0].subs) == 1
    assert np.max(np.abs(a.bodies_all()[:, 4:] - b.bodies_all()[:, 4:])) < 1e-7


def test_beta_scale_multiplies_the_trace_rule_and_rho():
    """A per-subsystem scale s_i gives beta_i = s_i Tr(A_i) / Tr(J_ci^T J_ci) (Sec. III-D's
    rule, computed here by hand), and s_i rho in the fixed mode."""
    rng = np.random.default_rng(7)
    A0, A1 = np.diag([1.0, 2.0, 3.0]), np.diag([4.0, 5.0])
    J0, J1 = rng.standard_normal((2, 3)), rng.standard_normal((2, 2))
    ifs = [sg.RowsIf(sg.EQUALITY, [0, 1], [J0, J1], np.zeros(2))]
    subs = [sg.GenericSub(A0, np.zeros(3)), sg.GenericSub(A1, np.zeros(2))]
    o = oracle.OracleScene(sg.Scene(subs, ifs), sg.Options(max_iters=1, tol_primal=-1))
    o.set_beta_scale(0, 0.25)
    o.set_beta_scale(1, 8.0)
    o.step()
    assert np.isclose(o.beta(0), 0.25 * 6.0 / np.sum(J0 ** 2), rtol=1e-14)
    assert np.isclose(o.beta(1), 8.0 * 9.0 / np.sum(J1 ** 2), rtol=1e-14)
    f = oracle.OracleScene(sg.Scene(subs, ifs), sg.Options(max_iters=1, tol_primal=-1,
                                                           beta_mode="fixed", rho=3.0))
    f.set_beta_scale(1, 0.5)
    f.step()
    assert f.beta(0) == 3.0 and f.beta(1) == 1.5


@pytest.mark.parametrize("seed", range(3))
def test_fixed_point_does_not_depend_on_beta_scales(seed):
    """Any positive beta_i leaves the ADMM fixed point unchanged: equality-only systems with
    random per-subsystem scales in [1/8, 8] still converge to the full KKT solution."""
    rng = np.random.default_rng(60 + seed)
    sc = sg.generic_scene(rng, n_sub=4, n_range=(6, 10), types=(sg.EQUALITY,), extra=2)
    A, b, J, e = _full_system(sc)
    m, n = J.shape
    KKT = np.block([[A, -J.T], [J, np.zeros((m, m))]])
    v_ref = np.linalg.solve(KKT, np.concatenate([b, -e]))[:n]
    o = oracle.OracleScene(sc, sg.Options(gravity=(0, 0, 0), warm="cold", tol_primal=1e-13,
                                          max_iters=400000))
    for i in range(len(sc.subs)):
        o.set_beta_scale(i, float(2.0 ** rng.uniform(-3, 3)))
    o.step()
    assert o.residuals()["converged"]
    assert np.max(np.abs(o.vhat_all() - v_ref)) / np.max(np.abs(v_ref)) < 1e-9
