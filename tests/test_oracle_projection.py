"""Pins of the oracle's z-step (Sec. III-C, Eq. admm-2j) against brute force and the
definitions of the constraint classes (Sec. II-A).  CPU only."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle

EQ, HARD, SOFT, CONTACT = 0, 1, 2, 3


def _z_from(lam, y, beta):
    # Eq. surrogate: beta_i z_ij = y_ij + lambda_j
    return (y + lam[None, :]) / beta[:, None]


def _brute(type_, beta, y, e, k=0.0, alpha=0.0):
    """Minimise Eq. admm-2j directly over z with a generic optimiser.

    objective  g_j(z) + sum_i beta_i/2 |z_i - y_i/beta_i|^2  (x - z + u/beta = y/beta - z)
    hard:      g = indicator(sum_i z_i + e >= 0)
    equality:  g = indicator(sum_i z_i + e == 0)
    soft:      g = the potential whose negative gradient is lambda = -k (e + alpha c),
               c = sum_i z_i, i.e. g(c) = k e c + k alpha c^2 / 2
    """
    ns, rows = y.shape

    def obj(zf):
        z = zf.reshape(ns, rows)
        val = 0.5 * np.sum(beta[:, None] * (z - y / beta[:, None]) ** 2)
        if type_ == SOFT:
            c = z.sum(0)
            val += np.sum(k * e * c + 0.5 * k * alpha * c * c)
        return val

    cons = []
    for r in range(rows):
        f = (lambda zf, r=r: zf.reshape(ns, rows)[:, r].sum() + e[r])
        if type_ == EQ:
            cons.append({"type": "eq", "fun": f})
        elif type_ == HARD:
            cons.append({"type": "ineq", "fun": f})
    z0 = (y / beta[:, None]).ravel()
    res = minimize(obj, z0, constraints=cons, method="SLSQP",
                   options={"ftol": 1e-15, "maxiter": 500})
    z = res.x.reshape(ns, rows)
    return beta[0] * z[0] - y[0]       # lambda from any side


@pytest.mark.parametrize("type_", [EQ, HARD, SOFT])
@pytest.mark.parametrize("seed", range(6))
def test_scalar_types_match_brute_force(type_, seed):
    rng = np.random.default_rng(seed)
    ns = 1 + seed % 3
    rows = 1 + (seed // 2) % 3
    beta = 10 ** rng.uniform(-1, 1, ns)
    y = rng.standard_normal((ns, rows))
    e = rng.standard_normal(rows)
    k, alpha = 10 ** rng.uniform(0, 1), 10 ** rng.uniform(-2, 0)
    lam = oracle.project(type_, beta, y, e, k, alpha)
    ref = _brute(type_, beta, y, e, k, alpha)
    assert np.allclose(lam, ref, atol=1e-6, rtol=1e-6), (lam, ref)
    # every side sees the same multiplier: beta_i z_i - y_i is side independent
    z = _z_from(lam, y, beta)
    lam_sides = beta[:, None] * z - y
    assert np.allclose(lam_sides, lam[None, :], atol=1e-12)


def test_hard_is_complementary():
    rng = np.random.default_rng(7)
    for _ in range(200):
        ns = int(rng.integers(1, 4))
        beta = 10 ** rng.uniform(-2, 2, ns)
        y = rng.standard_normal((ns, 1)) * 10
        e = rng.standard_normal(1) * 10
        lam = oracle.project(HARD, beta, y, e)
        c = _z_from(lam, y, beta).sum(0) + e
        # Eq. hard12: 0 <= lambda  perp  z_1 + z_2 + e >= 0
        assert lam[0] >= 0 and c[0] >= -1e-12 and abs(lam[0] * c[0]) < 1e-9


def test_equality_satisfies_constraint():
    rng = np.random.default_rng(3)
    beta = np.array([2.0, 0.5, 7.0])
    y = rng.standard_normal((3, 3))
    e = rng.standard_normal(3)
    lam = oracle.project(EQ, beta, y, e)
    c = _z_from(lam, y, beta).sum(0) + e
    assert np.allclose(c, 0.0, atol=1e-13)


def test_soft_satisfies_its_law():
    # Eq. soft12: lambda = -k (e + alpha (z_1 + z_2))
    rng = np.random.default_rng(4)
    for _ in range(50):
        ns = int(rng.integers(1, 4))
        beta = 10 ** rng.uniform(-1, 1, ns)
        y = rng.standard_normal((ns, 1))
        e = rng.standard_normal(1)
        k, alpha = 10 ** rng.uniform(-1, 2), 10 ** rng.uniform(-3, 0)
        lam = oracle.project(SOFT, beta, y, e, k, alpha)
        c = _z_from(lam, y, beta).sum(0)
        assert np.allclose(lam, -k * (e + alpha * c), rtol=1e-12, atol=1e-13)


def _contact_conditions(lam, c, mu, tol=1e-9):
    """Eq. contact12 checked on (lambda, c), c = z_1 + z_2 + e; returns the mode."""
    ln, lt = lam[0], lam[1:]
    cn, ct = c[0], c[1:]
    scale = max(1.0, np.abs(lam).max(), np.abs(c).max())
    tol = tol * scale
    assert ln >= -tol and cn >= -tol and abs(ln * cn) <= tol * scale
    nt = np.linalg.norm(lt)
    assert nt <= mu * ln + tol
    if ln <= tol:
        return "open"
    if np.linalg.norm(ct) <= tol:
        return "stick"
    # slip: delta lambda_t + mu lambda_n c_t = 0 with delta >= 0 -> c_t anti-parallel
    assert abs(nt - mu * ln) <= tol
    delta = -mu * ln * np.dot(ct, lt) / max(nt * nt, 1e-300)
    assert delta >= -tol
    assert np.allclose(delta * lt + mu * ln * ct, 0.0, atol=tol)
    return "slip"


def _enumerate_contact(s, w, mu):
    """All lambda solving Eq. contact12 with c = s lambda + w, by mode enumeration."""
    sols = []
    # open: lambda = 0, c = w, needs c_n >= 0
    if w[0] >= 0:
        sols.append(np.zeros(3))
    # stick: c = 0 -> lambda = -w/s, needs lambda_n >= 0 and |lambda_t| <= mu lambda_n
    lam = -w / s
    if lam[0] >= 0 and np.linalg.norm(lam[1:]) <= mu * lam[0]:
        sols.append(lam)
    # slip: c_n = 0 -> lambda_n = -w_n/s > 0;  |lambda_t| = mu lambda_n and
    # c_t = s lambda_t + w_t = -(delta/(mu lambda_n)) lambda_t with delta > 0
    ln = -w[0] / s
    wt = w[1:]
    if ln > 0 and np.linalg.norm(wt) > 0:
        d = -wt / np.linalg.norm(wt)
        delta = np.linalg.norm(wt) - s * mu * ln
        if delta > 0:
            sols.append(np.concatenate([[ln], mu * ln * d]))
    return sols


@pytest.mark.parametrize("seed", range(40))
def test_contact_matches_mode_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    ns = 1 + seed % 2
    beta = 10 ** rng.uniform(-1, 1, ns)
    y = rng.standard_normal((ns, 3))
    e = np.array([rng.standard_normal(), 0.0, 0.0])
    mu = rng.uniform(0.1, 1.2)
    lam = oracle.project(CONTACT, beta, y, e, mu=mu)
    s = np.sum(1 / beta)
    w = (y / beta[:, None]).sum(0) + e
    c = s * lam + w
    _contact_conditions(lam, c, mu)
    sols = _enumerate_contact(s, w, mu)
    assert len(sols) == 1, "Eq. contact12 has a unique solution under the s I metric"
    assert np.allclose(lam, sols[0], atol=1e-12)


def test_contact_modes_all_reached():
    seen = set()
    rng = np.random.default_rng(5)
    for _ in range(300):
        beta = np.array([1.0])
        y = rng.standard_normal((1, 3)) * 2
        e = np.zeros(3)
        lam = oracle.project(CONTACT, beta, y, e, mu=0.5)
        seen.add(_contact_conditions(lam, lam + y[0] + e, 0.5))
    assert seen == {"open", "stick", "slip"}


def test_contact_tangent_basis_invariance():
    rng = np.random.default_rng(9)
    for _ in range(100):
        beta = 10 ** rng.uniform(-1, 1, 2)
        y = rng.standard_normal((2, 3))
        e = np.array([rng.standard_normal() * 0.3, 0.0, 0.0])
        lam = oracle.project(CONTACT, beta, y, e, mu=0.7)
        a = rng.uniform(0, 2 * np.pi)
        Rt = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        y2 = y.copy()
        y2[:, 1:] = y[:, 1:] @ Rt.T
        lam2 = oracle.project(CONTACT, beta, y2, e, mu=0.7)
        assert np.isclose(lam2[0], lam[0], atol=1e-13)
        assert np.allclose(lam2[1:], Rt @ lam[1:], atol=1e-12)


def test_single_side_unit_beta_reduces_to_plain_projections():
    # |S_j| = 1, beta = 1: lambda = Pi(-(y + e))
    y = np.array([[0.3, -2.0, 0.5]])
    e = np.array([-1.0, 0.0, 0.0])
    assert np.allclose(oracle.project(EQ, [1.0], y, e), -(y[0] + e))
    assert np.allclose(oracle.project(HARD, [1.0], y, e), np.maximum(0, -(y[0] + e)))
    lam = oracle.project(CONTACT, [1.0], y, e, mu=0.5)
    ln = 0.7
    lt = -y[0, 1:]
    lt = lt * (0.5 * ln / np.linalg.norm(lt))
    assert np.allclose(lam, np.concatenate([[ln], lt]))
