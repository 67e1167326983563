"""Co-rotational linear elasticity in the oracle (the paper's beam model, Sec. IV-A): each
element's stiffness and force use the rotation R of its deformation gradient (polar
decomposition), so rigid motions produce no elastic force; without rotation it is the
linear model."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import scenegen as sg


def _one_tet(x=None, E=1e5, nu=0.45):
    X = np.array([[0.0, 0, 0], [0.01, 0, 0], [0, 0.012, 0], [0.002, 0.001, 0.011]])
    tets = np.array([[0, 1, 2, 3]])
    Ke, vol = sg.tet_stiffness(X, tets, E, nu)
    dof = np.arange(12)
    sub = sg.LinearSub(np.full(4, 1e-3), np.repeat(dof, 12), np.tile(dof, 12), Ke[0].ravel(),
                       np.zeros(12), X.ravel().copy(),
                       (X if x is None else x).ravel().copy(), np.zeros(12),
                       tets=tets, Ke=Ke, corot=True)
    o = oracle.OracleScene(sg.Scene([sub], []), sg.Options(gravity=(0, 0, 0)))
    return o, X, Ke[0]


def _blockrot(Q):
    return np.kron(np.eye(4), Q)


def test_rest_state_is_the_linear_model():
    o, X, K0 = _one_tet()
    f, K = o.elastic(0)
    assert np.max(np.abs(f)) == 0.0
    assert np.allclose(K, K0, rtol=1e-13, atol=1e-13 * np.abs(K0).max())


@pytest.mark.parametrize("seed", range(4))
def test_rigid_motion_has_no_elastic_force(seed):
    """x = Q X + t: F = Q, R = Q, the force -R K (R^T x - X) vanishes (K's kernel holds the
    rigid translations) and the stiffness is Q K Q^T per node block; the linear model would
    push back against the rotation."""
    rng = np.random.default_rng(seed)
    Q = Rotation.from_rotvec(rng.uniform(-2.5, 2.5, 3)).as_matrix()
    X = np.array([[0.0, 0, 0], [0.01, 0, 0], [0, 0.012, 0], [0.002, 0.001, 0.011]])
    x = X @ Q.T + rng.uniform(-1, 1, 3)
    o, _, K0 = _one_tet(x)
    f, K = o.elastic(0)
    scale = np.abs(K0).max() * np.abs(x).max()
    assert np.max(np.abs(f)) < 1e-11 * scale
    Qb = _blockrot(Q)
    assert np.allclose(K, Qb @ K0 @ Qb.T, rtol=0, atol=1e-12 * np.abs(K0).max())
    lin = -K0 @ (x - X).ravel()
    assert np.max(np.abs(lin)) > 1e-3 * scale          # what the linear model would do


@pytest.mark.parametrize("seed", range(4))
def test_forces_sum_to_zero_and_match_the_linear_model_without_rotation(seed):
    rng = np.random.default_rng(10 + seed)
    X = np.array([[0.0, 0, 0], [0.01, 0, 0], [0, 0.012, 0], [0.002, 0.001, 0.011]])
    # a large deformation: forces still balance (linear momentum)
    o, _, K0 = _one_tet(X + rng.uniform(-2e-3, 2e-3, X.shape))
    f, _ = o.elastic(0)
    assert np.max(np.abs(f.reshape(4, 3).sum(0))) < 1e-12 * np.abs(f).max()
    # a small symmetric (rotation-free) strain: F = I + eps S, R = I to O(eps^2)
    S = rng.standard_normal((3, 3)); S = 0.5 * (S + S.T)
    eps = 1e-7
    x = X @ (np.eye(3) + eps * S).T
    o, _, K0 = _one_tet(x)
    f, _ = o.elastic(0)
    lin = -K0 @ (x - X).ravel()
    assert np.max(np.abs(f - lin)) < 1e-5 * np.max(np.abs(lin))


def test_polar_rotation_properties():
    """For a general deformation the rotation the oracle uses is orthogonal with det 1 and
    R^T F is symmetric positive definite: checked through the stiffness it builds (R K R^T
    has K's eigenvalues) and against scipy's polar decomposition."""
    from scipy.linalg import polar
    rng = np.random.default_rng(3)
    X = np.array([[0.0, 0, 0], [0.01, 0, 0], [0, 0.012, 0], [0.002, 0.001, 0.011]])
    x = X + rng.uniform(-3e-3, 3e-3, X.shape)
    o, _, K0 = _one_tet(x)
    _, K = o.elastic(0)
    Dm = (X[1:] - X[0]).T
    Ds = (x[1:] - x[0]).T
    R, _ = polar(Ds @ np.linalg.inv(Dm))
    Rb = _blockrot(R)
    assert np.allclose(K, Rb @ K0 @ Rb.T, rtol=0, atol=1e-11 * np.abs(K0).max())
    assert np.allclose(np.linalg.eigvalsh(K), np.linalg.eigvalsh(K0), atol=1e-9 * np.abs(K0).max())


def test_corotational_beam_is_linear_beam_at_rest_and_steps():
    """A small co-rotational beam at rest assembles the linear beam's K (its first step is
    the linear model's step to rounding) and keeps stepping with finite states."""
    kw = dict(ny=3, nz=3, planes=8, slabs=3, length=0.03, width=0.01, height=0.01,
              tol_primal=-1, max_iters=30)
    a = oracle.run(sg.fem_beam(0, **kw), steps=1)[0]
    b = oracle.run(sg.fem_beam(0, corotational=True, **kw), steps=1)[0]
    assert np.max(np.abs(a.nodes_all() - b.nodes_all())) < 1e-12 * np.max(np.abs(a.nodes_all()))
    c = oracle.run(sg.fem_beam(0, corotational=True, **kw), steps=5)[0]
    assert np.all(np.isfinite(c.nodes_all()))
