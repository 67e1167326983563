"""Seeded synthetic scene generators.

This module only describes scenes: bodies, masses, initial poses, joint anchors and axes,
generic SPD blocks and random constraint rows.  It holds none of the method's arithmetic
(no dynamics assembly, no Jacobians, no projections, no ADMM): both the CPU oracle and the
CUDA library consume the descriptions built here, and each side does all of the method's
work in its own code.

Scene shapes follow the paper's examples (Sec. IV-A: rigid chains, articulated robots with
point contacts, split deformable blocks) at the sizes of the workloads this project
measures; every draw comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Projection types of a constraint (Sec. II-A: soft, hard, contact; hard covers equations
# and inequalities).
EQUALITY, HARD, SOFT, CONTACT = 0, 1, 2, 3
TYPE_NAMES = {EQUALITY: "equality", HARD: "hard", SOFT: "soft", CONTACT: "contact"}

# Interface sources: explicit rows, or a rigid-body model constraint whose rows are built
# from the bodies' state every step.
ROWS, BALL, REVOLUTE, ANGLE_PD, PLANE_CONTACT, SPHERE_CONTACT = 0, 1, 2, 3, 4, 5

WORLD = -1


@dataclass
class Body:
    """A rigid body in maximal coordinates.

    ``q`` is the unit quaternion (w, x, y, z) of the body-to-world rotation, ``v`` the
    world-frame linear velocity of the centre of mass, ``w`` the body-frame angular
    velocity.  The inertia is diagonal in the body frame (principal axes).
    """

    m: float
    I: np.ndarray
    p: np.ndarray
    q: np.ndarray
    v: np.ndarray
    w: np.ndarray


@dataclass
class GenericSub:
    """A subsystem given directly by its SPD block ``A`` (n x n) and vector ``b``."""

    A: np.ndarray
    b: np.ndarray

    @property
    def n(self) -> int:
        return int(self.b.shape[0])


@dataclass
class RigidSub:
    """A subsystem made of rigid bodies (6 DOF each: [v, w] per body)."""

    bodies: List[Body]

    @property
    def n(self) -> int:
        return 6 * len(self.bodies)


@dataclass
class LinearSub:
    """A linear elastic block of nodes (3 DOF each): lumped node masses, a symmetric
    stiffness K given by triplets (Ki, Kj, Kv), a constant force f, rest positions X0,
    positions x and velocities v (each 3 * nodes long)."""

    mass: np.ndarray
    Ki: np.ndarray
    Kj: np.ndarray
    Kv: np.ndarray
    f: np.ndarray
    X0: np.ndarray
    x: np.ndarray
    v: np.ndarray
    tets: Optional[np.ndarray] = None   # elements (T x 4 node indices), when known
    Ke: Optional[np.ndarray] = None     # their rest stiffness matrices (T x 12 x 12)
    corot: bool = False                 # co-rotational: K and force from the elements

    @property
    def nodes(self) -> int:
        return int(self.mass.shape[0])

    @property
    def n(self) -> int:
        return 3 * self.nodes

    def K_dense(self) -> np.ndarray:
        K = np.zeros((self.n, self.n))
        np.add.at(K, (self.Ki.astype(int), self.Kj.astype(int)), self.Kv)
        return K


def spring_stiffness(X: np.ndarray, edges, k: float):
    """Stiffness triplets of linear springs (stiffness k) along the rest directions of the
    given node pairs: each spring adds k d d^T to the (a,a), (b,b) blocks and -k d d^T to the
    (a,b), (b,a) blocks, d the unit rest direction."""
    acc = {}
    for a, b in edges:
        d = X[b] - X[a]
        d = d / np.linalg.norm(d)
        blk = k * np.outer(d, d)
        for (p, q, s) in ((a, a, 1.0), (b, b, 1.0), (a, b, -1.0), (b, a, -1.0)):
            for i in range(3):
                for j in range(3):
                    key = (3 * p + i, 3 * q + j)
                    acc[key] = acc.get(key, 0.0) + s * blk[i, j]
    keys = sorted(k_ for k_, v_ in acc.items() if v_ != 0.0)
    Ki = np.array([k_[0] for k_ in keys], dtype=np.int64)
    Kj = np.array([k_[1] for k_ in keys], dtype=np.int64)
    Kv = np.array([acc[k_] for k_ in keys])
    return Ki, Kj, Kv


_LATTICE_CACHE: dict = {}


def _lattice_stiffness(dims, spacing, k):
    key = (tuple(dims), float(spacing), float(k))
    if key not in _LATTICE_CACHE:
        nx, ny, nz = dims
        X = np.array([[i * spacing, j * spacing, l * spacing] for l in range(nz)
                      for j in range(ny) for i in range(nx)], dtype=np.float64)
        d = np.linalg.norm(X[None, :, :] - X[:, None, :], axis=2)
        a, b = np.nonzero(np.triu(d < 1.8 * spacing, 1))
        _LATTICE_CACHE[key] = (X, spring_stiffness(X, list(zip(a.tolist(), b.tolist())), k))
    return _LATTICE_CACHE[key]


def lattice_block(dims=(2, 2, 3), spacing=0.02, origin=(0.0, 0.0, 0.0), density=1000.0,
                  k=500.0, v=None) -> LinearSub:
    """Nodes on a dims grid joined by springs to their neighbours within one cell diagonal
    (a stand-in for a small linear FEM block); lumped mass = density * spacing^3 per node."""
    X, (Ki, Kj, Kv) = _lattice_stiffness(dims, spacing, k)
    X = X + np.asarray(origin, dtype=np.float64)
    nn = X.shape[0]
    mass = np.full(nn, density * spacing ** 3)
    vv = np.zeros(3 * nn) if v is None else np.tile(np.asarray(v, dtype=np.float64), nn)
    return LinearSub(mass, Ki, Kj, Kv, np.zeros(3 * nn), X.ravel().copy(), X.ravel().copy(), vv)


@dataclass
class RowsIf:
    """An interface given by explicit rows.

    ``subs[s]`` is the subsystem of side s; ``J[s]`` is (rows x n_subs[s]); the constraint
    value is sum_s J[s] v_subs[s] + e.  ``type`` is one of EQUALITY/HARD/SOFT/CONTACT;
    a contact has 3 rows ordered (normal, tangent 1, tangent 2).
    """

    type: int
    subs: List[int]
    J: List[np.ndarray]
    e: np.ndarray
    k: float = 0.0
    alpha: float = 0.0
    mu: float = 0.0

    @property
    def rows(self) -> int:
        return int(self.e.shape[0])


@dataclass
class JointIf:
    """A rigid-body model constraint between body ``a`` and body ``b`` (or the world).

    ``a`` and ``b`` are (subsystem, body index) pairs; ``b`` is None for the world, in which
    case ``anchor_b`` is a world point and ``axis_b``/``ref_b`` are world vectors.

    kind BALL:          anchor_a (a frame), anchor_b (b frame)                    3 rows
    kind REVOLUTE:      + axis_a, ref_a (a frame, ref_a orthogonal to axis_a),
                        axis_b (b frame)                                         5 rows
    kind ANGLE_PD:      axis_a, ref_a (a frame), ref_b (b frame), kp, kd, target 1 soft row
    kind PLANE_CONTACT: a sphere of radius radius_a (0: a point) about anchor_a (a frame)
                        against the plane {x : normal . x = plane_z} (normal: world,
                        default +z), mu                                         3 rows
    kind SPHERE_CONTACT: spheres about anchor_a (a frame) and anchor_b (b frame, or a
                        world point) of radii radius_a, radius_b; mu             3 rows
    """

    kind: int
    a: Tuple[int, int]
    b: Optional[Tuple[int, int]] = None
    anchor_a: np.ndarray = field(default_factory=lambda: np.zeros(3))
    anchor_b: np.ndarray = field(default_factory=lambda: np.zeros(3))
    axis_a: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    axis_b: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    ref_a: np.ndarray = field(default_factory=lambda: np.array([0.0, 1.0, 0.0]))
    ref_b: np.ndarray = field(default_factory=lambda: np.array([0.0, 1.0, 0.0]))
    kp: float = 0.0
    kd: float = 0.0
    target: float = 0.0
    plane_z: float = 0.0
    mu: float = 0.0
    normal: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, 1.0]))
    radius_a: float = 0.0
    radius_b: float = 0.0


@dataclass
class Scene:
    subs: list
    ifs: list


@dataclass
class Options:
    """Per-run settings shared by both implementations (each parses them itself)."""

    h: float = 1e-3
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.81)
    baumgarte: float = 0.2
    beta_mode: str = "trace"      # "trace": beta_i = Tr A_i / Tr(J_i^T J_i); "fixed": rho
    rho: float = 1e3
    warm: str = "prev"            # "cold" or "prev" (previous step's lambda and z)
    stop: str = "primal"          # "primal": r_p <= tol_primal; "theta": theta < theta_th
    tol_primal: float = 1e-6      # <= 0 runs exactly max_iters iterations
    theta_th: float = 1e-12
    max_iters: int = 1000
    solver: str = "admm"          # "admm" (the method) or "pj" (Projected Jacobi, the paper's
                                  # comparison solver: always exactly max_iters iterations)
    pj_omega: float = 1.0         # Projected Jacobi's relaxation factor


@dataclass
class Problem:
    scenes: List[Scene]
    options: Options
    name: str = ""


# ----------------------------------------------------------------------------------------
# small rotation helpers (input construction only)

def _quat_from_rotvec(r: np.ndarray) -> np.ndarray:
    th = float(np.linalg.norm(r))
    if th < 1e-300:
        return np.array([1.0, 0.0, 0.0, 0.0])
    a = np.asarray(r, dtype=np.float64) / th
    return np.concatenate([[np.cos(th / 2)], np.sin(th / 2) * a])


def _quat_mul(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    pw, px, py, pz = p
    qw, qx, qy, qz = q
    return np.array([
        pw * qw - px * qx - py * qy - pz * qz,
        pw * qx + px * qw + py * qz - pz * qy,
        pw * qy - px * qz + py * qw + pz * qx,
        pw * qz + px * qy - py * qx + pz * qw,
    ])


def _quat_to_mat(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def box_inertia(m: float, a: float, b: float, c: float) -> np.ndarray:
    """Principal inertia of a solid box with edges a (x), b (y), c (z)."""
    return np.array([m * (b * b + c * c) / 12.0, m * (a * a + c * c) / 12.0,
                     m * (a * a + b * b) / 12.0])


# ----------------------------------------------------------------------------------------
# Serial chain of 8 rigid links (shaped like the cable of Sec. IV-A): the 3D chain workload


def chain(seed: int = 0, n_links: int = 8, links_per_sub: int = 2, pinned: bool = True,
          gravity: bool = True, angle: float = 0.5, rho: Optional[float] = 1e3,
          h: float = 1e-3, max_iters: int = 100, tol_primal: float = -1.0,
          warm: str = "prev") -> Problem:
    """8 boxes 0.1 x 0.02 x 0.02 m, density 1000, ball joints at the box ends.

    The first link's -x end is pinned to the world origin (a one-sided ball joint).  The
    chain is split into subsystems of ``links_per_sub`` consecutive links: joints inside a
    subsystem are intra-subsystem constraints (|S_j| = 1), joints between subsystems are
    coupling interfaces (|S_j| = 2).  Initial joint rotation vectors are uniform in
    [-angle, angle]^3, composed along the chain; all velocities start at zero.
    """
    rng = np.random.default_rng(seed)
    L, wdt = 0.1, 0.02
    m = L * wdt * wdt * 1000.0
    I = box_inertia(m, L, wdt, wdt)
    half = np.array([L / 2, 0.0, 0.0])
    rv = rng.uniform(-angle, angle, size=(n_links, 3))
    bodies: List[Body] = []
    q = np.array([1.0, 0.0, 0.0, 0.0])
    end = np.zeros(3)
    for k in range(n_links):
        q = _quat_mul(q, _quat_from_rotvec(rv[k]))
        q = q / np.linalg.norm(q)
        R = _quat_to_mat(q)
        c = end + R @ half
        bodies.append(Body(m, I.copy(), c, q.copy(), np.zeros(3), np.zeros(3)))
        end = c + R @ half
    assert n_links % links_per_sub == 0
    n_sub = n_links // links_per_sub
    subs = [RigidSub(bodies[s * links_per_sub:(s + 1) * links_per_sub]) for s in range(n_sub)]

    def ref(k):
        return (k // links_per_sub, k % links_per_sub)

    ifs = []
    if pinned:
        ifs.append(JointIf(BALL, a=ref(0), b=None, anchor_a=-half, anchor_b=np.zeros(3)))
    for k in range(1, n_links):
        ifs.append(JointIf(BALL, a=ref(k - 1), b=ref(k), anchor_a=half.copy(), anchor_b=-half))
    opts = Options(h=h, gravity=(0.0, 0.0, -9.81) if gravity else (0.0, 0.0, 0.0),
                   beta_mode="fixed" if rho is not None else "trace",
                   rho=rho if rho is not None else 0.0, warm=warm,
                   tol_primal=tol_primal, max_iters=max_iters)
    return Problem([Scene(subs, ifs)], opts, name="chain8")


# ----------------------------------------------------------------------------------------
# Legged robots with point-foot contacts (articulated-with-contact workload)


def _rot_axis(axis: np.ndarray, ang: float) -> np.ndarray:
    return _quat_from_rotvec(np.asarray(axis, dtype=np.float64) * ang)


def legged_robot(rng: np.random.Generator, origin_xy=(0.0, 0.0), kp: float = 50.0,
                 kd: float = 1.0, mu: float = 0.8, offset: float = 0.2,
                 drop=(0.3, 0.5)) -> Scene:
    """A floating trunk plus 4 legs of 3 revolute joints (hip roll x, hip pitch y, knee y).

    One subsystem for the trunk (6 DOF) and one per leg (3 links, 18 DOF).  The hip-roll
    joint couples trunk and leg (|S_j| = 2); hip pitch and knee are intra-leg.  Every joint
    has a PD drive (soft row, Sec. II-A) towards its initial offset, drawn uniform in
    [-offset, offset]; each foot is a point contact with the plane z = 0.  The trunk starts
    level, with its lowest foot at a height uniform in ``drop`` above the plane.
    """
    rho = 1000.0
    tx, ty, tz = 0.3, 0.2, 0.08
    mt = tx * ty * tz * rho
    trunk = Body(mt, box_inertia(mt, tx, ty, tz), np.zeros(3), np.array([1.0, 0, 0, 0]),
                 np.zeros(3), np.zeros(3))
    lens = [0.05, 0.15, 0.15]
    lw = 0.04
    hips = [np.array([sx * 0.12, sy * 0.07, -tz / 2]) for sx in (1, -1) for sy in (1, -1)]
    ex, ey = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    refz = np.array([0.0, 0.0, 1.0])
    legs = []
    feet_world = []
    offsets = rng.uniform(-offset, offset, size=(4, 3))
    for lg in range(4):
        links = []
        q_par = trunk.q
        p_par = trunk.p
        anchor_par = hips[lg]
        axes = [ex, ey, ey]
        for k in range(3):
            qk = _quat_mul(q_par, _rot_axis(axes[k], offsets[lg, k]))
            Rk = _quat_to_mat(qk)
            joint_w = p_par + _quat_to_mat(q_par) @ anchor_par
            top = np.array([0.0, 0.0, lens[k] / 2])
            ck = joint_w - Rk @ top
            mk = lw * lw * lens[k] * rho
            links.append(Body(mk, box_inertia(mk, lw, lw, lens[k]), ck, qk, np.zeros(3),
                              np.zeros(3)))
            q_par, p_par, anchor_par = qk, ck, -top
        foot = np.array([0.0, 0.0, -lens[2] / 2])
        feet_world.append(links[2].p + _quat_to_mat(links[2].q) @ foot)
        legs.append(links)
    H = rng.uniform(*drop)
    zmin = min(f[2] for f in feet_world)
    shift = np.array([origin_xy[0], origin_xy[1], H - zmin])
    trunk.p = trunk.p + shift
    for links in legs:
        for b in links:
            b.p = b.p + shift
    subs = [RigidSub([trunk])] + [RigidSub(links) for links in legs]
    ifs = []
    for lg in range(4):
        s = lg + 1
        parents = [(0, 0), (s, 0), (s, 1)]
        children = [(s, 0), (s, 1), (s, 2)]
        axes = [ex, ey, ey]
        anchors_a = [hips[lg], np.array([0, 0, -lens[0] / 2]), np.array([0, 0, -lens[1] / 2])]
        for k in range(3):
            top = np.array([0.0, 0.0, lens[k] / 2])
            ax = axes[k]
            rf = refz if k == 0 else ex
            ifs.append(JointIf(REVOLUTE, a=parents[k], b=children[k], anchor_a=anchors_a[k],
                               anchor_b=top, axis_a=ax.copy(), axis_b=ax.copy(),
                               ref_a=rf.copy(), ref_b=rf.copy()))
            ifs.append(JointIf(ANGLE_PD, a=parents[k], b=children[k], axis_a=ax.copy(),
                               axis_b=ax.copy(), ref_a=rf.copy(), ref_b=rf.copy(), kp=kp,
                               kd=kd, target=float(offsets[lg, k])))
        ifs.append(JointIf(PLANE_CONTACT, a=(s, 2), anchor_a=np.array([0, 0, -lens[2] / 2]),
                           plane_z=0.0, mu=mu))
    return Scene(subs, ifs)


def robots(seed: int = 0, n_robots: int = 64, h: float = 2e-3, tol_primal: float = 1e-6,
           max_iters: int = 1000, warm: str = "prev", **kw) -> Problem:
    """``n_robots`` independent legged robots, one scene each, on a 1 m grid."""
    rng = np.random.default_rng(seed)
    side = int(np.ceil(np.sqrt(max(n_robots, 1))))
    scenes = [legged_robot(rng, origin_xy=(float(r % side), float(r // side)), **kw)
              for r in range(n_robots)]
    opts = Options(h=h, beta_mode="trace", warm=warm, tol_primal=tol_primal,
                   max_iters=max_iters)
    return Problem(scenes, opts, name=f"robots{n_robots}")


# ----------------------------------------------------------------------------------------
# Generic SPD blocks coupled by random rows (exercises every projection type and |S_j|)


def generic_scene(rng: np.random.Generator, n_sub: int = 4, n_range=(1, 12),
                  types: Sequence[int] = (EQUALITY, HARD, SOFT, CONTACT),
                  extra: int = 2, max_sides: int = 3, density: float = 1.0) -> Scene:
    """Random SPD blocks and a random constraint graph.

    Blocks: A = G G^T / n + diag(U[0.5, 2]) scaled by a per-block mass in [0.1, 10].
    Constraints: a random spanning tree (|S_j| = 2), ``extra`` further constraints on 1..
    ``max_sides`` distinct subsystems, and one intra constraint (|S_j| = 1) per block.
    Rows per constraint: 1..3 (contact: 3).  J entries N(0, 1) with the given density.
    """
    subs = []
    for _ in range(n_sub):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        G = rng.standard_normal((n, n))
        mass = 10.0 ** rng.uniform(-1, 1)
        A = mass * (G @ G.T / n + np.diag(rng.uniform(0.5, 2.0, n)))
        b = mass * rng.standard_normal(n)
        subs.append(GenericSub(A, b))
    edges: List[List[int]] = []
    for i in range(1, n_sub):
        edges.append([int(rng.integers(0, i)), i])
    for _ in range(extra):
        ns = int(rng.integers(1, min(max_sides, n_sub) + 1))
        edges.append([int(x) for x in rng.choice(n_sub, size=ns, replace=False)])
    for i in range(n_sub):
        edges.append([i])
    ifs = []
    for sides in edges:
        t = int(types[int(rng.integers(0, len(types)))])
        rows = 3 if t == CONTACT else int(rng.integers(1, 4))
        J = []
        for s in sides:
            M = rng.standard_normal((rows, subs[s].n))
            if density < 1.0:
                M = M * (rng.random(M.shape) < density)
            J.append(M)
        e = rng.standard_normal(rows)
        k = float(10.0 ** rng.uniform(0, 2))
        alpha = float(10.0 ** rng.uniform(-3, -1))
        mu = float(rng.uniform(0.2, 1.0))
        ifs.append(RowsIf(t, list(sides), J, e, k=k, alpha=alpha, mu=mu))
    return Scene(subs, ifs)


def generic(seed: int = 0, n_scenes: int = 4, tol_primal: float = -1.0, max_iters: int = 50,
            beta_mode: str = "trace", rho: float = 1.0, warm: str = "cold", **kw) -> Problem:
    rng = np.random.default_rng(seed)
    scenes = [generic_scene(rng, **kw) for _ in range(n_scenes)]
    opts = Options(h=1e-3, gravity=(0.0, 0.0, 0.0), beta_mode=beta_mode, rho=rho,
                   warm=warm, tol_primal=tol_primal, max_iters=max_iters)
    return Problem(scenes, opts, name="generic")


def hanging_scene(rng: np.random.Generator, n_blocks: int = 2, dims=(2, 2, 3),
                  with_body: bool = True, drop: float = 0.004) -> Scene:
    """Spring blocks pinned at two top nodes, one above the plane z = 0 with node contacts,
    and a rigid box hung from the first block by a ball joint (mixed rigid / linear scene)."""
    subs, ifs = [], []
    for b in range(n_blocks):
        blk = lattice_block(dims=dims, spacing=0.02, origin=(0.1 * b, 0.0, drop), k=400.0,
                            v=rng.uniform(-0.05, 0.05, 3))
        subs.append(blk)
    nn = subs[0].nodes
    top = nn - dims[0] * dims[1]
    for b in range(1, n_blocks):
        X = subs[b].X0
        ifs.append(JointIf(BALL, a=(b, top), b=None, anchor_b=X[3 * top:3 * top + 3].copy()))
        ifs.append(JointIf(BALL, a=(b, top + 1), b=None,
                           anchor_b=X[3 * (top + 1):3 * (top + 1) + 3].copy()))
    for k in range(dims[0] * dims[1]):        # the bottom layer of block 0 touches the plane
        ifs.append(JointIf(PLANE_CONTACT, a=(0, k), plane_z=0.0,
                           mu=float(rng.uniform(0.3, 1.0))))
    if with_body:
        X = subs[-1].X0
        pin = X[0:3]
        box = Body(0.05, box_inertia(0.05, 0.02, 0.02, 0.02), pin + np.array([0.0, 0.0, -0.03]),
                   np.array([1.0, 0.0, 0.0, 0.0]), np.zeros(3), np.zeros(3))
        subs.append(RigidSub([box]))
        ifs.append(JointIf(BALL, a=(len(subs) - 1, 0), b=(n_blocks - 1, 0),
                           anchor_a=np.array([0.0, 0.0, 0.03])))
    return Scene(subs, ifs)


# ----------------------------------------------------------------------------------------
# Linear tetrahedral FEM beam cut into slabs (rigid-deformable workload)

def lame(E: float, nu: float):
    """Lame parameters (lambda, mu) of an isotropic material."""
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def tet_stiffness(X: np.ndarray, tets: np.ndarray, E: float, nu: float):
    """Element stiffness matrices (T x 12 x 12) and volumes of linear (constant-strain)
    tetrahedra: K_e = V B^T C B with the strain-displacement matrix B of the barycentric
    shape functions and the isotropic elasticity matrix C in Voigt order
    (xx, yy, zz, 2yz, 2xz, 2xy)."""
    P = X[tets]                                    # T x 4 x 3
    Dm = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    vol = np.abs(np.linalg.det(Dm)) / 6.0
    Gi = np.linalg.inv(Dm)                         # rows: gradients of N1..N3
    grads = np.concatenate([-Gi.sum(axis=1, keepdims=True), Gi], axis=1)   # T x 4 x 3
    T = tets.shape[0]
    B = np.zeros((T, 6, 12))
    for a in range(4):
        bx, by, bz = grads[:, a, 0], grads[:, a, 1], grads[:, a, 2]
        c = 3 * a
        B[:, 0, c] = bx
        B[:, 1, c + 1] = by
        B[:, 2, c + 2] = bz
        B[:, 3, c + 1] = bz
        B[:, 3, c + 2] = by
        B[:, 4, c] = bz
        B[:, 4, c + 2] = bx
        B[:, 5, c] = by
        B[:, 5, c + 1] = bx
    lam, mu = lame(E, nu)
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2.0 * mu
    C[np.arange(3, 6), np.arange(3, 6)] = mu
    Ke = vol[:, None, None] * np.einsum("tji,jk,tkl->til", B, C, B)
    return Ke, vol


def kuhn_tets(cell_corners: np.ndarray) -> np.ndarray:
    """Split hexahedral cells (C x 8 corner ids, corner index = 4 i + 2 j + k for offsets
    (i, j, k) in {0, 1}^3) into 6 tetrahedra each around the 000-111 diagonal (Kuhn); the
    split is the same in every cell, so neighbouring cells share conforming faces."""
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        off = np.zeros(3, int)
        path = [0]
        for axis in perm:
            off[axis] = 1
            path.append(4 * off[0] + 2 * off[1] + off[2])
        tets.append(cell_corners[:, path])
    return np.concatenate(tets, axis=0)


def fem_slab(planes_x: np.ndarray, ny: int, nz: int, width: float, height: float,
             E: float, nu: float, rho: float, z0: float = 0.0):
    """One slab of the beam: node planes at x = planes_x, an ny x nz grid per plane over
    [0, width] x [z0, z0 + height].  Nodes are numbered plane-fastest,
    node = (iy nz + iz) k + p, which keeps the stiffness envelope narrow (slabs are only a
    few planes thick).  Returns the LinearSub (lumped mass, stiffness triplets) and the
    node index function."""
    k = len(planes_x)
    ys = np.linspace(0.0, width, ny)
    zs = np.linspace(z0, z0 + height, nz)

    def nid(p, iy, iz):
        return (iy * nz + iz) * k + p

    X = np.zeros((k * ny * nz, 3))
    for p in range(k):
        for iy in range(ny):
            for iz in range(nz):
                X[nid(p, iy, iz)] = (planes_x[p], ys[iy], zs[iz])
    cells = []
    for p in range(k - 1):
        for iy in range(ny - 1):
            for iz in range(nz - 1):
                cells.append([nid(p + i, iy + j, iz + l) for i in (0, 1) for j in (0, 1)
                              for l in (0, 1)])
    tets = kuhn_tets(np.array(cells, dtype=int))
    Ke, vol = tet_stiffness(X, tets, E, nu)
    dof = (3 * tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
    Ki = np.repeat(dof, 12, axis=1).ravel()
    Kj = np.tile(dof, (1, 12)).ravel()
    Kv = Ke.reshape(-1)
    # sum duplicate entries
    key = Ki.astype(np.int64) * (3 * X.shape[0]) + Kj
    uk, inv = np.unique(key, return_inverse=True)
    vals = np.zeros(uk.shape[0])
    np.add.at(vals, inv, Kv)
    Ki, Kj = (uk // (3 * X.shape[0])).astype(np.int64), (uk % (3 * X.shape[0])).astype(np.int64)
    mass = np.zeros(X.shape[0])
    np.add.at(mass, tets.ravel(), np.repeat(rho * vol / 4.0, 4))
    nn = X.shape[0]
    sub = LinearSub(mass, Ki, Kj, vals, np.zeros(3 * nn), X.ravel().copy(), X.ravel().copy(),
                    np.zeros(3 * nn), tets=tets.astype(np.int64), Ke=Ke)
    return sub, nid, tets


def gripper(anchor_w: np.ndarray, reach: float = 0.12, rho: float = 1000.0):
    """A 7-R arm in maximal coordinates (one subsystem of 7 boxes): a base turning about z
    on a world pivot above ``anchor_w``, a vertical chain of 4 links turning about y, and
    two paddles turning about x at the end, hanging down to ``anchor_w``.  Returns the
    subsystem, its joint and PD interfaces (joint i joins body i-1, or the world, to body
    i), and the paddles' body indices."""
    lw = 0.012
    lens = [0.02, reach / 4, reach / 4, reach / 4, reach / 4 - 0.02]
    top = np.asarray(anchor_w, float) + np.array([0.0, 0.0, sum(lens) + 0.02])
    bodies, joints = [], []
    ez, ey, ex = np.array([0.0, 0, 1]), np.array([0.0, 1, 0]), np.array([1.0, 0, 0])
    q0 = np.array([1.0, 0, 0, 0])
    z = top[2]
    axes = [ez, ey, ey, ey, ey]
    for k, L in enumerate(lens):
        c = np.array([top[0], top[1], z - L / 2])
        m = lw * lw * L * rho
        bodies.append(Body(m, box_inertia(m, lw, lw, L), c, q0.copy(), np.zeros(3), np.zeros(3)))
        joint_w = np.array([top[0], top[1], z])
        joints.append((k - 1, k, joint_w, axes[k]))
        z -= L
    # paddles: thin plates hanging either side of the anchor, hinged about x at the wrist
    pl = 0.02
    wrist = np.array([top[0], top[1], z])
    paddles = []
    for side in (-1, 1):
        c = wrist + np.array([0.0, side * 0.01, -pl / 2])
        m = 0.004 * 0.02 * pl * rho
        bodies.append(Body(m, box_inertia(m, 0.02, 0.004, pl), c, q0.copy(), np.zeros(3),
                           np.zeros(3)))
        joints.append((len(lens) - 1, len(bodies) - 1, wrist + np.array([0.0, side * 0.01, 0.0]), ex))
        paddles.append(len(bodies) - 1)
    return bodies, joints, paddles


def _arm(gs: int, anchor_w: np.ndarray, kp: float, kd: float, base_drive=None):
    """The 7-R arm stand-in of ``gripper`` as one rigid subsystem (index ``gs``) whose
    paddles hang down to ``anchor_w``: the subsystem, its revolute joints and PD drives
    (holding the initial pose), and the first paddle's body index.  ``base_drive`` =
    (kp, kd, angle) adds a PD drive of the base about the vertical that turns it by
    ``angle`` from its initial pose."""
    bodies, joints, paddles = gripper(anchor_w)
    ifs = []
    ex = np.array([1.0, 0, 0])
    for (pa, ch, jw, ax) in joints:
        ref = np.array([0.0, 0, 1.0]) if abs(ax[2]) < 0.5 else ex
        bc = bodies[ch]
        if pa < 0:
            ifs.append(JointIf(REVOLUTE, a=(gs, ch), b=None, anchor_a=jw - bc.p, anchor_b=jw.copy(),
                               axis_a=ax.copy(), axis_b=ax.copy(), ref_a=ref.copy(),
                               ref_b=ref.copy()))
            if base_drive is not None:
                bkp, bkd, angle = base_drive
                # the angle of the world's ref from the base's ref about the base's axis is
                # minus the base's turn
                ifs.append(JointIf(ANGLE_PD, a=(gs, ch), b=None, axis_a=ax.copy(),
                                   axis_b=ax.copy(), ref_a=ref.copy(), ref_b=ref.copy(),
                                   kp=bkp, kd=bkd, target=-angle))
            continue
        bp = bodies[pa]
        ifs.append(JointIf(REVOLUTE, a=(gs, pa), b=(gs, ch), anchor_a=jw - bp.p,
                           anchor_b=jw - bc.p, axis_a=ax.copy(), axis_b=ax.copy(),
                           ref_a=ref.copy(), ref_b=ref.copy()))
        ifs.append(JointIf(ANGLE_PD, a=(gs, pa), b=(gs, ch), axis_a=ax.copy(), axis_b=ax.copy(),
                           ref_a=ref.copy(), ref_b=ref.copy(), kp=kp, kd=kd, target=0.0))
    return RigidSub(bodies), ifs, paddles[0]


def cable(seed: int = 0, segments: int = 640, per_sub: int = 4, seg_len: float = 0.01,
          radius: float = 0.005, rho: float = 1200.0, bend_kp: float = 2e-3,
          twist_kp: float = 1e-3, damping: float = 2e-5, mu: float = 0.5, arms: bool = True,
          h: float = 1e-3, tol_primal: float = 1e-6, max_iters: int = 1000,
          warm: str = "prev") -> Problem:
    """A cable held by two arms, shaped like the paper's cable scene (Sec. IV-A: a Cosserat
    cable handled by two manipulators, 162 subsystems): ``segments`` rigid capsule segments
    along x, lying on the plane z = 0, joined end to end by ball joints, with the rod's
    bending (two axes normal to the segment) and twist (about it) as PD soft rows holding the
    straight rest shape -- a discrete elastic rod in maximal coordinates.  ``per_sub``
    consecutive segments form a subsystem; each segment has a speculative contact with the
    plane (friction mu).  With ``arms`` two 7-R arm stand-ins (as in the FEM beam scene) hold
    the cable's ends by ball joints between a paddle and the end segment.  The seed draws
    small initial lateral velocities of the segments (up to 2 cm/s).  The arms' and the
    cable's models are stand-ins: the paper's manipulator and cable models are not public."""
    rng = np.random.default_rng(seed)
    m = np.pi * radius ** 2 * seg_len * rho
    I = np.array([0.5 * m * radius ** 2, m * (3 * radius ** 2 + seg_len ** 2) / 12.0,
                  m * (3 * radius ** 2 + seg_len ** 2) / 12.0])
    q0 = np.array([1.0, 0.0, 0.0, 0.0])
    bodies = []
    for k in range(segments):
        c = np.array([(k + 0.5) * seg_len, 0.0, radius])
        v = np.array([0.0, rng.uniform(-0.02, 0.02), rng.uniform(0.0, 0.02)])
        bodies.append(Body(m, I.copy(), c, q0.copy(), v, np.zeros(3)))
    if segments % per_sub:
        raise ValueError("segments must be a multiple of per_sub")
    nsub = segments // per_sub
    subs = [RigidSub(bodies[s * per_sub:(s + 1) * per_sub]) for s in range(nsub)]

    def ref(k):
        return (k // per_sub, k % per_sub)

    ex, ey, ez = np.eye(3)
    half = np.array([seg_len / 2, 0.0, 0.0])
    ifs = []
    for k in range(1, segments):
        a, b = ref(k - 1), ref(k)
        ifs.append(JointIf(BALL, a=a, b=b, anchor_a=half.copy(), anchor_b=-half))
        for axis, rf, kp in ((ey, ex, bend_kp), (ez, ex, bend_kp), (ex, ey, twist_kp)):
            ifs.append(JointIf(ANGLE_PD, a=a, b=b, axis_a=axis.copy(), axis_b=axis.copy(),
                               ref_a=rf.copy(), ref_b=rf.copy(), kp=kp, kd=damping / seg_len,
                               target=0.0))
    for k in range(segments):
        ifs.append(JointIf(PLANE_CONTACT, a=ref(k), anchor_a=np.array([0.0, 0.0, -radius]),
                           plane_z=0.0, mu=mu))
    if arms:
        for end, k in ((0, 0), (1, segments - 1)):
            gs = len(subs)
            tip = bodies[k].p + (half if end else -half)
            arm, arm_ifs, paddle = _arm(gs, tip, kp=50.0, kd=1.0)
            subs.append(arm)
            ifs.extend(arm_ifs)
            pb = arm.bodies[paddle]
            ifs.append(JointIf(BALL, a=(gs, paddle), b=ref(k), anchor_a=tip - pb.p,
                               anchor_b=(half if end else -half)))
    opts = Options(h=h, beta_mode="trace", warm=warm, tol_primal=tol_primal, max_iters=max_iters)
    return Problem([Scene(subs, ifs)], opts, name=f"cable{segments}")


def fem_beam(seed: int = 0, ny: int = 10, nz: int = 10, planes: int = 137, slabs: int = 64,
             length: float = 0.5, width: float = 0.05, height: float = 0.05, E: float = 1e5,
             nu: float = 0.45, rho: float = 1000.0, mu: float = 0.5, drop: float = 0.002,
             with_gripper: bool = True, h: float = 1e-3, tol_primal: float = 1e-6,
             max_iters: int = 1000, warm: str = "prev", kp: float = 50.0, kd: float = 1.0,
             vary: bool = False, corotational: bool = False):
    """A linear-elastic tetrahedral beam (planes x ny x nz nodes, Kuhn split of every grid
    cell) cut into ``slabs`` subsystems: slab g holds 4 node planes when g is a multiple of
    8 and 3 otherwise, neighbouring slabs duplicate the cut plane, and each duplicated node
    pair is a node-node ball interface (equality, 3 rows).  Every node of the bottom face
    has a speculative contact with the plane z = 0 (friction mu); the beam starts ``drop``
    above it.  With the gripper, a 7-R arm (one rigid subsystem, PD drives holding its
    pose) holds the beam's x = 0 end by ball joints between its two paddles and the
    nearest side-face nodes.  With ``vary`` the seed draws a member of the workload's
    distribution: drop height U[1, 4] mm, friction U[0.3, 0.7], Young's modulus E 2^U[-1/2, 1/2]
    and PD gains kp 2^U[-1/2, 1/2]; otherwise the beam is the same for every seed.  With
    ``corotational`` the slabs are co-rotational (the paper's beam model, Sec. IV-A): their
    stiffness and elastic force come from the rotated elements at every step."""
    rng = np.random.default_rng(seed)
    if vary:
        drop = float(rng.uniform(0.001, 0.004))
        mu = float(rng.uniform(0.3, 0.7))
        E = float(E * 2.0 ** rng.uniform(-0.5, 0.5))
        kp = float(kp * 2.0 ** rng.uniform(-0.5, 0.5))
    ks = [4 if g % 8 == 0 else 3 for g in range(slabs)]
    if sum(k - 1 for k in ks) != planes - 1:
        raise ValueError("slab plane counts do not tile the beam")
    xs = np.linspace(0.0, length, planes)
    subs, ifs, nids = [], [], []
    p0 = 0
    for g in range(slabs):
        sub, nid, _ = fem_slab(xs[p0:p0 + ks[g]], ny, nz, width, height, E, nu, rho, z0=drop)
        sub.corot = corotational
        subs.append(sub)
        nids.append(nid)
        if g > 0:
            kp_prev = ks[g - 1]
            for iy in range(ny):
                for iz in range(nz):
                    ifs.append(JointIf(BALL, a=(g - 1, nids[g - 1](kp_prev - 1, iy, iz)),
                                       b=(g, nid(0, iy, iz))))
        for p in range(ks[g]):
            for iy in range(ny):
                ifs.append(JointIf(PLANE_CONTACT, a=(g, nid(p, iy, 0)), plane_z=0.0, mu=mu))
        p0 += ks[g] - 1
    if with_gripper:
        # hold the x = 0 end by its side faces, half-way up
        iz = nz // 2
        grip = [(0, nids[0](0, 0, iz)), (0, nids[0](1, 0, iz)),
                (0, nids[0](0, ny - 1, iz)), (0, nids[0](1, ny - 1, iz))]
        Xn = subs[0].X0.reshape(-1, 3)
        centre = 0.5 * (Xn[grip[0][1]] + Xn[grip[2][1]])
        bodies, joints, paddles = gripper(centre + np.array([0.0, 0.0, 0.015]))
        # paddles move to the side faces (y = -0.002 and y = width + 0.002)
        for pb, side_y in zip(paddles, (-0.002, width + 0.002)):
            bodies[pb].p = np.array([Xn[grip[0][1]][0] + 0.002, side_y, Xn[grip[0][1]][2]])
        gs = len(subs)
        subs.append(RigidSub(bodies))
        ex = np.array([1.0, 0, 0])
        for (pa, ch, jw, ax) in joints:
            ref = np.array([0.0, 0, 1.0]) if abs(ax[2]) < 0.5 else ex
            bc = bodies[ch]
            anchor_b = jw - bc.p
            if pa < 0:
                ifs.append(JointIf(REVOLUTE, a=(gs, ch), b=None, anchor_a=anchor_b,
                                   anchor_b=jw.copy(), axis_a=ax.copy(), axis_b=ax.copy(),
                                   ref_a=ref.copy(), ref_b=ref.copy()))
                continue
            bp = bodies[pa]
            ifs.append(JointIf(REVOLUTE, a=(gs, pa), b=(gs, ch), anchor_a=jw - bp.p,
                               anchor_b=anchor_b, axis_a=ax.copy(), axis_b=ax.copy(),
                               ref_a=ref.copy(), ref_b=ref.copy()))
            ifs.append(JointIf(ANGLE_PD, a=(gs, pa), b=(gs, ch), axis_a=ax.copy(),
                               axis_b=ax.copy(), ref_a=ref.copy(), ref_b=ref.copy(), kp=kp,
                               kd=kd, target=0.0))
        for j, (sg_, node) in enumerate(grip):
            pb = paddles[0] if j < 2 else paddles[1]
            ifs.append(JointIf(BALL, a=(gs, pb), b=(sg_, node), anchor_a=Xn[node] - bodies[pb].p))
    opts = Options(h=h, beta_mode="trace", warm=warm, tol_primal=tol_primal, max_iters=max_iters)
    return Problem([Scene(subs, ifs)], opts, name=f"fem_beam{slabs}")


def stir(seed: int = 0, n_side: int = 6, layers: int = 6, radius: float = 0.01,
         mass: float = 0.004, gap: float = 5e-4, mu: float = 0.5, tool_radius: float = 0.008,
         tool_offset: float = 0.03, sweep: float = 1.5, drive=(0.02, 0.002),
         arm: bool = True, neighbor: float = 1.5, h: float = 1e-2, tol_primal: float = 1e-6,
         max_iters: int = 1000, warm: str = "prev") -> Problem:
    """Granular stirring, shaped like the paper's stir scene (Sec. IV-A: 216 spheres of
    radius 1 cm and 4 g in a box, stirred by an arm's end effector; each sphere and the arm
    one subsystem, 217 in all; h = 10 ms as in the paper's experiments).

    ``n_side`` x ``n_side`` x ``layers`` spheres (one rigid subsystem each) start on a
    lattice of spacing 2 radius + gap above the floor z = 0, inside four walls, with seeded
    jitter (at most 0.2 gap per axis, so no two overlap), random orientations and small
    random velocities (up to 1 cm/s).  Contacts (friction mu), all speculative (an open one
    projects to zero): sphere-sphere for every pair whose centres start closer than
    ``neighbor`` diameters; the floor for the bottom layer and the facing wall for every
    sphere on the lattice's boundary (plane contacts with the sphere's radius).  With
    ``arm``, the 7-R arm stand-in (as in the cable and beam scenes) hangs from a world
    pivot ``tool_offset`` beside the box's axis and carries a tool sphere (``tool_radius``)
    in the top layer's central hollow; a PD drive (``drive`` = kp, kd) turns its base by
    ``sweep`` radians, sweeping the tool through the top layers, and the tool has a
    speculative contact with every sphere of the two top layers within reach of its
    circle.  The arm's model is a stand-in: the paper's manipulator model is not public."""
    rng = np.random.default_rng(seed)
    spacing = 2.0 * radius + gap
    I = 0.4 * mass * radius * radius
    half = 0.5 * (n_side - 1) * spacing
    centres, bodies = [], []
    for k in range(layers):
        for iy in range(n_side):
            for ix in range(n_side):
                c = np.array([ix * spacing - half, iy * spacing - half,
                              radius + 0.5 * gap + k * spacing])
                c = c + rng.uniform(-0.2 * gap, 0.2 * gap, 3)
                q = _random_rotation(rng)
                v = rng.uniform(-0.01, 0.01, 3)
                centres.append(c)
                bodies.append(Body(mass, np.array([I, I, I]), c, q, v, np.zeros(3)))
    subs = [RigidSub([b]) for b in bodies]
    N = len(bodies)
    P = np.array(centres)
    ifs = []
    cut = neighbor * 2.0 * radius
    for a in range(N):
        d = np.linalg.norm(P[a + 1:] - P[a], axis=1)
        for b in np.nonzero(d < cut)[0] + a + 1:
            ifs.append(JointIf(SPHERE_CONTACT, a=(a, 0), b=(int(b), 0), radius_a=radius,
                               radius_b=radius, mu=mu))
    wall = half + radius + gap
    for a in range(N):
        k, rem = divmod(a, n_side * n_side)
        iy, ix = divmod(rem, n_side)
        planes = []
        if k == 0:
            planes.append((np.array([0.0, 0.0, 1.0]), 0.0))
        if ix == 0:
            planes.append((np.array([1.0, 0.0, 0.0]), -wall))
        if ix == n_side - 1:
            planes.append((np.array([-1.0, 0.0, 0.0]), -wall))
        if iy == 0:
            planes.append((np.array([0.0, 1.0, 0.0]), -wall))
        if iy == n_side - 1:
            planes.append((np.array([0.0, -1.0, 0.0]), -wall))
        for nrm, off in planes:
            ifs.append(JointIf(PLANE_CONTACT, a=(a, 0), radius_a=radius, normal=nrm,
                               plane_z=off, mu=mu))
    if arm:
        ztop = radius + 0.5 * gap + (layers - 1) * spacing
        reach = radius + tool_radius + gap
        if n_side % 2 == 0:       # the central hollow between four top spheres
            dz = np.sqrt(max(reach * reach - 0.5 * spacing * spacing, 0.0))
        else:                     # on top of the central sphere
            dz = reach
        tool = np.array([0.0, 0.0, ztop + dz])
        axis_xy = np.array([-tool_offset, 0.0])
        gs = len(subs)
        arm_sub, arm_ifs, paddle = _arm(gs, np.array([axis_xy[0], 0.0, tool[2] + 0.02]),
                                        kp=50.0, kd=1.0,
                                        base_drive=(drive[0], drive[1], sweep))
        subs.append(arm_sub)
        ifs.extend(arm_ifs)
        pb = arm_sub.bodies[paddle]
        Rr = np.hypot(*(tool[:2] - axis_xy))
        band = radius + tool_radius + spacing
        for a in range(N):
            if P[a, 2] < ztop - spacing - 0.5 * gap:
                continue
            if abs(np.hypot(*(P[a, :2] - axis_xy)) - Rr) > band:
                continue
            ifs.append(JointIf(SPHERE_CONTACT, a=(gs, paddle), b=(a, 0), anchor_a=tool - pb.p,
                               radius_a=tool_radius, radius_b=radius, mu=mu))
    opts = Options(h=h, beta_mode="trace", warm=warm, tol_primal=tol_primal, max_iters=max_iters)
    return Problem([Scene(subs, ifs)], opts, name=f"stir{N}")


def _random_rotation(rng) -> np.ndarray:
    return _quat_from_rotvec(rng.uniform(-np.pi, np.pi, 3) * 0.3)


def _floating_chain(rng, links: int, L=0.05, w=0.01) -> RigidSub:
    """A straight chain of `links` boxes along a random direction (joined by ball joints at
    their ends, added by the caller)."""
    m = L * w * w * 1000.0
    I = box_inertia(m, L, w, w)
    q = _random_rotation(rng)
    R = _quat_to_mat(q)
    ax = R @ np.array([L, 0.0, 0.0])
    bodies = [Body(m, I.copy(), ax * k, q.copy(), np.zeros(3), np.zeros(3)) for k in range(links)]
    return RigidSub(bodies)


def _point_of(sub, idx, rng):
    """(anchor in the body frame or None for a node, world point) of an attachment site."""
    if isinstance(sub, RigidSub):
        b = sub.bodies[idx]
        anc = np.array([rng.choice([-0.025, 0.025]), 0.0, 0.0])
        return anc, b.p + _quat_to_mat(b.q) @ anc
    return None, sub.x[3 * idx:3 * idx + 3].copy()


def _shift(sub, d):
    if isinstance(sub, RigidSub):
        for b in sub.bodies:
            b.p = b.p + d
    else:
        sub.x = sub.x + np.tile(d, sub.nodes)
        sub.X0 = sub.X0 + np.tile(d, sub.nodes)


def _sites(sub) -> int:
    return len(sub.bodies) if isinstance(sub, RigidSub) else sub.nodes


def batched_scene(rng: np.random.Generator, n_sub=(2, 32), n_range=(6, 240), contacts=(0, 64),
                  mu=(0.3, 1.0)) -> Scene:
    """One scene of the batched workload: U{n_sub} subsystems with DOF log-uniform in
    n_range, half rigid floating chains (6 DOF per link, links joined by ball joints) and half
    spring blocks of 2 x 2 x k nodes (12 DOF per node layer); a random spanning tree of ball
    joints plus floor(N/4) chords, each anchored at points that coincide at t = 0; U{contacts}
    point contacts with the plane z = 0, friction uniform in mu."""
    N = int(rng.integers(n_sub[0], n_sub[1] + 1))
    subs, ifs = [], []
    for i in range(N):
        n_t = float(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))
        if rng.random() < 0.5:
            links = int(np.clip(round(n_t / 6), 1, n_range[1] // 6))
            sub = _floating_chain(rng, links)
            for k in range(1, links):
                ifs.append(JointIf(BALL, a=(i, k - 1), b=(i, k), anchor_a=np.array([0.025, 0, 0]),
                                   anchor_b=np.array([-0.025, 0, 0])))
        else:
            layers = int(np.clip(round(n_t / 12), 1, n_range[1] // 12))
            sub = lattice_block(dims=(2, 2, layers), spacing=0.02, k=400.0)
        subs.append(sub)
        if i > 0:
            parent = int(rng.integers(0, i))
            ip = int(rng.integers(0, _sites(subs[parent])))
            anc_p, P = _point_of(subs[parent], ip, rng)
            ic = int(rng.integers(0, _sites(sub)))
            anc_c, Pc = _point_of(sub, ic, rng)
            _shift(sub, P - Pc)
            ifs.append(JointIf(BALL, a=(i, ic), b=(parent, ip),
                               anchor_a=anc_c if anc_c is not None else np.zeros(3),
                               anchor_b=anc_p if anc_p is not None else np.zeros(3)))
    for _ in range(N // 4):
        a, b = (int(v) for v in rng.choice(N, size=2, replace=False))
        if not isinstance(subs[a], RigidSub):
            a, b = b, a
        if not isinstance(subs[a], RigidSub):
            continue                         # node-node chords would start violated
        ib = int(rng.integers(0, _sites(subs[b])))
        anc_b, P = _point_of(subs[b], ib, rng)
        ia = int(rng.integers(0, _sites(subs[a])))
        body = subs[a].bodies[ia]
        anc_a = _quat_to_mat(body.q).T @ (P - body.p)
        ifs.append(JointIf(BALL, a=(a, ia), b=(b, ib), anchor_a=anc_a,
                           anchor_b=anc_b if anc_b is not None else np.zeros(3)))
    # rest the scene just above the plane, then the contact sites
    zmin = min(min(b.p[2] for b in s.bodies) if isinstance(s, RigidSub) else s.x[2::3].min()
               for s in subs)
    lift = np.array([0.0, 0.0, -zmin + 0.03 + rng.uniform(0.0, 0.01)])
    for s in subs:
        _shift(s, lift)
    for _ in range(int(rng.integers(contacts[0], contacts[1] + 1))):
        i = int(rng.integers(0, N))
        k = int(rng.integers(0, _sites(subs[i])))
        anc = np.array([rng.choice([-0.025, 0.025]), 0.0, 0.0]) if isinstance(subs[i], RigidSub) \
            else np.zeros(3)
        ifs.append(JointIf(PLANE_CONTACT, a=(i, k), anchor_a=anc, plane_z=0.0,
                           mu=float(rng.uniform(*mu))))
    return Scene(subs, ifs)


def batched(seed: int = 0, n_scenes: int = 4096, h: float = 1e-3, tol_primal: float = 1e-6,
            max_iters: int = 1000, **kw) -> Problem:
    """The batched workload: many independent uneven scenes solved in one launch."""
    rng = np.random.default_rng(seed)
    scenes = [batched_scene(rng, **kw) for _ in range(n_scenes)]
    opts = Options(h=h, beta_mode="trace", warm="prev", tol_primal=tol_primal,
                   max_iters=max_iters)
    return Problem(scenes, opts, name=f"batched{n_scenes}")


def problem_sizes(p: Problem) -> dict:
    """Counts of subsystems, DOF, constraints, rows and side-rows (plain bookkeeping)."""
    n_sub = sum(len(s.subs) for s in p.scenes)
    dof = sum(sub.n for s in p.scenes for sub in s.subs)
    n_if = sum(len(s.ifs) for s in p.scenes)
    rows = 0
    side_rows = 0
    for s in p.scenes:
        for itf in s.ifs:
            if isinstance(itf, RowsIf):
                r, ns = itf.rows, len(itf.subs)
            else:
                r = {BALL: 3, REVOLUTE: 5, ANGLE_PD: 1, PLANE_CONTACT: 3,  # noqa
                     SPHERE_CONTACT: 3}[itf.kind]
                ns = 1 if (itf.b is None or itf.b[0] == itf.a[0]) else 2
            rows += r
            side_rows += r * ns
    return dict(scenes=len(p.scenes), subsystems=n_sub, dof=dof, interfaces=n_if, rows=rows,
                side_rows=side_rows)


def merged(problem: Problem) -> Problem:
    """The same scenes with every scene's subsystems merged into one: the full-system ADMM
    that the paper compares against (Sec. IV-B, "FADMM": one factorisation of the whole
    system per step, every constraint its own z-variable), run by the same solver.  Rigid
    scenes become one rigid subsystem (bodies concatenated), generic scenes one
    block-diagonal block; interfaces keep their rows, re-addressed to the merged subsystem.
    Scenes that mix kinds (or hold linear blocks) are rejected."""
    scenes = []
    for sc in problem.scenes:
        kinds = {type(s) for s in sc.subs}
        if kinds == {RigidSub}:
            off = np.cumsum([0] + [len(s.bodies) for s in sc.subs])
            sub = RigidSub([b for s in sc.subs for b in s.bodies])
            ifs = []
            for itf in sc.ifs:
                if not isinstance(itf, JointIf):
                    raise ValueError("explicit rows on rigid subsystems are not merged")
                a = (0, int(off[itf.a[0]] + itf.a[1]))
                b = None if itf.b is None else (0, int(off[itf.b[0]] + itf.b[1]))
                ifs.append(JointIf(**{**itf.__dict__, "a": a, "b": b}))
            scenes.append(Scene([sub], ifs))
        elif kinds == {GenericSub}:
            sizes = [s.n for s in sc.subs]
            off = np.cumsum([0] + sizes)
            N = int(off[-1])
            A = np.zeros((N, N))
            b = np.zeros(N)
            for s, o in zip(sc.subs, off):
                A[o:o + s.n, o:o + s.n] = s.A
                b[o:o + s.n] = s.b
            ifs = []
            for itf in sc.ifs:
                J = np.zeros((itf.rows, N))
                for s, Js in zip(itf.subs, itf.J):
                    J[:, off[s]:off[s] + sizes[s]] += np.asarray(Js)
                ifs.append(RowsIf(itf.type, [0], [J], np.asarray(itf.e).copy(), itf.k,
                                  itf.alpha, itf.mu))
            scenes.append(Scene([GenericSub(A, b)], ifs))
        else:
            raise ValueError("only all-rigid or all-generic scenes are merged")
    return Problem(scenes, problem.options, name=problem.name + "_merged")
