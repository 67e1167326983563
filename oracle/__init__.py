"""Python marshalling for the plain FP64 CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the package's smoke check and the benchmark's
CPU-baseline leg use it.  It shares no code with the CUDA library and never imports it.

``OracleScene`` mirrors one scene of a ``scenegen.Problem``; ``run(problem, steps)`` steps
every scene and returns per-scene results as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_PATH_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

D = C.c_double
PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)
VP = C.c_void_p

# type / source codes, as fixed in oracle.c
T_CODES = {0: 0, 1: 1, 2: 2, 3: 3}


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c with plain gcc (no FMA contraction) into oracle/_build/.  With
    ``openmp`` the same source is built with -fopenmp (the multi-core timing baseline)."""
    path = _LIB_PATH_OMP if openmp else _LIB_PATH
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-shared", "-fPIC",
                               *(["-fopenmp"] if openmp else []), _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, path)
    return path


def lib(openmp: bool = False):
    with _lock:
        if openmp not in _libs:
            L = C.CDLL(build(openmp=openmp))
            sig = {
                "orc_new": (VP, [PD]),
                "orc_add_generic": (C.c_int, [VP, C.c_int, PD, PD]),
                "orc_add_rigid": (C.c_int, [VP, C.c_int, PD]),
                "orc_add_linear": (C.c_int, [VP, C.c_int, PD]),
                "orc_get_node": (None, [VP, C.c_int, C.c_int, PD]),
                "orc_set_node": (None, [VP, C.c_int, C.c_int, PD]),
                "orc_add_rows": (C.c_int, [VP, C.c_int, C.c_int, C.c_int, PI, PD, PD, D, D, D]),
                "orc_add_joint": (C.c_int, [VP, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, PD]),
                "orc_step": (C.c_int, [VP]),
                "orc_assemble": (None, [VP]),
                "orc_set_trace": (None, [VP, PD, C.c_int]),
                "orc_set_pj": (C.c_int, [VP, C.c_int, D]),
                "orc_nsub": (C.c_int, [VP]),
                "orc_ncon": (C.c_int, [VP]),
                "orc_n": (C.c_int, [VP, C.c_int]),
                "orc_rows": (C.c_int, [VP, C.c_int]),
                "orc_nsides": (C.c_int, [VP, C.c_int]),
                "orc_con_sub": (C.c_int, [VP, C.c_int, C.c_int]),
                "orc_beta": (D, [VP, C.c_int]),
                "orc_get_vhat": (None, [VP, C.c_int, PD]),
                "orc_get_Ab": (None, [VP, C.c_int, PD, PD]),
                "orc_get_L": (None, [VP, C.c_int, PD]),
                "orc_get_lambda": (None, [VP, C.c_int, PD]),
                "orc_get_side": (None, [VP, C.c_int, C.c_int, PD]),
                "orc_get_rows": (None, [VP, C.c_int, PD, PD]),
                "orc_joint_phi": (None, [VP, C.c_int, PD]),
                "orc_get_body": (None, [VP, C.c_int, C.c_int, PD]),
                "orc_set_body": (None, [VP, C.c_int, C.c_int, PD]),
                "orc_set_generic": (None, [VP, C.c_int, PD, PD]),
                "orc_set_warm": (None, [VP, C.c_int, PD, PD]),
                "orc_set_beta_scale": (None, [VP, C.c_int, D]),
                "orc_set_corot": (C.c_int, [VP, C.c_int, C.c_int, PI, PD]),
                "orc_elastic": (None, [VP, C.c_int, PD, PD]),
                "orc_residuals": (None, [VP, PD]),
                "orc_chol_solve": (C.c_int, [C.c_int, PD, PD, PD]),
                "orc_project": (None, [C.c_int, C.c_int, C.c_int, PD, PD, PD, D, D, D, PD]),
                "orc_free": (None, [VP]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _libs[openmp] = L
    return _libs[openmp]


def _p(a: np.ndarray):
    return a.ctypes.data_as(PD)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def options_vector(o) -> np.ndarray:
    """Flatten a ``scenegen.Options``-like object into the oracle's option vector."""
    return _f64([o.h, o.gravity[0], o.gravity[1], o.gravity[2], o.baumgarte,
                 1.0 if o.beta_mode == "fixed" else 0.0, o.rho,
                 1.0 if o.warm == "prev" else 0.0, 1.0 if o.stop == "theta" else 0.0,
                 o.tol_primal, o.theta_th, float(o.max_iters)])


def body_record(b) -> np.ndarray:
    return _f64(np.concatenate([[b.m], b.I, b.p, b.q, b.v, b.w]))


def joint_params(j) -> np.ndarray:
    """The oracle's 23 parameters of a model constraint: a plane contact carries its normal
    in the axis_b slot and its radius in ref_a[0], a sphere contact its radii in ref_a[0] and
    ref_b[0]."""
    axis_b, ref_a, ref_b = j.axis_b, j.ref_a, j.ref_b
    if int(j.kind) == 4:
        axis_b = j.normal
        ref_a = [j.radius_a, 0.0, 0.0]
    elif int(j.kind) == 5:
        ref_a = [j.radius_a, 0.0, 0.0]
        ref_b = [j.radius_b, 0.0, 0.0]
    return _f64(np.concatenate([j.anchor_a, j.anchor_b, j.axis_a, axis_b, ref_a, ref_b,
                                [j.kp, j.kd, j.target, j.plane_z, j.mu]]))


class OracleScene:
    """One scene held by the oracle (subsystems and constraints in scene order)."""

    def __init__(self, scene, options, openmp: bool = False):
        L = lib(openmp)
        self.L = L
        ov = options_vector(options)
        self.h = L.orc_new(_p(ov))
        self.scene = scene
        for sub in scene.subs:
            if hasattr(sub, "bodies"):
                rec = _f64(np.concatenate([body_record(b) for b in sub.bodies]))
                rc = L.orc_add_rigid(self.h, len(sub.bodies), _p(rec))
            elif hasattr(sub, "Kv"):
                data = _f64(np.concatenate([sub.mass, sub.K_dense().ravel(), sub.f, sub.X0,
                                            sub.x, sub.v]))
                rc = L.orc_add_linear(self.h, sub.nodes, _p(data))
                if rc >= 0 and getattr(sub, "corot", False):
                    tets = np.ascontiguousarray(np.asarray(sub.tets, dtype=np.int32).ravel())
                    Ke = _f64(np.asarray(sub.Ke).ravel())
                    if L.orc_set_corot(self.h, rc, len(sub.tets), tets.ctypes.data_as(PI),
                                       _p(Ke)) < 0:
                        raise ValueError("oracle rejected the co-rotational elements")
            else:
                A, b = _f64(sub.A), _f64(sub.b)
                rc = L.orc_add_generic(self.h, sub.n, _p(A), _p(b))
            if rc < 0:
                raise ValueError("oracle rejected a subsystem")
        for itf in scene.ifs:
            if hasattr(itf, "J"):
                subs = np.ascontiguousarray(np.asarray(itf.subs, dtype=np.int32))
                J = _f64(np.concatenate([np.asarray(m, dtype=np.float64).ravel() for m in itf.J]))
                e = _f64(itf.e)
                rc = L.orc_add_rows(self.h, int(itf.type), itf.rows, len(itf.subs),
                                    subs.ctypes.data_as(PI), _p(J), _p(e), itf.k, itf.alpha,
                                    itf.mu)
            else:
                sb, bb = (itf.b if itf.b is not None else (-1, 0))
                prm = joint_params(itf)
                rc = L.orc_add_joint(self.h, int(itf.kind), itf.a[0], itf.a[1], sb, bb, _p(prm))
            if rc < 0:
                raise ValueError("oracle rejected an interface")
        if getattr(options, "solver", "admm") == "pj":
            if L.orc_set_pj(self.h, 1, float(options.pj_omega)) < 0:
                raise ValueError("oracle rejected the Projected Jacobi settings")
        self._trace = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.orc_free(self.h)
                self.h = None
        except Exception:
            pass

    # --- running
    def trace(self, cap: int):
        self._trace = np.full(3 * cap, np.nan)
        self.L.orc_set_trace(self.h, _p(self._trace), cap)

    def trace_array(self) -> np.ndarray:
        return self._trace.reshape(-1, 3)

    def step(self) -> int:
        return self.L.orc_step(self.h)

    def assemble(self):
        self.L.orc_assemble(self.h)

    # --- reading
    @property
    def nsub(self):
        return self.L.orc_nsub(self.h)

    @property
    def ncon(self):
        return self.L.orc_ncon(self.h)

    def n(self, i):
        return self.L.orc_n(self.h, i)

    def beta(self, i):
        return self.L.orc_beta(self.h, i)

    def vhat(self, i) -> np.ndarray:
        out = np.zeros(self.n(i))
        self.L.orc_get_vhat(self.h, i, _p(out))
        return out

    def Ab(self, i):
        n = self.n(i)
        A, b = np.zeros((n, n)), np.zeros(n)
        self.L.orc_get_Ab(self.h, i, _p(A), _p(b))
        return A, b

    def factor(self, i):
        n = self.n(i)
        Lm = np.zeros((n, n))
        self.L.orc_get_L(self.h, i, _p(Lm))
        return Lm

    def rows(self, j):
        return self.L.orc_rows(self.h, j)

    def sides(self, j):
        return [self.L.orc_con_sub(self.h, j, s) for s in range(self.L.orc_nsides(self.h, j))]

    def lam(self, j) -> np.ndarray:
        out = np.zeros(self.rows(j))
        self.L.orc_get_lambda(self.h, j, _p(out))
        return out

    def side(self, j, which: str) -> np.ndarray:
        code = {"x": 0, "z": 1, "u": 2, "y": 3}[which]
        ns = len(self.sides(j))
        out = np.zeros(ns * self.rows(j))
        self.L.orc_get_side(self.h, j, code, _p(out))
        return out.reshape(ns, self.rows(j))

    def con_rows(self, j):
        """(e, [J_s]) of constraint j as last assembled."""
        r = self.rows(j)
        subs = self.sides(j)
        e = np.zeros(r)
        J = np.zeros(sum(r * self.n(s) for s in subs))
        self.L.orc_get_rows(self.h, j, _p(e), _p(J))
        out, o = [], 0
        for s in subs:
            cnt = r * self.n(s)
            out.append(J[o:o + cnt].reshape(r, self.n(s)))
            o += cnt
        return e, out

    def phi(self, j) -> np.ndarray:
        out = np.zeros(5)
        self.L.orc_joint_phi(self.h, j, _p(out))
        return out[: self.rows(j)]

    def body(self, i, k) -> np.ndarray:
        out = np.zeros(17)
        self.L.orc_get_body(self.h, i, k, _p(out))
        return out

    def node(self, i, k) -> np.ndarray:
        out = np.zeros(6)
        self.L.orc_get_node(self.h, i, k, _p(out))
        return out

    def nodes_all(self) -> np.ndarray:
        out = []
        for i, sub in enumerate(self.scene.subs):
            if hasattr(sub, "Kv"):
                for k in range(sub.nodes):
                    out.append(self.node(i, k))
        return np.array(out).reshape(-1, 6)

    def set_body(self, i, k, rec):
        rec = _f64(rec)
        self.L.orc_set_body(self.h, i, k, _p(rec))

    def elastic(self, i):
        """(elastic force at the current positions, stiffness) of linear block i."""
        n = self.n(i)
        f, K = np.zeros(n), np.zeros((n, n))
        self.L.orc_elastic(self.h, i, _p(f), _p(K))
        return f, K

    def set_node(self, i, k, rec):
        self.L.orc_set_node(self.h, i, k, _p(_f64(rec)))

    def set_beta_scale(self, i, scale: float):
        """beta_i = scale x (trace rule or rho) from the next step on."""
        self.L.orc_set_beta_scale(self.h, i, float(scale))

    def set_warm(self, j, lam, z):
        """Constraint j's warm-start state (lambda per row, z per side and row)."""
        lam, z = _f64(lam), _f64(z)
        self.L.orc_set_warm(self.h, j, _p(lam), _p(z.ravel()))

    def set_generic(self, i, A=None, b=None):
        Aa = _f64(A) if A is not None else None
        ba = _f64(b) if b is not None else None
        self.L.orc_set_generic(self.h, i, _p(Aa) if Aa is not None else None,
                               _p(ba) if ba is not None else None)

    def residuals(self) -> dict:
        out = np.zeros(6)
        self.L.orc_residuals(self.h, _p(out))
        return dict(r_p=out[0], r_d=out[1], theta=out[2], iters=int(out[3]),
                    converged=bool(out[4]), status=int(out[5]))

    def vhat_all(self) -> np.ndarray:
        return np.concatenate([self.vhat(i) for i in range(self.nsub)])

    def lam_all(self) -> np.ndarray:
        return np.concatenate([self.lam(j) for j in range(self.ncon)]) if self.ncon else np.zeros(0)

    def bodies_all(self) -> np.ndarray:
        out = []
        for i, sub in enumerate(self.scene.subs):
            if hasattr(sub, "bodies"):
                for k in range(len(sub.bodies)):
                    out.append(self.body(i, k))
        return np.array(out).reshape(-1, 17)


def chol_solve(K, r) -> np.ndarray:
    K, r = _f64(K), _f64(r)
    x = np.zeros(r.shape[0])
    rc = lib().orc_chol_solve(r.shape[0], _p(K), _p(r), _p(x))
    if rc:
        raise np.linalg.LinAlgError("not SPD")
    return x


def project(type_: int, beta, y, e, k=0.0, alpha=0.0, mu=0.0) -> np.ndarray:
    """One constraint's z-step multiplier lambda.  y: (n_sides, rows)."""
    beta, y, e = _f64(beta), _f64(y), _f64(e)
    ns, rows = y.shape
    lam = np.zeros(rows)
    lib().orc_project(int(type_), rows, ns, _p(beta), _p(y.ravel()), _p(e), k, alpha, mu,
                      _p(lam))
    return lam


def run(problem, steps: int = 1, trace_cap: int = 0):
    """Step every scene of ``problem`` ``steps`` times; return the list of OracleScene."""
    out = []
    for sc in problem.scenes:
        o = OracleScene(sc, problem.options)
        if trace_cap:
            o.trace(trace_cap)
        for _ in range(steps):
            o.step()
        out.append(o)
    return out
