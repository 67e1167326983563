"""Python binding of libsubadmm (include/subadmm.h): argument marshalling only.

Every function named ``sim_*`` calls the C function of the same name and raises
``SimError`` on a negative status.  All of the method's work runs in the library's CUDA
kernels; this module never computes any of it.  Loading fails loudly when the library has
not been built (see ``paper_2302_14344_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

SIM_OK, SIM_NOT_CONVERGED = 0, 1
SIM_EINVAL, SIM_ENOMEM, SIM_ENOTSPD, SIM_ENAN, SIM_ECUDA = -1, -2, -3, -4, -5
SIM_SUB_GENERIC, SIM_SUB_RIGID, SIM_SUB_LINEAR = 0, 1, 2
SIM_IF_EQUALITY, SIM_IF_HARD, SIM_IF_SOFT, SIM_IF_CONTACT = 0, 1, 2, 3
SIM_IF_BALL, SIM_IF_REVOLUTE, SIM_IF_ANGLE_PD, SIM_IF_PLANE_CONTACT = 4, 5, 6, 7
SIM_IF_SPHERE_CONTACT = 8
SIM_BETA_TRACE, SIM_BETA_FIXED = 0, 1
SIM_WARM_COLD, SIM_WARM_PREV = 0, 1
SIM_STOP_PRIMAL, SIM_STOP_THETA = 0, 1
SIM_FP64, SIM_MIXED = 0, 1
SIM_GET_VHAT, SIM_GET_LAMBDA, SIM_GET_BODIES, SIM_GET_BETA, SIM_GET_Z, SIM_GET_NODES = range(6)

# exported symbols of include/subadmm.h
EXPORTS = ("sim_default_options", "sim_create", "sim_destroy", "sim_add_subsystem",
           "sim_add_interface", "sim_set_generic", "sim_step", "sim_residuals", "sim_get",
           "sim_read_state", "sim_read_state_noalloc", "sim_write_state", "sim_sizes",
           "sim_iteration_stats", "sim_scene_info", "sim_use_graph", "sim_launch_classes",
           "sim_autotune", "sim_grid_threshold", "sim_grid_staging", "sim_grid_blocks", "sim_tensor_cores", "sim_tc_factor", "sim_set_solver", "sim_keep_factors",
           "sim_set_beta_scale", "sim_set_corotational",
           "sim_probe_barrier", "sim_barrier_floor", "sim_gram_tc", "sim_interface_features",
           "sim_interface_targets", "sim_step_learned", "sim_phase_trace", "sim_sync",
           "sim_last_error")


class sim_options(C.Structure):
    _fields_ = [("h", C.c_double), ("gravity", C.c_double * 3), ("baumgarte", C.c_double),
                ("beta_mode", C.c_int), ("rho", C.c_double), ("warm", C.c_int),
                ("stop", C.c_int), ("tol_primal", C.c_double), ("theta_th", C.c_double),
                ("max_iters", C.c_int), ("precision", C.c_int), ("device", C.c_int),
                ("stream", C.c_void_p)]


class SimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_lock = threading.Lock()
_lib = None
PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)
PL = C.POINTER(C.c_longlong)
VP = C.c_void_p


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsubadmm.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libsubadmm.so is not built ({_build.LIB}); run "
                               "paper_2302_14344_gb300.build.build()")
        L = C.CDLL(_build.LIB)
        sig = {
            "sim_default_options": (None, [C.POINTER(sim_options)]),
            "sim_create": (C.c_int, [C.POINTER(sim_options), C.POINTER(VP)]),
            "sim_destroy": (None, [VP]),
            "sim_add_subsystem": (C.c_int, [VP, C.c_int, C.c_int, C.c_int, PD, PI]),
            "sim_add_interface": (C.c_int, [VP, C.c_int, C.c_int, C.c_int, C.c_int, PI, PD, PD,
                                            PD, PI]),
            "sim_set_generic": (C.c_int, [VP, C.c_int, PD, PD]),
            "sim_step": (C.c_int, [VP, C.c_int]),
            "sim_residuals": (C.c_int, [VP, C.c_int, PD]),
            "sim_get": (C.c_int, [VP, C.c_int, C.c_int, PD]),
            "sim_read_state": (C.c_int, [VP, VP]),
            "sim_read_state_noalloc": (C.c_int, [VP, VP]),
            "sim_write_state": (C.c_int, [VP, VP]),
            "sim_sizes": (C.c_int, [VP, PL]),
            "sim_iteration_stats": (C.c_int, [VP, PL, PL]),
            "sim_scene_info": (C.c_int, [VP, C.c_int, PL]),
            "sim_use_graph": (C.c_int, [VP, C.c_int]),
            "sim_launch_classes": (C.c_int, [VP, C.c_int, PL]),
            "sim_autotune": (C.c_int, [VP, C.c_int, C.c_int, PL]),
            "sim_grid_threshold": (C.c_int, [VP, C.c_int]),
            "sim_grid_staging": (C.c_int, [VP, C.c_int]),
            "sim_keep_factors": (C.c_int, [VP, C.c_int]),
            "sim_grid_blocks": (C.c_int, [VP, C.c_int]),
            "sim_tensor_cores": (C.c_int, [VP, C.c_int]),
            "sim_tc_factor": (C.c_int, [VP, C.c_int]),
            "sim_set_solver": (C.c_int, [VP, C.c_int, C.c_double]),
            "sim_set_beta_scale": (C.c_int, [VP, PD]),
            "sim_set_corotational": (C.c_int, [VP, C.c_int, C.c_int, PI, PD]),
            "sim_interface_features": (C.c_int, [VP, VP]),
            "sim_interface_targets": (C.c_int, [VP, VP, VP, VP]),
            "sim_step_learned": (C.c_int, [VP, VP, C.c_int]),
            "sim_probe_barrier": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, PI]),
            "sim_barrier_floor": (C.c_int, [C.c_int, C.c_int, PD]),
            "sim_gram_tc": (C.c_int, [C.c_int, C.c_int, C.POINTER(VP), PI, PI, PI,
                                      C.POINTER(VP), PI, C.c_int, C.POINTER(C.c_float)]),
            "sim_phase_trace": (C.c_int, [VP, C.c_int, PL]),
            "sim_sync": (C.c_int, [VP]),
            "sim_last_error": (C.c_char_p, [VP]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(h, rc: int) -> int:
    if rc < 0:
        msg = load().sim_last_error(h)
        raise SimError(rc, msg.decode() if msg else "error")
    return rc


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(PD)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --- thin wrappers, one per C function --------------------------------------------------

def sim_default_options() -> sim_options:
    o = sim_options()
    load().sim_default_options(C.byref(o))
    return o


def sim_create(opt: sim_options):
    h = VP()
    _check(None, load().sim_create(C.byref(opt), C.byref(h)))
    return h


def sim_destroy(h) -> None:
    load().sim_destroy(h)


def sim_add_subsystem(h, scene: int, kind: int, count: int, data) -> int:
    d = _f64(data)
    out = C.c_int(-1)
    _check(h, load().sim_add_subsystem(h, scene, kind, count, _dp(d), C.byref(out)))
    return out.value


def sim_add_interface(h, scene: int, kind: int, rows: int, n_sides: int, sides, J=None, e=None,
                      params=None) -> int:
    s = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    Jd = None if J is None else _f64(J)
    ed = None if e is None else _f64(e)
    pd = None if params is None else _f64(params)
    out = C.c_int(-1)
    _check(h, load().sim_add_interface(h, scene, kind, rows, n_sides, s.ctypes.data_as(PI),
                                       _dp(Jd), _dp(ed), _dp(pd), C.byref(out)))
    return out.value


def sim_set_generic(h, sub: int, A=None, b=None) -> None:
    Ad = None if A is None else _f64(A)
    bd = None if b is None else _f64(b)
    _check(h, load().sim_set_generic(h, sub, _dp(Ad), _dp(bd)))


def sim_step(h, n_steps: int = 1) -> None:
    _check(h, load().sim_step(h, n_steps))


def sim_residuals(h, scene: int) -> dict:
    out = np.zeros(6)
    rc = _check(h, load().sim_residuals(h, scene, _dp(out)))
    return dict(r_p=out[0], r_d=out[1], theta=out[2], iters=int(out[3]),
                converged=bool(out[4]), status=int(out[5]), rc=rc)


def sim_get(h, what: int, id_: int, count: int) -> np.ndarray:
    out = np.zeros(count)
    _check(h, load().sim_get(h, what, id_, _dp(out)))
    return out


def sim_read_state(h, dst_ptr: int) -> None:
    """dst_ptr: address of a host buffer of 13 doubles per body followed by 6 per node (e.g.
    a pinned tensor)."""
    _check(h, load().sim_read_state(h, VP(dst_ptr)))


def sim_read_state_noalloc(h, dst_ptr: int) -> None:
    """sim_read_state through the library's fixed device staging array: never allocates
    device memory (for callers that cannot); at most 131072 state doubles (10082 bodies);
    calls share the array."""
    _check(h, load().sim_read_state_noalloc(h, VP(dst_ptr)))


def sim_write_state(h, src_ptr: int) -> None:
    _check(h, load().sim_write_state(h, VP(src_ptr)))


def _class_rows(out, n: int) -> list:
    keys = ("scenes", "cached", "split", "smem_bytes", "ns_per_step")
    return [dict(zip(keys, (int(v) for v in out[5 * k:5 * k + 5]))) for k in range(n)]


def sim_launch_classes(h, max_classes: int = 64) -> list:
    out = (C.c_longlong * (5 * max_classes))()
    n = _check(h, load().sim_launch_classes(h, max_classes, out))
    return _class_rows(out, min(n, max_classes))


def sim_autotune(h, steps: int = 5, max_classes: int = 64) -> list:
    out = (C.c_longlong * (5 * max_classes))()
    n = _check(h, load().sim_autotune(h, steps, max_classes, out))
    return _class_rows(out, min(n, max_classes))


def sim_grid_threshold(h, side_rows: int) -> None:
    _check(h, load().sim_grid_threshold(h, side_rows))


def sim_grid_staging(h, enable: bool) -> None:
    _check(h, load().sim_grid_staging(h, 1 if enable else 0))


def sim_grid_blocks(h, blocks: int) -> None:
    _check(h, load().sim_grid_blocks(h, blocks))


def sim_set_corotational(h, sub: int, tets, Ke) -> None:
    t = np.ascontiguousarray(np.asarray(tets, dtype=np.int32).ravel())
    k = _f64(np.asarray(Ke).ravel())
    _check(h, load().sim_set_corotational(h, sub, len(t) // 4, t.ctypes.data_as(PI), _dp(k)))


def sim_set_beta_scale(h, scale) -> None:
    a = _f64(scale)
    _check(h, load().sim_set_beta_scale(h, _dp(a)))


def sim_tensor_cores(h, enable: bool) -> None:
    _check(h, load().sim_tensor_cores(h, 1 if enable else 0))


def sim_tc_factor(h, enable: bool) -> None:
    _check(h, load().sim_tc_factor(h, 1 if enable else 0))


SIM_SOLVER_ADMM, SIM_SOLVER_PJ = 0, 1


def sim_set_solver(h, solver: int, omega: float = 1.0) -> None:
    _check(h, load().sim_set_solver(h, solver, float(omega)))


def sim_keep_factors(h, enable: bool) -> None:
    _check(h, load().sim_keep_factors(h, 1 if enable else 0))


def sim_probe_barrier(device: int, blocks: int, expected: int, limit_s: float) -> dict:
    out = (C.c_int * 2)()
    rc = load().sim_probe_barrier(device, blocks, expected, limit_s, out)
    if rc < 0:
        raise SimError(rc, "sim_probe_barrier failed")
    return dict(timed_out=bool(out[0]), passed=int(out[1]))


def sim_barrier_floor(device: int, iters: int = 20000) -> dict:
    """Cycles and nanoseconds of one block-barrier round (the block kernel's per-iteration
    floor)."""
    out = (C.c_double * 2)()
    rc = load().sim_barrier_floor(device, iters, out)
    if rc < 0:
        raise SimError(rc, "sim_barrier_floor failed")
    return {"cycles": out[0], "ns": out[1]}


def sim_gram_tc(device: int, W_ptrs, n, cols, ldw, G_ptrs, ldg, reps: int = 1) -> float:
    """G_j = W_j^T W_j on the tensor cores for device arrays W_j (n_j x ldw_j floats) into
    G_j (cols_j x ldg_j floats); returns the mean ms per run over reps - 1 timed runs."""
    k = len(W_ptrs)
    arr = lambda t, v: (t * k)(*v)
    ms = C.c_float(0.0)
    rc = load().sim_gram_tc(device, k, arr(VP, W_ptrs), arr(C.c_int, n), arr(C.c_int, cols),
                            arr(C.c_int, ldw), arr(VP, G_ptrs), arr(C.c_int, ldg), reps,
                            C.byref(ms))
    if rc < 0:
        raise SimError(rc, "sim_gram_tc failed")
    return float(ms.value)


def sim_use_graph(h, enable: bool) -> None:
    _check(h, load().sim_use_graph(h, 1 if enable else 0))


def sim_sizes(h) -> dict:
    out = (C.c_longlong * 9)()
    _check(h, load().sim_sizes(h, out))
    keys = ("scenes", "subsystems", "dof", "interfaces", "rows", "side_rows", "bodies",
            "smem_bytes", "nodes")
    return {k: int(v) for k, v in zip(keys, out)}


def sim_scene_info(h, scene: int) -> dict:
    out = (C.c_longlong * 4)()
    _check(h, load().sim_scene_info(h, scene, out))
    return dict(global_workspace=bool(out[0]), placement=int(out[0]), smem_bytes=int(out[1]),
                subsystems=int(out[2]), work_bytes=int(out[3]))


def sim_iteration_stats(h, per_scene: bool = False) -> dict:
    """Totals since the last call (then cleared); with per_scene, also "per_scene": an
    array (scenes, 5) of [iterations, max iterations, not converged, scene-steps,
    fallbacks]."""
    out = (C.c_longlong * 5)()
    ps = None
    if per_scene:
        ps = np.zeros((sim_sizes(h)["scenes"], 5), dtype=np.int64)
    _check(h, load().sim_iteration_stats(h, out, None if ps is None else
                                         ps.ctypes.data_as(C.POINTER(C.c_longlong))))
    d = dict(total_iters=int(out[0]), max_iters=int(out[1]), not_converged=int(out[2]),
             scene_steps=int(out[3]), fallbacks=int(out[4]))
    if ps is not None:
        d["per_scene"] = ps
    return d


def sim_interface_features(h, x_ptr: int) -> None:
    _check(h, load().sim_interface_features(h, VP(x_ptr)))


def sim_interface_targets(h, x_ptr: int, t_ptr: int, mask_ptr: int) -> None:
    _check(h, load().sim_interface_targets(h, VP(x_ptr), VP(t_ptr), VP(mask_ptr)))


def sim_step_learned(h, net_handle, n_steps: int = 1) -> None:
    _check(h, load().sim_step_learned(h, net_handle, n_steps))


PHASES = ("assemble", "factor", "v_step", "z_step", "exit", "recover", "iterations",
          "scene_steps")


def sim_phase_trace(h, enable: bool) -> dict:
    """Counters since the last call (cycles per phase, iterations, scene-steps), then turn
    the device phase tracer on or off."""
    out = (C.c_longlong * 8)()
    _check(h, load().sim_phase_trace(h, 1 if enable else 0, out))
    return {k: int(v) for k, v in zip(PHASES, out)}


def sim_sync(h) -> None:
    _check(h, load().sim_sync(h))


def sim_last_error(h) -> str:
    m = load().sim_last_error(h)
    return m.decode() if m else ""


# --- convenience: a simulation built from a scene description ---------------------------

_KIND = {0: SIM_IF_EQUALITY, 1: SIM_IF_HARD, 2: SIM_IF_SOFT, 3: SIM_IF_CONTACT}
_MODEL = {1: SIM_IF_BALL, 2: SIM_IF_REVOLUTE, 3: SIM_IF_ANGLE_PD, 4: SIM_IF_PLANE_CONTACT,
          5: SIM_IF_SPHERE_CONTACT}


def model_params(itf) -> np.ndarray:
    """The 23 parameters of a rigid-model interface: a plane contact carries its normal in
    the axis_b slot and its radius in ref_a[0], a sphere contact its radii in ref_a[0] and
    ref_b[0]."""
    kind = _MODEL[int(itf.kind)]
    axis_b, ref_a, ref_b = itf.axis_b, itf.ref_a, itf.ref_b
    if kind == SIM_IF_PLANE_CONTACT:
        axis_b, ref_a = itf.normal, [itf.radius_a, 0.0, 0.0]
    elif kind == SIM_IF_SPHERE_CONTACT:
        ref_a, ref_b = [itf.radius_a, 0.0, 0.0], [itf.radius_b, 0.0, 0.0]
    return np.concatenate([itf.anchor_a, itf.anchor_b, itf.axis_a, axis_b, ref_a, ref_b,
                           [itf.kp, itf.kd, itf.target, itf.plane_z, itf.mu]]).astype(np.float64)


def options_from(o, stream: int = 0, device: int = 0, precision: int = SIM_FP64) -> sim_options:
    """sim_options from an object with the fields of ``scenegen.Options``."""
    opt = sim_default_options()
    opt.h = o.h
    for k in range(3):
        opt.gravity[k] = o.gravity[k]
    opt.baumgarte = o.baumgarte
    opt.beta_mode = SIM_BETA_FIXED if o.beta_mode == "fixed" else SIM_BETA_TRACE
    opt.rho = o.rho if o.beta_mode == "fixed" else 1e3
    opt.warm = SIM_WARM_PREV if o.warm == "prev" else SIM_WARM_COLD
    opt.stop = SIM_STOP_THETA if o.stop == "theta" else SIM_STOP_PRIMAL
    opt.tol_primal = o.tol_primal
    opt.theta_th = o.theta_th
    opt.max_iters = int(o.max_iters)
    opt.precision = precision
    opt.device = device
    opt.stream = stream or None
    return opt


class Simulation:
    """A libsubadmm simulation holding every scene of a problem description.

    ``problem`` has ``scenes`` (each with ``subs`` and ``ifs``) and ``options``, shaped like
    ``scenegen.Problem``.  Subsystem and interface ids are assigned in scene order."""

    def __init__(self, problem, stream: int = 0, device: int = 0, precision: int = SIM_FP64,
                 grid_side_rows: Optional[int] = None):
        self.h = sim_create(options_from(problem.options, stream, device, precision))
        if grid_side_rows is not None:
            sim_grid_threshold(self.h, grid_side_rows)
        if getattr(problem.options, "solver", "admm") == "pj":
            sim_set_solver(self.h, SIM_SOLVER_PJ, problem.options.pj_omega)
        self.sub_ids = []     # per scene: list of ids
        self.if_ids = []
        self.sub_n = []
        self.if_rows = []
        self.if_nsides = []
        self.rigid_subs = []
        self.linear_subs = []
        for sc_i, sc in enumerate(problem.scenes):
            ids = []
            for sub in sc.subs:
                if hasattr(sub, "bodies"):
                    rec = np.concatenate([np.concatenate([[b.m], b.I, b.p, b.q, b.v, b.w])
                                          for b in sub.bodies])
                    sid = sim_add_subsystem(self.h, sc_i, SIM_SUB_RIGID, len(sub.bodies), rec)
                    self.rigid_subs.append((sid, len(sub.bodies)))
                elif hasattr(sub, "Kv"):
                    trip = np.stack([np.asarray(sub.Ki, float), np.asarray(sub.Kj, float),
                                     np.asarray(sub.Kv, float)], axis=1).ravel()
                    data = np.concatenate([sub.mass, sub.f, sub.X0, sub.x, sub.v,
                                           [float(len(sub.Kv))], trip])
                    sid = sim_add_subsystem(self.h, sc_i, SIM_SUB_LINEAR, sub.nodes, data)
                    if getattr(sub, "corot", False):
                        sim_set_corotational(self.h, sid, sub.tets, sub.Ke)
                    self.linear_subs.append((sid, sub.nodes))
                else:
                    data = np.concatenate([np.asarray(sub.A, float).ravel(),
                                           np.asarray(sub.b, float)])
                    sid = sim_add_subsystem(self.h, sc_i, SIM_SUB_GENERIC, sub.n, data)
                ids.append(sid)
                self.sub_n.append(sub.n)
            self.sub_ids.append(ids)
            iids = []
            for itf in sc.ifs:
                if hasattr(itf, "J"):
                    sides = [ids[s] for s in itf.subs]
                    J = np.concatenate([np.asarray(m, float).ravel() for m in itf.J])
                    iid = sim_add_interface(self.h, sc_i, _KIND[int(itf.type)], itf.rows,
                                            len(sides), sides, J, itf.e,
                                            [itf.k, itf.alpha, itf.mu])
                    self.if_rows.append(itf.rows)
                    self.if_nsides.append(len(sides))
                else:
                    sb, bb = (ids[itf.b[0]], itf.b[1]) if itf.b is not None else (-1, 0)
                    prm = model_params(itf)
                    kind = _MODEL[int(itf.kind)]
                    iid = sim_add_interface(self.h, sc_i, kind, 0, 0,
                                            [ids[itf.a[0]], itf.a[1], sb, bb], None, None, prm)
                    rows = {SIM_IF_BALL: 3, SIM_IF_REVOLUTE: 5, SIM_IF_ANGLE_PD: 1,
                            SIM_IF_PLANE_CONTACT: 3, SIM_IF_SPHERE_CONTACT: 3}[kind]
                    self.if_rows.append(rows)
                    same = itf.b is None or itf.b[0] == itf.a[0]
                    self.if_nsides.append(1 if same else 2)
                iids.append(iid)
            self.if_ids.append(iids)
        self.n_scenes = len(problem.scenes)

    def close(self):
        if getattr(self, "h", None):
            sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        sim_step(self.h, n)

    def launch_classes(self) -> list:
        return sim_launch_classes(self.h)

    def autotune(self, steps: int = 5) -> list:
        return sim_autotune(self.h, steps)

    def use_graph(self, enable: bool = True) -> None:
        sim_use_graph(self.h, enable)

    def grid_staging(self, enable: bool = True) -> None:
        sim_grid_staging(self.h, enable)

    def grid_blocks(self, blocks: int) -> None:
        sim_grid_blocks(self.h, blocks)

    def set_beta_scale(self, scale) -> None:
        """One scale per subsystem id (sub_ids order): beta_i = scale x trace rule (or rho)."""
        sim_set_beta_scale(self.h, scale)

    def tensor_cores(self, enable: bool = True) -> None:
        sim_tensor_cores(self.h, enable)

    def tc_factor(self, enable: bool = True) -> None:
        """Blocked Cholesky with tensor-core Schur updates for the refactorised large blocks."""
        sim_tc_factor(self.h, enable)

    def keep_factors(self, enable: bool = True) -> None:
        sim_keep_factors(self.h, enable)

    def step_learned(self, net, n: int = 1) -> None:
        """n steps with the learned warm start of `net` (a warmstart.Network)."""
        sim_step_learned(self.h, net.h, n)

    def sync(self):
        sim_sync(self.h)

    def residuals(self, scene: int) -> dict:
        return sim_residuals(self.h, scene)

    def vhat(self, sid: int) -> np.ndarray:
        return sim_get(self.h, SIM_GET_VHAT, sid, self.sub_n[sid])

    def lam(self, iid: int) -> np.ndarray:
        return sim_get(self.h, SIM_GET_LAMBDA, iid, self.if_rows[iid])

    def z(self, iid: int) -> np.ndarray:
        return sim_get(self.h, SIM_GET_Z, iid, self.if_rows[iid] * self.if_nsides[iid]).reshape(
            self.if_nsides[iid], self.if_rows[iid])

    def beta(self, sid: int) -> float:
        return float(sim_get(self.h, SIM_GET_BETA, sid, 1)[0])

    def bodies(self, sid: int, nb: int) -> np.ndarray:
        return sim_get(self.h, SIM_GET_BODIES, sid, 17 * nb).reshape(nb, 17)

    def nodes(self, sid: int, nn: int) -> np.ndarray:
        return sim_get(self.h, SIM_GET_NODES, sid, 6 * nn).reshape(nn, 6)

    def scene_nodes(self, scene: int) -> np.ndarray:
        out = []
        for sid, nn in self.linear_subs:
            if sid in self.sub_ids[scene]:
                out.append(self.nodes(sid, nn))
        return np.concatenate(out) if out else np.zeros((0, 6))

    def scene_vhat(self, scene: int) -> np.ndarray:
        return np.concatenate([self.vhat(s) for s in self.sub_ids[scene]])

    def scene_lam(self, scene: int) -> np.ndarray:
        ids = self.if_ids[scene]
        return np.concatenate([self.lam(i) for i in ids]) if ids else np.zeros(0)

    def scene_bodies(self, scene: int) -> np.ndarray:
        out = []
        for sid, nb in self.rigid_subs:
            if sid in self.sub_ids[scene]:
                out.append(self.bodies(sid, nb))
        return np.concatenate(out) if out else np.zeros((0, 17))

    def sizes(self) -> dict:
        return sim_sizes(self.h)

    def iteration_stats(self, per_scene: bool = False) -> dict:
        return sim_iteration_stats(self.h, per_scene)
