"""Python binding of libpradmm (include/pradmm.h).

Argument marshalling only: every function here forwards to the C ABI of the
same name, and all arithmetic of the solver runs in the library's CUDA
kernels.  Importing this module does not load the library; the first call
does, and raises if `libpradmm.so` has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpradmm.so")

PRADMM_OK = 0
PRADMM_ERR_ARG = 1
PRADMM_ERR_INDEX = 2
PRADMM_ERR_SELFLOOP = 3
PRADMM_ERR_NONFINITE = 4
PRADMM_ERR_NOMEM = 5
PRADMM_ERR_CUDA = 6
PRADMM_ERR_TIMEOUT = 7
PRADMM_ERR_NOT_CONVERGED = 8
PRADMM_ERR_QUATERNION = 9
PRADMM_ERR_STATE = 10
PRADMM_FP64 = 0
PRADMM_FP32 = 1


class pradmm_params(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("relax", ctypes.c_double),
                ("gamma", ctypes.c_double * 4), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("fallback_eps", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("block", ctypes.c_int32), ("l2_window", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("inertia", ctypes.c_double)]


class PRADMMError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status} ({message})")
        self.status = status
        self.message = message


_lock = threading.Lock()
_lib = None

_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_i32 = _P(ctypes.c_int32)
_i64 = _P(ctypes.c_int64)
_h = ctypes.c_void_p

_SIGS = {
    "pradmm_default_params": (None, [_P(pradmm_params)]),
    "pradmm_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _i32, _i32, _d, _d, _d, _d, _P(pradmm_params),
                                     ctypes.c_void_p, _P(ctypes.c_void_p)]),
    "pradmm_create_device": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            _P(pradmm_params), ctypes.c_void_p, _P(ctypes.c_void_p)]),
    "pradmm_set_state": (ctypes.c_int, [_h, _d, _d]),
    "pradmm_set_state_full": (ctypes.c_int, [_h, _d, _d, _d, _d, _d, _d]),
    "pradmm_set_state_full_device": (ctypes.c_int, [_h, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pradmm_init_odometry": (ctypes.c_int, [_h]),
    "pradmm_autotune": (ctypes.c_int, [_h, ctypes.c_int32, _i32]),
    "pradmm_step": (ctypes.c_int, [_h, ctypes.c_int32, _d]),
    "pradmm_solve": (ctypes.c_int, [_h, _i32, _d]),
    "pradmm_objective": (ctypes.c_int, [_h, _d]),
    "pradmm_get_state": (ctypes.c_int, [_h, _d, _d, _d, _d, _d, _d]),
    "pradmm_get_state_device": (ctypes.c_int, [_h, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pradmm_get_poses": (ctypes.c_int, [_h, _d, _d]),
    "pradmm_iterations": (ctypes.c_int64, [_h]),
    "pradmm_set_trace": (ctypes.c_int, [_h, ctypes.c_int32]),
    "pradmm_profile_iterations": (ctypes.c_int, [_h, ctypes.c_int32, _d]),
    "pradmm_debug_set_neighbour": (ctypes.c_int, [_h, ctypes.c_int64, ctypes.c_int32]),
    "pradmm_get_trace": (ctypes.c_int, [_h, _d, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "pradmm_odometry_forest": (ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "pradmm_counters": (ctypes.c_int, [_h, _i64]),
    "pradmm_bytes_per_iteration": (ctypes.c_int, [_h, _d]),
    "pradmm_profile_sweeps": (ctypes.c_int, [_h, ctypes.c_int32, _d]),
    "pradmm_l2_window_info": (ctypes.c_int, [_h, _d]),
    "pradmm_set_sigma": (ctypes.c_int, [_h, _d, _d]),
    "pradmm_adjoint_record": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.c_int32]),
    "pradmm_adjoint_tape_info": (ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_int32), _d]),
    "pradmm_adjoint": (ctypes.c_int, [_h, _d, _d, _d, _d, _d, _d, _d]),
    "pradmm_adjoint_device": (ctypes.c_int, [_h] + [ctypes.c_void_p] * 7),
    "pradmm_objective_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 10),
    "pradmm_destroy": (None, [_h]),
    "pradmm_batch_create": (ctypes.c_int, [ctypes.c_int32, _i64, _i64, _i32, _i32, _d, _d, _d, _d, _P(pradmm_params),
                                           ctypes.c_void_p, _P(ctypes.c_void_p)]),
    "pradmm_batch_set_schedule": (ctypes.c_int, [_h, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32]),
    "pradmm_batch_get_schedule": (ctypes.c_int, [_h, _i32, _i32, _i32, _i32]),
    "pradmm_batch_autotune": (ctypes.c_int, [_h, ctypes.c_int32, _i32, _i32, _i32, _i32]),
    "pradmm_batch_autotune_profiled": (ctypes.c_int, [_h, ctypes.c_double, _i32, _i32, _i32, _i32]),
    "pradmm_batch_init_odometry": (ctypes.c_int, [_h]),
    "pradmm_batch_set_sigma": (ctypes.c_int, [_h, _d, _d]),
    "pradmm_batch_set_state": (ctypes.c_int, [_h, _d, _d]),
    "pradmm_batch_solve": (ctypes.c_int, [_h, ctypes.c_double, ctypes.c_int32, _i32, _d, _d, _i32]),
    "pradmm_batch_objectives": (ctypes.c_int, [_h, _d]),
    "pradmm_batch_spans": (ctypes.c_int, [_h, ctypes.POINTER(ctypes.c_uint64)]),
    "pradmm_batch_get_state": (ctypes.c_int, [_h, _d, _d, _d, _d, _d, _d]),
    "pradmm_batch_destroy": (None, [_h]),
    "pradmm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pradmm_last_error": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Loads libpradmm.so (built by `paper_2601_15684_gb300.build_lib.build()`)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libpradmm.so not built at {path}; "
                                   "build it with paper_2601_15684_gb300.build_lib.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != PRADMM_OK:
        lib = load()
        msg = lib.pradmm_last_error().decode() or lib.pradmm_status_string(status).decode()
        raise PRADMMError(status, where, msg)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_d)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


# ---- same-name wrappers of the C ABI ---------------------------------------------

def pradmm_default_params() -> pradmm_params:
    p = pradmm_params()
    load().pradmm_default_params(ctypes.byref(p))
    return p


def pradmm_create(n, src, dst, q_meas, t_meas, kappa=None, omega=None, params=None, stream=None):
    """Returns a handle (int).  Arrays are host numpy arrays; see pradmm.h."""
    lib = load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    q_meas = _f64(q_meas, (m, 4))
    t_meas = _f64(t_meas, (m, 3))
    kappa = _f64(kappa)
    omega = _f64(omega)
    prm = params if params is not None else pradmm_default_params()
    h = ctypes.c_void_p()
    st = lib.pradmm_create(int(n), m, src.ctypes.data_as(_i32), dst.ctypes.data_as(_i32), _dp(q_meas), _dp(t_meas),
                           _dp(kappa), _dp(omega), ctypes.byref(prm), ctypes.c_void_p(stream or 0), ctypes.byref(h))
    _check(st, "pradmm_create")
    return h.value


def pradmm_create_device(n, m, src_ptr, dst_ptr, q_ptr, t_ptr, kappa_ptr=0, omega_ptr=0, params=None, stream=None):
    """Device-pointer variant (e.g. torch tensors' data_ptr())."""
    lib = load()
    prm = params if params is not None else pradmm_default_params()
    h = ctypes.c_void_p()
    st = lib.pradmm_create_device(int(n), int(m), ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr),
                                  ctypes.c_void_p(q_ptr), ctypes.c_void_p(t_ptr), ctypes.c_void_p(kappa_ptr or 0),
                                  ctypes.c_void_p(omega_ptr or 0), ctypes.byref(prm), ctypes.c_void_p(stream or 0),
                                  ctypes.byref(h))
    _check(st, "pradmm_create_device")
    return h.value


def pradmm_set_state(h, q, t, n):
    q, t = _f64(q, (n, 4)), _f64(t, (n, 3))
    _check(load().pradmm_set_state(h, _dp(q), _dp(t)), "pradmm_set_state")


def pradmm_set_state_full(h, st: dict, n):
    a = {k: _f64(st[k], (n, 4) if k in ("p", "q", "lam") else (n, 3)) for k in ("p", "q", "t", "s", "lam", "z")}
    _check(load().pradmm_set_state_full(h, _dp(a["p"]), _dp(a["q"]), _dp(a["t"]), _dp(a["s"]), _dp(a["lam"]),
                                        _dp(a["z"])), "pradmm_set_state_full")


def pradmm_set_state_full_device(h, p, q, t, s, lam=0, z=0):
    """Device-pointer variant of pradmm_set_state_full (addresses of FP64
    device arrays, e.g. torch tensors' data_ptr(); lam, z may be 0)."""
    _check(load().pradmm_set_state_full_device(h, ctypes.c_void_p(p), ctypes.c_void_p(q), ctypes.c_void_p(t),
                                               ctypes.c_void_p(s), ctypes.c_void_p(lam or 0),
                                               ctypes.c_void_p(z or 0)), "pradmm_set_state_full_device")


def pradmm_autotune(h, iters: int) -> int:
    """CTA size of the sweeps chosen by timing `iters` iterations (state restored)."""
    b = ctypes.c_int32(0)
    _check(load().pradmm_autotune(h, int(iters), ctypes.byref(b)), "pradmm_autotune")
    return int(b.value)


def pradmm_init_odometry(h):
    _check(load().pradmm_init_odometry(h), "pradmm_init_odometry")


def pradmm_step(h, iters: int) -> float:
    e = ctypes.c_double(0.0)
    _check(load().pradmm_step(h, int(iters), ctypes.byref(e)), "pradmm_step")
    return e.value


def pradmm_solve(h):
    """Returns (converged, iterations, e_final)."""
    it = ctypes.c_int32(0)
    e = ctypes.c_double(0.0)
    st = load().pradmm_solve(h, ctypes.byref(it), ctypes.byref(e))
    if st not in (PRADMM_OK, PRADMM_ERR_NOT_CONVERGED):
        _check(st, "pradmm_solve")
    return st == PRADMM_OK, it.value, e.value


def pradmm_objective(h) -> float:
    F = ctypes.c_double(0.0)
    _check(load().pradmm_objective(h, ctypes.byref(F)), "pradmm_objective")
    return F.value


def pradmm_get_state(h, n) -> dict:
    out = {"p": np.zeros((n, 4)), "q": np.zeros((n, 4)), "t": np.zeros((n, 3)), "s": np.zeros((n, 3)),
           "lam": np.zeros((n, 4)), "z": np.zeros((n, 3))}
    _check(load().pradmm_get_state(h, _dp(out["p"]), _dp(out["q"]), _dp(out["t"]), _dp(out["s"]), _dp(out["lam"]),
                                   _dp(out["z"])), "pradmm_get_state")
    return out


def pradmm_get_state_device(h, p=0, q=0, t=0, s=0, lam=0, z=0):
    _check(load().pradmm_get_state_device(h, ctypes.c_void_p(p), ctypes.c_void_p(q), ctypes.c_void_p(t),
                                          ctypes.c_void_p(s), ctypes.c_void_p(lam), ctypes.c_void_p(z)),
           "pradmm_get_state_device")


def pradmm_get_poses(h, n, q_out=None, t_out=None):
    q = q_out if q_out is not None else np.zeros((n, 4))
    t = t_out if t_out is not None else np.zeros((n, 3))
    _check(load().pradmm_get_poses(h, _dp(q), _dp(t)), "pradmm_get_poses")
    return q, t


def pradmm_iterations(h) -> int:
    return int(load().pradmm_iterations(h))


def pradmm_debug_set_neighbour(h, slot: int, value: int):
    _check(load().pradmm_debug_set_neighbour(h, int(slot), int(value)), "pradmm_debug_set_neighbour")


def pradmm_profile_iterations(h, iters: int):
    """(iters x 4) ms: q/lambda, t, s/z+p kernel and iteration time of each iteration."""
    out = np.zeros((int(iters), 4))
    _check(load().pradmm_profile_iterations(h, int(iters), _dp(out)), "pradmm_profile_iterations")
    return out


def pradmm_set_trace(h, capacity: int):
    _check(load().pradmm_set_trace(h, int(capacity)), "pradmm_set_trace")


def pradmm_odometry_forest(h, n):
    """(parent, tree-edge code) of every vertex, int32; see pradmm.h."""
    par = np.zeros(n, dtype=np.int32)
    pedge = np.zeros(n, dtype=np.int32)
    i32 = ctypes.POINTER(ctypes.c_int32)
    _check(load().pradmm_odometry_forest(h, par.ctypes.data_as(i32), pedge.ctypes.data_as(i32)),
           "pradmm_odometry_forest")
    return par, pedge


def pradmm_get_trace(h, capacity: int):
    """(first iteration number, e^k array oldest first)."""
    out = np.zeros(max(int(capacity), 1))
    first = ctypes.c_int64(0)
    cnt = ctypes.c_int32(0)
    _check(load().pradmm_get_trace(h, _dp(out), ctypes.byref(first), ctypes.byref(cnt)), "pradmm_get_trace")
    return int(first.value), out[:cnt.value].copy()


def pradmm_counters(h) -> dict:
    out = np.zeros(4, dtype=np.int64)
    _check(load().pradmm_counters(h, out.ctypes.data_as(_i64)), "pradmm_counters")
    return {"fallbacks": int(out[0]), "zero_u": int(out[1]), "iterations": int(out[2]), "stopped": int(out[3])}


def pradmm_bytes_per_iteration(h) -> dict:
    out = np.zeros(4)
    _check(load().pradmm_bytes_per_iteration(h, _dp(out)), "pradmm_bytes_per_iteration")
    return {"total": out[0], "k_q": out[1], "k_t": out[2], "k_sp": out[3]}


def pradmm_l2_window_info(h) -> dict:
    out = np.zeros(3)
    _check(load().pradmm_l2_window_info(h, _dp(out)), "pradmm_l2_window_info")
    return {"window_bytes": out[0], "hit_ratio": out[1], "set_aside_bytes": out[2]}


def pradmm_profile_sweeps(h, iters: int) -> dict:
    out = np.zeros(4)
    _check(load().pradmm_profile_sweeps(h, int(iters), _dp(out)), "pradmm_profile_sweeps")
    return {"k_q": out[0], "k_t": out[1], "k_sp": out[2], "iteration": out[3]}


def pradmm_set_sigma(h, Sigma1=None, Sigma2=None):
    """General 4x4 weight matrices (row-major); both None returns to Sigma = I."""
    S1 = None if Sigma1 is None else _f64(Sigma1, (4, 4))
    S2 = None if Sigma2 is None else _f64(Sigma2, (4, 4))
    _check(load().pradmm_set_sigma(h, _dp(S1), _dp(S2)), "pradmm_set_sigma")


def pradmm_adjoint_record(h, iters: int, ckpt_every: int = 0):
    _check(load().pradmm_adjoint_record(h, int(iters), int(ckpt_every)), "pradmm_adjoint_record")


def pradmm_adjoint_tape_info(h):
    """(checkpoint spacing, tape bytes) of the current recording."""
    c = ctypes.c_int32(0)
    b = np.zeros(1)
    _check(load().pradmm_adjoint_tape_info(h, ctypes.byref(c), _dp(b)), "pradmm_adjoint_tape_info")
    return int(c.value), float(b[0])


_X0 = (("p", 4), ("q", 4), ("t", 3), ("s", 3), ("lam", 4), ("z", 3))


def pradmm_adjoint(h, n, m, p_bar=None, t_bar=None, x0=False) -> dict:
    """Gradients of L(p^K, t^K) given p_bar = dL/dp^K, t_bar = dL/dt^K (host
    arrays): dict with q_meas (m x 4), t_meas (m x 3), kappa (m), omega (m)
    and, if x0, the adjoint of the recorded initial state (dict of p .. z)."""
    pb = _f64(p_bar, (n, 4)) if p_bar is not None else None
    tb = _f64(t_bar, (n, 3)) if t_bar is not None else None
    out = {"q_meas": np.zeros((m, 4)), "t_meas": np.zeros((m, 3)), "kappa": np.zeros(m), "omega": np.zeros(m)}
    x0buf = np.zeros(21 * n) if x0 else None
    _check(load().pradmm_adjoint(h, _dp(pb), _dp(tb), _dp(out["q_meas"]), _dp(out["t_meas"]), _dp(out["kappa"]),
                                 _dp(out["omega"]), _dp(x0buf)), "pradmm_adjoint")
    if x0:
        o, d = 0, {}
        for key, w in _X0:
            d[key] = x0buf[o:o + w * n].reshape(n, w)
            o += w * n
        out["x0"] = d
    return out


def pradmm_adjoint_device(h, p_bar_ptr, t_bar_ptr, q_meas_bar_ptr, t_meas_bar_ptr, kappa_bar_ptr, omega_bar_ptr,
                          x0_bar_ptr=0):
    args = [ctypes.c_void_p(x or 0) for x in (p_bar_ptr, t_bar_ptr, q_meas_bar_ptr, t_meas_bar_ptr, kappa_bar_ptr,
                                              omega_bar_ptr, x0_bar_ptr)]
    _check(load().pradmm_adjoint_device(h, *args), "pradmm_adjoint_device")


def pradmm_objective_noalloc(n, m, src_ptr, dst_ptr, q_meas_ptr, t_meas_ptr, kappa_ptr, omega_ptr, q_ptr, t_ptr,
                             F_ptr, stream=None):
    """F of Eq. (1) from device arrays into the device double at F_ptr, with no
    allocation (for callers that cannot allocate device memory at that point;
    see pradmm.h).  Pointers are raw device addresses (e.g. tensor.data_ptr());
    kappa_ptr / omega_ptr may be 0 for unit weights."""
    args = [ctypes.c_void_p(x or 0) for x in (src_ptr, dst_ptr, q_meas_ptr, t_meas_ptr, kappa_ptr, omega_ptr, q_ptr,
                                              t_ptr, F_ptr, stream)]
    _check(load().pradmm_objective_noalloc(int(n), int(m), *args), "pradmm_objective_noalloc")


def pradmm_destroy(h):
    if h:
        load().pradmm_destroy(h)


def pradmm_status_string(st: int) -> str:
    return load().pradmm_status_string(int(st)).decode()


# ---- convenience object ------------------------------------------------------------

class Solver:
    """Owns one handle for a `synth.PoseGraph`-like object (fields n, src, dst,
    q_meas, t_meas, kappa, omega)."""

    def __init__(self, graph, params: pradmm_params | None = None, stream=None, **overrides):
        prm = params if params is not None else pradmm_default_params()
        for k, v in overrides.items():
            if k == "gamma":
                for i in range(4):
                    prm.gamma[i] = v[i]
            else:
                setattr(prm, k, v)
        self.params = prm
        self.n = int(graph.n)
        self.m = int(len(graph.src))
        self.h = pradmm_create(graph.n, graph.src, graph.dst, graph.q_meas, graph.t_meas, graph.kappa, graph.omega,
                               prm, stream)

    def close(self):
        if self.h:
            pradmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, q, t):
        pradmm_set_state(self.h, q, t, self.n)

    def set_state_full(self, st):
        pradmm_set_state_full(self.h, st, self.n)

    def set_state_device(self, p, q, t, s, lam=None, z=None):
        """Full state from CUDA float64 tensors (n x 4 for p, q, lam; n x 3 for
        t, s, z; contiguous); the caller's stream must have finished writing them."""
        def ptr(x, width, name, optional=False):
            if x is None and optional:
                return 0
            if (x is None or not x.is_cuda or x.dtype.itemsize != 8 or not x.dtype.is_floating_point
                    or not x.is_contiguous() or tuple(x.shape) != (self.n, width)):
                raise ValueError(f"{name}: need a contiguous CUDA float64 tensor of shape ({self.n}, {width})")
            return x.data_ptr()
        pradmm_set_state_full_device(self.h, ptr(p, 4, "p"), ptr(q, 4, "q"), ptr(t, 3, "t"), ptr(s, 3, "s"),
                                     ptr(lam, 4, "lam", True), ptr(z, 3, "z", True))

    def init_odometry(self):
        pradmm_init_odometry(self.h)

    def odometry_forest(self):
        """(parent, tree-edge code) per vertex of the odometry start's forest."""
        return pradmm_odometry_forest(self.h, self.n)

    def autotune(self, iters=20):
        return pradmm_autotune(self.h, iters)

    def step(self, iters=1):
        return pradmm_step(self.h, iters)

    def solve(self):
        return pradmm_solve(self.h)

    def objective(self):
        return pradmm_objective(self.h)

    def state(self):
        return pradmm_get_state(self.h, self.n)

    def poses(self):
        return pradmm_get_poses(self.h, self.n)

    def set_sigma(self, Sigma1=None, Sigma2=None):
        pradmm_set_sigma(self.h, Sigma1, Sigma2)

    def adjoint_record(self, iters, ckpt_every=0):
        pradmm_adjoint_record(self.h, iters, ckpt_every)

    def adjoint_tape_info(self):
        return pradmm_adjoint_tape_info(self.h)

    def adjoint(self, p_bar=None, t_bar=None, x0=False):
        return pradmm_adjoint(self.h, self.n, self.m, p_bar, t_bar, x0)

    def iterations(self):
        return pradmm_iterations(self.h)

    def set_trace(self, capacity):
        self._trace_cap = int(capacity)
        pradmm_set_trace(self.h, capacity)

    def trace(self):
        return pradmm_get_trace(self.h, getattr(self, "_trace_cap", 1))

    def counters(self):
        return pradmm_counters(self.h)

    def bytes_per_iteration(self):
        return pradmm_bytes_per_iteration(self.h)

    def profile(self, iters):
        return pradmm_profile_sweeps(self.h, iters)


# ---- batched solver ---------------------------------------------------------------

class Batch:
    """Many independent graphs (a list of synth.PoseGraph-like objects) solved
    together by the batched entry points of pradmm.h."""

    def __init__(self, graphs, params: pradmm_params | None = None, stream=None, **overrides):
        lib = load()
        prm = params if params is not None else pradmm_default_params()
        for k, v in overrides.items():
            if k == "gamma":
                for i in range(4):
                    prm.gamma[i] = v[i]
            else:
                setattr(prm, k, v)
        self.params = prm
        self.G = len(graphs)
        self.n_g = np.array([g.n for g in graphs], dtype=np.int64)
        self.m_g = np.array([g.m for g in graphs], dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.n_g)])
        self.N = int(self.offsets[-1])
        src = np.ascontiguousarray(np.concatenate([g.src for g in graphs]), dtype=np.int32)
        dst = np.ascontiguousarray(np.concatenate([g.dst for g in graphs]), dtype=np.int32)
        qm = _f64(np.concatenate([g.q_meas for g in graphs]))
        tm = _f64(np.concatenate([g.t_meas for g in graphs]))
        ka = _f64(np.concatenate([g.kappa for g in graphs]))
        om = _f64(np.concatenate([g.omega for g in graphs]))
        h = ctypes.c_void_p()
        st = lib.pradmm_batch_create(self.G, self.n_g.ctypes.data_as(_i64), self.m_g.ctypes.data_as(_i64),
                                     src.ctypes.data_as(_i32), dst.ctypes.data_as(_i32), _dp(qm), _dp(tm), _dp(ka),
                                     _dp(om), ctypes.byref(prm), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        _check(st, "pradmm_batch_create")
        self.h = h.value

    def close(self):
        if self.h:
            load().pradmm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_schedule(self, block, warp_max_n, cluster=1, cluster_min_n=0):
        _check(load().pradmm_batch_set_schedule(self.h, int(block), int(warp_max_n), int(cluster), int(cluster_min_n)),
               "pradmm_batch_set_schedule")

    def schedule(self):
        """(block, warp_max_n, cluster, cluster_min_n)"""
        v = [ctypes.c_int32(0) for _ in range(4)]
        _check(load().pradmm_batch_get_schedule(self.h, *[ctypes.byref(x) for x in v]), "pradmm_batch_get_schedule")
        return tuple(x.value for x in v)

    def autotune(self, iters=20):
        """Returns the chosen (block, warp_max_n, cluster, cluster_min_n)."""
        v = [ctypes.c_int32(0) for _ in range(4)]
        _check(load().pradmm_batch_autotune(self.h, int(iters), *[ctypes.byref(x) for x in v]),
               "pradmm_batch_autotune")
        return tuple(x.value for x in v)

    def autotune_profiled(self, work_fraction=0.05):
        """Schedule search on probes that run each graph for work_fraction of its
        iterations in the last solve; returns (block, warp_max_n, cluster, cluster_min_n)."""
        v = [ctypes.c_int32(0) for _ in range(4)]
        _check(load().pradmm_batch_autotune_profiled(self.h, float(work_fraction), *[ctypes.byref(x) for x in v]),
               "pradmm_batch_autotune_profiled")
        return tuple(x.value for x in v)

    def init_odometry(self):
        _check(load().pradmm_batch_init_odometry(self.h), "pradmm_batch_init_odometry")

    def set_sigma(self, Sigma1=None, Sigma2=None):
        """General 4x4 weight matrices for every graph; both None: Sigma = I."""
        S1 = None if Sigma1 is None else _f64(Sigma1, (4, 4))
        S2 = None if Sigma2 is None else _f64(Sigma2, (4, 4))
        _check(load().pradmm_batch_set_sigma(self.h, _dp(S1), _dp(S2)), "pradmm_batch_set_sigma")

    def set_state(self, q, t):
        q, t = _f64(q, (self.N, 4)), _f64(t, (self.N, 3))
        _check(load().pradmm_batch_set_state(self.h, _dp(q), _dp(t)), "pradmm_batch_set_state")

    def solve(self, rel_tol=1e-6, max_iter=3000):
        """Returns dict of per-graph arrays: iters, e_first, e_last, status."""
        it = np.zeros(self.G, dtype=np.int32)
        e1 = np.zeros(self.G)
        ek = np.zeros(self.G)
        stt = np.zeros(self.G, dtype=np.int32)
        st = load().pradmm_batch_solve(self.h, float(rel_tol), int(max_iter), it.ctypes.data_as(_i32), _dp(e1),
                                       _dp(ek), stt.ctypes.data_as(_i32))
        if st not in (PRADMM_OK, PRADMM_ERR_NOT_CONVERGED):
            _check(st, "pradmm_batch_solve")
        return {"iters": it, "e_first": e1, "e_last": ek, "status": stt, "all_converged": st == PRADMM_OK}

    def objectives(self):
        F = np.zeros(self.G)
        _check(load().pradmm_batch_objectives(self.h, _dp(F)), "pradmm_batch_objectives")
        return F

    def spans(self):
        """(G, 2) uint64: device start / end time (ns) of each graph in the last solve."""
        out = np.zeros((self.G, 2), dtype=np.uint64)
        _check(load().pradmm_batch_spans(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))),
               "pradmm_batch_spans")
        return out

    def state(self):
        N = self.N
        out = {"p": np.zeros((N, 4)), "q": np.zeros((N, 4)), "t": np.zeros((N, 3)), "s": np.zeros((N, 3)),
               "lam": np.zeros((N, 4)), "z": np.zeros((N, 3))}
        _check(load().pradmm_batch_get_state(self.h, _dp(out["p"]), _dp(out["q"]), _dp(out["t"]), _dp(out["s"]),
                                             _dp(out["lam"]), _dp(out["z"])), "pradmm_batch_get_state")
        return out



# ---- torch autograd wrapper of the reverse mode ---------------------------------------

class _Handle:
    """Destroys its handle when the autograd graph that holds it is freed."""

    def __init__(self, h):
        self.h = h

    def __del__(self):
        try:
            pradmm_destroy(self.h)
        except Exception:
            pass


def unrolled_poses(n, src, dst, q_meas, t_meas, kappa=None, omega=None, iters=200, ckpt_every=0, params=None,
                   init=None):
    """(p^K, t^K) after `iters` iterations of Algorithm 1, differentiable with
    respect to q_meas (m x 4), t_meas (m x 3), kappa (m), omega (m): CUDA
    float64 tensors; src, dst CUDA int32 tensors.  The start is the odometry
    initialisation (init=None) or init=(q0, t0) host arrays, held fixed.
    ckpt_every: checkpoint spacing of the tape (0: chosen from the free device
    memory, every iterate kept where it fits).  Forward and backward run in libpradmm's kernels on torch's current stream
    (pradmm_adjoint_record / pradmm_adjoint_device)."""
    import torch

    class _Unrolled(torch.autograd.Function):
        @staticmethod
        def forward(ctx, qm, tm, ka, om):
            m = int(qm.shape[0])
            stream = torch.cuda.current_stream(qm.device).cuda_stream
            h = pradmm_create_device(n, m, src.data_ptr(), dst.data_ptr(), qm.data_ptr(), tm.data_ptr(),
                                     ka.data_ptr(), om.data_ptr(), params, stream)
            hold = _Handle(h)
            if init is None:
                pradmm_init_odometry(h)
            else:
                pradmm_set_state(h, init[0], init[1], n)
            pradmm_adjoint_record(h, iters, ckpt_every)
            p = torch.empty((n, 4), dtype=torch.float64, device=qm.device)
            t = torch.empty((n, 3), dtype=torch.float64, device=qm.device)
            pradmm_get_state_device(h, p=p.data_ptr(), t=t.data_ptr())
            ctx.hold = hold
            ctx.m = m
            return p, t

        @staticmethod
        def backward(ctx, gp, gt):
            dev = gp.device if gp is not None else gt.device
            gp = None if gp is None else gp.contiguous().to(torch.float64)
            gt = None if gt is None else gt.contiguous().to(torch.float64)
            m = ctx.m
            dq = torch.empty((m, 4), dtype=torch.float64, device=dev)
            dt = torch.empty((m, 3), dtype=torch.float64, device=dev)
            dk = torch.empty((m,), dtype=torch.float64, device=dev)
            do = torch.empty((m,), dtype=torch.float64, device=dev)
            pradmm_adjoint_device(ctx.hold.h, 0 if gp is None else gp.data_ptr(), 0 if gt is None else gt.data_ptr(),
                                  dq.data_ptr(), dt.data_ptr(), dk.data_ptr(), do.data_ptr())
            return dq, dt, dk, do

    m = int(q_meas.shape[0])
    ones = None
    if kappa is None or omega is None:
        ones = torch.ones(m, dtype=torch.float64, device=q_meas.device)
    return _Unrolled.apply(q_meas.contiguous(), t_meas.contiguous(), ones if kappa is None else kappa.contiguous(),
                           ones if omega is None else omega.contiguous())
