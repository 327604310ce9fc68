"""FP64 CPU oracle for PRADMM (arXiv 2601.15684) -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library and the library
never calls it.

`pradmm_oracle.c` holds the iteration itself (Section 3.2 Eq. (3),
Algorithm 1, Appendix B closed forms, Appendix E.1 residual) as plain double
precision loops; this module only loads it and marshals numpy arrays.
`matrix_form.py` is a second, independent statement of the same iteration
built from the literal 4x4 matrices M(.), W(.), D of Appendix A.2/B.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pradmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("tau", ctypes.c_double),
                ("gamma", ctypes.c_double * 4)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lib_omp = None
_SRC_F32 = os.path.join(_HERE, "pradmm_oracle_f32.c")
_SO_F32 = os.path.join(_BUILD, "liboracle_f32.so")
_lib_f32 = None


class Params32(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("tau", ctypes.c_float),
                ("gamma", ctypes.c_float * 4)]


def build_f32(force: bool = False) -> str:
    """The checker's source with its real type set to float: a tolerance
    reference (pradmm_oracle_f32.c), never the checker."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_F32))
    if force or not os.path.exists(_SO_F32) or os.path.getmtime(_SO_F32) < newest:
        tmp = _SO_F32 + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                               "-fsingle-precision-constant", "-o", tmp, _SRC_F32, "-lm"])
        os.replace(tmp, _SO_F32)
    return _SO_F32


def lib_f32():
    global _lib_f32
    with _lock:
        if _lib_f32 is None:
            build_f32()
            L = ctypes.CDLL(_SO_F32)
            P = ctypes.POINTER
            f, i32, i64 = P(ctypes.c_float), P(ctypes.c_int32), ctypes.c_int64
            L.orc_iterate.restype = ctypes.c_int64
            L.orc_iterate.argtypes = [i64, i64, i32, i32, f, f, f, f, P(Params32), f, f, f, f, f, f, f]
            L.orc_iterate_inertial.restype = ctypes.c_int64
            L.orc_iterate_inertial.argtypes = [i64, i64, i32, i32, f, f, f, f, P(Params32), ctypes.c_float,
                                               f, f, f, f, f, f, f, f, f, f, f]
            _lib_f32 = L
    return _lib_f32


def _params32(p: Params) -> Params32:
    q = Params32()
    q.beta1, q.beta2, q.tau = p.beta1, p.beta2, p.tau
    for k in range(4):
        q.gamma[k] = p.gamma[k]
    return q


_KEYS = ("p", "q", "t", "s", "lam", "z")


def iterate_f32(g, params: Params, state: dict, iters: int = 1):
    """`iters` iterations of the oracle executed in single precision from the
    state rounded to FP32; returns the state as float64 arrays."""
    f = ctypes.POINTER(ctypes.c_float)
    a = [np.ascontiguousarray(x, dtype=np.float32) for x in (g.q_meas, g.t_meas, g.kappa, g.omega)]
    src = np.ascontiguousarray(g.src, dtype=np.int32)
    dst = np.ascontiguousarray(g.dst, dtype=np.int32)
    st = {k: np.array(state[k], dtype=np.float32) for k in _KEYS}
    res = np.zeros(5, np.float32)
    p32 = _params32(params)
    F = lambda x: x.ctypes.data_as(f)
    L = lib_f32()
    for _ in range(iters):
        L.orc_iterate(g.n, src.shape[0], _i(src), _i(dst), *[F(x) for x in a], ctypes.byref(p32),
                      *[F(st[k]) for k in _KEYS], F(res))
    return {k: v.astype(np.float64) for k, v in st.items()}


def iterate_inertial_f32(g, params: Params, state: dict, theta: float, iters: int = 1, prev: dict | None = None):
    """The inertial iteration executed in single precision (state and x^{k-1}
    in FP32); returns (state, prev) as float64 arrays."""
    f = ctypes.POINTER(ctypes.c_float)
    a = [np.ascontiguousarray(x, dtype=np.float32) for x in (g.q_meas, g.t_meas, g.kappa, g.omega)]
    src = np.ascontiguousarray(g.src, dtype=np.int32)
    dst = np.ascontiguousarray(g.dst, dtype=np.int32)
    st = {k: np.array(state[k], dtype=np.float32) for k in _KEYS}
    pv = {k: np.array((prev if prev is not None else state)[k], dtype=np.float32) for k in ("p", "q", "t", "s")}
    res = np.zeros(5, np.float32)
    p32 = _params32(params)
    F = lambda x: x.ctypes.data_as(f)
    L = lib_f32()
    for _ in range(iters):
        L.orc_iterate_inertial(g.n, src.shape[0], _i(src), _i(dst), *[F(x) for x in a], ctypes.byref(p32),
                               ctypes.c_float(theta), *[F(st[k]) for k in _KEYS],
                               *[F(pv[k]) for k in ("p", "q", "t", "s")], F(res))
    return ({k: v.astype(np.float64) for k, v in st.items()}, {k: v.astype(np.float64) for k, v in pv.items()})


def build_omp(force: bool = False) -> str:
    """The OpenMP timing build: the same source with -DORC_OPENMP -fopenmp.
    A CPU baseline for the benchmark, never the checker."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < os.path.getmtime(_SRC):
        tmp = _SO_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                               "-fopenmp", "-DORC_OPENMP", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


def lib_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            build_omp()
            L = ctypes.CDLL(_SO_OMP)
            P = ctypes.POINTER
            d, i32, i64 = P(ctypes.c_double), P(ctypes.c_int32), ctypes.c_int64
            L.orc_iterate_omp.restype = ctypes.c_int64
            L.orc_iterate_omp.argtypes = [i64, i64, i32, i32, d, d, d, d, P(Params), P(ctypes.c_int64), i32,
                                          P(ctypes.c_int64), i32, d, d, d, d, d, d, d]
            L.orc_omp_threads.restype = ctypes.c_int
            L.orc_omp_threads.argtypes = []
            _lib_omp = L
    return _lib_omp


def omp_threads() -> int:
    """Threads the OpenMP timing build runs on (OMP_NUM_THREADS, else all cores)."""
    return int(lib_omp().orc_omp_threads())


def vertex_edges(g):
    """Each vertex's out-edges (tail i) and in-edges (head i) in input order:
    (out_ptr, out_eid, in_ptr, in_eid) for iterate_omp."""
    src = np.asarray(g.src, dtype=np.int64)
    dst = np.asarray(g.dst, dtype=np.int64)
    out_eid = np.argsort(src, kind="stable").astype(np.int32)
    in_eid = np.argsort(dst, kind="stable").astype(np.int32)
    out_ptr = np.zeros(g.n + 1, np.int64)
    in_ptr = np.zeros(g.n + 1, np.int64)
    np.cumsum(np.bincount(src, minlength=g.n), out=out_ptr[1:])
    np.cumsum(np.bincount(dst, minlength=g.n), out=in_ptr[1:])
    return out_ptr, out_eid, in_ptr, in_eid


def iterate_omp(g, params: Params, state: dict, iters: int = 1, edges=None):
    """`iters` iterations of the OpenMP timing build (state bitwise equal to
    iterate's; the residuals are summed in another order)."""
    keep, a = _graph_args(g)
    out_ptr, out_eid, in_ptr, in_eid = edges if edges is not None else vertex_edges(g)
    st = copy_state(state)
    res = np.zeros(5)
    trace = np.zeros(iters)
    pi = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    L = lib_omp()
    for k in range(iters):
        r = L.orc_iterate_omp(*a, ctypes.byref(params), pi(out_ptr), _i(out_eid), pi(in_ptr), _i(in_eid),
                              _d(st["p"]), _d(st["q"]), _d(st["t"]), _d(st["s"]), _d(st["lam"]), _d(st["z"]),
                              _d(res))
        if r < 0:
            raise MemoryError("oracle OpenMP iteration: allocation failed")
        trace[k] = res[0]
    return st, trace


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.POINTER
            d, i32, i64 = P(ctypes.c_double), P(ctypes.c_int32), ctypes.c_int64
            L.orc_iterate.restype = ctypes.c_int64
            L.orc_iterate.argtypes = [i64, i64, i32, i32, d, d, d, d, P(Params), d, d, d, d, d, d, d]
            L.orc_iterate_inertial.restype = ctypes.c_int64
            L.orc_iterate_inertial.argtypes = [i64, i64, i32, i32, d, d, d, d, P(Params), ctypes.c_double,
                                               d, d, d, d, d, d, d, d, d, d, d]
            L.orc_solve.restype = ctypes.c_int64
            L.orc_solve.argtypes = [i64, i64, i32, i32, d, d, d, d, P(Params), i64, ctypes.c_double,
                                    d, d, d, d, d, d, d, d]
            L.orc_objective.restype = ctypes.c_double
            L.orc_objective.argtypes = [i64, i64, i32, i32, d, d, d, d, d, d]
            L.orc_split_objective.restype = None
            L.orc_split_objective.argtypes = [i64, i64, i32, i32, d, d, d, d, d, d, d, d, d, d]
            L.orc_lagrangian.restype = ctypes.c_double
            L.orc_lagrangian.argtypes = [i64, i64, i32, i32, d, d, d, d, P(Params), d, d, d, d, d, d]
            L.orc_init_odometry.restype = ctypes.c_int
            L.orc_init_odometry.argtypes = [i64, i64, i32, i32, d, d, d, d]
            L.orc_odometry_forest.restype = ctypes.c_int
            L.orc_odometry_forest.argtypes = [i64, i64, i32, i32, i32, i32]
            L.orc_adjoint.restype = ctypes.c_int
            L.orc_adjoint.argtypes = [i64, i64, i32, i32, d, d, d, d, P(Params), i64, d, d, d, d, d, d, d, d,
                                      d, d, d, d, d, d, d]
            L.orc_adjoint_inertial.restype = ctypes.c_int
            L.orc_adjoint_inertial.argtypes = [i64, i64, i32, i32, d, d, d, d, P(Params), ctypes.c_double, i64,
                                               d, d, d, d, d, d, d, d, d, d, d, d, d, d, d]
            L.orc_block.restype = ctypes.c_int64
            L.orc_block.argtypes = [ctypes.c_int, i64, i64, i32, i32, d, d, d, d, P(Params), d, d, d, d, d, d, d]
            L.orc_qmul.restype = None
            L.orc_qmul.argtypes = [d, d, d]
            L.orc_qrotate.restype = None
            L.orc_qrotate.argtypes = [d, d, d]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(beta1=10.0, beta2=10.0, tau=1.5, gamma=(1.0, 1e-3, 1e-3, 1e-3)) -> Params:
    p = Params()
    p.beta1, p.beta2, p.tau = beta1, beta2, tau
    for k in range(4):
        p.gamma[k] = gamma[k]
    return p


def _graph_args(g):
    src = np.ascontiguousarray(g.src, dtype=np.int32)
    dst = np.ascontiguousarray(g.dst, dtype=np.int32)
    qe = _f64(g.q_meas)
    te = _f64(g.t_meas)
    ka = _f64(g.kappa)
    om = _f64(g.omega)
    keep = (src, dst, qe, te, ka, om)
    return keep, (g.n, src.shape[0], _i(src), _i(dst), _d(qe), _d(te), _d(ka), _d(om))


def init_state(q0, t0):
    """Initial ADMM state of reading R8: p = q = q0, s = t = t0, multipliers zero."""
    q0, t0 = _f64(q0), _f64(t0)
    n = q0.shape[0]
    return {"p": q0.copy(), "q": q0.copy(), "t": t0.copy(), "s": t0.copy(),
            "lam": np.zeros((n, 4)), "z": np.zeros((n, 3))}


def copy_state(st):
    return {k: _f64(v).copy() for k, v in st.items()}


def init_odometry(g):
    keep, a = _graph_args(g)
    q = np.zeros((g.n, 4))
    t = np.zeros((g.n, 3))
    rc = lib().orc_init_odometry(*a[:6], _d(q), _d(t))
    if rc != 0:
        raise MemoryError("oracle init_odometry")
    return q, t


def odometry_forest(g):
    """The spanning forest of init_odometry: (parent, tree-edge code) per
    vertex, int32; parent -1 for a root; the code is e when the vertex is the
    head of its tree edge e, -(e + 2) when it is the tail, -1 for a root."""
    keep, a = _graph_args(g)
    par = np.zeros(g.n, dtype=np.int32)
    pedge = np.zeros(g.n, dtype=np.int32)
    if lib().orc_odometry_forest(*a[:4], _i(par), _i(pedge)) != 0:
        raise MemoryError("oracle odometry_forest")
    return par, pedge


def iterate(g, params: Params, state: dict, iters: int = 1):
    """Runs `iters` iterations of Algorithm 1 in place on a copy of `state`.
    Returns (new_state, residual parts [e, |dlam|^2, |dz|^2, |dq|^2, |dt|^2] of
    the last iteration, number of zero-|u| vertices over all iterations)."""
    st = copy_state(state)
    keep, a = _graph_args(g)
    res = np.zeros(5)
    nz = 0
    for _ in range(iters):
        r = lib().orc_iterate(*a, ctypes.byref(params), _d(st["p"]), _d(st["q"]), _d(st["t"]),
                              _d(st["s"]), _d(st["lam"]), _d(st["z"]), _d(res))
        if r < 0:
            raise MemoryError("oracle iterate")
        nz += int(r)
    return st, res.copy(), nz


def iterate_inertial(g, params: Params, state: dict, theta: float, iters: int = 1, prev: dict | None = None):
    """Inertial PRADMM (reading R27): `iters` iterations whose proximal anchors
    are x^k + theta (x^k - x^{k-1}) for x = p, q, t, s.  `prev` holds x^{k-1}
    (p, q, t, s); None means x^{-1} = x^0.  Returns (new_state, new_prev,
    residual parts of the last iteration, zero-|u| count)."""
    st = copy_state(state)
    pv = {k: st[k].copy() for k in ("p", "q", "t", "s")} if prev is None else copy_state(prev)
    keep, a = _graph_args(g)
    res = np.zeros(5)
    nz = 0
    for _ in range(iters):
        r = lib().orc_iterate_inertial(*a, ctypes.byref(params), float(theta), _d(st["p"]), _d(st["q"]),
                                       _d(st["t"]), _d(st["s"]), _d(st["lam"]), _d(st["z"]), _d(pv["p"]),
                                       _d(pv["q"]), _d(pv["t"]), _d(pv["s"]), _d(res))
        if r < 0:
            raise MemoryError("oracle iterate_inertial")
        nz += int(r)
    return st, pv, res.copy(), nz


BLOCKS = {"p": 0, "q": 1, "c": 2, "t": 3, "s": 4, "duals": 5}


def block(g, params: Params, state: dict, which: str, c):
    """One block of Algorithm 1 in place on `state` (arrays of float64,
    modified): "p", "q", "c" (c_e into c, m x 3), "t", "s", "duals".  Run in
    that order the blocks are one iteration of `iterate`, bitwise."""
    keep, a = _graph_args(g)
    r = lib().orc_block(BLOCKS[which], *a, ctypes.byref(params), _d(state["p"]), _d(state["q"]), _d(state["t"]),
                        _d(state["s"]), _d(state["lam"]), _d(state["z"]), _d(c))
    if r < 0:
        raise MemoryError("oracle block")
    return int(r)


def solve(g, params: Params, state: dict, max_iter: int, tol: float):
    st = copy_state(state)
    keep, a = _graph_args(g)
    e = np.zeros(1)
    trace = np.zeros(max(max_iter, 1))
    k = lib().orc_solve(*a, ctypes.byref(params), int(max_iter), float(tol), _d(st["p"]), _d(st["q"]),
                        _d(st["t"]), _d(st["s"]), _d(st["lam"]), _d(st["z"]), _d(e), _d(trace))
    return st, int(k), float(e[0]), trace[:k].copy()


def adjoint(g, params: Params, state: dict, iters: int, p_bar, t_bar):
    """Reverse-mode gradient of a loss L(p^K, t^K) through `iters` iterations
    of Algorithm 1 started at `state` (held fixed), given p_bar = dL/dp^K
    (n x 4) and t_bar = dL/dt^K (n x 3).  Returns a dict with the gradients
    with respect to the measurements ("q_meas" m x 4, "t_meas" m x 3,
    "kappa" m, "omega" m), the adjoint of the initial state ("x0": dict of
    p, q, t, s, lam, z) and the final "p", "t"."""
    n, m = g.n, g.m
    st = copy_state(state)
    keep, a = _graph_args(g)
    pb, tb = _f64(p_bar), _f64(t_bar)
    out = {"p": np.zeros((n, 4)), "t": np.zeros((n, 3)), "q_meas": np.zeros((m, 4)), "t_meas": np.zeros((m, 3)),
           "kappa": np.zeros(m), "omega": np.zeros(m)}
    x0 = np.zeros(21 * n)
    rc = lib().orc_adjoint(*a, ctypes.byref(params), int(iters), _d(st["p"]), _d(st["q"]), _d(st["t"]),
                           _d(st["s"]), _d(st["lam"]), _d(st["z"]), _d(pb), _d(tb), _d(out["p"]), _d(out["t"]),
                           _d(out["q_meas"]), _d(out["t_meas"]), _d(out["kappa"]), _d(out["omega"]), _d(x0))
    if rc != 0:
        raise MemoryError("oracle adjoint")
    sizes = (("p", 4), ("q", 4), ("t", 3), ("s", 3), ("lam", 4), ("z", 3))
    o, x0d = 0, {}
    for key, w in sizes:
        x0d[key] = x0[o:o + w * n].reshape(n, w)
        o += w * n
    out["x0"] = x0d
    return out


def adjoint_inertial(g, params: Params, state: dict, iters: int, theta: float, p_bar, t_bar):
    """adjoint() for the inertial iteration (reading R27) started with
    x^{-1} = x^0: the gradients of L(p^K, t^K) through `iters` inertial
    iterations with anchors x^k + theta (x^k - x^{k-1}).  Same outputs."""
    n, m = g.n, g.m
    st = copy_state(state)
    keep, a = _graph_args(g)
    pb, tb = _f64(p_bar), _f64(t_bar)
    out = {"p": np.zeros((n, 4)), "t": np.zeros((n, 3)), "q_meas": np.zeros((m, 4)), "t_meas": np.zeros((m, 3)),
           "kappa": np.zeros(m), "omega": np.zeros(m)}
    x0 = np.zeros(21 * n)
    rc = lib().orc_adjoint_inertial(*a, ctypes.byref(params), float(theta), int(iters), _d(st["p"]), _d(st["q"]),
                                    _d(st["t"]), _d(st["s"]), _d(st["lam"]), _d(st["z"]), _d(pb), _d(tb),
                                    _d(out["p"]), _d(out["t"]), _d(out["q_meas"]), _d(out["t_meas"]),
                                    _d(out["kappa"]), _d(out["omega"]), _d(x0))
    if rc != 0:
        raise MemoryError("oracle adjoint_inertial")
    sizes = (("p", 4), ("q", 4), ("t", 3), ("s", 3), ("lam", 4), ("z", 3))
    o, x0d = 0, {}
    for key, w in sizes:
        x0d[key] = x0[o:o + w * n].reshape(n, w)
        o += w * n
    out["x0"] = x0d
    return out


def objective(g, q, t) -> float:
    """Eq. (1) at (q, t)."""
    keep, a = _graph_args(g)
    q, t = _f64(q), _f64(t)
    return float(lib().orc_objective(*a, _d(q), _d(t)))


def split_objective(g, st) -> tuple[float, float]:
    keep, a = _graph_args(g)
    f = np.zeros(1)
    gg = np.zeros(1)
    s = copy_state(st)
    lib().orc_split_objective(*a, _d(s["p"]), _d(s["q"]), _d(s["t"]), _d(s["s"]), _d(f), _d(gg))
    return float(f[0]), float(gg[0])


def lagrangian(g, params: Params, st) -> float:
    keep, a = _graph_args(g)
    s = copy_state(st)
    return float(lib().orc_lagrangian(*a, ctypes.byref(params), _d(s["p"]), _d(s["q"]), _d(s["t"]),
                                      _d(s["s"]), _d(s["lam"]), _d(s["z"])))


def qmul(a, b):
    a, b = _f64(a), _f64(b)
    o = np.zeros(4)
    lib().orc_qmul(_d(a), _d(b), _d(o))
    return o


def qrotate(q, t):
    q, t = _f64(q), _f64(t)
    o = np.zeros(3)
    lib().orc_qrotate(_d(q), _d(t), _d(o))
    return o
