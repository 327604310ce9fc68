"""Element-wise comparison of a state against the FP64 oracle.

For every vertex i and state array X the per-element error is

    err_i(X) = |X_gpu,i - X_orc,i| / max(|X_orc,i|, scale_X,i)

(|.| the Euclidean norm of the vertex's row), and a check asserts the
maximum over vertices.  The floor scale_X,i keeps an entry whose own value
is near zero from demanding more than its inputs can give:

- p, q (unit quaternions, and q near unit length): 1;
- t, s (positions): the translation magnitude of the graph, the root mean
  square of the oracle's |t_i|; a position near the origin is formed from
  neighbours that far apart, so its FP32 rounding is of that size;
- lam: tau*beta1 (|p_i| + |q_i|), the size of the terms tau*beta1 (p - q)
  it accumulates;
- z: tau*beta2 (|t_i| + |s_i|), floored by tau*beta2 times the
  translation magnitude for the same reason as t.

The per-array relative error |X_gpu - X_orc|_2 / |X_orc|_2 is reported
beside it; a localized mistake (one vertex's wrong CSR slot, a race on a
few vertices) shows in the per-element maximum where the per-array norm
over a million vertices hides it.
"""
import numpy as np

STATE_KEYS = ("p", "q", "t", "s", "lam", "z")


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def translation_scale(orc):
    t = np.asarray(orc["t"])
    if t.size == 0:
        return 1.0
    return max(float(np.sqrt(np.mean(np.sum(t * t, axis=1)))), 1e-300)


def element_errors(gpu, orc, tau=1.5, beta1=1.0, beta2=1.0, keys=STATE_KEYS):
    """{key: per-vertex error array} with the floors above."""
    rn = lambda a: np.linalg.norm(np.asarray(a, dtype=np.float64), axis=1)
    ts = translation_scale(orc)
    floors = {
        "p": np.ones(len(orc["p"])),
        "q": np.ones(len(orc["q"])),
        "t": np.full(len(orc["t"]), ts),
        "s": np.full(len(orc["s"]), ts),
    }
    if "lam" in orc:
        floors["lam"] = tau * beta1 * (rn(orc["p"]) + rn(orc["q"]))
    if "z" in orc:
        floors["z"] = tau * beta2 * np.maximum(rn(orc["t"]) + rn(orc["s"]), ts)
    out = {}
    for k in keys:
        if k not in orc:
            continue
        d = rn(np.asarray(gpu[k]) - np.asarray(orc[k]))
        out[k] = d / np.maximum(rn(orc[k]), floors[k])
    return out


def max_element_errors(gpu, orc, **kw):
    return {k: (float(v.max()) if v.size else 0.0) for k, v in element_errors(gpu, orc, **kw).items()}


def check_elements(gpu, orc, tol, what="", tau=1.5, beta1=1.0, beta2=1.0, keys=STATE_KEYS, verbose=True):
    """Assert max_i err_i(X) <= tol for every array; returns the maxima."""
    errs = element_errors(gpu, orc, tau=tau, beta1=beta1, beta2=beta2, keys=keys)
    mx = {}
    for k, v in errs.items():
        m = float(v.max()) if v.size else 0.0
        mx[k] = m
        if verbose:
            arg = int(np.argmax(v)) if v.size else -1
            print(f"{what}: {k}: max element error {m:.3e} (vertex {arg}), array relerr {relerr(gpu[k], orc[k]):.3e}")
    for k, m in mx.items():
        assert m <= tol, (what, k, m, tol)
    return mx


# Per-element bounds against the FP64 oracle.
# FP64: rounding-order differences only (1 and 10 iterations).
# FP32: every element within ELEM_FLOOR_FP32 of its scale, within
# ELEM_FACTOR_FP32 times the deviation d_i of an FP32 reference run from the
# same start (the largest of the references given), or within
# ELEM_SPREAD_FP32 times the root mean square of d over the vertices,
# whichever is largest (the last term grows with the iterations as the
# typical FP32 deviation does; two FP32 executions that round in different
# orders leave errors of that size at vertices where one of them happens to
# stay small).  The
# references are the checker's own algorithm executed in single precision
# (oracle.iterate_f32) and, where that build does not cover a form, the FP64
# oracle with its state stored in FP32 (fp32_storage_run).  A vertex whose
# update is ill conditioned amplifies FP32 rounding by itself; no FP32
# implementation can be held closer to the FP64 iterates there than an FP32
# execution of the same iteration gets.
ELEM_TOL_FP64 = 1e-10
ELEM_FLOOR_FP32 = 1e-4
ELEM_FACTOR_FP32 = 32.0
ELEM_SPREAD_FP32 = 32.0


def to_fp32(st):
    """A state rounded to FP32 (and held in double)."""
    return {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in st.items()}


def fp32_storage_run(step, st0, iters):
    """The oracle's iterates with the state stored in FP32: starting from
    to_fp32(st0), each iteration runs the FP64 oracle step and rounds its
    result to FP32.  step(state) -> state after one iteration."""
    st = to_fp32(st0)
    for _ in range(iters):
        st = to_fp32(step(st))
    return st


def check_elements_fp32(gpu, orc, refs, what="", tau=1.5, beta1=1.0, beta2=1.0, keys=STATE_KEYS,
                        floor=ELEM_FLOOR_FP32, factor=ELEM_FACTOR_FP32, spread=ELEM_SPREAD_FP32):
    """FP32 per-element rule: err_i(gpu) <= max(floor, factor * d_i,
    spread * rms(d)) with d_i = max_r err_i(r) over the FP32 references r (a
    state or a list of states), every vertex and array, errors against the
    FP64 oracle orc."""
    if isinstance(refs, dict):
        refs = [refs]
    eg = element_errors(gpu, orc, tau=tau, beta1=beta1, beta2=beta2, keys=keys)
    er = [element_errors(r, orc, tau=tau, beta1=beta1, beta2=beta2, keys=keys) for r in refs]
    worst = {}
    for k in eg:
        if eg[k].size == 0:
            continue
        d = np.max(np.stack([e[k] for e in er]), axis=0)
        bound = np.maximum(max(floor, spread * float(np.sqrt(np.mean(d * d)))), factor * d)
        r = eg[k] / bound
        i = int(np.argmax(r))
        worst[k] = float(r[i])
        print(f"{what}: {k}: max element error {eg[k].max():.3e} (FP32 reference {d.max():.3e}); "
              f"worst error / bound {r[i]:.3f} at vertex {i} ({eg[k][i]:.3e} vs {bound[i]:.3e}); "
              f"array relerr {relerr(gpu[k], orc[k]):.3e}")
    for k, r in worst.items():
        assert r <= 1.0, (what, k, r)
    return worst
