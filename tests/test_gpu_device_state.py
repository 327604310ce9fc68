"""State set and read through device pointers (pradmm_set_state_full_device,
pradmm_get_state_device) against the host-pointer calls: the same packing
kernels run on the same values, so the states agree bit for bit."""
import numpy as np
import pytest

from paper_2601_15684_gb300 import synth

pytestmark = pytest.mark.gpu
KEYS = ("p", "q", "t", "s", "lam", "z")


@pytest.fixture(scope="module")
def P():
    from paper_2601_15684_gb300 import build_lib
    from paper_2601_15684_gb300 import pradmm
    build_lib.build()
    pradmm.load()
    return pradmm


def _cuda(st):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to("cuda:0") for k, v in st.items()}


@pytest.mark.parametrize("precision", [0, 1])
def test_device_state_equals_host_state(P, precision):
    import torch
    g = synth.random_graph(333, 1000, seed=31, isolated=3)
    st = synth.random_state(np.random.default_rng(5), g.n)
    dev = _cuda(st)
    torch.cuda.synchronize()
    out = []
    for via_device in (False, True):
        with P.Solver(g, precision=precision, inertia=0.3) as S:
            if via_device:
                S.set_state_device(dev["p"], dev["q"], dev["t"], dev["s"], dev["lam"], dev["z"])
            else:
                S.set_state_full(st)
            a = S.state()
            S.step(5)
            out.append((a, S.state()))
    for k in KEYS:
        np.testing.assert_array_equal(out[0][0][k], out[1][0][k])
        np.testing.assert_array_equal(out[0][1][k], out[1][1][k])


def test_device_state_without_multipliers_is_set_state(P):
    import torch
    g = synth.random_graph(120, 400, seed=32)
    st = synth.random_state(np.random.default_rng(6), g.n)
    dev = _cuda(st)
    torch.cuda.synchronize()
    with P.Solver(g, precision=0) as S:
        S.set_state(st["q"], st["t"])
        a = S.state()
        S.set_state_device(dev["q"], dev["q"], dev["t"], dev["t"])
        b = S.state()
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k])
    assert not b["lam"].any() and not b["z"].any()


def test_get_state_device_round_trip(P):
    import torch
    g = synth.random_graph(250, 700, seed=33)
    st = synth.random_state(np.random.default_rng(7), g.n)
    with P.Solver(g, precision=1) as S:
        S.set_state_full(st)
        S.step(3)
        host = S.state()
        d = {k: torch.empty((g.n, 4 if k in ("p", "q", "lam") else 3), dtype=torch.float64, device="cuda:0")
             for k in KEYS}
        P.pradmm_get_state_device(S.h, **{k: d[k].data_ptr() for k in KEYS})
        torch.cuda.synchronize()
        for k in KEYS:
            np.testing.assert_array_equal(d[k].cpu().numpy(), host[k])
        with pytest.raises(ValueError):
            S.set_state_device(d["p"][:10], d["q"], d["t"], d["s"])
        with pytest.raises(ValueError):
            S.set_state_device(d["p"].float(), d["q"], d["t"], d["s"])


def test_create_from_device_arrays_equals_host_create(P):
    """pradmm_create_device copies the edge arrays device to device and runs
    the same validation and build: the odometry start and the iterates agree
    bit for bit with a handle created from the host arrays, and a bad edge
    gives the host path's status and message."""
    import torch
    g = synth.random_graph(2000, 7000, seed=41, isolated=5)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to("cuda:0")
         for k, v in (("src", g.src), ("dst", g.dst), ("q", g.q_meas), ("t", g.t_meas), ("k", g.kappa),
                      ("w", g.omega))}
    torch.cuda.synchronize()
    prm = P.pradmm_default_params()
    out = []
    for via_device in (False, True):
        if via_device:
            h = P.pradmm_create_device(g.n, g.m, d["src"].data_ptr(), d["dst"].data_ptr(), d["q"].data_ptr(),
                                       d["t"].data_ptr(), d["k"].data_ptr(), d["w"].data_ptr(), prm)
        else:
            h = P.pradmm_create(g.n, g.src, g.dst, g.q_meas, g.t_meas, g.kappa, g.omega, prm)
        try:
            P.pradmm_init_odometry(h)
            P.pradmm_step(h, 7)
            q = np.zeros((g.n, 4))
            t = np.zeros((g.n, 3))
            P.pradmm_get_poses(h, g.n, q, t)
            out.append((q, t))
        finally:
            P.pradmm_destroy(h)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    for e, v, code in ((4321, g.n, P.PRADMM_ERR_INDEX), (1234, "self", P.PRADMM_ERR_SELFLOOP)):
        dst = g.dst.copy()
        dst[e] = g.src[e] if v == "self" else v
        msgs = []
        for via_device in (False, True):
            with pytest.raises(P.PRADMMError) as ei:
                if via_device:
                    dd = torch.from_numpy(dst).to("cuda:0")
                    P.pradmm_create_device(g.n, g.m, d["src"].data_ptr(), dd.data_ptr(), d["q"].data_ptr(),
                                           d["t"].data_ptr(), d["k"].data_ptr(), d["w"].data_ptr(), prm)
                else:
                    P.pradmm_create(g.n, g.src, dst, g.q_meas, g.t_meas, g.kappa, g.omega, prm)
            assert ei.value.status == code
            msgs.append(ei.value.message)
        assert msgs[0] == msgs[1] and f"edge {e}" in msgs[0], msgs
