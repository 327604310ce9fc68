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
