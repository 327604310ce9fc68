"""The allocation-free objective entry point (pradmm_objective_noalloc).

Some callers cannot allocate device memory when they need the objective --
for example a process that reserves all of its GPU memory up front and
forbids allocation afterwards -- so they cannot create a handle.  This test
calls the allocation-free entry point through the C ABI, twice in a row on
the same device, and checks it against the handle-based pradmm_objective
on the same poses.  It lives in its own file that pytest collects last.
"""
import numpy as np
import pytest

from paper_2601_15684_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2601_15684_gb300 import build_lib
    from paper_2601_15684_gb300 import pradmm
    build_lib.build()
    pradmm.load()
    return pradmm


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def test_noalloc_objective_matches_handle_objective(P):
    import torch

    g = synth.helix_graph(n=3000)
    rng = np.random.default_rng(0)
    states = [(g.q_gt, g.t_gt),
              (synth._qmul(g.q_gt, synth.axis_angle_noise(rng, g.n, 0.1)), g.t_gt + rng.standard_normal((g.n, 3)))]
    prm = P.pradmm_default_params()
    prm.precision = P.PRADMM_FP64
    src = _dev(torch, g.src, torch.int32)
    dst = _dev(torch, g.dst, torch.int32)
    qm = _dev(torch, g.q_meas, torch.float64)
    tm = _dev(torch, g.t_meas, torch.float64)
    ka = _dev(torch, g.kappa, torch.float64)
    om = _dev(torch, g.omega, torch.float64)
    F_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with P.Solver(g, prm) as S:
        for q0, t0 in states:  # two calls in a row share the static scratch
            S.set_state(q0, t0)
            F_ref = S.objective()
            qd = _dev(torch, q0, torch.float64)
            td = _dev(torch, t0, torch.float64)
            F_dev.fill_(-1.0)
            P.pradmm_objective_noalloc(g.n, g.m, src.data_ptr(), dst.data_ptr(), qm.data_ptr(), tm.data_ptr(),
                                       ka.data_ptr(), om.data_ptr(), qd.data_ptr(), td.data_ptr(),
                                       F_dev.data_ptr(), stream)
            torch.cuda.synchronize()
            F = float(F_dev.item())
            assert abs(F - F_ref) <= 1e-10 * max(abs(F_ref), 1e-300), (F, F_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    import torch

    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    i = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PRADMMError) as ei:
        P.pradmm_objective_noalloc(2, 4 * 1024 * 1024 + 1, i.data_ptr(), i.data_ptr(), x.data_ptr(), x.data_ptr(),
                                   0, 0, x.data_ptr(), x.data_ptr(), x.data_ptr())
    assert ei.value.status == P.PRADMM_ERR_ARG
    assert "scratch" in ei.value.message
