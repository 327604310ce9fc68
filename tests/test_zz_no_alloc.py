"""The allocation-free objective entry point (pradmm_objective_noalloc).

Some callers cannot allocate device memory when they need the objective --
for example a process that reserves all of its GPU memory up front and
forbids allocation afterwards -- so they cannot create a handle.  These
tests call the allocation-free entry point through the C ABI, twice in a
row on the same device, and check it against the handle-based
pradmm_objective and the FP64 oracle's Eq. (1) on the same poses; at the
1M-pose lattice's 2,580,580 edges (about 2,500 chunk partials of the 4,096
the static scratch holds), check that a call after the first allocates no
device memory, and that an out-of-range endpoint gives NaN without reading
any pose.  The file is collected last.
"""
import numpy as np
import pytest

import oracle
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


class _Edges:
    def __init__(self, torch, g):
        self.src = _dev(torch, g.src, torch.int32)
        self.dst = _dev(torch, g.dst, torch.int32)
        self.qm = _dev(torch, g.q_meas, torch.float64)
        self.tm = _dev(torch, g.t_meas, torch.float64)
        self.ka = _dev(torch, g.kappa, torch.float64)
        self.om = _dev(torch, g.omega, torch.float64)


def _call(P, torch, g, E, qd, td, F_dev, m=None, src=None):
    F_dev.fill_(-1.0)
    P.pradmm_objective_noalloc(g.n, g.m if m is None else m, (src if src is not None else E.src).data_ptr(),
                               E.dst.data_ptr(), E.qm.data_ptr(), E.tm.data_ptr(), E.ka.data_ptr(),
                               E.om.data_ptr(), qd.data_ptr(), td.data_ptr(), F_dev.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return float(F_dev.item())


def test_noalloc_objective_matches_handle_objective_and_oracle(P):
    import torch

    g = synth.helix_graph(n=3000)
    rng = np.random.default_rng(0)
    states = [(g.q_gt, g.t_gt),
              (synth._qmul(g.q_gt, synth.axis_angle_noise(rng, g.n, 0.1)), g.t_gt + rng.standard_normal((g.n, 3)))]
    prm = P.pradmm_default_params()
    prm.precision = P.PRADMM_FP64
    E = _Edges(torch, g)
    F_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    with P.Solver(g, prm) as S:
        for q0, t0 in states:  # two calls in a row share the static scratch
            S.set_state(q0, t0)
            F_ref = S.objective()
            F_orc = oracle.objective(g, q0, t0)
            F = _call(P, torch, g, E, _dev(torch, q0, torch.float64), _dev(torch, t0, torch.float64), F_dev)
            assert abs(F - F_ref) <= 1e-10 * max(abs(F_ref), 1e-300), (F, F_ref)
            assert abs(F - F_orc) <= 1e-10 * max(abs(F_orc), 1e-300), (F, F_orc)


def test_noalloc_objective_at_lattice_size_allocates_nothing(P):
    # 2,580,580 edges: 2,521 chunk partials, summed by the last CTA
    import torch

    g = synth.workload("lattice1m")
    rng = np.random.default_rng(1)
    q1 = synth._qmul(g.q_gt, synth.axis_angle_noise(rng, g.n, 0.05))
    t1 = g.t_gt + 0.3 * rng.standard_normal((g.n, 3))
    E = _Edges(torch, g)
    F_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    poses = [(_dev(torch, g.q_gt, torch.float64), _dev(torch, g.t_gt, torch.float64)),
             (_dev(torch, q1, torch.float64), _dev(torch, t1, torch.float64))]
    F_orc = [oracle.objective(g, g.q_gt, g.t_gt), oracle.objective(g, q1, t1)]
    _call(P, torch, g, E, *poses[0], F_dev)  # the first call on this device: start-up
    free0, _ = torch.cuda.mem_get_info()
    for k in (1, 0, 1):
        F = _call(P, torch, g, E, *poses[k], F_dev)
        assert abs(F - F_orc[k]) <= 1e-10 * F_orc[k], (k, F, F_orc[k])
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_out_of_range_endpoint_gives_nan(P):
    import torch

    g = synth.random_graph(500, 3000, seed=3)
    E = _Edges(torch, g)
    q0 = synth.random_unit_quaternions(np.random.default_rng(2), g.n)
    t0 = np.random.default_rng(3).standard_normal((g.n, 3))
    qd, td = _dev(torch, q0, torch.float64), _dev(torch, t0, torch.float64)
    F_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    F_orc = oracle.objective(g, q0, t0)
    for bad in (g.n, -1, 2 ** 31 - 1):
        src = g.src.copy()
        src[1234] = bad
        F = _call(P, torch, g, E, qd, td, F_dev, src=_dev(torch, src, torch.int32))
        assert np.isnan(F), (bad, F)
        # the next call rewrites every partial it reads: no NaN left behind
        F = _call(P, torch, g, E, qd, td, F_dev)
        assert abs(F - F_orc) <= 1e-10 * F_orc, (F, F_orc)


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    import torch

    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    i = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PRADMMError) as ei:
        P.pradmm_objective_noalloc(2, 4 * 1024 * 1024 + 1, i.data_ptr(), i.data_ptr(), x.data_ptr(), x.data_ptr(),
                                   0, 0, x.data_ptr(), x.data_ptr(), x.data_ptr())
    assert ei.value.status == P.PRADMM_ERR_ARG
    assert "scratch" in ei.value.message
