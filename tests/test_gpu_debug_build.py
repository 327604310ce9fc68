"""The index-checked build (libpradmm_debug.so): the plain sweeps with every
neighbour index and CSR row bound range-checked on the device.  In a child
process that loads that library: a clean run agrees with the FP64 oracle
(the checks find nothing), and a neighbour index planted one past the end of
the vertex range is caught, replaced in bounds and reported as
PRADMM_ERR_INDEX; the release library refuses to plant."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle
from paper_2601_15684_gb300 import build_lib, pradmm as P, synth
P.load(build_lib.LIB_DEBUG)
g = synth.random_graph(2000, 7000, seed=12, isolated=3)
st0 = synth.random_state(np.random.default_rng(1), g.n)
prm = P.pradmm_default_params()
prm.precision = P.PRADMM_FP64
prm.beta1, prm.beta2, prm.relax = 1.0, 1.0, 1.5
with P.Solver(g, prm) as S:
    S.set_state_full(st0)
    S.step(10)
    gpu = S.state()
orc, _, _ = oracle.iterate(g, oracle.make_params(beta1=1.0, beta2=1.0, tau=1.5), st0, 10)
for k in ("p", "q", "t", "s", "lam", "z"):
    e = np.linalg.norm(gpu[k] - orc[k]) / np.linalg.norm(orc[k])
    assert e <= 1e-10, (k, e)
with P.Solver(g, prm) as S:
    S.set_state_full(st0)
    P.pradmm_debug_set_neighbour(S.h, 123, g.n)
    try:
        S.step(2)
        raise SystemExit("planted index not reported")
    except P.PRADMMError as ex:
        assert ex.status == P.PRADMM_ERR_INDEX, ex
        assert "out of range" in str(ex) and str(g.n) in str(ex), str(ex)
print("debug build ok")
'''


def test_index_checked_build_runs_clean_and_catches_a_planted_index():
    from paper_2601_15684_gb300 import build_lib
    build_lib.build(debug=True)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                       text=True, timeout=600)
    assert r.returncode == 0 and "debug build ok" in r.stdout, r.stdout[-3000:]


def test_release_build_refuses_to_plant():
    from paper_2601_15684_gb300 import build_lib
    from paper_2601_15684_gb300 import pradmm as P
    from paper_2601_15684_gb300 import synth
    build_lib.build()
    P.load()
    g = synth.random_graph(50, 150, seed=1)
    with P.Solver(g) as S:
        with pytest.raises(P.PRADMMError) as ei:
            P.pradmm_debug_set_neighbour(S.h, 0, 3)
        assert ei.value.status == P.PRADMM_ERR_STATE
