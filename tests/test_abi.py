"""The C ABI: the library builds, loads, and exports every function that
include/pradmm.h declares; host-only entry points work without a GPU; the
binding refuses to run without the library (no fallback path)."""
import ctypes
import os
import re

import pytest

from paper_2601_15684_gb300 import build_lib
from paper_2601_15684_gb300 import pradmm as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pradmm_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return P.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pradmm_create" in names and "pradmm_step" in names and "pradmm_solve" in names
    so = ctypes.CDLL(build_lib.LIB)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    for n in _declared():
        assert n in P._SIGS, n


def test_host_only_entry_points(lib):
    prm = P.pradmm_default_params()
    assert prm.beta1 == 1.0 and prm.beta2 == 1.0 and prm.relax == 1.5
    assert list(prm.gamma) == [1.0, 1e-3, 1e-3, 1e-3]
    assert prm.tol == 1e-4 and prm.max_iter == 300 and prm.precision == P.PRADMM_FP32
    assert P.pradmm_status_string(P.PRADMM_ERR_SELFLOOP) == "self-loop edge"
    assert ctypes.sizeof(P.pradmm_params) == 104 and prm.inertia == 0.0


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        P._lib_backup = P._lib
        try:
            P._lib = None
            P.load(str(tmp_path / "absent.so"))
        finally:
            P._lib = P._lib_backup


def test_header_is_plain_c():
    """No C++ or torch types cross the boundary."""
    txt = open(os.path.join(ROOT, "include", "pradmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    for bad in ("torch", "at::", "std::", "template", "cudaStream_t"):
        assert bad not in txt
