"""CPU checks of the C ABI library: it builds, loads without a GPU, exports
every function that include/ppmlr.h declares, the binding covers them all,
and argument errors are reported before any CUDA call.  Also checks that the
GPU library and the oracle share no code."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ppmlr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1607_02214_gb300 import build, ppmlr
    build.build()
    return ppmlr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ppmlr_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1607_02214_gb300 import ppmlr
    assert sorted(n for n, _, _ in ppmlr.SIGNATURES) == declared_functions()


def test_invalid_arguments_rejected_on_host(lib):
    from paper_1607_02214_gb300 import ppmlr
    out = ctypes.c_void_p(123)
    assert lib.ppmlr_create(None, 5 / 3, None, 0, None, ctypes.byref(out)) == ppmlr.PPMLR_E_INVALID
    assert out.value is None
    assert lib.ppmlr_step(None, 1.0) == ppmlr.PPMLR_E_INVALID
    assert lib.ppmlr_check(None) == ppmlr.PPMLR_E_INVALID
    assert lib.ppmlr_last_error(None) == b"null context"
    # bad grid (non-ascending edges) and bad gamma are rejected before CUDA is touched
    import numpy as np
    e = np.array([0.0, 1.0, 0.5])
    g = ppmlr.ppmlr_grid()
    for d in range(3):
        g.n[d] = 2
        g.edges[d] = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    bc = ppmlr.ppmlr_bc()
    assert lib.ppmlr_create(ctypes.byref(g), 5 / 3, ctypes.byref(bc), 0, None, ctypes.byref(out)) == 1
    ok = np.array([0.0, 0.5, 1.0])
    for d in range(3):
        g.edges[d] = ok.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.ppmlr_create(ctypes.byref(g), 1.0, ctypes.byref(bc), 0, None, ctypes.byref(out)) == 1
    bc.face[0][0] = 1  # outflow on one face, periodic on the other: invalid
    assert lib.ppmlr_create(ctypes.byref(g), 5 / 3, ctypes.byref(bc), 0, None, ctypes.byref(out)) == 1


def test_oracle_and_library_share_no_code():
    csrc = os.path.join(ROOT, "paper_1607_02214_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower() or f == "inputs.py" and "import oracle" not in txt, f
    otxt = open(os.path.join(ROOT, "oracle", "ppmlr_oracle.c")).read()
    assert "ppmlr.h" not in otxt and "csrc" not in otxt
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            assert "paper_1607_02214_gb300" not in open(os.path.join(ROOT, "oracle", f)).read()
