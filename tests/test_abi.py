"""The C-ABI library builds, loads and exports every function include/mpbjac.h declares
(no GPU needed: nothing is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            name = m.group(1)
            if name not in ("if", "while", "sizeof"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2407_15973_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("bjac_setup", "pcg_solve", "bjac_destroy", "bjac_last_error", "bjac_spmv", "bjac_apply",
               "bjac_residual", "bjac_export", "bjac_import_inverse", "bjac_info", "bjac_mlp_param_count"):
        assert fn in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_validation_without_gpu(libpath):
    # argument checks run on the host before any CUDA call
    from paper_2407_15973_gb300 import binding as B
    L = B.lib()
    out = ctypes.c_void_p()
    assert L.bjac_setup(None, None, 0, None, ctypes.byref(out)) == B.ERR_INVALID_ARG
    assert b"NULL" in L.bjac_last_error()
    csr = B.bjac_csr(0, 0, None, None, None)
    pol = B.bjac_policy()
    assert L.bjac_setup(ctypes.byref(csr), None, 1, ctypes.byref(pol), ctypes.byref(out)) == B.ERR_INVALID_ARG
    assert L.pcg_solve(None, None, None, 1e-10, 10, None, None) == B.ERR_INVALID_ARG
    assert L.bjac_mlp_param_count() == 5187 + 24
