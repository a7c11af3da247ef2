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
    assert L.bjac_l2_residency(2) == B.ERR_INVALID_ARG
    assert L.bjac_batch_force_timeout(None, 1) == B.ERR_INVALID_ARG
    assert L.bjac_l2_residency(0) == 1 and L.bjac_l2_residency(1) == 0     # default on; restored


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a small C program compiled with gcc."""
    import subprocess
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpbjac.h"\nint main(void) {\n'
                   f'  printf("%zu\\n", sizeof({struct}));\n{body}  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("name", ["bjac_policy", "pcg_stats", "bjac_csr"])
def test_binding_structs_match_header(name, tmp_path):
    from paper_2407_15973_gb300 import binding as B
    cls = getattr(B, name)
    fields = [f for f, _ in cls._fields_]
    got = _c_layout(name, fields, tmp_path)
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in fields]


def test_invalid_spmv_format_rejected_on_host(libpath):
    # checked before any CUDA call: the (never dereferenced) device pointers may be fake
    from paper_2407_15973_gb300 import binding as B
    import numpy as np
    L = B.lib()
    csr = B.bjac_csr(64, 64, 16, 16, 16)
    bp = np.array([0, 32, 64], np.int32)
    pol = B.bjac_policy()
    pol.select, pol.spmv_format = B.SELECT_UNIFORM, 4
    out = ctypes.c_void_p()
    rc = L.bjac_setup(ctypes.byref(csr), bp.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(pol), ctypes.byref(out))
    assert rc == B.ERR_INVALID_ARG
    assert b"spmv_format" in L.bjac_last_error()
    pol.spmv_format, pol.flexible = 0, 2
    rc = L.bjac_setup(ctypes.byref(csr), bp.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(pol), ctypes.byref(out))
    assert rc == B.ERR_INVALID_ARG
    assert b"flexible" in L.bjac_last_error()
