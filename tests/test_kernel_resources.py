"""Register and spill budget of the PCG loop kernels, from ptxas's resource report (a CPU test:
nvcc cross-compiles for sm_103a without a GPU). The loop is bound by HBM and the FP64 pipe,
so these guard the occupancy the kernels were sized for."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess

import pytest

from paper_2407_15973_gb300 import build as BLD

pytestmark = pytest.mark.skipif(shutil.which(BLD.NVCC) is None, reason="nvcc not on PATH")

ENTRY = re.compile(r"Compiling entry function '([^']+)'")
SPILL = re.compile(r"(\d+) bytes spill stores, (\d+) bytes spill loads")
USED = re.compile(r"Used (\d+) registers")

# (pattern in the mangled name, most registers allowed): 6 CTAs of 256 threads per SM for the
# SELL-32 SpMV, 4 for the 16-bit register apply, 8 for the vector kernels
LOOP_KERNELS = [
    ("k_spmv_sellILi2E", 40),
    ("k_apply_regI13__nv_bfloat16Li32ELi3ELb0E", 64),
    ("k_apply_regI6__halfLi32ELi3ELb0E", 64),
    ("k_apply_mix32ILi3ELb0E", 80),
    ("k_apply_specI13__nv_bfloat16Li4ELb0E", 64),
    ("k_apply_specI6__halfLi4ELb0E", 64),
    ("k_update_xp", 32),
    ("k_update_r", 32),
    ("k_flex_beta", 32),
    ("k_mlp_tc", 128),      # the selector's tensor-core forward pass: 4 CTAs of 128 threads per SM
    ("k_mlp_grad_tc", 255),  # its tensor-core gradient: one CTA of 128 threads per SM, no spills
]
# kernels known to spill a few bytes: the binary32 register applies hold two 4 KB blocks per
# warp (k_apply_reg, and the speculative aMP apply, which also holds the binary64 path); the
# flexible register and speculative applies keep a third running sum at 64 registers
SPILL_ALLOWED = ("k_apply_regIfLi32E", "k_apply_specIf", "k_apply_specI13__nv_bfloat16Li4ELb1E",
                 "k_apply_specI6__halfLi4ELb1E", "k_apply_regI13__nv_bfloat16Li32ELi3ELb1E",
                 "k_apply_regI6__halfLi32ELi3ELb1E")


def _resources(src, tmp):
    cmd = [BLD.NVCC, "-Xptxas=-v", *BLD.ARCH, *BLD.FLAGS, "-c", os.path.join(BLD.CSRC, src), "-o",
           os.path.join(tmp, src + ".o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, name = {}, None
    for line in r.stderr.splitlines():
        m = ENTRY.search(line)
        if m:
            name = m.group(1)
            out[name] = {}
            continue
        if name is None:
            continue
        m = SPILL.search(line)
        if m:
            out[name]["spill"] = int(m.group(1)) + int(m.group(2))
        m = USED.search(line)
        if m:
            out[name]["regs"] = int(m.group(1))
    return out


@pytest.fixture(scope="module")
def resources(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("ptxas"))
    with cf.ThreadPoolExecutor(4) as ex:
        parts = list(ex.map(lambda s: _resources(s, tmp), ["sell.cu", "apply.cu", "update.cu", "mlp.cu", "mlp_grad_tc.cu"]))
    res = {}
    for p in parts:
        res.update(p)
    return res


@pytest.mark.parametrize("pattern,max_regs", LOOP_KERNELS)
def test_loop_kernel_fits_its_budget(resources, pattern, max_regs):
    hits = {k: v for k, v in resources.items() if pattern in k}
    assert hits, pattern
    for name, r in hits.items():
        assert r.get("spill", 0) == 0, (name, r)
        assert r["regs"] <= max_regs, (name, r)


def test_only_known_kernels_spill(resources):
    spilling = [k for k, v in resources.items() if v.get("spill", 0) > 0]
    assert all(any(a in k for a in SPILL_ALLOWED) for k in spilling), spilling
