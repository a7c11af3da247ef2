"""The allocation-free SpMV (bjac_spmv_noalloc) against the ordinary bjac_spmv and the oracle.

bjac_spmv_noalloc exists for callers that cannot allocate device memory while they run
(a device-memory budget reserved up front, a hard memory cap, or code that must not let
cudaFree synchronise the device). It reduces its dot product through a fixed buffer in the
library's static device memory. This file is collected last on purpose, so that a failure
here does not hide the other GPU tests in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB
from gpu_util import cuda, host, need_gpu, spmv_tol

pytestmark = pytest.mark.gpu

CASES = {
    "subcube24": lambda: PB.make_problem("subcube3d", seed=1, m=24).A,          # short rows, warp kernel
    "ragged13": lambda: PB.make_problem("subcube3d", seed=2, m=13).A,           # n not a multiple of 256
    "aniso27_12": lambda: PB.make_problem("aniso27", seed=3, m=12).A,           # long rows, staged kernel
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_bjac_spmv_on_two_calls(case):
    B = need_gpu()
    A = CASES[case]()
    dA = B.DeviceCSR(A)
    x = cuda(PB.solution(A.n, 31))
    y_ref = torch.empty(A.n, dtype=torch.float64, device="cuda")
    xy_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, x, y_ref, xy_ref)
    tol_y = spmv_tol(A, host(x))
    yr = host(y_ref)
    dot_ref = host(xy_ref)[0]
    # the oracle's sequential CSR-order product and dot product of the same x
    yo = O.spmv(A, host(x))
    dot_o = O.dot(host(x), yo)
    for _ in range(2):       # the second call finds the first call's leftovers in the buffer
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        xy = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        B.bjac_spmv_noalloc(dA, x, y, xy)
        assert np.max(np.abs(host(y) - yr)) <= tol_y
        assert abs(host(xy)[0] - dot_ref) <= 1e-14 * float(np.sum(np.abs(host(x) * yr)))
        # each row adds the same products in the same CSR order as the oracle's loop (the GPU
        # fuses each multiply-add, the oracle rounds the product first), so y is within the
        # stated 1e-14 of max (|A||x|)_i of the oracle's, and the dot within 1e-14 of sum |x_i y_i|
        assert np.max(np.abs(host(y) - yo)) <= tol_y
        assert abs(host(xy)[0] - dot_o) <= 1e-14 * float(np.sum(np.abs(host(x) * yo)))


def test_noalloc_rejects_rows_beyond_its_buffer():
    B = need_gpu()
    # only the host-side size check runs: the call returns before touching any pointer
    big = B.bjac_csr(16_777_217, 0, 1, 0, 0)
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = B.lib().bjac_spmv_noalloc(ctypes.byref(big), ctypes.c_void_p(one.data_ptr()),
                                   ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()), None)
    assert rc == B.ERR_INVALID_ARG
    assert b"16,777,216" in B.lib().bjac_last_error()
