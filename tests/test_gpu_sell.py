"""The SELL-32 layout of the loop SpMV through a handle: same bits as the CSR kernels, the
same PCG trajectory, the stated padding, and the layout choice reported."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB
from gpu_util import cuda, host, need_gpu, spmv_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    return need_gpu()


def _entries(A):
    """Stored SELL-32 entries: every slice of 32 rows padded to its longest row."""
    lens = np.diff(np.asarray(A.rowptr, dtype=np.int64))
    ns = (A.n + 31) // 32
    pad = np.zeros(ns * 32, np.int64)
    pad[:A.n] = lens
    return int(32 * pad.reshape(ns, 32).max(axis=1).sum())


CASES = {
    "poisson2d_64_bs8": lambda: (PB.make_problem("poisson2d", seed=0, m=64, bs=8), B_FP32),
    "subcube_ragged_13": lambda: (PB.make_problem("subcube3d", seed=4, m=13, bs=32), B_BF16),
    "aniso27_12_bs64": lambda: (PB.make_problem("aniso27", seed=5, m=12, bs=64), B_FP32),
    "voronoi_uneven_16": lambda: (PB.make_problem("voronoi3d", seed=6, m=16), B_FP16S),
}
B_FP32, B_BF16, B_FP16S = 1, 2, 3


@pytest.mark.parametrize("layout", [2, 3])
@pytest.mark.parametrize("case", list(CASES))
def test_handle_spmv_sell_matches_csr_bits(B, case, layout):
    pr, fmt = CASES[case]()
    A = pr.A
    dA = B.DeviceCSR(A)
    x = cuda(PB.solution(A.n, 31))
    y_csr = torch.empty(A.n, dtype=torch.float64, device="cuda")
    xy_csr = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, x, y_csr, xy_csr)
    hs = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=fmt, spmv_format=layout)
    hc = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=fmt, spmv_format=1)
    try:
        fs, fc = hs.spmv_format(), hc.spmv_format()
        assert fs["format"] == {2: "sell32", 3: "sell32-prefetch"}[layout] and fs["entries"] == _entries(A)
        assert fc["format"] == "csr" and fc["entries"] == 0
        y = torch.empty(A.n, dtype=torch.float64, device="cuda")
        xy = torch.zeros(1, dtype=torch.float64, device="cuda")
        hs.spmv(x, y, xy)
        assert np.array_equal(host(y).view(np.uint64), host(y_csr).view(np.uint64))
        ref = O.spmv(A, host(x))
        assert np.max(np.abs(host(y) - ref)) <= spmv_tol(A, host(x))
        assert abs(host(xy)[0] - O.dot(host(x), ref)) <= 1e-14 * np.sum(np.abs(host(x) * ref))
        # the PCG loop runs the same arithmetic in both layouts: same iterations, same x bits
        b = torch.empty(A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(dA, cuda(pr.x_star), b)
        xs = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        xc = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        ss = hs.solve(b, xs, tol=1e-10, maxit=5000)
        sc = hc.solve(b, xc, tol=1e-10, maxit=5000)
        assert ss["converged"] and sc["converged"]
        assert ss["iters"] == sc["iters"]
        assert np.array_equal(host(xs).view(np.uint64), host(xc).view(np.uint64))
        assert ss["true_relres"] <= 1e-10
    finally:
        hs.close()
        hc.close()


def test_default_layout_is_timed_and_reported(B):
    pr = PB.make_problem("subcube3d", seed=7, m=48, bs=32)
    dA = B.DeviceCSR(pr.A)
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=B.BF16)
    try:
        f = h.spmv_format()
        assert all(t > 0 for t in f["ms"])
        ms = f["ms"]
        best = 1 if ms[1] < ms[0] else 0
        if ms[2] < 0.97 * ms[best]:
            best = 2
        assert f["format"] == ["csr", "sell32", "sell32-prefetch"][best]
        assert f["entries"] == (_entries(pr.A) if f["format"] != "csr" else 0)
    finally:
        h.close()


def test_padding_limit_keeps_csr(B):
    # one dense row in a slice of short rows: padding far above 1.5 nnz, so the default keeps CSR
    n = 256
    rows, cols, vals = [], [], []
    for i in range(n):
        c = np.arange(n) if i == 0 else np.array(sorted({0, i}))
        for j in c:
            rows.append(i)
            cols.append(j)
            vals.append(float(n + 1) if i == j else -1.0 / n)
    import scipy.sparse as sp
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    M = ((M + M.T) * 0.5).tocsr()
    M.sort_indices()
    A = PB.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    dA = B.DeviceCSR(A)
    bp = np.arange(0, n + 1, 32, dtype=np.int32)
    h = B.bjac_setup(dA, bp, select=B.SELECT_FIXED, fixed_fmt=B.FP32)
    try:
        assert h.spmv_format()["format"] == "csr"
    finally:
        h.close()
    for layout in (2, 3):
        h = B.bjac_setup(dA, bp, select=B.SELECT_FIXED, fixed_fmt=B.FP32, spmv_format=layout)
        try:
            assert h.spmv_format()["entries"] == _entries(A)
            x = cuda(PB.solution(n, 3))
            y = torch.empty(n, dtype=torch.float64, device="cuda")
            h.spmv(x, y)
            assert np.max(np.abs(host(y) - O.spmv(A, host(x)))) <= spmv_tol(A, host(x))
        finally:
            h.close()


def test_invalid_layout_rejected(B):
    pr = PB.make_problem("poisson2d", seed=0, m=16, bs=8)
    dA = B.DeviceCSR(pr.A)
    with pytest.raises(B.MpbjacError):
        B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_UNIFORM, spmv_format=4)
