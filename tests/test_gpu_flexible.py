"""Flexible PCG (the Polak-Ribiere direction coefficient of flexible CG, Golub-Ye 1999 and
Notay 2000) through the C ABI, against the oracle's flexible PCG."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB
from gpu_util import cuda, host, need_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    return need_gpu()


CASES = {
    "subcube24_bs32_fmp_bf16": (lambda: PB.make_problem("subcube3d", seed=1, m=24, bs=32), 2, O.POLICY_FMP, 10.0),
    "voronoi24_hl_fp16s": (lambda: PB.make_problem("voronoi3d", seed=4, m=24), 3, O.POLICY_HL, 1e-2),
    "ragged13_lh_bf16": (lambda: PB.make_problem("subcube3d", seed=5, m=13, bs=32), 2, O.POLICY_LH, 1e-3),
    "aniso27_hl_fp32": (lambda: PB.make_problem("aniso27", seed=3, m=12, bs=64), 1, O.POLICY_HL, 1e-4),
}


def _policy(B, fmt, policy, adp):
    temporal = {O.POLICY_FMP: B.TEMPORAL_NONE, O.POLICY_HL: B.TEMPORAL_HL, O.POLICY_LH: B.TEMPORAL_LH}[policy]
    return dict(select=B.SELECT_FIXED, fixed_fmt=fmt, temporal=temporal, adp_tol=adp)


def _solve(B, pr, b, maxit=5000, tol=TOL, **pol):
    h = B.bjac_setup(B.DeviceCSR(pr.A), pr.block_ptr, **pol)
    x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
    st = h.solve(cuda(b), x, tol=tol, maxit=maxit)
    h.close()
    st["x"] = host(x)
    return st


@pytest.mark.parametrize("case", list(CASES))
def test_flexible_pcg_vs_oracle(B, case):
    make, fmt, policy, adp = CASES[case]
    pr = make()
    b = O.spmv(pr.A, pr.x_star)
    P = O.Preconditioner(pr.A, pr.block_ptr, fmt=fmt)
    ref = O.pcg(pr.A, P, b, tol=TOL, maxit=5000, policy=policy, adp_tol=adp, flexible=True)
    got = _solve(B, pr, b, flexible=True, **_policy(B, fmt, policy, adp))
    assert ref["converged"] and got["converged"] and got["true_relres"] <= TOL
    assert abs(got["iters"] - ref["iters"]) <= max(3, 0.05 * ref["iters"]), (got["iters"], ref["iters"])
    assert abs(got["low_applies"] - ref["low_applies"]) <= 3
    err = np.linalg.norm(got["x"] - pr.x_star) / np.linalg.norm(pr.x_star)
    ref_err = np.linalg.norm(ref["x"] - pr.x_star) / np.linalg.norm(pr.x_star)
    assert err <= 10 * ref_err + 1e-12


def test_flexible_equals_standard_with_binary64_blocks(B):
    pr = PB.make_problem("voronoi3d", seed=4, m=24)
    b = O.spmv(pr.A, pr.x_star)
    std = _solve(B, pr, b, select=B.SELECT_UNIFORM)
    flex = _solve(B, pr, b, select=B.SELECT_UNIFORM, flexible=True)
    assert std["converged"] and flex["converged"] and abs(std["iters"] - flex["iters"]) <= 1
    assert std["kernel_launches"] < flex["kernel_launches"]       # one more kernel per iteration


def test_flexible_keeps_consecutive_steps_conjugate(B):
    # the property that defines the flexible coefficient, on the GPU's own iterates: with the
    # precision switch of aMP(hl) inside the first 12 iterations, consecutive steps
    # x_{k+1} - x_k stay A-conjugate to rounding with flexible=1 and not with flexible=0
    pr = PB.make_problem("voronoi3d", seed=4, m=12)
    A = sp.csr_matrix((pr.A.val, pr.A.colidx, pr.A.rowptr), shape=(pr.A.n, pr.A.n))
    b = O.spmv(pr.A, pr.x_star)
    dA = B.DeviceCSR(pr.A)
    out = {}
    for flex in (0, 1):
        h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=B.BF16, temporal=B.TEMPORAL_HL,
                         adp_tol=1e-2, flexible=bool(flex))
        xs = [np.zeros(pr.A.n)]
        for k in range(1, 13):
            x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
            st = h.solve(cuda(b), x, tol=1e-14, maxit=k)
            assert st["iters"] == k
            xs.append(host(x))
        h.close()
        d = [xs[k + 1] - xs[k] for k in range(12)]
        out[flex] = np.array([abs(d[k + 1] @ (A @ d[k])) / np.sqrt((d[k + 1] @ (A @ d[k + 1])) * (d[k] @ (A @ d[k])))
                              for k in range(11)])
    assert out[1].max() < 1e-11, out[1]
    assert out[0].max() > 1e3 * out[1].max(), (out[0], out[1])


def test_flexible_kt_vs_oracle(B):
    pr = PB.make_problem("subcube3d", seed=11, m=16)
    bp = np.linspace(0, pr.A.n, 9).astype(np.int32)
    b = O.spmv(pr.A, pr.x_star)
    ref = O.pcg_kt(pr.A, bp, b, k=2, t=2, tol=TOL, maxit=5000, policy=O.POLICY_HL, adp_tol=1e-3, flexible=True)
    h = B.bjac_setup(B.DeviceCSR(pr.A), bp, select=B.SELECT_KT, fixed_fmt=B.FP32, temporal=B.TEMPORAL_HL,
                     adp_tol=1e-3, flexible=True)
    x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
    st = h.solve(cuda(b), x, tol=TOL, maxit=5000)
    h.close()
    assert ref["converged"] and st["converged"] and st["true_relres"] <= TOL
    assert abs(st["iters"] - ref["iters"]) <= max(3, 0.05 * ref["iters"])
    assert abs(st["low_applies"] - ref["low_applies"]) <= 3


def test_flexible_eager_loop_matches_graph(B):
    pr = PB.make_problem("subcube3d", seed=1, m=24, bs=32)
    b = O.spmv(pr.A, pr.x_star)
    pol = dict(select=B.SELECT_FIXED, fixed_fmt=B.BF16, temporal=B.TEMPORAL_HL, adp_tol=1e-3, flexible=True)
    g = _solve(B, pr, b, graph_mode=0, **pol)
    e = _solve(B, pr, b, graph_mode=1, **pol)
    assert g["iters"] == e["iters"] and np.array_equal(g["x"], e["x"])
