"""Full-size (128^3, n = 2,097,152) checks in the launch configuration bench.py times.

Iteration counts are compared with the oracle's full-size solves stored in
oracle/full_size_reference.json (written by oracle/reference_runs.py, which calls only the
oracle); SpMV and apply outputs are compared element by element on sampled rows the oracle
computes directly.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB
from gpu_util import cuda, host, need_gpu

pytestmark = pytest.mark.gpu
REF = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "full_size_reference.json")


@pytest.fixture(scope="module")
def full():
    B = need_gpu()
    pr = PB.make_problem("subcube3d", seed=0, m=128, bs=32)
    dA = B.DeviceCSR(pr.A)
    xs = cuda(pr.x_star)
    b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, xs, b)
    with open(REF) as f:
        ref = json.load(f)
    return B, pr, dA, b, ref


def test_full_size_spmv_sampled_rows(full):
    B, pr, dA, b, _ = full
    A = pr.A
    bh = host(b)
    rows = np.unique(np.concatenate([np.arange(0, 64), np.arange(A.n - 64, A.n),
                                     np.random.default_rng(0).integers(0, A.n, 4000)]))
    for i in rows:
        lo, hi = A.rowptr[i], A.rowptr[i + 1]
        terms = A.val[lo:hi] * pr.x_star[A.colidx[lo:hi]]
        exact = 0.0
        for t in terms:          # sequential CSR-order sum, as the oracle's SpMV forms it
            exact += t
        assert abs(bh[i] - exact) <= 1e-14 * np.sum(np.abs(terms))


@pytest.mark.parametrize("fmt", [1, 2])
def test_full_size_apply_sampled_blocks(full, fmt):
    B, pr, dA, b, _ = full
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=fmt, fp64_fallback=True)
    ex = h.export()
    r = PB.solution(pr.A.n, 77) * 1e3
    z = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
    h.apply(cuda(r), z, set=1)
    zd = host(z)
    h.close()
    rng = np.random.default_rng(fmt)
    blocks = np.unique(np.concatenate([[0, pr.nb - 1], rng.integers(0, pr.nb, 300)]))
    for bk in blocks:
        s, e = pr.block_ptr[bk], pr.block_ptr[bk + 1]
        bp = np.array([0, e - s], np.int32)
        nbytes = (e - s) ** 2 * (4 if fmt == 1 else 2)
        pool = ex["pool"][ex["qoff"][bk]:ex["qoff"][bk] + nbytes].copy()
        zo = O.apply(bp, np.array([fmt], np.uint8), pool, np.array([0, nbytes], np.int64),
                     ex["scale"][bk:bk + 1], r[s:e], mode=1)
        assert np.array_equal(zd[s:e], zo), bk


@pytest.mark.parametrize("policy", ["uniform", "fp32", "bf16"])
def test_full_size_iterations_match_oracle(full, policy):
    B, pr, dA, b, ref = full
    r = ref[f"m128_bs32_{policy}"]
    pol = dict(select=B.SELECT_UNIFORM) if policy == "uniform" else \
        dict(select=B.SELECT_FIXED, fixed_fmt={"fp32": B.FP32, "bf16": B.BF16}[policy])
    h = B.bjac_setup(dA, pr.block_ptr, **pol)
    x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
    st = h.solve(b, x, tol=1e-10, maxit=20000)
    h.close()
    assert st["converged"] and st["true_relres"] <= 1e-10
    slack = 2 if policy == "uniform" else max(3, 0.05 * r["iters"])
    assert abs(st["iters"] - r["iters"]) <= slack, (st["iters"], r["iters"])
    err = float(torch.linalg.norm(x - cuda(pr.x_star)) / torch.linalg.norm(cuda(pr.x_star)))
    assert err <= 10 * r["x_rel_err"] + 1e-9


KT_REF = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "kt_reference.json")


@pytest.mark.parametrize("law", ["const", "ani", "dis", "rand"])
def test_full_size_paper_bjac_k2t2_vs_oracle(law):
    """The paper's configuration (BJAC(2, 2) with 32 blocks, Diff3D laws at 128^3) against the
    oracle's full-size solves in oracle/kt_reference.json (written by oracle/kt_reference_runs.py)."""
    B = need_gpu()
    with open(KT_REF) as f:
        ref = json.load(f)
    pr = PB.make_problem(f"diff3d-{law}", seed=0, m=128)
    bp = np.linspace(0, pr.A.n, 33).astype(np.int32)
    dA = B.DeviceCSR(pr.A)
    b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, cuda(pr.x_star), b)
    for fmt, pol in ((B.FP64, "uniform"), (B.FP32, "fp32")):
        r = ref[f"{law}_m128_nb32_k2t2_{pol}"]
        h = B.bjac_setup(dA, bp, select=B.SELECT_KT, fixed_fmt=fmt)
        x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
        st = h.solve(b, x, tol=1e-10, maxit=5000)
        h.close()
        assert st["converged"] and st["true_relres"] <= 1e-10
        slack = 2 if pol == "uniform" else max(3, 0.05 * r["iters"])
        assert abs(st["iters"] - r["iters"]) <= slack, (law, pol, st["iters"], r["iters"])
        err = float(torch.linalg.norm(x - cuda(pr.x_star)) / np.linalg.norm(pr.x_star))
        assert err <= 10 * r["x_rel_err"] + 1e-12
