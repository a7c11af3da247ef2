"""BJAC(k, t) of Eq. 3-2 / 3-3 (the paper's inexact block Jacobi: inner Jacobi sweeps inside the
blocks, outer block-Jacobi sweeps on A) through the C ABI, against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB
from gpu_util import cuda, host, need_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    return need_gpu()


def _layouts():
    a = PB.make_problem("subcube3d", seed=11, m=16)
    b = PB.make_problem("subcube3d", seed=12, m=13)             # ragged: n = 2197
    c = PB.make_problem("aniso27", seed=13, m=10)
    rng = np.random.default_rng(5)
    cuts = np.sort(rng.choice(np.arange(1, b.A.n), 6, replace=False))
    return {
        "subcube16_8blocks": (a, np.linspace(0, a.A.n, 9).astype(np.int32)),
        "ragged13_uneven": (b, np.concatenate([[0], cuts, [b.A.n]]).astype(np.int32)),
        "aniso27_4blocks": (c, np.linspace(0, c.A.n, 5).astype(np.int32)),
        "subcube16_one_block": (a, np.array([0, a.A.n], np.int32)),
    }


LAYOUTS = _layouts()


@pytest.mark.parametrize("kt", [(1, 1), (2, 2), (3, 2), (2, 3)])
@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_kt_apply_bitwise_vs_oracle(B, layout, kt):
    pr, bp = LAYOUTS[layout]
    k, t = kt
    dA = B.DeviceCSR(pr.A)
    r = PB.solution(pr.A.n, 41) * 3.0
    h = B.bjac_setup(dA, bp, select=B.SELECT_KT, fixed_fmt=B.FP32, kt_outer=k, kt_inner=t)
    try:
        for prec in (0, 1):
            z = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
            rz = torch.zeros(1, dtype=torch.float64, device="cuda")
            h.apply(cuda(r), z, set=prec, rz=rz)
            ref = O.kt_apply(pr.A, bp, k, t, r, prec=prec)
            got = host(z)
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (layout, kt, prec)
            assert abs(host(rz)[0] - np.dot(r, ref)) <= 1e-13 * np.sum(np.abs(r * ref))
    finally:
        h.close()


@pytest.mark.parametrize("layout", ["subcube16_8blocks", "ragged13_uneven", "aniso27_4blocks"])
def test_kt_pcg_vs_oracle(B, layout):
    pr, bp = LAYOUTS[layout]
    dA = B.DeviceCSR(pr.A)
    b = O.spmv(pr.A, pr.x_star)
    for fmt, pol in ((B.FP64, O.POLICY_UNIFORM), (B.FP32, O.POLICY_FMP)):
        h = B.bjac_setup(dA, bp, select=B.SELECT_KT, fixed_fmt=fmt)
        x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
        st = h.solve(cuda(b), x, tol=TOL, maxit=5000)
        h.close()
        ref = O.pcg_kt(pr.A, bp, b, k=2, t=2, policy=pol, tol=TOL, maxit=5000)
        if not ref["converged"]:
            # the Jacobi sweeps diverge on this (non-M-matrix) operator, M-hat^-1 is not positive
            # definite and PCG breaks down at once; the library reports the same
            assert ref["status"] == -5 and st["status"] == B.ERR_BREAKDOWN and not st["converged"]
            assert st["iters"] == ref["iters"]
            continue
        assert st["converged"] and st["true_relres"] <= TOL
        slack = 2 if fmt == B.FP64 else max(3, 0.05 * ref["iters"])
        assert abs(st["iters"] - ref["iters"]) <= slack, (layout, fmt, st["iters"], ref["iters"])
        err = np.linalg.norm(host(x) - pr.x_star) / np.linalg.norm(pr.x_star)
        ref_err = np.linalg.norm(ref["x"] - pr.x_star) / np.linalg.norm(pr.x_star)
        assert err <= 10 * ref_err + 1e-12


def test_kt_amp_limits(B):
    # Section 4.3.2: hl -> uniform as adp_tol -> 0 and -> fMP as adp_tol -> inf; lh the reverse
    pr, bp = LAYOUTS["subcube16_8blocks"]
    dA = B.DeviceCSR(pr.A)
    b = cuda(O.spmv(pr.A, pr.x_star))

    def run(**pol):
        h = B.bjac_setup(dA, bp, select=B.SELECT_KT, **pol)
        x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
        st = h.solve(b, x, tol=TOL, maxit=5000)
        h.close()
        return st, host(x)

    uni, xu = run(fixed_fmt=B.FP64)
    fmp, xf = run(fixed_fmt=B.FP32)
    for temporal, adp, ref, xr in ((B.TEMPORAL_HL, 1e-30, uni, xu), (B.TEMPORAL_HL, 1e30, fmp, xf),
                                   (B.TEMPORAL_LH, 1e-30, fmp, xf), (B.TEMPORAL_LH, 1e30, uni, xu)):
        st, x = run(fixed_fmt=B.FP32, temporal=temporal, adp_tol=adp)
        assert st["iters"] == ref["iters"] and np.array_equal(x, xr), (temporal, adp)
        assert st["low_applies"] + st["high_applies"] == ref["low_applies"] + ref["high_applies"]


def test_kt_point_jacobi_equals_blocks_of_one(B):
    # k = t = 1 is diagonal scaling (Section 3.1), i.e. exact block Jacobi with blocks of one row
    pr = PB.make_problem("subcube3d", seed=14, m=12)
    dA = B.DeviceCSR(pr.A)
    b = cuda(O.spmv(pr.A, pr.x_star))
    res = []
    for pol, bp in ((dict(select=B.SELECT_KT, fixed_fmt=B.FP64, kt_outer=1, kt_inner=1),
                     np.array([0, pr.A.n], np.int32)),
                    (dict(select=B.SELECT_UNIFORM), np.arange(pr.A.n + 1, dtype=np.int32))):
        h = B.bjac_setup(dA, bp, **pol)
        x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
        res.append(h.solve(b, x, tol=TOL, maxit=5000)["iters"])
        h.close()
    assert abs(res[0] - res[1]) <= 2, res


def test_kt_rejects_bad_inputs(B):
    pr, bp = LAYOUTS["subcube16_8blocks"]
    dA = B.DeviceCSR(pr.A)
    for kw in (dict(fixed_fmt=B.BF16), dict(fixed_fmt=B.FP64, temporal=B.TEMPORAL_HL), dict(kt_outer=65)):
        with pytest.raises(B.MpbjacError):
            B.bjac_setup(dA, bp, select=B.SELECT_KT, **{"fixed_fmt": B.FP32, **kw})
    A = PB.CSR(pr.A.n, pr.A.rowptr, pr.A.colidx, pr.A.val.copy())
    A.val[A.rowptr[5]:A.rowptr[6]][A.colidx[A.rowptr[5]:A.rowptr[6]] == 5] = -1.0
    with pytest.raises(B.MpbjacError) as e:
        B.bjac_setup(B.DeviceCSR(A), bp, select=B.SELECT_KT, fixed_fmt=B.FP32)
    assert e.value.code == B.ERR_NOT_SPD
