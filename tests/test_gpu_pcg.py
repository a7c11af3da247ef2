"""Solver-level parity: GPU PCG with the BJAC policies against the oracle's PCG."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB
from gpu_util import cuda, host, need_gpu
from pcg_cases import PROBLEMS, uniform_iteration_band

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    return need_gpu()


_cache = {}


def _problem(name):
    if name not in _cache:
        pr = PROBLEMS[name]()
        b = O.spmv(pr.A, pr.x_star)
        _cache[name] = (pr, b, O.Preconditioner(pr.A, pr.block_ptr))
    return _cache[name]


def _gpu_solve(B, pr, b, maxit=3000, hist=False, **pol):
    dA = B.DeviceCSR(pr.A)
    h = B.bjac_setup(dA, pr.block_ptr, **pol)
    x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
    hh = torch.full((maxit + 1,), float("nan"), dtype=torch.float64, device="cuda") if hist else None
    st = h.solve(cuda(b), x, tol=TOL, maxit=maxit, hist=hh)
    xs = host(x)
    h.close()
    st["x"] = xs
    if hist:
        st["hist"] = host(hh)[:st["iters"] + 1]
    return st


def _err(x, xs):
    return np.linalg.norm(x - xs) / np.linalg.norm(xs)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_uniform_fp64_iterations(B, name):
    pr, b, P = _problem(name)
    ref = O.pcg(pr.A, P, b, tol=TOL, maxit=3000)
    got = _gpu_solve(B, pr, b, select=B.SELECT_UNIFORM, hist=True)
    assert ref["converged"] and got["converged"]
    # +-2 around the band of counts the oracle itself gives under five valid summation orders
    # of its dot products (test_oracle_pins.py::test_uniform_iteration_band_over_summation_orders:
    # one count on every system here but the 27-point anisotropic one, 326 ... 334 there)
    lo, hi = uniform_iteration_band(pr, b, P)
    assert lo - 2 <= got["iters"] <= hi + 2, (got["iters"], lo, hi)
    assert got["true_relres"] <= TOL
    assert abs(_err(got["x"], pr.x_star) - _err(ref["x"], pr.x_star)) <= 10 * _err(ref["x"], pr.x_star) + 1e-12
    k = min(got["iters"], ref["iters"], 20)
    assert np.allclose(got["hist"][:k], ref["hist"][:k], rtol=1e-6)
    assert got["high_applies"] > 0 and got["low_applies"] == 0


@pytest.mark.parametrize("fmt", [1, 2, 3])
@pytest.mark.parametrize("name", ["poisson2d_bs8", "subcube24_bs32", "subcube24_bs64", "voronoi24_uneven",
                                  "aniso27_12_bs64"])
def test_fmp_iterations(B, name, fmt):
    pr, b, P = _problem(name)
    P.set_formats(fmt)
    ref = O.pcg(pr.A, P, b, tol=TOL, maxit=3000, policy=O.POLICY_FMP, mode=1)
    got = _gpu_solve(B, pr, b, select=B.SELECT_FIXED, fixed_fmt=fmt)
    assert got["converged"] and got["true_relres"] <= TOL
    if ref["converged"]:
        assert abs(got["iters"] - ref["iters"]) <= max(3, 0.05 * ref["iters"])
    assert got["blocks_per_fmt"][fmt] == P.nb


@pytest.mark.parametrize("temporal,adp,limit", [(1, 1e-30, "uniform"), (1, 1e30, "fmp"),
                                                (2, 1e30, "uniform"), (2, 1e-30, "fmp")])
def test_amp_limits(B, temporal, adp, limit):
    # Section 4.3.2: hl -> uniform (adp_tol -> 0) and fMP (adp_tol -> inf); lh the reverse
    pr, b, P = _problem("subcube24_bs32")
    uni = _gpu_solve(B, pr, b, select=B.SELECT_UNIFORM)
    fmp = _gpu_solve(B, pr, b, select=B.SELECT_FIXED, fixed_fmt=B.BF16)
    got = _gpu_solve(B, pr, b, select=B.SELECT_FIXED, fixed_fmt=B.BF16, temporal=temporal, adp_tol=adp)
    ref = uni if limit == "uniform" else fmp
    assert abs(got["iters"] - ref["iters"]) <= 1
    assert got["converged"]
    if limit == "uniform":
        assert got["low_applies"] == 0
    else:
        assert got["high_applies"] == 0


# blocks of 64: separate residual-update and apply kernels; blocks of 32: the speculative
# application with its redo (k_apply_spec)
@pytest.mark.parametrize("name", ["subcube24_bs64", "subcube24_bs32"])
@pytest.mark.parametrize("temporal,adp", [(1, 10.0), (1, 1e-4), (2, 1e-5), (2, 1e-2)])
def test_amp_against_oracle(B, temporal, adp, name):
    pr, b, P = _problem(name)
    P.set_formats(O.BF16)
    pol = O.POLICY_HL if temporal == 1 else O.POLICY_LH
    ref = O.pcg(pr.A, P, b, tol=TOL, maxit=3000, policy=pol, adp_tol=adp, mode=1)
    got = _gpu_solve(B, pr, b, hist=True, select=B.SELECT_FIXED, fixed_fmt=B.BF16, temporal=temporal, adp_tol=adp)
    assert got["converged"] and got["true_relres"] <= TOL
    assert abs(got["iters"] - ref["iters"]) <= max(3, 0.05 * ref["iters"])
    assert abs(got["low_applies"] - ref["low_applies"]) <= 3
    # the switch follows the relres of the residual being preconditioned: applications happen
    # after iterations 0 .. iters-1 (none after the converging one)
    if got["restarts"] == 0:
        h = got["hist"][:got["iters"]]
        expect_low = int(np.sum(h < adp)) if temporal == 1 else int(np.sum(h >= adp))
        assert got["low_applies"] == expect_low
        assert got["low_applies"] + got["high_applies"] == got["iters"]


def test_rule_and_fallback(B):
    pr, b, P = _problem("voronoi24_uneven")
    got = _gpu_solve(B, pr, b, select=B.SELECT_RULE, fp64_fallback=True)
    assert got["converged"] and got["true_relres"] <= TOL
    assert sum(got["blocks_per_fmt"]) == P.nb


def test_zero_rhs_and_maxit(B):
    pr, b, P = _problem("poisson2d_bs8")
    dA = B.DeviceCSR(pr.A)
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=B.FP32)
    x = torch.ones(pr.A.n, dtype=torch.float64, device="cuda")
    st = h.solve(torch.zeros(pr.A.n, dtype=torch.float64, device="cuda"), x)
    assert st["status"] == 0 and st["iters"] == 0 and torch.all(x == 0)
    x.zero_()
    st = h.solve(cuda(b), x, maxit=5)
    assert st["status"] == B.NOT_CONVERGED and st["iters"] == 5 and not st["converged"]
    # warm start from the exact solution: nothing to do
    x = cuda(pr.x_star)
    st = h.solve(cuda(b), x)
    assert st["iters"] <= 1
    h.close()


def test_repeat_solves_identical(B):
    pr, b, P = _problem("subcube24_bs32")
    dA = B.DeviceCSR(pr.A)
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=B.FP16S)
    xs = []
    for _ in range(3):
        x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
        st = h.solve(cuda(b), x)
        xs.append((st["iters"], host(x)))
    h.close()
    assert xs[0][0] == xs[1][0] == xs[2][0]
    assert np.array_equal(xs[0][1], xs[1][1]) and np.array_equal(xs[0][1], xs[2][1])


@pytest.mark.parametrize("select", ["bf16", "rule", "hl"])
def test_l2_residency_changes_no_bits(B, select):
    # the evict_last policy on the loop's vector accesses is a cache hint: same iterates
    pr, b, P = _problem("subcube24_bs32")
    dA = B.DeviceCSR(pr.A)
    pol = {"bf16": dict(select=B.SELECT_FIXED, fixed_fmt=B.BF16), "rule": dict(select=B.SELECT_RULE),
           "hl": dict(select=B.SELECT_FIXED, fixed_fmt=B.FP32, temporal=B.TEMPORAL_HL, adp_tol=1e-4)}[select]
    h = B.bjac_setup(dA, pr.block_ptr, **pol)
    out = []
    try:
        for keep in (0, 1):
            old = B.bjac_l2_residency(keep)
            x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
            st = h.solve(cuda(b), x)
            B.bjac_l2_residency(old)
            out.append((st["iters"], st["low_applies"], host(x)))
    finally:
        h.close()
    assert out[0][:2] == out[1][:2] and np.array_equal(out[0][2], out[1][2])
    with pytest.raises(B.MpbjacError):
        B.bjac_l2_residency(2)


@pytest.mark.parametrize("temporal", [0, 1])
def test_eager_loop_matches_graph(B, temporal):
    # the host-driven loop enqueues exactly the kernels of the graph's loop body
    pr, b, P = _problem("subcube24_bs32")
    outs = []
    for mode in (0, 1):
        st = _gpu_solve(B, pr, b, select=B.SELECT_FIXED, fixed_fmt=B.BF16, temporal=temporal, adp_tol=1e-3,
                        graph_mode=mode)
        outs.append(st)
    assert outs[0]["iters"] == outs[1]["iters"] and outs[0]["converged"] and outs[1]["converged"]
    assert np.array_equal(outs[0]["x"], outs[1]["x"])
    assert outs[1]["graph_launches"] == 0


@pytest.mark.parametrize("flexible", [False, True])
@pytest.mark.parametrize("temporal,adp", [(1, 1e-4), (2, 1e-4), (1, 10.0), (2, 1e-5)])
def test_amp_speculative_matches_separate_kernels(B, temporal, adp, flexible):
    # the speculative application (default for 32-row blocks) against the separate residual
    # update + generic apply (apply_variant 1): the same choice of set at every application and
    # counts within the +-2 that regrouped partial sums allow
    pr = PB.make_problem("subcube3d", seed=3, m=64, bs=32)      # 8,192 blocks
    b = O.spmv(pr.A, pr.x_star)
    pol = dict(select=B.SELECT_FIXED, fixed_fmt=B.BF16, temporal=temporal, adp_tol=adp, flexible=flexible)
    spec = _gpu_solve(B, pr, b, hist=True, **pol)
    sep = _gpu_solve(B, pr, b, hist=True, apply_variant=1, **pol)
    for got in (spec, sep):
        assert got["converged"] and got["true_relres"] <= TOL
        if got["restarts"] == 0:
            h = got["hist"][:got["iters"]]
            expect_low = int(np.sum(h < adp)) if temporal == 1 else int(np.sum(h >= adp))
            assert got["low_applies"] == expect_low
            assert got["low_applies"] + got["high_applies"] == got["iters"]
    assert abs(spec["iters"] - sep["iters"]) <= 2
    k = min(spec["iters"], sep["iters"], 15)
    assert np.allclose(spec["hist"][:k], sep["hist"][:k], rtol=1e-8)


@pytest.mark.parametrize("temporal,adp", [(1, 1e-4), (2, 1e-4)])
def test_amp_speculative_graph_equals_eager(B, temporal, adp):
    # the redo launch runs inside the graph's loop as it does from the host: same bits
    pr, b, P = _problem("subcube24_bs32")
    pol = dict(select=B.SELECT_FIXED, fixed_fmt=B.BF16, temporal=temporal, adp_tol=adp)
    g = _gpu_solve(B, pr, b, hist=True, **pol)
    e = _gpu_solve(B, pr, b, hist=True, graph_mode=1, **pol)
    assert g["iters"] == e["iters"] and g["low_applies"] == e["low_applies"]
    assert np.array_equal(g["x"], e["x"]) and np.array_equal(g["hist"], e["hist"])


@pytest.mark.parametrize("layout", [1, 2])      # CSR, SELL-32
@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
def test_alpha_paths_agree(B, fmt, layout):
    # In front of the generic apply the loop SpMV's last CTA sums the per-CTA partials of p.q
    # into sigma and alpha; in front of the register and TMA applies every CTA of the apply sums
    # them itself (loop_alpha). The applies give the same z bits but run different grids, so
    # their own sums of r.z and r.r, and with them the iterates, differ in the last bits: the
    # three solves must take the same iterations and agree to rounding (a partial left out of
    # alpha, or a stale one, moves the iterates far more than that).
    pr, b, _ = _problem("subcube24_bs32")
    f = {"fp32": B.FP32, "bf16": B.BF16}[fmt]
    runs = [_gpu_solve(B, pr, b, select=B.SELECT_FIXED, fixed_fmt=f, apply_variant=v, spmv_format=layout)
            for v in (1, 2, 3)]     # generic, TMA, register
    for st in runs:
        assert st["converged"] and st["true_relres"] <= TOL
    for st in runs[1:]:
        assert abs(st["iters"] - runs[0]["iters"]) <= 1, (st["iters"], runs[0]["iters"])
        assert np.max(np.abs(st["x"] - runs[0]["x"])) <= 1e-10 * np.max(np.abs(runs[0]["x"]))
