"""Batched solver (one persistent cooperative launch for many systems) against the
single-system GPU solver and the oracle."""
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


@pytest.fixture(scope="module")
def systems():
    out = PB.batch2d(count=10, seed=3, side_lo=12, side_hi=48)
    out.append(PB.make_problem("subcube3d", seed=4, m=12, bs=32))
    out.append(PB.make_problem("poisson2d", m=20, bs=16))
    return out


def _solve_batch(B, systems, rhs, **pol):
    dAs = [B.DeviceCSR(p.A) for p in systems]
    bt = B.Batch(dAs, [p.block_ptr for p in systems], **pol)
    bs = [cuda(b) for b in rhs]
    xs = [torch.zeros(p.A.n, dtype=torch.float64, device="cuda") for p in systems]
    rc, st = bt.solve(bs, xs, tol=TOL, maxit=5000)
    info = bt.info()
    bt.close()
    return rc, st, [host(x) for x in xs], info


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_batched_matches_single_and_oracle(B, systems, fmt):
    rhs = [O.spmv(p.A, p.x_star) for p in systems]
    pol = dict(select=B.SELECT_UNIFORM) if fmt == 0 else dict(select=B.SELECT_FIXED, fixed_fmt=fmt)
    rc, st, xs, info = _solve_batch(B, systems, rhs, **pol)
    assert rc == 0 and info["tile_rows"] in (32, 64) and info["ntiles"] > len(systems)
    for p, b, s, x in zip(systems, rhs, st, xs):
        assert s["converged"] and s["true_relres"] <= TOL
        dA = B.DeviceCSR(p.A)
        h = B.bjac_setup(dA, p.block_ptr, **pol)
        xg = torch.zeros(p.A.n, dtype=torch.float64, device="cuda")
        sg = h.solve(cuda(b), xg, tol=TOL, maxit=5000)
        h.close()
        assert abs(sg["iters"] - s["iters"]) <= 2, (p.name, sg["iters"], s["iters"])
        P = O.Preconditioner(p.A, p.block_ptr, fmt=None if fmt == 0 else fmt)
        ref = O.pcg(p.A, P, b, tol=TOL, maxit=5000, policy=O.POLICY_UNIFORM if fmt == 0 else O.POLICY_FMP, mode=1)
        slack = 2 if fmt == 0 else max(3, 0.05 * ref["iters"])
        assert abs(ref["iters"] - s["iters"]) <= slack, (p.name, ref["iters"], s["iters"])
        err = np.linalg.norm(x - p.x_star) / np.linalg.norm(p.x_star)
        ref_err = np.linalg.norm(ref["x"] - p.x_star) / np.linalg.norm(p.x_star)
        assert err <= 10 * ref_err + 1e-12


def test_batched_zero_rhs_and_rule(B, systems):
    rhs = [O.spmv(p.A, p.x_star) for p in systems]
    rhs[2] = np.zeros_like(rhs[2])           # this system is solved by x = 0
    rc, st, xs, info = _solve_batch(B, systems, rhs, select=B.SELECT_RULE)
    assert rc == 0
    assert st[2]["iters"] == 0 and np.all(xs[2] == 0)
    assert all(s["converged"] for s in st)


def test_batched_repeatable(B, systems):
    # one batch solved twice gives bit-identical results (fixed tiles, fixed reduction order)
    rhs = [O.spmv(p.A, p.x_star) for p in systems]
    dAs = [B.DeviceCSR(p.A) for p in systems]
    bt = B.Batch(dAs, [p.block_ptr for p in systems], select=B.SELECT_FIXED, fixed_fmt=B.FP32)
    runs = []
    for _ in range(2):
        xs = [torch.zeros(p.A.n, dtype=torch.float64, device="cuda") for p in systems]
        rc, st = bt.solve([cuda(b) for b in rhs], xs, tol=TOL, maxit=5000)
        runs.append(([s["iters"] for s in st], [host(x) for x in xs]))
    bt.close()
    assert runs[0][0] == runs[1][0]
    for x1, x2 in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(x1, x2)


def test_batched_barrier_timeout_reports_and_recovers(B, systems):
    # the failure path of the persistent kernel: its grid barriers are bounded waits. With the
    # test hook each barrier waits for one CTA more than the grid holds, so every wait expires
    # (2 s), the kernel leaves and the call reports TIMEOUT; nothing faults or hangs, and the
    # next normal solve on the same batch (same context) converges
    import time
    sub = systems[:3]
    rhs = [cuda(O.spmv(p.A, p.x_star)) for p in sub]
    bt = B.Batch([B.DeviceCSR(p.A) for p in sub], [p.block_ptr for p in sub], select=B.SELECT_FIXED,
                 fixed_fmt=B.FP32)
    try:
        bt.force_timeout(True)
        xs = [torch.zeros(p.A.n, dtype=torch.float64, device="cuda") for p in sub]
        t0 = time.time()
        with pytest.raises(B.MpbjacError) as e:
            bt.solve(rhs, xs, tol=TOL, maxit=5000)
        assert e.value.code == B.ERR_TIMEOUT
        assert 1.5 < time.time() - t0 < 60
        bt.force_timeout(False)
        xs = [torch.zeros(p.A.n, dtype=torch.float64, device="cuda") for p in sub]
        rc, st = bt.solve(rhs, xs, tol=TOL, maxit=5000)
        assert rc == 0 and all(s["converged"] and s["true_relres"] <= TOL for s in st)
    finally:
        bt.close()


def test_batched_given_formats_match_single_and_oracle(B, systems):
    # per-block formats named by the caller (every block of every system, in order): the same
    # systems as the single-system solver with SELECT_GIVEN and the oracle with those formats
    rng = np.random.default_rng(17)
    fmts = [rng.integers(0, 4, len(p.block_ptr) - 1).astype(np.uint8) for p in systems]
    rhs = [O.spmv(p.A, p.x_star) for p in systems]
    rc, st, xs, info = _solve_batch(B, systems, rhs, select=B.SELECT_GIVEN, block_fmt=np.concatenate(fmts))
    assert rc == 0
    for p, b, s, fm in zip(systems, rhs, st, fmts):
        assert s["converged"] and s["true_relres"] <= TOL
        assert s["blocks_per_fmt"] == np.bincount(np.concatenate(fmts), minlength=4).tolist()
        dA = B.DeviceCSR(p.A)
        h = B.bjac_setup(dA, p.block_ptr, select=B.SELECT_GIVEN, block_fmt=fm)
        xg = torch.zeros(p.A.n, dtype=torch.float64, device="cuda")
        sg = h.solve(cuda(b), xg, tol=TOL, maxit=5000)
        h.close()
        assert abs(sg["iters"] - s["iters"]) <= max(2, 0.03 * sg["iters"]), (p.name, sg["iters"], s["iters"])
        P = O.Preconditioner(p.A, p.block_ptr, fmt=fm)
        ref = O.pcg(p.A, P, b, tol=TOL, maxit=5000, policy=O.POLICY_FMP, mode=1)
        assert abs(ref["iters"] - s["iters"]) <= max(3, 0.05 * ref["iters"]), (p.name, ref["iters"], s["iters"])


def test_batched_given_needs_formats(B, systems):
    dAs = [B.DeviceCSR(p.A) for p in systems[:2]]
    with pytest.raises(B.MpbjacError):
        B.Batch(dAs, [p.block_ptr for p in systems[:2]], select=B.SELECT_GIVEN)
    bad = np.full(sum(len(p.block_ptr) - 1 for p in systems[:2]), 7, np.uint8)
    with pytest.raises(B.MpbjacError):
        B.Batch(dAs, [p.block_ptr for p in systems[:2]], select=B.SELECT_GIVEN, block_fmt=bad)


# a batch of the 256-system workload's law whose sides reach 496 and 507 (seed 6: sides 34 ... 507,
# 912,201 rows), solved with every kernel variant forced
_big = {}


def _big_batch(B):
    if not _big:
        systems = PB.batch2d(count=12, seed=6, side_lo=32, side_hi=512)
        assert max(p.meta["side"] for p in systems) >= 496
        rhs = [O.spmv(p.A, p.x_star) for p in systems]
        single = []
        for p, b in zip(systems, rhs):
            dA = B.DeviceCSR(p.A)
            h = B.bjac_setup(dA, p.block_ptr, select=B.SELECT_FIXED, fixed_fmt=B.FP32)
            xg = torch.zeros(p.A.n, dtype=torch.float64, device="cuda")
            single.append(h.solve(cuda(b), xg, tol=TOL, maxit=20000)["iters"])
            h.close()
        order = np.argsort([p.A.n for p in systems])
        oracle = {}
        for i in order[:3]:                      # the three smallest against the oracle
            p = systems[i]
            P = O.Preconditioner(p.A, p.block_ptr, fmt=O.FP32)
            oracle[int(i)] = O.pcg(p.A, P, rhs[i], tol=TOL, maxit=20000, policy=O.POLICY_FMP, mode=1)["iters"]
        _big.update(systems=systems, rhs=rhs, single=single, oracle=oracle)
    return _big


@pytest.mark.parametrize("variant", range(8))
def test_every_kernel_variant_on_large_sides(B, variant):
    big = _big_batch(B)
    systems, rhs = big["systems"], big["rhs"]
    dAs = [B.DeviceCSR(p.A) for p in systems]
    bt = B.Batch(dAs, [p.block_ptr for p in systems], select=B.SELECT_FIXED, fixed_fmt=B.FP32)
    try:
        bt.set_variant(variant)
        bs = [cuda(b) for b in rhs]
        xs = [torch.zeros(p.A.n, dtype=torch.float64, device="cuda") for p in systems]
        rc, st = bt.solve(bs, xs, tol=TOL, maxit=20000)
        info = bt.info()
    finally:
        bt.close()
    assert rc == 0 and info["tile_rows"] == (32 if variant < 3 else 64 if variant < 6 else 128)
    for i, (p, s, x) in enumerate(zip(systems, st, xs)):
        assert s["converged"] and s["true_relres"] <= TOL, (i, s)
        assert abs(s["iters"] - big["single"][i]) <= max(2, 0.03 * big["single"][i]), (i, s["iters"], big["single"][i])
        err = np.linalg.norm(host(x) - p.x_star) / np.linalg.norm(p.x_star)
        assert err < 1e-5, (i, err)
    for i, it in big["oracle"].items():
        assert abs(st[i]["iters"] - it) <= max(3, 0.05 * it), (i, st[i]["iters"], it)


def test_set_variant_rejects_bad_values(B, systems):
    dAs = [B.DeviceCSR(p.A) for p in systems[:2]]
    bt = B.Batch(dAs, [p.block_ptr for p in systems[:2]], select=B.SELECT_FIXED, fixed_fmt=B.FP32)
    try:
        for v in (-1, 8):
            with pytest.raises(B.MpbjacError):
                bt.set_variant(v)
    finally:
        bt.close()
