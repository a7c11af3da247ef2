"""What the trained selector gains, on held-out systems (training used seeds >= 1000), against
the methods without it: fixed BF16 (the cheapest format), fixed FP32 (the paper's low
precision), the condition-number rule and uniform binary64. The measure is the modelled time
to solution: iterations x the bytes one PCG iteration moves with the chosen formats (SpMV,
vectors, block inverses; selector.iteration_bytes).

* On laws where no storage format delays the solve (the 7-point subcube diffusion, the 27-point
  anisotropic FEM with blocks of 64, the Voronoi materials, Diff3D-Rand(1000)) the best any
  per-block choice can do is 16-bit everywhere; the selector must match fixed BF16.
* On the multiscale core (the Rand law of Section 4.1.1 with s = 1e10 on the central cube,
  Eq. 4-5 multiscale strength up to 1e10) fixed BF16 breaks down, and the selector must beat
  fixed FP32, the rule and binary64.
"""
import os

import numpy as np
import pytest
import torch

from paper_2407_15973_gb300 import problems as PB
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _compare(B, selector, law, m, bs, seeds=range(5)):
    params = selector.load()
    theta = selector.load_safety_theta()
    pols = {"fp64": dict(select=B.SELECT_UNIFORM), "fp32": dict(select=B.SELECT_FIXED, fixed_fmt=B.FP32),
            "bf16": dict(select=B.SELECT_FIXED, fixed_fmt=B.BF16), "rule": dict(select=B.SELECT_RULE),
            "mlp": dict(select=B.SELECT_MLP, mlp_params=params, safety_theta=theta)}
    out = {k: {"time": 0.0, "iters": 0, "bytes": 0.0, "converged": 0} for k in pols}
    for seed in seeds:
        pr = PB.make_problem(law, seed=seed, m=m, bs=bs)
        dA = B.DeviceCSR(pr.A)
        xs = torch.as_tensor(pr.x_star).cuda()
        b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(dA, xs, b)
        for name, pol in pols.items():
            h = B.bjac_setup(dA, pr.block_ptr, **pol)
            fm = h.formats().astype(np.int64)
            x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
            st = h.solve(b, x, tol=1e-10, maxit=30000)
            h.close()
            ok = st["converged"] and st["true_relres"] <= 1e-10
            o = out[name]
            o["converged"] += int(ok)
            o["iters"] += st["iters"]
            o["bytes"] += selector.iteration_bytes(pr, fm)
            o["time"] += st["iters"] * selector.iteration_bytes(pr, fm) if ok else float("inf")
    return out


@pytest.fixture(scope="module")
def ctx():
    B = need_gpu()
    from paper_2407_15973_gb300 import selector
    if not os.path.exists(selector.DEFAULT_WEIGHTS):
        pytest.fail("trained weights missing: run python -m paper_2407_15973_gb300.selector")
    return B, selector


@pytest.mark.parametrize("law,m,bs", [("subcube3d", 32, 32), ("aniso27", 20, 64), ("voronoi3d", 32, None),
                                      ("diff3d-rand", 32, 32)])
def test_selector_matches_fixed_bf16_where_nothing_delays(ctx, law, m, bs):
    B, selector = ctx
    r = _compare(B, selector, law, m, bs)
    assert r["mlp"]["converged"] == 5 and r["bf16"]["converged"] == 5, r
    # 16-bit (nearly) everywhere: bytes per iteration within 2 % of fixed BF16, the same count
    # within the rounding noise of the solve, and not slower in the model
    assert r["mlp"]["bytes"] <= 1.02 * r["bf16"]["bytes"], r
    assert r["mlp"]["iters"] <= r["bf16"]["iters"] + max(5, 0.01 * r["bf16"]["iters"]), r
    assert r["mlp"]["time"] <= 1.03 * r["bf16"]["time"], r
    # and clearly ahead of the rule, FP32 and binary64 on these laws
    for other in ("rule", "fp32", "fp64"):
        assert r["mlp"]["time"] < 0.9 * r[other]["time"], (other, r)


@pytest.mark.parametrize("m", [32, 48])
def test_selector_beats_every_fixed_format_and_the_rule_on_the_multiscale_core(ctx, m):
    B, selector = ctx
    r = _compare(B, selector, "mscore3d", m, 32)
    assert r["mlp"]["converged"] == 5, r
    assert r["bf16"]["converged"] < 5, r                      # BF16 everywhere breaks down
    # measured when the committed weights were trained (modelled time): about 8 % below FP32,
    # 13 % below the rule and 28 % below binary64 at side 32, similar at 48
    for other, frac in (("fp32", 0.97), ("rule", 0.95), ("fp64", 0.8)):
        assert r[other]["converged"] == 5, (other, r)
        assert r["mlp"]["time"] < frac * r[other]["time"], (other, r)
