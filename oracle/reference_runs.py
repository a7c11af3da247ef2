"""Full-size oracle solves whose results the GPU tests and the benchmark's CPU leg use.

Runs the CPU oracle (unchanged, single thread) on the 128^3 subcube diffusion system
(seed 0, blocks of 32) with the uniform binary64 preconditioner and with fMP in the
binary32-emulation mode, and writes iteration counts, final residuals and the per-iteration
wall time to oracle/full_size_reference.json. Only oracle/ and the input generator are
used. Takes tens of minutes per policy.

    python oracle/reference_runs.py [--m 128] [--bs 32] [--policies uniform,bf16,fp32]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2407_15973_gb300 import problems as PB  # noqa: E402

FMT = {"fp32": O.FP32, "bf16": O.BF16, "fp16s": O.FP16S}


def run(m, bs, policy):
    pr = PB.make_problem("subcube3d", seed=0, m=m, bs=bs)
    b = O.spmv(pr.A, pr.x_star)
    t0 = time.perf_counter()
    P = O.Preconditioner(pr.A, pr.block_ptr, fmt=None if policy == "uniform" else FMT[policy])
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = O.pcg(pr.A, P, b, tol=1e-10, maxit=20000,
                policy=O.POLICY_UNIFORM if policy == "uniform" else O.POLICY_FMP, mode=1)
    t_solve = time.perf_counter() - t0
    err = float(np.linalg.norm(res["x"] - pr.x_star) / np.linalg.norm(pr.x_star))
    return {"workload": f"subcube3d m={m} seed=0", "block_size": bs, "policy": policy, "iters": res["iters"],
            "converged": res["converged"], "true_relres": res["true_relres"], "relres": res["relres"],
            "restarts": res["restarts"], "x_rel_err": err, "setup_s": t_setup, "solve_s": t_solve,
            "hist_every_100": [float(v) for v in res["hist"][::100]]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=128)
    ap.add_argument("--bs", type=int, default=32)
    ap.add_argument("--policies", default="uniform,bf16,fp32")
    ap.add_argument("--out", default=os.path.join(HERE, "full_size_reference.json"))
    a = ap.parse_args()
    data = {}
    if os.path.exists(a.out):
        with open(a.out) as f:
            data = json.load(f)
    for pol in a.policies.split(","):
        key = f"m{a.m}_bs{a.bs}_{pol}"
        data[key] = run(a.m, a.bs, pol)
        with open(a.out + ".tmp", "w") as f:
            json.dump(data, f, indent=1)
        os.replace(a.out + ".tmp", a.out)
        print(key, data[key]["iters"], data[key]["true_relres"], flush=True)


if __name__ == "__main__":
    main()
