"""Full-size oracle solves with the paper's inexact BJAC(k, t) (Eq. 3-2 / 3-3) on the Diff3D laws.

Runs the CPU oracle (unchanged, single thread) on the 128^3 Diff3D-Const / Ani(1000) / Dis(1000)
/ Rand(1000) systems of Section 4.1.1 (seed 0, b = A x*), with 32 contiguous blocks and
k = t = 2 as in the paper's experiments (Section 4.2), with the binary64 preconditioner and with
fMP in binary32 (Algorithm 3.1), and writes iteration counts and final residuals to
oracle/kt_reference.json. Only oracle/ and the input generator are used. About a minute per
solve.

    python oracle/kt_reference_runs.py [--m 128] [--laws const,ani,dis,rand]
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


def run(law, m, policy, nblocks=32, k=2, t=2):
    pr = PB.make_problem(f"diff3d-{law}", seed=0, m=m)
    bp = np.linspace(0, pr.A.n, nblocks + 1).astype(np.int32)
    b = O.spmv(pr.A, pr.x_star)
    t0 = time.perf_counter()
    res = O.pcg_kt(pr.A, bp, b, k=k, t=t, tol=1e-10, maxit=5000,
                   policy=O.POLICY_UNIFORM if policy == "uniform" else O.POLICY_FMP)
    secs = time.perf_counter() - t0
    err = float(np.linalg.norm(res["x"] - pr.x_star) / np.linalg.norm(pr.x_star))
    return {"workload": f"diff3d-{law} m={m} seed=0", "blocks": nblocks, "k": k, "t": t, "policy": policy,
            "iters": res["iters"], "converged": res["converged"], "true_relres": res["true_relres"],
            "x_rel_err": err, "solve_s": secs}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=128)
    ap.add_argument("--laws", default="const,ani,dis,rand")
    ap.add_argument("--out", default=os.path.join(HERE, "kt_reference.json"))
    a = ap.parse_args()
    data = {}
    if os.path.exists(a.out):
        with open(a.out) as f:
            data = json.load(f)
    for law in a.laws.split(","):
        for pol in ("uniform", "fp32"):
            key = f"{law}_m{a.m}_nb32_k2t2_{pol}"
            data[key] = run(law, a.m, pol)
            print(key, data[key], flush=True)
            with open(a.out + ".tmp", "w") as f:
                json.dump(data, f, indent=1)
            os.replace(a.out + ".tmp", a.out)


if __name__ == "__main__":
    main()
