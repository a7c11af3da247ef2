"""The paper's feature studies (Section 4.3-4.5) on the synthetic Diff3D laws, with the paper's
preconditioner configuration: BJAC(k = 2, t = 2) of Eq. 3-2 / 3-3 with 32 contiguous blocks,
binary64 (uniform) against binary32 (fMP, aMP), on one GPU through the C ABI.

  * adp_tol study (Table 4.2): aMP-BJAC(hl) and (lh) iterations for adp_tol = 10 ... 1e-5
    on Diff3D-Const and Diff3D-Dis(1000).
  * anisotropy study (Section 4.5.1, Figure 4.6): Diff3D-Ani(s), s = 1000, 100, 10, 4, 2, 1:
    iterations of uniform and fMP, and the relative residual at which the two residual
    histories part (the paper's "bifurcation").
  * diagonal-dominance study (Section 4.5.2, Figure 4.8): a_ii += P_diag sum_{j!=i} |a_ij| on
    Diff3D-Dis(1000) (the RHD3D matrices are not available), iter_o = iter_fMP / iter_uniform.

The same two relationships with the library's own configuration, exact inverses of blocks of
32 rows stored in binary32, bfloat16 or scaled binary16 (fMP), where they can be seen: with
BJAC(2, 2) the binary32 set causes no delay on these laws.

  * multiscale study (Section 4.5.1, Eq. 4-5): Diff3D-Rand(s), s = 1e2 ... 1e12, where the
    largest multiscale strength tau_i grows with s: iter_o per storage format, or the failure
    (breakdown or no convergence) of the solve.
  * diagonal-dominance study on Diff3D-Rand(1e10) with P_diag = 0 ... 2.

    python -m paper_2407_15973_gb300.experiments [--m 128] [--m-exact 64] [--out experiments.json]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import binding as B
from . import problems as PB

TOL = 1e-10
MAXIT = 5000


def _system(A, m, nblocks=32):
    dA = B.DeviceCSR(A)
    xs = torch.as_tensor(PB.solution(A.n, 0)).cuda()
    b = torch.empty(A.n, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, xs, b)
    bp = np.linspace(0, A.n, nblocks + 1).astype(np.int32)
    return dA, bp, b


def _solve(dA, bp, b, hist=False, **pol):
    h = B.bjac_setup(dA, bp, select=B.SELECT_KT, **pol)
    x = torch.zeros(dA.n, dtype=torch.float64, device="cuda")
    hv = torch.full((MAXIT + 1,), float("nan"), dtype=torch.float64, device="cuda") if hist else None
    st = h.solve(b, x, tol=TOL, maxit=MAXIT, hist=hv)
    h.close()
    out = {"iters": st["iters"], "converged": st["converged"], "true_relres": st["true_relres"],
           "low_applies": st["low_applies"], "high_applies": st["high_applies"], "solve_ms": round(st["solve_ms"], 2)}
    if hist:
        out["hist"] = hv[:st["iters"] + 1].cpu().numpy()
    return out


def adp_tol_study(m):
    res = {}
    for law in ("const", "dis"):
        dA, bp, b = _system(PB.diff3d(m, law, 1000.0, 0), m)
        row = {"uniform": _solve(dA, bp, b, fixed_fmt=B.FP64)["iters"],
               "fp32-fMP": _solve(dA, bp, b, fixed_fmt=B.FP32)["iters"], "hl": {}, "lh": {}}
        for tol in (10.0, 5.0, 1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
            row["hl"][str(tol)] = _solve(dA, bp, b, fixed_fmt=B.FP32, temporal=B.TEMPORAL_HL, adp_tol=tol)["iters"]
            row["lh"][str(tol)] = _solve(dA, bp, b, fixed_fmt=B.FP32, temporal=B.TEMPORAL_LH, adp_tol=tol)["iters"]
        res[f"diff3d-{law}"] = row
    return res


def anisotropy_study(m):
    res = {}
    for s in (1000.0, 100.0, 10.0, 4.0, 2.0, 1.0):
        dA, bp, b = _system(PB.diff3d(m, "ani", s, 0), m)
        u = _solve(dA, bp, b, hist=True, fixed_fmt=B.FP64)
        f = _solve(dA, bp, b, hist=True, fixed_fmt=B.FP32)
        k = min(len(u["hist"]), len(f["hist"]))
        apart = np.abs(np.log10(f["hist"][:k]) - np.log10(u["hist"][:k])) > 0.1
        split = int(np.argmax(apart)) if apart.any() else None
        res[f"ani{int(s)}"] = {"uniform": u["iters"], "fp32-fMP": f["iters"],
                               "histories_part_at_relres": None if split is None else float(u["hist"][split]),
                               "histories_part_at_iteration": split}
    return res


def dominance_study(m):
    res = {}
    base = PB.diff3d(m, "dis", 1000.0, 0)
    for pd in (0.0, 0.5, 1.0, 2.0, 4.0, 8.0):
        dA, bp, b = _system(PB.diag_boost(base, pd), m)
        u = _solve(dA, bp, b, fixed_fmt=B.FP64)["iters"]
        f = _solve(dA, bp, b, fixed_fmt=B.FP32)["iters"]
        res[f"pdiag{pd:g}"] = {"uniform": u, "fp32-fMP": f, "iter_o": round(f / u, 4)}
    return res


FORMATS = {"fp32": 1, "bf16": 2, "fp16s": 3}


def _solve_exact(A, bs=32, maxit=50000, **pol):
    dA = B.DeviceCSR(A)
    xs = torch.as_tensor(PB.solution(A.n, 0)).cuda()
    b = torch.empty(A.n, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, xs, b)
    h = B.bjac_setup(dA, PB.uniform_blocks(A.n, bs), **pol)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st = h.solve(b, x, tol=TOL, maxit=maxit)
    h.close()
    return {"iters": st["iters"], "converged": st["converged"], "status": st["status"],
            "true_relres": st["true_relres"], "solve_ms": round(st["solve_ms"], 2)}


def _format_row(A):
    u = _solve_exact(A, select=B.SELECT_UNIFORM)
    row = {"uniform": u["iters"], "uniform_converged": u["converged"]}
    for name, f in FORMATS.items():
        r = _solve_exact(A, select=B.SELECT_FIXED, fixed_fmt=f, maxit=max(4 * u["iters"], 100))
        row[name] = {"iters": r["iters"], "converged": r["converged"], "status": r["status"],
                     "iter_o": round(r["iters"] / u["iters"], 4) if r["converged"] and u["iters"] else None}
    return row


def _tau(A, bs=32):
    """(max, mean) of log10 tau_i (Eq. 4-5) over the rows, from the library's block features
    (per block: max and mean of log10 tau_i over its rows; blocks of equal size)."""
    h = B.bjac_setup(B.DeviceCSR(A), PB.uniform_blocks(A.n, bs), select=B.SELECT_UNIFORM)
    feat = h.export()["feat"]
    h.close()
    return float(feat[:, 6].max()), float(feat[:, 7].mean())


def multiscale_study(m, svals=(1e2, 1e4, 1e6, 1e8, 1e10, 1e12)):
    res = {}
    for s in svals:
        A = PB.diff3d(m, "rand", s, 0)
        row = _format_row(A)
        mx, mean = _tau(A)
        row["max_log10_tau"] = round(mx, 2)
        row["mean_log10_tau"] = round(mean, 2)
        res[f"rand{s:g}"] = row
    return res


def dominance_study_exact(m, pdvals=(0.0, 0.01, 0.1, 0.5, 1.0, 2.0)):
    base = PB.diff3d(m, "rand", 1e10, 0)
    return {f"pdiag{pd:g}": _format_row(PB.diag_boost(base, pd)) for pd in pdvals}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=128)
    ap.add_argument("--m-exact", type=int, default=64)
    ap.add_argument("--out", default="experiments.json")
    a = ap.parse_args()
    B.lib()
    t0 = time.time()
    out = {"config": {"m": a.m, "blocks": 32, "k": 2, "t": 2, "tol": TOL, "x_star_seed": 0,
                      "m_exact": a.m_exact, "exact_block_rows": 32},
           "adp_tol_table_4_2": adp_tol_study(a.m),
           "anisotropy_figure_4_6": anisotropy_study(a.m),
           "diagonal_dominance_figure_4_8": dominance_study(a.m),
           "multiscale_exact_blocks": multiscale_study(a.m_exact),
           "diagonal_dominance_exact_blocks": dominance_study_exact(a.m_exact)}
    out["seconds"] = round(time.time() - t0, 1)
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
