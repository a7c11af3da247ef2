"""Learned per-block format selector: label generation and training (on the GPU).

Labels come from the method itself: for a training system, the blocks are split into 8
groups by the octiles of their log10 condition number; for each group and each candidate
class (FP32, 16-bit) only that group is demoted (all other blocks binary64) and the system
is solved; the group's label is the cheapest class whose solve converges with a delay of
at most max(3, 1.5 % of the all-binary64 count) iterations (class 0 = FP64 otherwise). On
these ill-conditioned systems any perturbation of the rounding moves the count by a few
iterations, so a tighter bound would label noise. The
12-64-64-3 MLP is then trained by the library's own forward/backward kernels (full-batch
Adam, bfloat16 forward weights, binary32 masters).

    python -m paper_2407_15973_gb300.selector --systems 96 --out paper_2407_15973_gb300/selector_weights.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import binding as B
from . import problems as PB

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "selector_weights.json")
L2 = math.log10(2.0)
NPARAM = 5187 + 24


def sixteen_bit(feat: np.ndarray) -> np.ndarray:
    """16-bit format per block: scaled binary16 when G's dynamic range fits 2^29, else bfloat16."""
    return np.where(feat[:, 8] <= 29 * L2, B.FP16S, B.BF16).astype(np.uint8)


def solve_given(dA, pr, b, fmts, tol=1e-10, maxit=20000):
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_GIVEN, block_fmt=fmts)
    x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
    st = h.solve(b, x, tol=tol, maxit=maxit)
    h.close()
    return st


def label_problem(pr, groups: int = 8, tol: float = 1e-10):
    """(features [nb, 12], labels [nb], info) for one system."""
    dA = B.DeviceCSR(pr.A)
    xs = torch.as_tensor(pr.x_star).cuda()
    b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, xs, b)
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_UNIFORM)
    feat = h.export()["feat"]
    x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
    base = h.solve(b, x, tol=tol, maxit=20000)
    h.close()
    nb = pr.nb
    order = np.argsort(feat[:, 0], kind="stable")
    grp = np.zeros(nb, np.int32)
    for g, idx in enumerate(np.array_split(order, groups)):
        grp[idx] = g
    sixteen = sixteen_bit(feat)
    labels = np.zeros(nb, np.int32)
    monotone_violations = 0
    for g in range(groups):
        sel = grp == g
        if not sel.any():
            continue
        ok = {}
        for cls in (1, 2):
            fm = np.zeros(nb, np.uint8)
            fm[sel] = B.FP32 if cls == 1 else sixteen[sel]
            st = solve_given(dA, pr, b, fm, tol)
            ok[cls] = st["converged"] and st["iters"] - base["iters"] <= max(3, 0.015 * base["iters"])
        if ok[2] and not ok[1]:
            monotone_violations += 1
        labels[sel] = 2 if ok[2] else (1 if ok[1] else 0)
    return feat, labels, dict(base_iters=base["iters"], monotone_violations=monotone_violations)


def init_params(feat: np.ndarray, seed: int = 0) -> np.ndarray:
    """He-style seeded initial weights; feature mean / deviation from the training data."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM, np.float32)
    o = 0
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 3)):
        w = rng.standard_normal((fan_out, fan_in)) * math.sqrt(2.0 / fan_in)
        p[o:o + w.size] = w.ravel()
        o += w.size + fan_out          # biases stay zero
    mu = feat.mean(axis=0)
    sd = feat.std(axis=0)
    sd[sd < 1e-6] = 1.0
    p[5187:5199] = mu
    p[5199:5211] = sd
    return p


def train(feat: np.ndarray, labels: np.ndarray, epochs: int = 400, lr: float = 3e-3, seed: int = 0):
    fd = torch.as_tensor(np.ascontiguousarray(feat, dtype=np.float64)).cuda()
    ld = torch.as_tensor(np.ascontiguousarray(labels, dtype=np.int32)).cuda()
    p0 = init_params(feat, seed)
    params, hist = B.bjac_mlp_train(p0, fd, ld, epochs=epochs, lr=lr)
    logits = B.bjac_mlp_logits(params, fd)
    acc = float(np.mean(np.argmax(logits, axis=1) == labels))
    return params, hist, acc


def save(params, path=DEFAULT_WEIGHTS, meta=None):
    with open(path, "w") as f:
        json.dump({"params": [float(v) for v in params], "meta": meta or {}}, f)


def load(path=DEFAULT_WEIGHTS) -> np.ndarray:
    with open(path) as f:
        return np.asarray(json.load(f)["params"], dtype=np.float32)


def training_systems(count: int, seed0: int = 1000, m_lo: int = 12, m_hi: int = 18):
    """The 27-point anisotropic law (kappa_e lognormal, anisotropy 1e4 in z), blocks of 64."""
    out = []
    for i in range(count):
        s = seed0 + i
        m = m_lo + int(PB.uniform(s, 71, 1)[0] * (m_hi - m_lo + 1))
        out.append(PB.make_problem("aniso27", seed=s, m=min(m, m_hi), bs=64))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=96)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    a = ap.parse_args()
    t0 = time.time()
    feats, labels, viol, base = [], [], 0, []
    for pr in training_systems(a.systems):
        f, l, info = label_problem(pr)
        feats.append(f)
        labels.append(l)
        viol += info["monotone_violations"]
        base.append(info["base_iters"])
    F = np.concatenate(feats)
    L = np.concatenate(labels)
    t1 = time.time()
    params, hist, acc = train(F, L, a.epochs, a.lr)
    meta = dict(systems=a.systems, samples=int(len(L)), label_counts=np.bincount(L, minlength=3).tolist(),
                monotone_violations=viol, label_seconds=round(t1 - t0, 1), train_seconds=round(time.time() - t1, 1),
                final_loss=float(hist[-1]), train_accuracy=acc, epochs=a.epochs, lr=a.lr,
                law="aniso27 m=12..18, blocks of 64, seeds 1000..")
    save(params, a.out, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
