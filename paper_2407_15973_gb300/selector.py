"""Learned per-block format selector: label generation, training (on the GPU), the safety
threshold.

Labels come from the method itself. For a training system the blocks are split into 8 groups
by the octiles of their log10 condition number; for each group and each candidate class
(FP32, 16-bit) only that group is demoted, all other blocks binary64, and the system is
solved. The label is cost-aware: the class with the least modelled time to solution, where the
time of a solve is its iteration count times the bytes one PCG iteration moves (the SpMV, the
vector updates and the block inverses in their formats: 12 nnz + 92 n + sum_b bs_b^2 bytes_b),
among the solves that converge; a demotion whose delay costs more than the bytes it saves keeps
the group in binary64. The 17
solves of a system run on the batched solver (blocks of 32 rows) together with those of the
other systems of a chunk: one launch solves every system with all blocks binary64, a second
one every demotion, stopped at twice the binary64 count (demoting one group never saves half
the bytes of an iteration, so a longer solve cannot pay). Systems
with blocks of 64 rows, which the batched solver does not take, are labelled with single
solves.

The training mix (seeded, sizes log-uniform, sides 20..32, 24..64 for the multiscale core): five
laws with blocks of 32 -- the subcube
diffusion of the 128^3 workload, the multiscale-core law (the Rand law of Section 4.1.1 with
s = 1e10 on the central cube, 1e2 elsewhere), the Voronoi materials, the 27-point anisotropic
FEM and Diff3D-Rand(1000) -- plus the 27-point anisotropic law with blocks of 64.

The 12-64-64-3 MLP is trained by the library's own forward / backward kernels (full-batch Adam,
bfloat16 forward weights, binary32 masters). Its choice is only ever promoted by the safety
rule kappa_1 u_f <= safety_theta. safety_theta comes from data: its cap is twice the 99th
percentile of kappa_1 u_16 over the blocks labelled 16-bit (beyond it the labels rarely
tolerate 16-bit storage); below the cap it is lowered in steps of 10^0.2 until every system of
a held-out validation set of the multiscale core (seeds 100..109 at side 32, 100..103 at 48)
converges with the selector.

    python -m paper_2407_15973_gb300.selector --systems 2000 --out paper_2407_15973_gb300/selector_weights.json
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
GROUPS = 8
BATCH_LAWS = ("subcube3d", "mscore3d", "voronoi3d", "aniso27", "diff3d-rand")
U16 = {B.BF16: 2.0 ** -8, B.FP16S: 2.0 ** -11}


def sixteen_bit(feat: np.ndarray) -> np.ndarray:
    """16-bit format per block: scaled binary16 when G's dynamic range fits 2^29, else bfloat16."""
    return np.where(feat[:, 8] <= 29 * L2, B.FP16S, B.BF16).astype(np.uint8)


FMT_BYTES = np.array([8, 4, 2, 2])


def iteration_bytes(pr, fmts: np.ndarray) -> float:
    """Bytes one PCG iteration moves with these block formats: the SpMV (12 per nonzero, row
    pointers, p and q), the vectors of the apply and the updates (r, q, z, x, p: 72 per row) and
    the stored inverses (bs^2 entries of each block in its format)."""
    bs = np.diff(np.asarray(pr.block_ptr, dtype=np.int64))
    return 12.0 * pr.A.nnz + 92.0 * pr.A.n + float(np.sum(bs * bs * FMT_BYTES[fmts]))


def modelled_time(st, pr, fmts) -> float:
    """Iterations x bytes per iteration of a solve that converged, else infinity."""
    if not st["converged"]:
        return math.inf
    return st["iters"] * iteration_bytes(pr, fmts)


def groups_of(feat: np.ndarray, groups: int = GROUPS) -> np.ndarray:
    """Group of every block: the octile of its log10 kappa_1."""
    order = np.argsort(feat[:, 0], kind="stable")
    grp = np.zeros(len(feat), np.int32)
    for g, idx in enumerate(np.array_split(order, groups)):
        grp[idx] = g
    return grp


def demotions(feat: np.ndarray, grp: np.ndarray, groups: int = GROUPS):
    """[(group, class, formats)] of the 2 x groups demoted solves (other blocks binary64)."""
    sixteen = sixteen_bit(feat)
    out = []
    for g in range(groups):
        sel = grp == g
        if not sel.any():
            continue
        for cls in (1, 2):
            fm = np.zeros(len(feat), np.uint8)
            fm[sel] = B.FP32 if cls == 1 else sixteen[sel]
            out.append((g, cls, fm))
    return out


def labels_from(pr, grp: np.ndarray, base, results) -> tuple[np.ndarray, int]:
    """(label per block, number of non-monotone groups: 16-bit pays, FP32 does not).
    results[(group, class)] = (stats, formats) of the demoted solves; base = stats of the
    all-binary64 solve."""
    t0 = modelled_time(base, pr, np.zeros(len(grp), np.int64))
    labels = np.zeros(len(grp), np.int32)
    viol = 0
    for g in sorted({g for g, _ in results}):
        t = {0: t0}
        for cls in (1, 2):
            if (g, cls) in results:
                st, fm = results[(g, cls)]
                t[cls] = modelled_time(st, pr, fm.astype(np.int64))
        pays = {c: t.get(c, math.inf) < t0 for c in (1, 2)}
        if pays[2] and not pays[1]:
            viol += 1
        labels[grp == g] = min(t, key=lambda c: (t[c], -c))
    return labels, viol


def system_features(dA, pr):
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_UNIFORM)
    feat = h.export()["feat"]
    h.close()
    return feat


def _batched(entries, tol, maxit):
    """Stats of one batched launch over entries [(DeviceCSR, problem, b, formats)]."""
    fmts = np.concatenate([e[3] for e in entries])
    bt = B.Batch([e[0] for e in entries], [e[1].block_ptr for e in entries], select=B.SELECT_GIVEN, block_fmt=fmts)
    xs = [torch.zeros(e[1].A.n, dtype=torch.float64, device="cuda") for e in entries]
    rc, st = bt.solve([e[2] for e in entries], xs, tol=tol, maxit=maxit)
    bt.close()
    return st


def label_batch(problems, tol: float = 1e-10, maxit: int = 20000):
    """Labels of several systems (blocks of <= 32 rows) from two batched launches: every system
    with all blocks binary64, then every (system, group, class) demotion."""
    prep = []
    for pr in problems:
        dA = B.DeviceCSR(pr.A)
        xs = torch.as_tensor(pr.x_star).cuda()
        b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(dA, xs, b)
        feat = system_features(dA, pr)
        prep.append((dA, pr, b, feat, groups_of(feat)))
    base = _batched([(dA, pr, b, np.zeros(pr.nb, np.uint8)) for dA, pr, b, _, _ in prep], tol, maxit)
    keep = [(p, st) for p, st in zip(prep, base) if st["converged"]]     # binary64 must solve it
    if not keep:
        return []
    # a demoted solve saves at most half the bytes per iteration, so it cannot pay beyond twice
    # the binary64 count: stop there
    cap = max(2 * st["iters"] + 1 for _, st in keep)
    entries, keys = [], []
    for k, ((dA, pr, b, feat, grp), st) in enumerate(keep):
        for g, cls, fm in demotions(feat, grp):
            entries.append((dA, pr, b, fm))
            keys.append((k, g, cls))
    dem = _batched(entries, tol, min(cap, maxit))
    res = [dict() for _ in keep]
    for (k, g, cls), st, e in zip(keys, dem, entries):
        res[k][(g, cls)] = (st, e[3])
    out = []
    for k, ((dA, pr, b, feat, grp), st) in enumerate(keep):
        labels, viol = labels_from(pr, grp, st, res[k])
        out.append((feat, labels, dict(base_iters=st["iters"], monotone_violations=viol, groups=len(res[k]) // 2)))
    return out


def label_problem(pr, groups: int = GROUPS, tol: float = 1e-10):
    """(features [nb, 12], labels [nb], info) for one system, with single solves (any block
    size up to 128)."""
    dA = B.DeviceCSR(pr.A)
    xs = torch.as_tensor(pr.x_star).cuda()
    b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, xs, b)

    def solve(**pol):
        h = B.bjac_setup(dA, pr.block_ptr, **pol)
        x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
        st = h.solve(b, x, tol=tol, maxit=20000)
        h.close()
        return st

    feat = system_features(dA, pr)
    base = solve(select=B.SELECT_UNIFORM)
    grp = groups_of(feat, groups)
    results = {(g, cls): (solve(select=B.SELECT_GIVEN, block_fmt=fm), fm) for g, cls, fm in demotions(feat, grp, groups)}
    labels, viol = labels_from(pr, grp, base, results)
    return feat, labels, dict(base_iters=base["iters"], monotone_violations=viol, groups=groups)


def kappa_u16(feat: np.ndarray) -> np.ndarray:
    """kappa_1 u_16 of every block, u_16 of the 16-bit format the block would take."""
    fmt16 = sixteen_bit(feat)
    u = np.where(fmt16 == B.FP16S, U16[B.FP16S], U16[B.BF16])
    return np.power(10.0, feat[:, 0]) * u


def safety_theta_from(feat: np.ndarray, labels: np.ndarray, margin: float = 2.0, q: float = 99.0) -> float:
    """Twice the q-th percentile of kappa_1 u_16 over the blocks labelled 16-bit: beyond it the
    labels rarely say that 16-bit storage was tolerated. A percentile, not the largest value:
    binary64 and 16-bit labels overlap for kappa_1 u_16 between about 1e4 and 1e6 (groups
    whose demotion happened to pay), and the 99.9th percentile still let core blocks of the
    multiscale law through to a breakdown on a held-out system."""
    sel = labels == 2
    if not sel.any():
        return 0.5
    return float(margin * np.percentile(kappa_u16(feat)[sel], q))


# held-out validation of the safety threshold (training seeds start at 1000, the gain tests use
# 0..4): the multiscale core, the law where 16-bit storage can break a solve down
VALIDATION = tuple((32, s) for s in range(100, 110)) + tuple((48, s) for s in range(100, 104))


def validate_theta(params: np.ndarray, theta_max: float, step: float = 0.2, floor: float = 0.5):
    """The largest safety_theta on the grid theta_max * 10^(-step k), k = 0, 1, ..., at which
    every validation system (VALIDATION, multiscale core) converges with the selector; returns
    (theta, [(theta, converged count)])."""
    systems = []
    for m, seed in VALIDATION:
        pr = PB.make_problem("mscore3d", seed=seed, m=m, bs=32)
        dA = B.DeviceCSR(pr.A)
        xs = torch.as_tensor(pr.x_star).cuda()
        b = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
        B.bjac_spmv(dA, xs, b)
        systems.append((pr, dA, b))
    trail = []
    theta = theta_max
    while theta >= floor:
        ok = 0
        for pr, dA, b in systems:
            h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_MLP, mlp_params=params, safety_theta=theta)
            x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
            st = h.solve(b, x, tol=1e-10, maxit=40000)
            h.close()
            ok += int(st["converged"] and st["true_relres"] <= 1e-10)
        trail.append((theta, ok))
        if ok == len(systems):
            return theta, trail
        theta *= 10.0 ** -step
    return floor, trail


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


def load_safety_theta(path=DEFAULT_WEIGHTS) -> float:
    """The safety threshold derived from the labels the weights were trained on (0.5 if the
    file predates it)."""
    with open(path) as f:
        return float(json.load(f)["meta"].get("safety_theta", 0.5))


def _side(seed: int, m_lo: int, m_hi: int) -> int:
    u = PB.uniform(seed, 71, 1)[0]
    return int(round(math.exp(math.log(m_lo) + (math.log(m_hi) - math.log(m_lo)) * u)))


# sides of the multiscale-core law: up to 64, so that blocks of 32 rows lying wholly inside the
# core (an x-line of the core is 16 nodes at side 32, 32 at side 64) appear in the labels
CORE_SIDES = (24, 64)


def training_systems(count: int, seed0: int = 1000, m_lo: int = 20, m_hi: int = 32):
    """The batched part of the training mix: the five laws in turn, blocks of 32, side
    log-uniform in [m_lo, m_hi] (CORE_SIDES for the multiscale core), seeds seed0, seed0 + 1, ..."""
    out = []
    for i in range(count):
        law = BATCH_LAWS[i % len(BATCH_LAWS)]
        lo, hi = CORE_SIDES if law == "mscore3d" else (m_lo, m_hi)
        out.append(PB.make_problem(law, seed=seed0 + i, m=_side(seed0 + i, lo, hi), bs=32))
    return out


def training_systems_bs64(count: int, seed0: int = 5000, m_lo: int = 12, m_hi: int = 18):
    """The part with blocks of 64 rows (single solves): the 27-point anisotropic law."""
    return [PB.make_problem("aniso27", seed=seed0 + i, m=_side(seed0 + i, m_lo, m_hi), bs=64) for i in range(count)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=2000, help="systems in all (the last --bs64 with blocks of 64)")
    ap.add_argument("--bs64", type=int, default=100)
    ap.add_argument("--chunk", type=int, default=16, help="systems labelled per pair of batched launches")
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--validate-only", action="store_true",
                    help="keep the weights and labels of --out; only choose the safety threshold again")
    a = ap.parse_args()
    if a.validate_only:
        with open(a.out) as f:
            saved = json.load(f)
        params = np.asarray(saved["params"], dtype=np.float32)
        meta = saved["meta"]
        cap = meta.get("safety_theta_cap", meta["safety_theta"])
        theta, trail = validate_theta(params, cap)
        meta.update(safety_theta=theta, safety_theta_cap=cap, safety_validation=[[round(t, 1), c] for t, c in trail])
        save(params, a.out, meta)
        print(json.dumps(meta))
        return
    t0 = time.time()
    feats, labels, viol, groups, per_law = [], [], 0, 0, {}
    nb32 = a.systems - a.bs64
    systems = training_systems(nb32)
    for c in range(0, nb32, a.chunk):
        chunk = systems[c:c + a.chunk]
        for pr, (f, l, info) in zip(chunk, label_batch(chunk)):
            feats.append(f)
            labels.append(l)
            viol += info["monotone_violations"]
            groups += info["groups"]
            law = per_law.setdefault(pr.name, np.zeros(3, np.int64))
            law += np.bincount(l, minlength=3)
    for pr in training_systems_bs64(a.bs64):
        f, l, info = label_problem(pr)
        feats.append(f)
        labels.append(l)
        viol += info["monotone_violations"]
        groups += info["groups"]
        law = per_law.setdefault(pr.name + "-bs64", np.zeros(3, np.int64))
        law += np.bincount(l, minlength=3)
    F = np.concatenate(feats)
    L = np.concatenate(labels)
    t1 = time.time()
    params, hist, acc = train(F, L, a.epochs, a.lr)
    theta_cap = safety_theta_from(F, L)
    theta, trail = validate_theta(params, theta_cap)
    ku = np.log10(kappa_u16(F))
    q = {f"label{c}": [round(float(np.percentile(ku[L == c], p)), 2) for p in (50, 90, 99, 99.9, 100)]
         for c in range(3) if (L == c).any()}
    meta = dict(systems=len(feats), samples=int(len(L)), label_counts=np.bincount(L, minlength=3).tolist(),
                label_counts_per_law={k: v.tolist() for k, v in per_law.items()},
                groups=groups, monotone_violations=viol, label_seconds=round(t1 - t0, 1),
                train_seconds=round(time.time() - t1, 1), final_loss=float(hist[-1]), train_accuracy=acc,
                epochs=a.epochs, lr=a.lr, safety_theta=theta, safety_theta_cap=theta_cap,
                safety_validation=[[round(t, 1), c] for t, c in trail],
                log10_kappa_u16_percentiles_50_90_99_99p9_100=q,
                laws=f"{nb32} systems of {', '.join(BATCH_LAWS)} in turn, blocks of 32, sides 20..32 "
                     f"({CORE_SIDES[0]}..{CORE_SIDES[1]} for mscore3d), seeds 1000..; "
                     f"{a.bs64} of aniso27 with blocks of 64, sides 12..18, seeds 5000..")
    save(params, a.out, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
