"""Host logic of the selector's labels (no GPU): the cost-aware choice of a group's class, the
monotonicity count, the safety threshold, and the statistics of the committed training labels."""
import json
import math
import os
from types import SimpleNamespace

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2407_15973_gb300 import selector as SEL  # noqa: E402


def _pr(nblocks=8, bs=32, nnz_per_row=7):
    n = nblocks * bs
    A = SimpleNamespace(n=n, nnz=nnz_per_row * n)
    return SimpleNamespace(A=A, block_ptr=np.arange(0, n + 1, bs, dtype=np.int32), nb=nblocks)


def _st(iters, converged=True):
    return {"iters": iters, "converged": converged}


def test_iteration_bytes_model():
    pr = _pr()
    n = pr.A.n
    fm = np.zeros(8, np.int64)
    assert SEL.iteration_bytes(pr, fm) == 12 * 7 * n + 92 * n + 8 * 32 * 32 * 8
    fm[:] = 2
    assert SEL.iteration_bytes(pr, fm) == 12 * 7 * n + 92 * n + 8 * 32 * 32 * 2


def test_label_is_the_class_of_least_modelled_time():
    pr = _pr()
    grp = np.repeat(np.arange(4), 2).astype(np.int32)          # 4 groups of 2 blocks
    base = _st(100)
    bytes0 = SEL.iteration_bytes(pr, np.zeros(8, np.int64))

    def dem(g, cls):
        fm = np.zeros(8, np.uint8)
        fm[grp == g] = 1 if cls == 1 else 2
        return fm

    res = {}
    # group 0: no delay in either class -> 16-bit (fewest bytes)
    res[(0, 1)] = (_st(100), dem(0, 1))
    res[(0, 2)] = (_st(100), dem(0, 2))
    # group 1: 16-bit fails to converge, FP32 no delay -> FP32
    res[(1, 1)] = (_st(100), dem(1, 1))
    res[(1, 2)] = (_st(40, False), dem(1, 2))
    # group 2: a delay that costs more than the saved bytes in both classes -> binary64
    res[(2, 1)] = (_st(130), dem(2, 1))
    res[(2, 2)] = (_st(140), dem(2, 2))
    # group 3: 16-bit pays, FP32 does not (a non-monotone group) -> 16-bit, counted
    b16 = SEL.iteration_bytes(pr, dem(3, 2).astype(np.int64))
    it16 = int(math.floor(100 * bytes0 / b16))                 # just below break-even
    res[(3, 1)] = (_st(150), dem(3, 1))
    res[(3, 2)] = (_st(it16), dem(3, 2))
    labels, viol = SEL.labels_from(pr, grp, base, res)
    assert labels.tolist() == [2, 2, 1, 1, 0, 0, 2, 2]
    assert viol == 1


def test_safety_theta_from_labels():
    feat = np.zeros((4, 12))
    feat[:, 0] = [1.0, 3.0, 5.0, 7.0]          # log10 kappa_1
    feat[:, 8] = [1.0, 1.0, 10.0, 1.0]         # dynamic range: block 2 needs bfloat16
    labels = np.array([2, 2, 2, 0])
    # 16-bit formats: FP16S (u = 2^-11) for blocks 0, 1, 3 and BF16 (u = 2^-8) for block 2
    theta = SEL.safety_theta_from(feat, labels, q=100.0)
    assert theta == pytest.approx(2 * 1e5 * 2.0 ** -8)
    ku = np.array([10 * 2.0 ** -11, 1e3 * 2.0 ** -11, 1e5 * 2.0 ** -8])
    assert SEL.safety_theta_from(feat, labels) == pytest.approx(2 * np.percentile(ku, 99))
    assert SEL.safety_theta_from(feat, np.zeros(4, int)) == 0.5


def test_committed_labels():
    # statistics the training run wrote beside the weights: the labels are mostly monotone
    # (16-bit paying while FP32 does not is rare), the laws where no storage format delays
    # the solve are labelled 16-bit, the multiscale core keeps binary64 / binary32 blocks
    with open(SEL.DEFAULT_WEIGHTS) as f:
        meta = json.load(f)["meta"]
    assert meta["systems"] == 2000 and meta["groups"] >= 15000
    assert meta["monotone_violations"] <= 0.05 * meta["groups"]
    per = meta["label_counts_per_law"]
    for law in ("subcube3d", "voronoi3d", "diff3d-rand"):
        c = np.array(per[law])
        assert c[2] >= 0.99 * c.sum(), (law, c)
    core = np.array(per["mscore3d"])
    assert core[0] + core[1] >= 0.1 * core.sum() and core[2] >= 0.2 * core.sum(), core
    assert 0.5 < meta["safety_theta"] < math.inf
    assert meta["train_accuracy"] >= 0.9
