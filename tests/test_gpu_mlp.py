"""The selector's GPU forward / backward kernels against the oracle's binary64 MLP."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import cuda, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    return need_gpu()


def _data(seed, n=300):
    rng = np.random.default_rng(seed)
    feat = rng.standard_normal((n, 12)) * rng.uniform(0.5, 3, 12) + rng.uniform(-2, 2, 12)
    params = np.zeros(5187 + 24, np.float32)
    params[:5187] = (rng.standard_normal(5187) * 0.3).astype(np.float32)
    params[5187:5199] = feat.mean(0)
    params[5199:5211] = feat.std(0)
    label = rng.integers(0, 3, n).astype(np.int32)
    return feat, params, label


def _xin(feat, params):
    mu = params[5187:5199].astype(np.float64)
    sd = params[5199:5211].astype(np.float64)
    return (feat - mu) / sd


def _bf16(w):
    return O.decode(O.BF16, O.round_bits(O.BF16, w.astype(np.float64)))


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_fp32_weights_match_oracle(B, seed):
    feat, params, label = _data(seed)
    loss, g = B.bjac_mlp_grad(params, cuda(feat), cuda(label, torch.int32), bf16_weights=False)
    lo, go = O.mlp_loss_grad(params[:5187].astype(np.float64), _xin(feat, params), label)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    assert np.max(np.abs(g[big] - go[big]) / np.abs(go[big])) <= 1e-3


@pytest.mark.parametrize("tensor_cores", [True, False])
def test_gradient_bf16_weights(B, tensor_cores):
    feat, params, label = _data(2)
    loss, g = B.bjac_mlp_grad(params, cuda(feat), cuda(label, torch.int32), bf16_weights=True,
                              tensor_cores=tensor_cores)
    # the weights inference uses: each one rounded to bfloat16
    w16 = _bf16(params[:5187])
    lo16, go16 = O.mlp_loss_grad(w16, _xin(feat, params), label)
    assert abs(loss - lo16) <= 1e-5 * abs(lo16)
    assert np.linalg.norm(g - go16) <= 1e-4 * np.linalg.norm(go16)
    # and against the unrounded binary32 weights (the stated 2e-2)
    lo, go = O.mlp_loss_grad(params[:5187].astype(np.float64), _xin(feat, params), label)
    assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go)


@pytest.mark.parametrize("n", [1, 127, 128, 129, 5000, 200_003])
def test_tensor_core_gradient(B, n):
    # the tcgen05 gradient (layer 2's forward product, back-propagation and weight gradient as
    # BF16 MMAs; 128-sample tiles, a ragged last tile, and at 200,003 samples several tiles per
    # CTA accumulated in TMEM) against the oracle's binary64 gradient with the same rounded
    # weights, block by block of the parameter vector so that a wrong operand in one product
    # (W2's gradient comes only from the MMA, b2 and W1 only through it) fails on its own.
    # Taking hi.hi alone for the weight gradient would leave a relative error near 2^-9.
    rng = np.random.default_rng(100 + n)
    feat = rng.standard_normal((n, 12)) * rng.uniform(0.5, 3, 12) + rng.uniform(-2, 2, 12)
    _, params, _ = _data(11)
    label = rng.integers(0, 3, n).astype(np.int32)
    loss, g = B.bjac_mlp_grad(params, cuda(feat), cuda(label, torch.int32))
    lo16, go16 = O.mlp_loss_grad(_bf16(params[:5187]), _xin(feat, params), label)
    assert np.all(np.isfinite(g))
    assert abs(loss - lo16) <= 1e-5 * abs(lo16)
    parts = {"W1": (0, 768), "b1": (768, 832), "W2": (832, 4928), "b2": (4928, 4992), "W3": (4992, 5184),
             "b3": (5184, 5187)}
    for name, (a, b) in parts.items():
        ref = go16[a:b]
        assert np.linalg.norm(g[a:b] - ref) <= 1e-4 * np.linalg.norm(ref) + 1e-9, name
    # the same weights on CUDA cores
    _, gc = B.bjac_mlp_grad(params, cuda(feat), cuda(label, torch.int32), tensor_cores=False)
    assert np.linalg.norm(g - gc) <= 1e-4 * np.linalg.norm(gc)


def test_gradient_rejects_unknown_mode(B):
    feat, params, label = _data(3)
    g = np.zeros(5187, np.float32)
    dfeat, dlabel = cuda(feat), cuda(label, torch.int32)
    for mode in (-1, 3):
        rc = B.lib().bjac_mlp_grad(params.ctypes.data, mode, dfeat.data_ptr(), dlabel.data_ptr(), len(feat),
                                   g.ctypes.data, None, None)
        assert rc == B.ERR_INVALID_ARG


def test_logits_match_oracle(B):
    feat, params, label = _data(3)
    out = B.bjac_mlp_logits(params, cuda(feat), bf16_weights=False)
    ref = O.mlp_forward(params[:5187].astype(np.float64), _xin(feat, params))
    assert np.max(np.abs(out - ref)) <= 1e-5 * max(1.0, np.abs(ref).max())
    out16 = B.bjac_mlp_logits(params, cuda(feat), bf16_weights=True)
    ref16 = O.mlp_forward(_bf16(params[:5187]), _xin(feat, params))
    assert np.max(np.abs(out16 - ref16)) <= 1e-5 * max(1.0, np.abs(ref16).max())


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 200_003])
def test_tensor_core_logits(B, n):
    # the tcgen05 forward pass (bfloat16 weights; 128-sample tiles, a ragged last tile, and at
    # 200,003 rows several tiles per CTA) against the oracle's binary64 forward pass with the same
    # rounded weights, and against the CUDA-core kernel. Dropping the low bfloat16 part of the
    # hidden values would leave a relative error near 2^-9, far above the bound.
    rng = np.random.default_rng(n)
    feat, params, _ = _data(7, n=max(n, 300))
    feat = feat[rng.permutation(len(feat))[:n]] if n <= len(feat) else feat
    feat = np.ascontiguousarray(feat[:n])
    out = B.bjac_mlp_logits(params, cuda(feat))
    ref = O.mlp_forward(_bf16(params[:5187]), _xin(feat, params))
    assert np.all(np.isfinite(out))
    assert np.max(np.abs(out - ref)) <= 1e-5 * max(1.0, np.abs(ref).max())
    cc = B.bjac_mlp_logits(params, cuda(feat), tensor_cores=False)
    assert np.max(np.abs(out - cc)) <= 1e-5 * max(1.0, np.abs(cc).max())


def test_logits_rejects_unknown_mode(B):
    feat, params, _ = _data(3)
    dfeat = cuda(feat)
    out = np.zeros(3 * len(feat), np.float32)
    for mode in (-1, 3):
        rc = B.lib().bjac_mlp_logits(params.ctypes.data, mode, dfeat.data_ptr(), len(feat), out.ctypes.data, None)
        assert rc == B.ERR_INVALID_ARG


def test_training_learns_a_separable_rule(B):
    rng = np.random.default_rng(9)
    feat = rng.standard_normal((2000, 12))
    label = np.where(feat[:, 0] > 0.5, 2, np.where(feat[:, 1] > 0, 1, 0)).astype(np.int32)
    from paper_2407_15973_gb300 import selector
    params, hist, acc = selector.train(feat, label, epochs=300, lr=1e-2)
    assert hist[-1] < 0.5 * hist[0]
    assert acc > 0.95


def test_setup_mlp_selection_follows_the_network(B):
    from paper_2407_15973_gb300 import problems as PB
    from paper_2407_15973_gb300 import selector
    pr = PB.make_problem("aniso27", seed=5, m=14, bs=64)
    dA = B.DeviceCSR(pr.A)
    hu = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_UNIFORM)
    feat = hu.export()["feat"]
    hu.close()
    rng = np.random.default_rng(4)
    params = selector.init_params(feat, seed=3)
    params[5187 - 3:5187] = rng.standard_normal(3).astype(np.float32)     # move the class biases
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_MLP, mlp_params=params, safety_theta=1e30)
    got = h.export()["fmt"]
    h.close()
    cls = np.argmax(B.bjac_mlp_logits(params, cuda(feat)), axis=1)
    expect = np.where(cls == 0, B.FP64, np.where(cls == 1, B.FP32, selector.sixteen_bit(feat)))
    assert np.array_equal(got, expect)
