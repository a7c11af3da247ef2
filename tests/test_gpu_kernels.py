"""Kernel-level parity of the CUDA path (through the C ABI) against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB
from gpu_util import csr_from_dense, cuda, host, need_gpu, spmv_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    return need_gpu()


def _long_row_matrix():
    # 6000 rows; row 7 is dense (spans several staging chunks), rows 100..109 are empty
    n = 6000
    rng = np.random.default_rng(0)
    rows, cols, vals = [], [], []
    for i in range(n):
        if 100 <= i < 110:
            continue
        if i == 7:
            c = np.arange(n)
        else:
            c = np.unique(np.concatenate([[i], rng.integers(0, n, 5)]))
        rows += [i] * len(c)
        cols += list(c)
        vals += list(rng.standard_normal(len(c)))
    import scipy.sparse as sp
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    M.sort_indices()
    return PB.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


SPMV_CASES = {
    "subcube24": lambda: PB.make_problem("subcube3d", seed=1, m=24).A,
    "ragged13": lambda: PB.make_problem("subcube3d", seed=2, m=13).A,
    "aniso27_12": lambda: PB.make_problem("aniso27", seed=3, m=12).A,
    "long_and_empty_rows": _long_row_matrix,
    "single_row": lambda: PB.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5])),
}


def test_spmv_integer_exact(B):
    A = PB.poisson2d_5pt_int(64)
    x = np.floor(PB.uniform(5, 7, A.n) * 2001) - 1000.0
    dA = B.DeviceCSR(A)
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    xy = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.bjac_spmv(dA, cuda(x), y, xy)
    ref = O.spmv(A, x)
    assert np.array_equal(host(y), ref)
    assert host(xy)[0] == float(np.dot(x, ref))    # integers below 2^53: exact in any order


@pytest.mark.parametrize("variant", [1, 2, 5])
@pytest.mark.parametrize("case", list(SPMV_CASES))
def test_spmv_parity(B, case, variant):
    A = SPMV_CASES[case]()
    x = PB.solution(A.n, 17)
    dA = B.DeviceCSR(A)
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    xy = torch.zeros(1, dtype=torch.float64, device="cuda")
    old = B.bjac_spmv_kernel(variant)
    try:
        B.bjac_spmv(dA, cuda(x), y, xy)
        ref = O.spmv(A, x)
        got = host(y)
        r = torch.empty(A.n, dtype=torch.float64, device="cuda")
        B.bjac_residual(dA, cuda(ref), cuda(x), r)
        res = host(r)
    finally:
        B.bjac_spmv_kernel(old)
    assert np.max(np.abs(got - ref)) <= spmv_tol(A, x)
    assert abs(host(xy)[0] - O.dot(x, ref)) <= 1e-14 * np.sum(np.abs(x * ref)) + 1e-300
    assert np.max(np.abs(res)) <= spmv_tol(A, x)


@pytest.mark.parametrize("case", list(SPMV_CASES))
def test_spmv_layouts_bitwise_equal(B, case):
    """Every SpMV kernel (two CSR kernels, the SELL-32 copy) sums each row as the same FMA
    chain in CSR order, so all give the same bits."""
    A = SPMV_CASES[case]()
    x = cuda(PB.solution(A.n, 23))
    dA = B.DeviceCSR(A)
    outs = []
    for variant in (1, 2, 5):
        y = torch.empty(A.n, dtype=torch.float64, device="cuda")
        old = B.bjac_spmv_kernel(variant)
        try:
            B.bjac_spmv(dA, x, y)
        finally:
            B.bjac_spmv_kernel(old)
        outs.append(host(y))
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint64), outs[0].view(np.uint64))


def _conversion_inputs():
    f32 = np.finfo(np.float32)
    tiny = float(f32.smallest_subnormal)
    vals = [0.0, -0.0, 1.0, -1.0, np.pi, 1.0 / 3.0, float(f32.max), -float(f32.max),
            float(f32.max) * (1 + 2.0 ** -25), float(f32.max) * (1 + 2.0 ** -24), 2.0 ** 128, 1e300, -1e300,
            float(f32.tiny), float(f32.tiny) * (1 - 2.0 ** -30), tiny, tiny * 0.5, tiny * 0.5000001, tiny * 1.5,
            tiny * 2.5, tiny * 0.49, 1e-50, -1e-50, 5e-324, -5e-324, 2.2250738585072014e-308,
            np.inf, -np.inf, np.nan,
            1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52, 1.0 - 2.0 ** -25]
    rng = np.random.default_rng(11)
    mag = 10.0 ** rng.uniform(-50, 40, 4000)
    rand = mag * rng.choice([-1.0, 1.0], 4000)
    sub = rng.integers(1, 2 ** 23, 2000) * tiny * rng.uniform(0.5, 1.5, 2000)    # around binary32 subnormals
    return np.concatenate([np.array(vals), rand, sub])


def test_integer_conversions_match_hardware_and_oracle(B):
    """The apply kernels' integer-only binary64 -> binary32 rounding and widening agree bit for
    bit with the hardware conversion and with the oracle's rounding (written independently
    from the IEEE 754 layout), across normal, subnormal, overflowing, infinite and NaN inputs."""
    x = _conversion_inputs()
    dx = cuda(x)
    f, w = B.bjac_convert(dx)
    fb = host(f).view(np.uint32)
    hw = host(dx.to(torch.float32)).view(np.uint32)
    nan = np.isnan(x)
    assert np.array_equal(fb[~nan], hw[~nan])
    assert np.all(np.isnan(host(f)[nan]))
    orc = O.round_bits(O.FP32, x)
    assert np.array_equal(fb[~nan], orc[~nan])
    wb = host(w)
    assert np.array_equal(wb[~nan].view(np.uint64), host(f.to(torch.float64))[~nan].view(np.uint64))
    assert np.all(np.isnan(wb[nan]))
    # widening alone: every binary32 class, including subnormal inputs
    fin = np.concatenate([np.array([0.0, -0.0, np.inf, -np.inf], np.float32),
                          (np.arange(1, 4096, dtype=np.uint32) * 2047).view(np.float32),
                          np.random.default_rng(12).standard_normal(3000).astype(np.float32) * 1e30])
    f2, w2 = B.bjac_convert(cuda(fin.astype(np.float64)))
    assert np.array_equal(host(f2).view(np.uint32), fin.view(np.uint32))
    assert np.array_equal(host(w2).view(np.uint64), fin.astype(np.float64).view(np.uint64))


def test_residual_parity(B):
    A = SPMV_CASES["subcube24"]()
    x, b = PB.solution(A.n, 3), PB.solution(A.n, 4) * 1e4
    dA = B.DeviceCSR(A)
    r = torch.empty(A.n, dtype=torch.float64, device="cuda")
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.bjac_residual(dA, cuda(b), cuda(x), r, rr)
    ref = O.residual(A, b, x)
    assert np.max(np.abs(host(r) - ref)) <= spmv_tol(A, x)
    assert abs(host(rr)[0] - O.dot(ref, ref)) <= 1e-12 * O.dot(ref, ref)


# ------------------------------------------------------------------------------------------
# setup: binary64 inverses, features, formats
# ------------------------------------------------------------------------------------------
LAYOUTS = {
    "bs32": lambda: PB.make_problem("subcube3d", seed=5, m=16, bs=32),
    "bs64": lambda: PB.make_problem("subcube3d", seed=6, m=16, bs=64),
    "bs16": lambda: PB.make_problem("subcube3d", seed=7, m=16, bs=16),
    "bs8_poisson": lambda: PB.make_problem("poisson2d", bs=8),
    "ragged_bs32": lambda: PB.make_problem("subcube3d", seed=8, m=13, bs=32),
    "uneven_voronoi": lambda: PB.make_problem("voronoi3d", seed=9, m=20),
    "bs128_aniso": lambda: PB.make_problem("aniso27", seed=10, m=10, bs=128),
}


@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_setup_inverse_parity(B, layout):
    pr = LAYOUTS[layout]()
    P = O.Preconditioner(pr.A, pr.block_ptr)
    feat_o = O.features(pr.A, P)
    dA = B.DeviceCSR(pr.A)
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_UNIFORM)
    ex = h.export()
    assert np.all(ex["fmt"] == B.FP64)
    kap = 10.0 ** feat_o[:, 0]
    u = 2.0 ** -53
    for b in range(P.nb):
        bs = pr.block_ptr[b + 1] - pr.block_ptr[b]
        g_o = O.block_of(P.G, P.goff, pr.block_ptr, b)
        g_d = ex["G"][P.goff[b]:P.goff[b + 1]].reshape(bs, bs)
        assert np.array_equal(g_d, g_d.T)
        assert np.max(np.abs(g_d - g_o)) <= 8 * bs * kap[b] * u * np.abs(g_o).max(), b
    # features: CSR-derived ones to 1e-12 relative; the two from G within the inverse error
    fd = ex["feat"]
    for k in (1, 2, 3, 4, 5, 6, 7, 9, 10, 11):
        assert np.allclose(fd[:, k], feat_o[:, k], rtol=1e-12, atol=1e-12), k
    bsz = np.diff(pr.block_ptr)
    assert np.all(np.abs(fd[:, 0] - feat_o[:, 0]) <= 1e-12 + 8 * bsz * kap * u)
    # log10 dynamic range uses the smallest entry of G, whose relative error can be larger
    assert np.allclose(fd[:, 8], feat_o[:, 8], rtol=0, atol=1e-2)
    h.close()


def _hard_residual(n):
    """Random residual with binary32 rounding ties, near-ties, zeros and values outside the
    normal binary32 range mixed in, so that ConvertPrecision's edge cases are exercised."""
    r = PB.solution(n, 21) * 1e3
    rng = np.random.default_rng(7)
    k = n // 8
    idx = rng.choice(n, size=min(n, 6 * k), replace=False)
    e = rng.integers(-20, 20, k).astype(float)
    mant = rng.integers(0, 2 ** 23, k)
    base = (1 + mant / 2.0 ** 23) * 2.0 ** e
    half = 2.0 ** (e - 24)
    vals = [base + half, -(base + half), base + half * (1 + 2.0 ** -29), base + half * (1 - 2.0 ** -29),
            np.zeros(k), np.full(k, 1e-40)]
    r[idx] = np.concatenate(vals)[:len(idx)]
    r[idx[:2]] = [3e39, 5e-46]     # binary32 overflow to inf and underflow to zero
    return r


@pytest.mark.parametrize("fmt", [1, 2, 3])
@pytest.mark.parametrize("layout", ["bs32", "bs64", "bs16", "uneven_voronoi", "ragged_bs32", "bs128_aniso"])
def test_pack_and_apply_bitwise(B, fmt, layout):
    """Same binary64 inverses on both sides -> identical format bits, scales and z."""
    pr = LAYOUTS[layout]()
    P = O.Preconditioner(pr.A, pr.block_ptr, fmt=fmt)
    dA = B.DeviceCSR(pr.A)
    outs = []
    for variant in (0, 1, 2, 3):     # autotuned, generic, TMA-staged, register-direct kernel
        h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_FIXED, fixed_fmt=fmt, fp64_fallback=True,
                         apply_variant=variant)
        h.import_inverse(P.G)
        ex = h.export()
        assert np.array_equal(ex["scale"], P.scale)
        for b in range(P.nb):
            bs = pr.block_ptr[b + 1] - pr.block_ptr[b]
            nbytes = bs * bs * (4 if fmt == 1 else 2)
            assert np.array_equal(ex["pool"][ex["qoff"][b]:ex["qoff"][b] + nbytes],
                                  P.pool[P.qoff[b]:P.qoff[b] + nbytes]), b
        r = _hard_residual(pr.A.n)
        z = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
        rz = torch.zeros(1, dtype=torch.float64, device="cuda")
        h.apply(cuda(r), z, set=1, rz=rz)
        zo = O.apply(P.block_ptr, P.fmt, P.pool, P.qoff, P.scale, r, mode=1)
        zd = host(z)
        assert np.array_equal(zd, zo, equal_nan=True)
        fin = np.isfinite(zo)
        assert fin.mean() > 0.85       # one block holds the overflowing entry
        if fin.all():
            assert abs(host(rz)[0] - O.dot(r, zo)) <= 1e-13 * np.sum(np.abs(r * zo))
        outs.append(zd)
        h.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o, equal_nan=True)


@pytest.mark.parametrize("layout", ["bs32", "bs64", "uneven_voronoi"])
def test_apply_fp64_set(B, layout):
    pr = LAYOUTS[layout]()
    P = O.Preconditioner(pr.A, pr.block_ptr)
    dA = B.DeviceCSR(pr.A)
    h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_UNIFORM)
    h.import_inverse(P.G)
    r = PB.solution(pr.A.n, 22)
    z = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
    h.apply(cuda(r), z, set=0)
    zo = O.apply_fp64(P.block_ptr, P.G, P.goff, r)
    bound = np.zeros(pr.A.n)
    for b in range(P.nb):
        s, e = pr.block_ptr[b], pr.block_ptr[b + 1]
        bound[s:e] = 2 * (e - s) * 2.0 ** -53 * (np.abs(O.block_of(P.G, P.goff, pr.block_ptr, b)) @ np.abs(r[s:e]))
    assert np.all(np.abs(host(z) - zo) <= bound)
    h.close()


def test_rule_formats_match_oracle(B):
    # coefficient 10^U[0,2] per node, no time-step shift: block condition numbers straddle
    # the bfloat16 / binary32 boundary of the rule (kappa_1 = 25.6 at theta = 0.1)
    A = PB.fdm3d_7pt(*(3 * [np.power(10.0, 2 * PB.uniform(4, 61, 16 ** 3)).reshape(16, 16, 16)]))
    bp = PB.uniform_blocks(A.n, 16)
    P = O.Preconditioner(A, bp)
    feat = O.features(A, P)
    ref = O.select_rule(feat, 0.1)
    h = B.bjac_setup(B.DeviceCSR(A), bp, select=B.SELECT_RULE, theta=0.1)
    got = h.export()["fmt"]
    l2 = np.log10(2.0)
    lk, ldr = feat[:, 0], feat[:, 8]
    near = np.zeros(len(ref), bool)
    for t in (np.log10(0.1) + 11 * l2, np.log10(0.1) + 8 * l2, np.log10(0.1) + 24 * l2):
        near |= np.abs(lk - t) < 1e-9
    near |= np.abs(ldr - 29 * l2) < 1e-6
    assert np.array_equal(got[~near], ref[~near])
    assert len(set(ref.tolist())) >= 2      # the case really exercises several formats
    h.close()


# ------------------------------------------------------------------------------------------
# argument and numerical errors (all detected without faulting the GPU)
# ------------------------------------------------------------------------------------------
def test_not_spd_block_is_reported(B):
    D = np.diag([2.0, -1.0, 3.0, 4.0])
    h = None
    with pytest.raises(B.MpbjacError) as e:
        h = B.bjac_setup(B.DeviceCSR(csr_from_dense(D)), np.array([0, 2, 4], np.int32), select=B.SELECT_UNIFORM)
    assert e.value.code == B.ERR_NOT_SPD and h is None


def test_invalid_inputs_rejected(B):
    A = PB.poisson2d_5pt_int(8)
    dA = B.DeviceCSR(A)
    for bp in ([0, 32, 63], [1, 64], [0, 0, 64], [0, 200, 64]):
        with pytest.raises(B.MpbjacError) as e:
            B.bjac_setup(dA, np.array(bp, np.int32))
        assert e.value.code == B.ERR_INVALID_ARG
    bad = PB.CSR(A.n, A.rowptr, A.colidx.copy(), A.val)
    bad.colidx[5] = A.n + 3
    with pytest.raises(B.MpbjacError) as e:
        B.bjac_setup(B.DeviceCSR(bad), PB.uniform_blocks(A.n, 8))
    assert e.value.code == B.ERR_INVALID_ARG


@pytest.mark.parametrize("m", [16, 32])
def test_mixed_format_register_apply_bitwise(B, m):
    """Per-block formats (as the kappa rule or the learned selector assign them) on 32-row blocks:
    the mixed-format register kernel gives the generic kernel's z bit for bit, and both give the
    oracle's z bit for bit on the low-precision blocks (binary32 products in natural order) and
    within the binary64 dot-product bound on the binary64 blocks (the kernels contract with FMA)."""
    pr = PB.make_problem("subcube3d", seed=30 + m, m=m, bs=32)
    fmt = np.random.default_rng(m).integers(0, 4, len(pr.block_ptr) - 1).astype(np.uint8)
    fmt[:4] = [0, 1, 2, 3]
    P = O.Preconditioner(pr.A, pr.block_ptr, fmt=fmt)
    dA = B.DeviceCSR(pr.A)
    r = _hard_residual(pr.A.n)
    zo = O.apply(P.block_ptr, P.fmt, P.pool, P.qoff, P.scale, r, mode=1)
    row_fmt = np.repeat(fmt, 32)
    low = row_fmt != 0
    bound = np.zeros(pr.A.n)
    for b in np.nonzero(fmt == 0)[0]:
        s, e = pr.block_ptr[b], pr.block_ptr[b + 1]
        bound[s:e] = 2 * 32 * 2.0 ** -53 * (np.abs(O.block_of(P.G, P.goff, pr.block_ptr, b)) @ np.abs(r[s:e]))
    kinds, outs = [], []
    for variant in (4, 1, 0):
        h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_GIVEN, block_fmt=fmt, apply_variant=variant,
                         fp64_fallback=True)    # keeps the binary64 set that import_inverse overwrites
        try:
            h.import_inverse(P.G)
            kinds.append(h.apply_kernel()[0])
            z = torch.empty(pr.A.n, dtype=torch.float64, device="cuda")
            rz = torch.zeros(1, dtype=torch.float64, device="cuda")
            h.apply(cuda(r), z, set=1, rz=rz)
            zd = host(z)
            assert np.array_equal(zd[low], zo[low], equal_nan=True), variant
            assert np.all(np.abs(zd[~low] - zo[~low]) <= bound[~low]), variant
            fin = np.isfinite(zo)
            if fin.all():
                assert abs(host(rz)[0] - O.dot(r, zo)) <= 1e-13 * np.sum(np.abs(r * zo))
            outs.append(zd)
        finally:
            h.close()
    assert kinds == ["mixed", "generic", "mixed"], kinds
    for o in outs[1:]:
        assert np.array_equal(outs[0], o, equal_nan=True)


def test_mixed_format_register_pcg(B):
    """PCG with per-block formats through the mixed-format register kernel against the oracle."""
    pr = PB.make_problem("subcube3d", seed=44, m=24, bs=32)
    fmt = np.random.default_rng(3).integers(0, 4, len(pr.block_ptr) - 1).astype(np.uint8)
    P = O.Preconditioner(pr.A, pr.block_ptr, fmt=fmt)
    b = O.spmv(pr.A, pr.x_star)
    ref = O.pcg(pr.A, P, b, tol=1e-10, maxit=5000, policy=O.POLICY_FMP)
    dA = B.DeviceCSR(pr.A)
    iters = []
    for variant in (4, 1):
        h = B.bjac_setup(dA, pr.block_ptr, select=B.SELECT_GIVEN, block_fmt=fmt, apply_variant=variant)
        x = torch.zeros(pr.A.n, dtype=torch.float64, device="cuda")
        st = h.solve(cuda(b), x, tol=1e-10, maxit=5000)
        h.close()
        assert st["converged"] and st["true_relres"] <= 1e-10
        iters.append(st["iters"])
    assert ref["converged"]
    for it in iters:
        assert abs(it - ref["iters"]) <= max(3, 0.02 * ref["iters"]), (iters, ref["iters"])
