"""Pins for the CPU oracle against facts fixed outside it (no GPU).

Each test checks the oracle against something it does not compute itself: closed forms,
brute force on tiny inputs, an independent library routine (numpy / scipy), or numbers
printed in the paper (tests/golden/).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2407_15973_gb300 import problems as PB

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# SpMV (working-precision product of PCG, Section 3.2)
# ---------------------------------------------------------------------------------------
def test_spmv_exact_on_integers(oracle):
    A = PB.poisson2d_5pt_int(64)
    x = np.floor(PB.uniform(3, 7, A.n) * 2001) - 1000.0
    dense = A.to_scipy().toarray()
    assert np.array_equal(oracle.spmv(A, x), dense @ x)


def test_spmv_laplacian_eigenvector(oracle):
    # integer 5-point stencil on an m x m grid: v(i,j) = sin(p pi (i+1)/(m+1)) sin(q pi (j+1)/(m+1))
    # is an eigenvector with lambda = 4 sin^2(p pi / (2(m+1))) + 4 sin^2(q pi / (2(m+1)))
    m = 40
    A = PB.poisson2d_5pt_int(m)
    idx = np.arange(m * m)
    i, j = idx % m, idx // m
    for p, q in [(1, 1), (3, 7), (40, 1), (17, 23)]:
        v = np.sin(p * math.pi * (i + 1) / (m + 1)) * np.sin(q * math.pi * (j + 1) / (m + 1))
        lam = 4 * math.sin(p * math.pi / (2 * (m + 1))) ** 2 + 4 * math.sin(q * math.pi / (2 * (m + 1))) ** 2
        assert np.max(np.abs(oracle.spmv(A, v) - lam * v)) < 1e-13


def test_spmv_rounding_bound_exact_rational(oracle):
    pr = PB.make_problem("subcube3d", seed=2, m=16)
    A = pr.A
    x = pr.x_star
    y = oracle.spmv(A, x)
    u = 2.0 ** -53
    for row in range(0, A.n, 97):
        lo, hi = A.rowptr[row], A.rowptr[row + 1]
        exact = sum(Fraction(float(A.val[k])) * Fraction(float(x[A.colidx[k]])) for k in range(lo, hi))
        absrow = sum(abs(float(A.val[k]) * float(x[A.colidx[k]])) for k in range(lo, hi))
        k = hi - lo
        gamma = k * u / (1 - k * u)
        assert abs(Fraction(float(y[row])) - exact) <= Fraction(gamma * absrow * 1.0000001)


# ---------------------------------------------------------------------------------------
# Block inverses (Eq. 3-1 with exact D_b^-1)
# ---------------------------------------------------------------------------------------
def _cheb_u(k, t):
    if k < 0:
        return 0.0
    u0, u1 = 1.0, 2 * t
    if k == 0:
        return u0
    for _ in range(k - 1):
        u0, u1 = u1, 2 * t * u1 - u0
    return u1


def test_block_inverse_tridiagonal_closed_form(oracle):
    # the blocks of 8 rows of the 64x64 integer Poisson matrix lie inside one grid line,
    # so each is tridiag(-1, 4, -1); (T^-1)_ij = U_{i-1}(2) U_{8-j}(2) / U_8(2), i <= j (1-based)
    pr = PB.make_problem("poisson2d")
    G, goff, _, bad = oracle.block_inverse(pr.A, pr.block_ptr)
    assert bad == 0
    m, t = 8, 2.0
    T = np.zeros((m, m))
    for i in range(1, m + 1):
        for j in range(1, m + 1):
            a, c = min(i, j), max(i, j)
            T[i - 1, j - 1] = _cheb_u(a - 1, t) * _cheb_u(m - c, t) / _cheb_u(m, t)
    for b in (0, 1, 17, pr.nb - 1):
        Gb = oracle.block_of(G, goff, pr.block_ptr, b)
        assert np.max(np.abs(Gb - T)) < 1e-15


@pytest.mark.parametrize("name,kw", [("poisson2d", {}), ("subcube3d", {"m": 16}), ("subcube3d", {"m": 16, "bs": 64})])
def test_block_inverse_identity(oracle, name, kw):
    pr = PB.make_problem(name, seed=1, **kw)
    G, goff, _, bad = oracle.block_inverse(pr.A, pr.block_ptr)
    assert bad == 0
    dense = pr.A.to_scipy()
    for b in range(0, pr.nb, max(1, pr.nb // 40)):
        s, e = pr.block_ptr[b], pr.block_ptr[b + 1]
        B = dense[s:e, s:e].toarray()
        Gb = oracle.block_of(G, goff, pr.block_ptr, b)
        assert np.array_equal(Gb, Gb.T)
        scale = np.abs(Gb).max() * np.abs(B).max()
        assert np.max(np.abs(Gb @ B - np.eye(e - s))) <= 1e-13 * max(1.0, scale / 1.0) * 1.0
        # independent library inverse
        Ginv = np.linalg.inv(B)
        assert np.max(np.abs(Gb - Ginv)) <= 1e-12 * np.abs(Ginv).max() * np.linalg.cond(B, 1) / 1e2 + 1e-300


def test_block_inverse_random_spd_vs_numpy(oracle):
    rng = np.random.default_rng(5)
    sizes = [1, 3, 16, 37, 64, 128]
    rows, cols, vals, bp = [], [], [], [0]
    off = 0
    for bs in sizes:
        Q = rng.standard_normal((bs, bs))
        B = Q @ Q.T + bs * np.eye(bs)
        r, c = np.nonzero(np.ones((bs, bs)))
        rows.append(r + off); cols.append(c + off); vals.append(B[r, c])
        off += bs
        bp.append(off)
    import scipy.sparse as sp
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(off, off))
    M.sort_indices()
    A = PB.CSR(off, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    G, goff, n1, bad = oracle.block_inverse(A, np.array(bp, np.int32))
    assert bad == 0
    for b, bs in enumerate(sizes):
        s = bp[b]
        B = M[s:s + bs, s:s + bs].toarray()
        Gb = oracle.block_of(G, goff, np.array(bp), b)
        ref = np.linalg.inv(B)
        assert np.allclose(Gb, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
        assert n1[b] == pytest.approx(np.abs(B).sum(axis=0).max(), rel=1e-15)


def test_block_inverse_singular_block_reported(oracle):
    # a 2x2 block [[1,1],[1,1]] is singular
    A = PB.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.ones(4))
    _, _, _, bad = oracle.block_inverse(A, np.array([0, 2], np.int32))
    assert bad == 1


# ---------------------------------------------------------------------------------------
# ConvertPrecision (Algorithm 3.1) from the bit layouts
# ---------------------------------------------------------------------------------------
def _hard_doubles(rng, count):
    """Random doubles plus exact ties / near-ties of the 32/16-bit grids and edge values."""
    x = rng.standard_normal(count) * np.exp(rng.uniform(-30, 30, count))
    ties = []
    for mb, lo, hi in [(23, -140, 120), (10, -24, 15), (7, -130, 120)]:
        e = rng.integers(lo, hi, 200)
        mant = rng.integers(0, 2 ** mb, 200)
        base = (1 + mant / 2.0 ** mb) * 2.0 ** e
        half = 2.0 ** (e - mb - 1)
        ties += list(base + half) + list(base + half * (1 + 2.0 ** -30)) + list(base + half * (1 - 2.0 ** -30))
    special = [0.0, -0.0, 65504.0, 65519.99, 65520.0, 2.0 ** -24, 2.0 ** -25, 2.0 ** -25 * 1.0000001,
               3.4028234663852886e38, 3.4028235677973366e38, 1e-45, 1.4e-45, 7e-46, 1e300, -1e300,
               2.0 ** -149, 2.0 ** -150, 2.0 ** -126, 1.1754942e-38]
    return np.concatenate([x, np.array(ties), np.array(special), -np.array(ties)])


def test_round_fp32_matches_numpy(oracle):
    x = _hard_doubles(np.random.default_rng(0), 20000)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).view(np.uint32)
    assert np.array_equal(oracle.round_bits(oracle.FP32, x), ref)


def test_round_fp16_matches_numpy_direct_rounding(oracle):
    x = _hard_doubles(np.random.default_rng(1), 20000)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(oracle.round_bits(oracle.FP16S, x), ref)
    # a value just above a binary16 tie must not be double-rounded through binary32
    assert oracle.decode(oracle.FP16S, oracle.round_bits(oracle.FP16S, np.array([1 + 2 ** -11 + 2 ** -40])))[0] == 1 + 2 ** -10


def _bf16_brute(x: float) -> int:
    """Nearest bfloat16 by exact rational comparison over the two neighbouring candidates."""
    if x == 0:
        return 0x8000 if math.copysign(1, x) < 0 else 0
    sign = 0x8000 if x < 0 else 0
    a = Fraction(abs(x))
    best = None
    # candidates: truncation toward zero of the binary32 pattern and its successor
    import struct
    f32 = struct.unpack("<I", struct.pack("<f", np.float32(abs(x)) if abs(x) < 3.4e38 else np.float32(3.4e38)))[0]
    base = f32 >> 16
    cands = [c for c in (base - 1, base, base + 1, base + 2) if 0 <= c <= 0x7F80]

    def val(c):
        if c == 0x7F80:
            return None
        e, mnt = c >> 7, c & 0x7F
        if e == 0:
            return Fraction(mnt, 2 ** 7) * Fraction(2) ** (-126)
        return (1 + Fraction(mnt, 2 ** 7)) * Fraction(2) ** (e - 127)

    for c in cands:
        v = val(c)
        if v is None:
            continue
        d = abs(v - a)
        if best is None or d < best[0] or (d == best[0] and (c & 1) == 0):
            best = (d, c)
    return sign | best[1]


def test_round_bf16_matches_brute_force(oracle):
    rng = np.random.default_rng(2)
    x = _hard_doubles(rng, 3000)
    x = x[np.abs(x) < 3.0e38]
    got = oracle.round_bits(oracle.BF16, x)
    for xi, gi in zip(x.tolist(), got.tolist()):
        assert gi == _bf16_brute(xi), (xi, hex(gi))


def test_decode_roundtrip(oracle):
    bits = np.arange(0, 0x7C00, 37, dtype=np.uint16)
    vals = oracle.decode(oracle.FP16S, bits)
    assert np.array_equal(vals, bits.view(np.float16).astype(np.float64))
    assert np.array_equal(oracle.round_bits(oracle.FP16S, vals), bits)


# ---------------------------------------------------------------------------------------
# Packing and apply (Algorithm 3.1)
# ---------------------------------------------------------------------------------------
def test_pack_scale_and_accuracy(oracle):
    pr = PB.make_problem("subcube3d", seed=3, m=16)
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    for f, u in [(oracle.FP32, 2.0 ** -24), (oracle.BF16, 2.0 ** -8), (oracle.FP16S, 2.0 ** -11)]:
        P.set_formats(f)
        for b in range(0, P.nb, 17):
            bs = pr.block_ptr[b + 1] - pr.block_ptr[b]
            raw = P.pool[P.qoff[b]:P.qoff[b + 1]]
            bits = raw.view(np.uint32 if f == oracle.FP32 else np.uint16)
            Q = oracle.decode(f, bits).reshape(bs, bs)
            Gb = oracle.block_of(P.G, P.goff, pr.block_ptr, b)
            s = float(P.scale[b])
            if f in (oracle.BF16, oracle.FP16S):
                assert 2 ** 14 <= np.abs(Q).max() < 2 ** 15
                assert math.log2(s) == int(math.log2(s))
            else:
                assert s == 1.0
            big = np.abs(Gb) >= np.abs(Gb).max() * 2.0 ** -20
            assert np.all(np.abs(Q * s - Gb)[big] <= u * np.abs(Gb)[big])
            assert np.array_equal(Q, Q.T)


def test_apply_point_jacobi_and_inverse(oracle):
    pr = PB.make_problem("subcube3d", seed=4, m=8, bs=1)
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    r = PB.solution(pr.A.n, 9)
    diag = pr.A.to_scipy().diagonal()
    assert np.allclose(oracle.apply_fp64(P.block_ptr, P.G, P.goff, r), r / diag, rtol=1e-15, atol=0)
    pr = PB.make_problem("subcube3d", seed=4, m=16)
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    dense = pr.A.to_scipy()
    Bd = np.zeros(pr.A.n)
    x = PB.solution(pr.A.n, 10)
    for b in range(P.nb):
        s, e = pr.block_ptr[b], pr.block_ptr[b + 1]
        Bd[s:e] = dense[s:e, s:e] @ x[s:e]
    assert np.allclose(oracle.apply_fp64(P.block_ptr, P.G, P.goff, Bd), x, rtol=0, atol=1e-12)


def test_apply_fp32_emulation_within_bound(oracle):
    pr = PB.make_problem("subcube3d", seed=5, m=16, bs=64)
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    r = PB.solution(pr.A.n, 11) * 1e3
    for f in (oracle.FP32, oracle.BF16, oracle.FP16S):
        P.set_formats(f)
        z0 = oracle.apply(P.block_ptr, P.fmt, P.pool, P.qoff, P.scale, r, mode=0)
        z1 = oracle.apply(P.block_ptr, P.fmt, P.pool, P.qoff, P.scale, r, mode=1)
        rh = r.astype(np.float32).astype(np.float64)
        for b in range(0, P.nb, 5):
            s, e = pr.block_ptr[b], pr.block_ptr[b + 1]
            bs = e - s
            raw = P.pool[P.qoff[b]:P.qoff[b + 1]]
            Q = oracle.decode(f, raw.view(np.uint32 if f == oracle.FP32 else np.uint16)).reshape(bs, bs)
            bound = (bs + 2) * 2.0 ** -24 * float(P.scale[b]) * (np.abs(Q) @ np.abs(rh[s:e]))
            assert np.all(np.abs(z1[s:e] - z0[s:e]) <= bound)
            assert np.allclose(z0[s:e], float(P.scale[b]) * (Q @ rh[s:e]), rtol=1e-13, atol=0)


# ---------------------------------------------------------------------------------------
# PCG with BJAC and the precision policies (Algorithms 3.1-3.3, Section 4.2)
# ---------------------------------------------------------------------------------------
def test_pcg_block_size_one_is_point_jacobi_scipy(oracle):
    import scipy.sparse.linalg as spla
    pr = PB.make_problem("subcube3d", seed=6, m=12, bs=1)
    b = oracle.spmv(pr.A, pr.x_star)
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    res = oracle.pcg(pr.A, P, b, tol=1e-10, maxit=5000)
    M = pr.A.to_scipy()
    dinv = 1.0 / M.diagonal()
    count = [0]
    x, info = spla.cg(M, b, rtol=1e-10, atol=0.0, maxiter=5000,
                      M=spla.LinearOperator(M.shape, matvec=lambda v: dinv * v),
                      callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert info == 0 and res["converged"]
    assert abs(res["iters"] - count[0]) <= 1
    assert np.linalg.norm(res["x"] - x) <= 1e-8 * np.linalg.norm(x)


def test_pcg_single_block_converges_in_one_iteration(oracle):
    A = PB.poisson2d_5pt_int(20)     # n = 400 <= 1024
    x_star = PB.solution(A.n, 12)
    b = oracle.spmv(A, x_star)
    P = oracle.Preconditioner(A, np.array([0, A.n], np.int32))
    res = oracle.pcg(A, P, b, tol=1e-10, maxit=50)
    assert res["converged"] and res["iters"] == 1
    assert np.max(np.abs(res["x"] - x_star)) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_pcg_tiny_spd_within_n_iterations(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 17))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    # CG ends within n steps in exact arithmetic; in binary64 the loss of orthogonality
    # adds a few steps that grow with kappa, so the eigenvalues span at most 1e2 here
    lam = np.exp(rng.uniform(0, math.log(1e2), n))
    D = (Q * lam) @ Q.T
    D = 0.5 * (D + D.T)
    import scipy.sparse as sp
    M = sp.csr_matrix(D)
    A = PB.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    x_star = rng.uniform(-1, 1, n)
    b = oracle.spmv(A, x_star)
    for bp in (np.arange(n + 1, dtype=np.int32), np.array([0, n // 2, n], np.int32),
               np.array([0, n], np.int32)):
        P = oracle.Preconditioner(A, bp)
        res = oracle.pcg(A, P, b, tol=1e-10, maxit=200)
        assert res["converged"] and res["iters"] <= n + 2
        if len(bp) == 2:
            assert res["iters"] == 1


def test_pcg_laplacian_iteration_bound(oracle):
    # point Jacobi on the constant 5-point Laplacian is CG on a scaled identity preconditioner:
    # kappa = sin^2(64 pi h / 2) / sin^2(pi h / 2), h = 1/65, and
    # k <= ln(2 sqrt(kappa) / tol) / ln((sqrt(kappa)+1)/(sqrt(kappa)-1)) = 567.5 at tol 1e-10.
    # For this M-matrix the block-Jacobi (bs = 8) spectral radius is no larger (Varga), so the
    # same bound holds.
    h = 1 / 65
    kappa = math.sin(64 * math.pi * h / 2) ** 2 / math.sin(math.pi * h / 2) ** 2
    sk = math.sqrt(kappa)
    bound = math.log(2 * sk / 1e-10) / math.log((sk + 1) / (sk - 1))
    assert 567 < bound < 568
    pr = PB.make_problem("poisson2d")
    b = oracle.spmv(pr.A, pr.x_star)
    for bs in (1, 8):
        P = oracle.Preconditioner(pr.A, PB.uniform_blocks(pr.A.n, bs))
        res = oracle.pcg(pr.A, P, b, tol=1e-10, maxit=2000)
        assert res["converged"] and res["iters"] <= bound
        assert res["true_relres"] <= 1e-10


def test_policy_limits_match_uniform_and_fmp(oracle):
    # Section 4.3.2: hl -> uniform as adp_tol -> 0 and -> fMP as adp_tol -> inf; lh reverse.
    pr = PB.make_problem("subcube3d", seed=7, m=16)
    b = oracle.spmv(pr.A, pr.x_star)
    P = oracle.Preconditioner(pr.A, pr.block_ptr, fmt=oracle.BF16)
    uni = oracle.pcg(pr.A, P, b, policy=oracle.POLICY_UNIFORM)
    fmp = oracle.pcg(pr.A, P, b, policy=oracle.POLICY_FMP)
    cases = [(oracle.POLICY_HL, 1e-30, uni), (oracle.POLICY_HL, 1e30, fmp),
             (oracle.POLICY_LH, 1e30, uni), (oracle.POLICY_LH, 1e-30, fmp)]
    for pol, tol, ref in cases:
        got = oracle.pcg(pr.A, P, b, policy=pol, adp_tol=tol)
        assert got["iters"] == ref["iters"]
        assert np.array_equal(got["hist"], ref["hist"])
        assert np.array_equal(got["x"], ref["x"])


def test_fp64_format_fmp_equals_uniform(oracle):
    # Section 4.3 / 4.4: fMP with fp64 as the "low" format reproduces the uniform solver
    pr = PB.make_problem("subcube3d", seed=8, m=16)
    b = oracle.spmv(pr.A, pr.x_star)
    P = oracle.Preconditioner(pr.A, pr.block_ptr, fmt=oracle.FP64)
    uni = oracle.pcg(pr.A, P, b, policy=oracle.POLICY_UNIFORM)
    fmp = oracle.pcg(pr.A, P, b, policy=oracle.POLICY_FMP)
    assert np.array_equal(uni["hist"], fmp["hist"]) and np.array_equal(uni["x"], fmp["x"])


def test_hl_switches_on_current_relres(oracle):
    pr = PB.make_problem("subcube3d", seed=9, m=16)
    b = oracle.spmv(pr.A, pr.x_star)
    P = oracle.Preconditioner(pr.A, pr.block_ptr, fmt=oracle.FP32)
    res = oracle.pcg(pr.A, P, b, policy=oracle.POLICY_HL, adp_tol=1e-4)
    h, low = res["hist"], res["low_used"]
    k = res["iters"]
    # each preconditioner application after iteration j (j < k) uses low iff relres_j < adp_tol
    for j in range(k):
        assert bool(low[j]) == (h[j] < 1e-4)
    assert res["converged"] and res["true_relres"] <= 1e-10


def test_zero_rhs_and_maxit(oracle):
    pr = PB.make_problem("poisson2d")
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    res = oracle.pcg(pr.A, P, np.zeros(pr.A.n), x0=np.ones(pr.A.n))
    assert res["iters"] == 0 and res["converged"] and np.all(res["x"] == 0)
    b = oracle.spmv(pr.A, pr.x_star)
    res = oracle.pcg(pr.A, P, b, maxit=5)
    assert res["iters"] == 5 and not res["converged"] and res["status"] == 1


# ---------------------------------------------------------------------------------------
# Summation order of the dot products: every order is a valid evaluation of PCG
# ---------------------------------------------------------------------------------------
def test_dot_orders_within_error_bound(oracle):
    # every order rounds each product once and adds in binary64: the textbook bound
    # |computed - exact| <= gamma_n sum |a_i b_i| holds for each; the compensated one is
    # within 2u |exact| + gamma_n^2 sum |a_i b_i| (Neumaier 1974)
    rng = np.random.default_rng(21)
    u = 2.0 ** -53
    for n in (1, 7, 100, 5000):
        a = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
        b = rng.standard_normal(n)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        absum = float(np.sum(np.abs(a * b)))
        gamma = n * u / (1 - n * u)
        got = {}
        old = oracle.set_dot_order(0)
        try:
            for order in range(5):
                oracle.set_dot_order(order)
                got[order] = oracle.dot(a, b)
        finally:
            oracle.set_dot_order(old)
        for order in range(4):
            assert abs(Fraction(got[order]) - exact) <= Fraction(gamma * absum * 1.0000001)
        assert abs(Fraction(got[4]) - exact) <= Fraction(2 * u * abs(float(exact)) + gamma ** 2 * absum * 2)
        if n == 5000:
            assert len(set(got.values())) > 1     # the orders really differ
    # the default order is the plain loop from index 0
    x = np.array([1e16, 1.0, -1e16, 1.0])
    assert oracle.dot(x, np.ones(4)) == 1.0


@pytest.mark.parametrize("name", ["poisson2d_bs8", "subcube24_bs32", "subcube24_bs64", "aniso27_12_bs64",
                                  "voronoi24_uneven", "ragged13_bs32"])
def test_uniform_iteration_band_over_summation_orders(oracle, name):
    # How far the binary64 BJAC-PCG iteration count moves when only the summation order of the
    # dot products changes. On the well-conditioned systems every order gives the same count;
    # on the ill-conditioned 27-point anisotropic system (not an M-matrix, kappa(M^-1 A) large)
    # the five orders give 326 ... 334. The GPU parity test accepts the band the orders span,
    # widened by the stated +-2, so its tolerance stays +-2 where the band is one count.
    import pcg_cases
    pr = pcg_cases.PROBLEMS[name]()
    b = oracle.spmv(pr.A, pr.x_star)
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    lo, hi = pcg_cases.uniform_iteration_band(pr, b, P)
    if name == "aniso27_12_bs64":
        assert (lo, hi) == (326, 334)
    else:
        assert hi - lo == 0


# ---------------------------------------------------------------------------------------
# Multiscale strength (Eq. 4-5) against Tables 4.3 and 4.4
# ---------------------------------------------------------------------------------------
def _percent(tau, bins):
    edges = [float(b) if b != "inf" else math.inf for b in bins]
    out = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        out.append(100.0 * np.count_nonzero((tau >= lo) & (tau < hi)) / len(tau))
    return np.array(out)


@pytest.fixture(scope="module")
def golden_tables():
    with open(os.path.join(GOLDEN, "multiscale_tables.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("col,kind,tol", [("const", "const", 0.0), ("ani1000", "ani", 0.0),
                                          ("dis1000", "dis", 0.005), ("rand1000", "rand", 0.5)])
def test_table_4_3_multiscale(oracle, golden_tables, col, kind, tol):
    t = golden_tables["table_4_3"]
    A = PB.diff3d(128, kind, 1000.0, seed=0)
    assert A.n == 2097152 and A.nnz == 14581760          # Table 4.1
    got = _percent(oracle.multiscale(A), t["bins"])
    assert np.max(np.abs(got - np.array(t[col]))) <= tol + 1e-9, got


@pytest.mark.parametrize("s", [1000, 100, 10, 4, 2, 1])
def test_table_4_4_multiscale_ani(oracle, golden_tables, s):
    t = golden_tables["table_4_4"]
    A = PB.diff3d(32, "ani", float(s))
    got = _percent(oracle.multiscale(A), t["bins"])
    assert np.array_equal(got, np.array(t[f"ani{s}"], dtype=float)), got


def test_diag_boost_definition(oracle):
    A = PB.poisson2d_5pt_int(6)
    B = oracle.diag_boost(A, 2.0)
    D = A.to_scipy().toarray()
    E = B.to_scipy().toarray()
    off = np.abs(D).sum(1) - np.abs(np.diag(D))
    assert np.array_equal(np.diag(E), np.diag(D) + 2.0 * off)
    assert np.array_equal(E - np.diag(np.diag(E)), D - np.diag(np.diag(D)))


# ---------------------------------------------------------------------------------------
# Features, selection rule, MLP
# ---------------------------------------------------------------------------------------
def _csr_from_dense(D):
    import scipy.sparse as sp
    M = sp.csr_matrix(D)
    M.sort_indices()
    return PB.CSR(D.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def test_features_hand_built(oracle):
    # block 0: diag(1, 10^3) (kappa_1 = 1e3, no off-diagonals); block 1: 2x2 [[4,-1],[-1,4]]
    # coupled to block 2 through a_23 = a_32 = -2; block 2: 1x1 [5].
    D = np.zeros((5, 5))
    D[0, 0], D[1, 1] = 1.0, 1e3
    D[2, 2], D[2, 3], D[3, 2], D[3, 3] = 4.0, -1.0, -1.0, 4.0
    D[3, 4] = D[4, 3] = -2.0
    D[4, 4] = 5.0
    A = _csr_from_dense(D)
    bp = np.array([0, 2, 4, 5], np.int32)
    P = oracle.Preconditioner(A, bp)
    f = oracle.features(A, P)
    assert f[0, 0] == pytest.approx(3.0)                      # kappa_1 = 1e3 * 1
    assert f[0, 1] == pytest.approx(0.5 * math.log10(1 + 1e6))
    assert f[0, 2] == 1e6 and f[0, 3] == 1e6                  # no off-diagonals: capped
    assert f[0, 4] == pytest.approx(1e-3)
    assert f[0, 5] == 0.0 and f[0, 6] == 0.0 and f[0, 8] == pytest.approx(3.0)
    assert f[0, 9] == 2 / 128 and f[0, 10] == 1.0 and f[0, 11] == 1.0
    # block 1: B = [[4,-1],[-1,4]], kappa_1 = 5 * (5/15) = 5/3; rows: d = 4/1, 4/3
    assert f[1, 0] == pytest.approx(math.log10(5 / 3))
    assert f[1, 2] == pytest.approx(4 / 3) and f[1, 3] == pytest.approx((4 + 4 / 3) / 2)
    assert f[1, 5] == pytest.approx(2 / (5 + 7))
    assert f[1, 6] == pytest.approx(math.log10(2.0)) and f[1, 7] == pytest.approx(math.log10(2.0) / 2)
    assert f[1, 8] == pytest.approx(math.log10(4.0))
    assert f[1, 11] == pytest.approx(((4 - 1) / 4 + (4 - 3) / 4) / 2)
    # block 2: [5] with off-block -2: d = 2.5, coupling 2/7
    assert f[2, 0] == pytest.approx(0.0) and f[2, 2] == pytest.approx(2.5) and f[2, 5] == pytest.approx(2 / 7)


@pytest.mark.parametrize("p,expect", [(0, 3), (2, 3), (2.3, 3), (2.32, 1), (4, 1), (6.2, 1), (6.23, 0), (9, 0)])
def test_rule_classes_from_known_kappa(oracle, p, expect):
    # diag(1, 10^p): kappa_1 = 10^p; FP16S needs kappa <= 0.1 * 2^11 = 204.8 (log 2.311),
    # FP32 needs kappa <= 0.1 * 2^24 = 1.68e6 (log 6.225), otherwise FP64.
    D = np.diag([1.0, 10.0 ** p])
    A = _csr_from_dense(D)
    P = oracle.Preconditioner(A, np.array([0, 2], np.int32))
    f = oracle.features(A, P)
    assert oracle.select_rule(f, 0.1)[0] == expect


def test_rule_bf16_when_dynamic_range_is_wide(oracle):
    # tridiag(eps, 1, eps) of size 8: kappa ~ 1 but G's entries decay like eps^|i-j|
    eps = 1e-5
    D = np.eye(8) + eps * (np.eye(8, k=1) + np.eye(8, k=-1))
    A = _csr_from_dense(D)
    P = oracle.Preconditioner(A, np.array([0, 8], np.int32))
    f = oracle.features(A, P)
    assert f[0, 8] > 29 * math.log10(2)
    assert oracle.select_rule(f, 0.1)[0] == oracle.BF16


def test_mlp_gradient_central_differences(oracle):
    rng = np.random.default_rng(3)
    npar = oracle.mlp_nparam()
    assert npar == 64 * 12 + 64 + 64 * 64 + 64 + 3 * 64 + 3
    w = rng.standard_normal(npar) * 0.3
    x = rng.standard_normal((7, 12))
    y = rng.integers(0, 3, 7)
    loss, g = oracle.mlp_loss_grad(w, x, y)
    h = 1e-6
    for k in rng.choice(npar, 60, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        num = (oracle.mlp_loss_grad(wp, x, y)[0] - oracle.mlp_loss_grad(wm, x, y)[0]) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-8


def _mlp_params(W1, b1, W2, b2, W3, b3):
    """Parameter vector in the oracle's layout W1[64][12] b1 W2[64][64] b2 W3[3][64] b3."""
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def test_mlp_forward_hand_computed(oracle):
    # Integer weights, few nonzeros; every value below is worked out by hand.
    #   x = (1, -2, 0, ..., 0)
    #   layer 1 (W1 x + b1, then ReLU):
    #     unit 0: 1*1 + 1*(-2) + 0   = -1  -> 0   (cut by the ReLU)
    #     unit 1: 2*1 + 1            =  3  -> 3
    #     unit 2: -1*(-2) - 1        =  1  -> 1
    #     unit 3: 0.5*(-2) + 3       =  2  -> 2   (bias before the ReLU: ReLU(-1) + 3 would be 3)
    #     units 4..63: bias 0        =  0  -> 0
    #   layer 2 (W2 h1 + b2, then ReLU), W2[out][in]:
    #     unit 0: 5*h1_0 + 1*h1_1 - 4*h1_2 + 0 = 0 + 3 - 4   = -1 -> 0 (cut)
    #     unit 1: 1*h1_0 + 2*h1_1 - 1          = 0 + 6 - 1   =  5 -> 5
    #     unit 2: 3*h1_2 + 1*h1_3 + 0.5        = 3 + 2 + 0.5 = 5.5 -> 5.5
    #     unit 3: -2*h1_0 + 1*h1_1 + 1*h1_2    = 0 + 3 + 1   =  4 -> 4
    #     unit 4: 1*h1_3 - 3                   = 2 - 3       = -1 -> 0 (cut)
    #   logits (W3 h2 + b3):
    #     0: 7*h2_0 + 1*h2_1 + 2*h2_4 + 0.25 = 0 + 5 + 0 + 0.25 = 5.25
    #     1: 2*h2_2 - 1*h2_3 - 1             = 11 - 4 - 1        = 6
    #     2: 1*h2_0 - 1*h2_1 + 1*h2_2 + 1*h2_3 = 0 - 5 + 5.5 + 4  = 4.5
    # A missing ReLU (layer 1: unit 0 = -1 reaches layer 2; layer 2: units 0, 4 = -1 reach the
    # logits), a bias added after the ReLU, or W2 / W3 read transposed each change the logits.
    W1 = np.zeros((64, 12)); b1 = np.zeros(64)
    W1[0, 0], W1[0, 1] = 1, 1
    W1[1, 0], b1[1] = 2, 1
    W1[2, 1], b1[2] = -1, -1
    W1[3, 1], b1[3] = 0.5, 3
    W2 = np.zeros((64, 64)); b2 = np.zeros(64)
    W2[0, 0], W2[0, 1], W2[0, 2] = 5, 1, -4
    W2[1, 0], W2[1, 1], b2[1] = 1, 2, -1
    W2[2, 2], W2[2, 3], b2[2] = 3, 1, 0.5
    W2[3, 0], W2[3, 1], W2[3, 2] = -2, 1, 1
    W2[4, 3], b2[4] = 1, -3
    W3 = np.zeros((3, 64)); b3 = np.array([0.25, -1.0, 0.0])
    W3[0, 0], W3[0, 1], W3[0, 4] = 7, 1, 2
    W3[1, 2], W3[1, 3] = 2, -1
    W3[2, 0], W3[2, 1], W3[2, 2], W3[2, 3] = 1, -1, 1, 1
    w = _mlp_params(W1, b1, W2, b2, W3, b3)
    x = np.zeros((2, 12))
    x[0, 0], x[0, 1] = 1, -2
    # second sample: every input 0, so only the biases act: h1 = ReLU(b1) = (0, 1, 0, 3, 0...),
    # h2 = ReLU(W2 h1 + b2) = (1, 2 - 1, 3 + 0.5, 1, 3 - 3) = (1, 1, 3.5, 1, 0),
    # logits = (7 + 1 + 0 + 0.25, 7 - 1 - 1, 1 - 1 + 3.5 + 1) = (8.25, 5, 4.5)
    got = oracle.mlp_forward(w, x)
    assert np.array_equal(got, np.array([[5.25, 6.0, 4.5], [8.25, 5.0, 4.5]]))


def test_mlp_forward_random_weights_vs_matrix_products(oracle):
    # the same network written as three matrix products with numpy (ReLU as np.maximum)
    rng = np.random.default_rng(11)
    W1, b1 = rng.standard_normal((64, 12)), rng.standard_normal(64)
    W2, b2 = rng.standard_normal((64, 64)) * 0.2, rng.standard_normal(64)
    W3, b3 = rng.standard_normal((3, 64)) * 0.2, rng.standard_normal(3)
    x = rng.standard_normal((40, 12))
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    ref = h2 @ W3.T + b3
    assert (h1 == 0).any() and (h2 == 0).any()          # the ReLUs act in both layers
    got = oracle.mlp_forward(_mlp_params(W1, b1, W2, b2, W3, b3), x)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_mlp_softmax_ce_closed_form(oracle):
    # with W3 = 0 the logits are b3 for every sample: dL/db3 = softmax(b3) - mean onehot
    npar = oracle.mlp_nparam()
    rng = np.random.default_rng(4)
    w = rng.standard_normal(npar)
    w[-(3 * 64 + 3):-3] = 0.0
    b3 = np.array([0.3, -1.2, 2.0])
    w[-3:] = b3
    x = rng.standard_normal((5, 12))
    y = np.array([0, 2, 2, 1, 0])
    loss, g = oracle.mlp_loss_grad(w, x, y)
    p = np.exp(b3 - b3.max()) / np.exp(b3 - b3.max()).sum()
    onehot = np.eye(3)[y].mean(0)
    assert np.allclose(g[-3:], p - onehot, atol=1e-15)
    assert loss == pytest.approx(-np.mean(np.log(p[y])), rel=1e-14)
    assert np.allclose(oracle.mlp_forward(w, x), np.tile(b3, (5, 1)), atol=0)


# ------------------------------------------------------------------------------------------
# BJAC(k, t) of Eq. 3-2 / 3-3 (inner Jacobi sweeps inside the blocks, outer sweeps on A)
# ------------------------------------------------------------------------------------------
def _spd_blocks(n=24, bs=8, seed=3, dominance=1.5):
    """Random sparse symmetric matrix with positive diagonal, diagonally dominant by `dominance`."""
    rng = np.random.default_rng(seed)
    M = np.zeros((n, n))
    for _ in range(3 * n):
        i, j = rng.integers(0, n, 2)
        if i != j:
            v = -rng.uniform(0.1, 1.0)
            M[i, j] += v
            M[j, i] += v
    np.fill_diagonal(M, dominance * np.abs(M).sum(axis=1) + rng.uniform(0.5, 1.5, n))
    from gpu_util import csr_from_dense
    return M, csr_from_dense(M), np.arange(0, n + 1, bs, dtype=np.int32)


def _dense_kt(M, bp, k, t):
    """M-hat^-1 of Eq. 3-2 / 3-3 as explicit matrix polynomials."""
    n = M.shape[0]
    D = np.diag(np.diag(M))
    Dinv = np.diag(1.0 / np.diag(M))
    Abd = np.zeros_like(M)
    for b in range(len(bp) - 1):
        s, e = bp[b], bp[b + 1]
        Abd[s:e, s:e] = M[s:e, s:e]
    I = np.eye(n)
    Dh = sum(np.linalg.matrix_power(I - Dinv @ Abd, i) for i in range(t)) @ Dinv
    return sum(np.linalg.matrix_power(I - Dh @ M, j) for j in range(k)) @ Dh


def test_kt_k1_t1_is_diagonal_scaling(oracle):
    # Eq. 3-2 with k = t = 1 degenerates to D^-1 (Section 3.1)
    pr = PB.make_problem("subcube3d", seed=2, m=10, bs=32)
    r = PB.solution(pr.A.n, 4)
    z = oracle.kt_apply(pr.A, pr.block_ptr, 1, 1, r)
    d = np.array([pr.A.val[pr.A.rowptr[i]:pr.A.rowptr[i + 1]][pr.A.colidx[pr.A.rowptr[i]:pr.A.rowptr[i + 1]] == i].sum()
                  for i in range(pr.A.n)])
    assert np.array_equal(z, (1.0 / d) * r)


@pytest.mark.parametrize("k,t", [(1, 2), (2, 1), (2, 2), (3, 2), (2, 3), (4, 4)])
def test_kt_matches_dense_matrix_polynomials(oracle, k, t):
    M, A, bp = _spd_blocks()
    r = np.random.default_rng(k * 10 + t).standard_normal(M.shape[0])
    ref = _dense_kt(M, bp, k, t) @ r
    z = oracle.kt_apply(A, bp, k, t, r)
    assert np.max(np.abs(z - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_kt_many_inner_sweeps_reach_the_exact_block_inverse(oracle):
    # t -> inf: D-hat^-1 -> A_bd^-1 when the inner Jacobi converges; with k = 1 this is the
    # exact block Jacobi of the rest of the oracle (LU inverses)
    M, A, bp = _spd_blocks(dominance=3.0)
    r = np.random.default_rng(9).standard_normal(M.shape[0])
    z = oracle.kt_apply(A, bp, 1, 60, r)
    P = oracle.Preconditioner(A, bp)
    ref = oracle.apply_fp64(bp, P.G, P.goff, r)
    assert np.max(np.abs(z - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_kt_preconditioner_is_symmetric(oracle):
    pr = PB.make_problem("subcube3d", seed=3, m=12, bs=32)
    bp = np.linspace(0, pr.A.n, 5).astype(np.int32)
    r1, r2 = PB.solution(pr.A.n, 5), PB.solution(pr.A.n, 6)
    a = np.dot(r1, oracle.kt_apply(pr.A, bp, 2, 2, r2))
    b = np.dot(r2, oracle.kt_apply(pr.A, bp, 2, 2, r1))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_kt_binary32_emulation(oracle):
    pr = PB.make_problem("subcube3d", seed=4, m=12, bs=32)
    bp = np.linspace(0, pr.A.n, 5).astype(np.int32)
    r = PB.solution(pr.A.n, 7)
    z64 = oracle.kt_apply(pr.A, bp, 2, 2, r, prec=0)
    z32 = oracle.kt_apply(pr.A, bp, 2, 2, r, prec=1)
    assert np.all(z32 == z32.astype(np.float32).astype(np.float64))      # binary32 values
    assert np.max(np.abs(z32 - z64)) <= 1e-5 * np.max(np.abs(z64))
    # k = t = 1: RN32(RN32(1/a_ii) * RN32(r_i)), one rounding per operation
    z1 = oracle.kt_apply(pr.A, bp, 1, 1, r, prec=1)
    d = np.array([pr.A.val[pr.A.rowptr[i]:pr.A.rowptr[i + 1]][pr.A.colidx[pr.A.rowptr[i]:pr.A.rowptr[i + 1]] == i].sum()
                  for i in range(pr.A.n)])
    ref = ((1.0 / d).astype(np.float32) * r.astype(np.float32)).astype(np.float64)
    assert np.array_equal(z1, ref)


def test_kt_pcg_point_jacobi_equals_blocks_of_one(oracle):
    pr = PB.make_problem("poisson2d", seed=0)
    b = oracle.spmv(pr.A, pr.x_star)
    ref = oracle.pcg(pr.A, oracle.Preconditioner(pr.A, np.arange(pr.A.n + 1, dtype=np.int32)), b, maxit=2000)
    got = oracle.pcg_kt(pr.A, pr.block_ptr, b, k=1, t=1, maxit=2000)
    assert got["iters"] == ref["iters"] and np.array_equal(got["x"], ref["x"])


def test_kt_pcg_policy_limits(oracle):
    # Section 4.3.2: hl -> uniform as adp_tol -> 0 and -> fMP as adp_tol -> inf; lh the reverse
    pr = PB.make_problem("subcube3d", seed=5, m=12, bs=32)
    bp = np.linspace(0, pr.A.n, 9).astype(np.int32)
    b = oracle.spmv(pr.A, pr.x_star)
    uni = oracle.pcg_kt(pr.A, bp, b, policy=oracle.POLICY_UNIFORM, maxit=3000)
    fmp = oracle.pcg_kt(pr.A, bp, b, policy=oracle.POLICY_FMP, maxit=3000)
    assert uni["converged"] and fmp["converged"] and uni["true_relres"] <= 1e-10
    for pol, tol, ref in ((oracle.POLICY_HL, 1e-30, uni), (oracle.POLICY_HL, 1e30, fmp),
                          (oracle.POLICY_LH, 1e-30, fmp), (oracle.POLICY_LH, 1e30, uni)):
        got = oracle.pcg_kt(pr.A, bp, b, policy=pol, adp_tol=tol, maxit=3000)
        assert got["iters"] == ref["iters"] and np.array_equal(got["x"], ref["x"])


def test_diag_boost_input_matches_oracle_definition(oracle):
    # Section 4.5.2: a_ii += P_diag * sum_{j != i} |a_ij| (input of the P_diag experiment)
    pr = PB.make_problem("subcube3d", seed=8, m=10)
    for pd in (0.0, 1.0, 8.0):
        got = PB.diag_boost(pr.A, pd)
        ref = oracle.diag_boost(pr.A, pd)
        assert np.allclose(got.val, ref.val, rtol=1e-15, atol=0)


def _step_conjugacy(oracle, pr, solve, steps=12):
    """|d_{k+1}^T A d_k| / (||d_{k+1}||_A ||d_k||_A) for the steps d_k = x_{k+1} - x_k (= alpha_k p_k)
    of the first iterations, each x_k from a separate run stopped after k iterations."""
    import scipy.sparse as sp
    A = sp.csr_matrix((pr.A.val, pr.A.colidx, pr.A.rowptr), shape=(pr.A.n, pr.A.n))
    xs = [np.zeros(pr.A.n)] + [solve(k)["x"] for k in range(1, steps + 1)]
    d = [xs[k + 1] - xs[k] for k in range(steps)]
    return np.array([abs(d[k + 1] @ (A @ d[k])) / np.sqrt((d[k + 1] @ (A @ d[k + 1])) * (d[k] @ (A @ d[k])))
                     for k in range(steps - 1)])


@pytest.mark.parametrize("fmt", [2, 3])
@pytest.mark.parametrize("policy,adp", [(2, 1e-2), (3, 1e-2), (1, 1.0)])
def test_flexible_pcg_keeps_consecutive_directions_conjugate(oracle, fmt, policy, adp):
    # Flexible CG (Golub-Ye 1999, Notay 2000): the Polak-Ribiere beta makes p_{k+1} A-conjugate
    # to p_k whatever the preconditioner does between iterations; the Fletcher-Reeves beta of
    # standard PCG loses that at aMP's precision switch and under a low-precision apply.
    pr = PB.make_problem("voronoi3d", seed=4, m=12)
    P = oracle.Preconditioner(pr.A, pr.block_ptr, fmt=fmt)
    b = oracle.spmv(pr.A, pr.x_star)

    def run(flexible):
        return lambda k: oracle.pcg(pr.A, P, b, tol=1e-14, maxit=k, policy=policy, adp_tol=adp,
                                    flexible=flexible)
    flex = _step_conjugacy(oracle, pr, run(True))
    std = _step_conjugacy(oracle, pr, run(False))
    low = oracle.pcg(pr.A, P, b, tol=1e-14, maxit=12, policy=policy, adp_tol=adp)["low_used"]
    if policy != 1:
        assert 0 < low[:12].sum() < 12          # the switch happens inside the window
    assert flex.max() < 1e-12, flex
    assert std.max() > 1e3 * flex.max(), (std, flex)


@pytest.mark.parametrize("name,kw", [("voronoi3d", dict(seed=4, m=12)), ("poisson2d", dict(bs=8))])
def test_flexible_pcg_equals_standard_for_a_fixed_preconditioner(oracle, name, kw):
    # binary64 blocks: a fixed SPD preconditioner, so z_{k+1}^T r_k = 0 and both betas agree
    pr = PB.make_problem(name, **kw)
    P = oracle.Preconditioner(pr.A, pr.block_ptr)
    b = oracle.spmv(pr.A, pr.x_star)
    std = oracle.pcg(pr.A, P, b, maxit=3000)
    flex = oracle.pcg(pr.A, P, b, maxit=3000, flexible=True)
    assert std["converged"] and flex["converged"]
    assert abs(std["iters"] - flex["iters"]) <= 1
    k = min(std["iters"], flex["iters"], 30)
    assert np.allclose(std["hist"][:k], flex["hist"][:k], rtol=1e-8)
    assert np.linalg.norm(std["x"] - flex["x"]) <= 1e-9 * np.linalg.norm(pr.x_star)
    # and for BJAC(k, t), whose M-hat^-1 is fixed and symmetric in binary64
    bp = np.linspace(0, pr.A.n, 5).astype(np.int32)
    s2 = oracle.pcg_kt(pr.A, bp, b, maxit=3000)
    f2 = oracle.pcg_kt(pr.A, bp, b, maxit=3000, flexible=True)
    if s2["converged"]:
        assert f2["converged"] and abs(s2["iters"] - f2["iters"]) <= 1


def test_flexible_pcg_kt_keeps_consecutive_directions_conjugate(oracle):
    # the same property with BJAC(2, 2) applied in binary32 (Algorithm 3.1 with Eq. 3-2 / 3-3)
    pr = PB.make_problem("voronoi3d", seed=4, m=12)
    bp = np.linspace(0, pr.A.n, 9).astype(np.int32)
    b = oracle.spmv(pr.A, pr.x_star)
    flex = _step_conjugacy(oracle, pr, lambda k: oracle.pcg_kt(pr.A, bp, b, tol=1e-14, maxit=k,
                                                               policy=oracle.POLICY_HL, adp_tol=1e-2, flexible=True))
    std = _step_conjugacy(oracle, pr, lambda k: oracle.pcg_kt(pr.A, bp, b, tol=1e-14, maxit=k,
                                                              policy=oracle.POLICY_HL, adp_tol=1e-2))
    assert flex.max() < 1e-12 and std.max() > 1e3 * flex.max(), (std, flex)


def test_oracle_rounds_every_product_and_sum(oracle):
    # the oracle's sums are sequential with each product rounded before it is added (no fused
    # multiply-add): (1 + 2^-30)(1 - 2^-30) = 1 - 2^-60 rounds to 1, so -1 + that product is 0;
    # a fused evaluation would give -2^-60
    c, d = 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -30
    assert oracle.dot(np.array([-1.0, c]), np.array([1.0, d])) == 0.0
    A = PB.CSR(1, np.array([0, 2], np.int32), np.array([0, 0], np.int32), np.array([-1.0, c]))
    assert oracle.spmv(A, np.array([1.0]))[0] == c - 1.0            # -1 * 1 + c * 1, each rounded
    A2 = PB.CSR(2, np.array([0, 2, 2], np.int32), np.array([0, 1], np.int32), np.array([-1.0, c]))
    assert oracle.spmv(A2, np.array([1.0, d]))[0] == 0.0
