"""The seeded input recipe (paper Section 4.1 laws and the workloads built on them): the
counter-based generator against SplitMix64's published outputs, and the structural facts
the recipe states for each workload."""
import numpy as np
import pytest

from paper_2407_15973_gb300 import problems as PB


def test_splitmix64_published_outputs():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first outputs of the reference
    # generator, whose state advances by the golden gamma before each output
    g = 0x9E3779B97F4A7C15
    z = np.array([0, g, (2 * g) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    got = [int(v) for v in PB._splitmix64(z)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_is_counter_based():
    a = PB.uniform(7, 3, 1000)
    assert np.array_equal(a[400:], PB.uniform(7, 3, 600, start=400))      # no dependence on what came before
    assert np.all((a >= 0.0) & (a < 1.0)) and abs(a.mean() - 0.5) < 0.05
    assert not np.array_equal(a, PB.uniform(7, 4, 1000)) and not np.array_equal(a, PB.uniform(8, 3, 1000))
    assert np.all(a * 2.0 ** 53 == np.floor(a * 2.0 ** 53))               # 53-bit values


def _entries(A, i):
    s, e = A.rowptr[i], A.rowptr[i + 1]
    return A.colidx[s:e], A.val[s:e]


def test_subcube_workload_recipe():
    # 7-point FDM, coefficient constant on 8^3 subcubes and log-uniform in [1e-3, 1e3],
    # faces by harmonic mean, operator scaled by 1/h^2, plus the time-step shift 1/dt = 100
    m = 16
    A = PB.make_problem("subcube3d", seed=5, m=m).A
    h2 = 1.0 / (m + 1) ** 2
    assert A.n == m ** 3 and A.nnz == 7 * m ** 3 - 6 * m ** 2
    idx = lambda x, y, z: (z * m + y) * m + x
    for (sx, sy, sz) in [(0, 0, 0), (1, 0, 1), (1, 1, 1)]:
        ks = set()
        for z in range(8 * sz + 1, 8 * sz + 7):
            for y in range(8 * sy + 1, 8 * sy + 7):
                for x in range(8 * sx + 1, 8 * sx + 7):
                    c, v = _entries(A, idx(x, y, z))
                    off = -v[c != idx(x, y, z)] * h2
                    ks.update(np.round(off, 12).tolist())
                    # inside a subcube: diagonal = 6 k / h^2 + 1/dt
                    assert np.isclose(v[c == idx(x, y, z)][0], 6 * off[0] / h2 + 100.0, rtol=1e-13)
        assert len(ks) == 1                                            # one coefficient per subcube
        k = ks.pop()
        assert 1e-3 <= k <= 1e3
    # a face between two subcubes carries the harmonic mean of their coefficients
    i, j = idx(7, 3, 3), idx(8, 3, 3)
    c, v = _entries(A, i)
    ki = -v[c == idx(6, 3, 3)][0] * h2
    kj = -_entries(A, j)[1][_entries(A, j)[0] == idx(9, 3, 3)][0] * h2
    kij = -v[c == j][0] * h2
    assert np.isclose(kij, 2 * ki * kj / (ki + kj), rtol=1e-13)


def test_voronoi_blocks_follow_the_materials():
    # cut at every material change and every 128 rows; a piece under 16 rows joins the
    # previous block when the result stays <= 128
    pr = PB.make_problem("voronoi3d", seed=0, m=24)
    bp, mat = pr.block_ptr, pr.meta["material"]
    sizes = np.diff(bp)
    assert bp[0] == 0 and bp[-1] == pr.A.n and np.all(sizes >= 1) and np.all(sizes <= 128)
    for b in range(len(bp) - 1):
        s, e = bp[b], bp[b + 1]
        changes = np.flatnonzero(mat[s + 1:e] != mat[s:e - 1]) + s + 1
        for c in changes:          # a change inside a block only where a short piece was merged in
            nxt = changes[changes > c]
            piece_end = nxt[0] if len(nxt) else e
            assert piece_end - c < 16
    # and every block end is a material change or a multiple of 128 rows into a uniform run
    change_all = np.flatnonzero(mat[1:] != mat[:-1]) + 1
    run_start = np.concatenate([[0], change_all])
    for c in bp[1:-1]:
        r0 = run_start[np.searchsorted(run_start, c, side="right") - 1]
        assert (c - r0) % 128 == 0
    assert 0.0 < np.mean(sizes < 16) < 0.2          # short blocks exist but are rare


def test_batched_workload_recipe():
    # 256 systems, side log-uniform in [32, 512], 5-point FDM or 9-point Q1 by draw, blocks of
    # 16 or 32 rows: the totals the benchmark reports
    sys_ = PB.batch2d(256, seed=0)
    sides = np.array([p.meta["side"] for p in sys_])
    assert len(sys_) == 256 and sides.min() >= 32 and sides.max() <= 512
    assert all(p.A.n == p.meta["side"] ** 2 for p in sys_)
    assert {p.meta["bs"] for p in sys_} == {16, 32} and 0.3 < np.mean([p.meta["nine"] for p in sys_]) < 0.7
    for p in sys_[:20]:
        expect = 9 * p.meta["side"] ** 2 - 12 * p.meta["side"] + 4 if p.meta["nine"] else 5 * p.meta["side"] ** 2 - 4 * p.meta["side"]
        assert p.A.nnz == expect
    assert sum(p.A.n for p in sys_) == 11037723 and sum(p.A.nnz for p in sys_) == 78749967


def test_aniso27_workload_recipe():
    # Q1 trilinear elements on (m+1)^3 elements: 27-point stencil on m^3 interior nodes,
    # symmetric positive definite, but with positive off-diagonal entries (not an M-matrix)
    m = 6
    A = PB.make_problem("aniso27", seed=3, m=m).A
    assert A.n == m ** 3 and A.nnz == (3 * m - 2) ** 3
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n)).toarray()
    assert np.allclose(M, M.T, rtol=1e-14, atol=0)
    assert np.linalg.eigvalsh(M).min() > 0
    off = M - np.diag(np.diag(M))
    assert (off > 0).any()
