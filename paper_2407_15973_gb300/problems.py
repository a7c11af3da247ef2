"""Seeded synthetic inputs: sparse SPD matrices (CSR), block partitions, exact solutions.

This module only builds inputs. It holds none of the solver's arithmetic (no SpMV,
no block inverse, no rounding, no Krylov step), so that the CPU oracle and the CUDA
path can both be fed from it without sharing any of the method's code.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to
``base(seed, stream) + index``, so every value depends only on (seed, stream, index)
and not on the platform, the array order or how much was drawn before.

Discretisations (paper Section 4.1, Eq. 4-1 and Table 4.1):

* 3D node-based finite differences on the unit cube with Dirichlet boundary, m^3
  interior nodes, h = 1/(m+1); the coefficient between two nodes is the harmonic
  mean of their coefficients, a face to a boundary node uses the node's own value;
  7-point stencil scaled by 1/h^2, optional diagonal shift 1/dt (the time-step term
  of Section 4.5.2).
* Diff3D-Const / Ani(s) / Dis(s) / Rand(s): the four coefficient laws of Section 4.1.1.
* 3D Q1 (trilinear) finite elements, elementwise diagonal coefficient tensor:
  27-point stencil.
* 2D 5-point FDM and 2D 9-point Q1 FEM for the batched workload.
* 3D multi-material Voronoi problem with material-aligned uneven blocks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z += _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _base(seed: int, stream: int) -> np.uint64:
    s = np.array([(int(seed) & 0xFFFFFFFF) << 32 | (int(stream) & 0xFFFFFFFF)], dtype=np.uint64)
    return _splitmix64(_splitmix64(s))[0]


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of SplitMix64(base + index)."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        bits = _splitmix64(idx + _base(seed, stream))
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, stream, count)
    u2 = uniform(seed, stream + 0x10000, count)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class CSR:
    """Compressed sparse rows: int32 row pointers / column indices, float64 values."""
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colidx, self.rowptr), shape=(self.n, self.n))


@dataclass
class Problem:
    name: str
    A: CSR
    block_ptr: np.ndarray          # int32[nb+1], contiguous row blocks
    x_star: np.ndarray             # float64[n], the exact solution (b = A x_star)
    meta: dict = field(default_factory=dict)

    @property
    def nb(self) -> int:
        return len(self.block_ptr) - 1


def _compress(vals: np.ndarray, cols: np.ndarray, mask: np.ndarray) -> CSR:
    """Build CSR from per-row slot arrays (n, s) whose slots are in ascending column order."""
    n = vals.shape[0]
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    return CSR(n=n, rowptr=rowptr.astype(np.int32), colidx=cols[mask].astype(np.int32),
               val=np.ascontiguousarray(vals[mask], dtype=np.float64))


def _hmean(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    with np.errstate(divide="ignore", invalid="ignore"):
        h = 2.0 * a * b / (a + b)
    return np.where(a == b, a, h)


# ----------------------------------------------------------------------------------------
# 2D 5-point Poisson with the integer stencil (4, -1): entries are small integers, so any
# summation order of an SpMV on integer-valued vectors is exact.
# ----------------------------------------------------------------------------------------
def poisson2d_5pt_int(m: int) -> CSR:
    n = m * m
    idx = np.arange(n)
    i, j = idx % m, idx // m
    offs = [-m, -1, 0, 1, m]
    ok = [j > 0, i > 0, np.ones(n, bool), i < m - 1, j < m - 1]
    vals = np.stack([np.full(n, -1.0), np.full(n, -1.0), np.full(n, 4.0),
                     np.full(n, -1.0), np.full(n, -1.0)], axis=1)
    cols = np.stack([idx + o for o in offs], axis=1)
    mask = np.stack(ok, axis=1)
    return _compress(vals, cols, mask)


# ----------------------------------------------------------------------------------------
# 3D 7-point node-based FDM, coefficient arrays indexed [z, y, x]
# ----------------------------------------------------------------------------------------
def fdm3d_7pt(kx: np.ndarray, ky: np.ndarray, kz: np.ndarray, shift: float = 0.0) -> CSR:
    m = kx.shape[0]
    assert kx.shape == ky.shape == kz.shape == (m, m, m)
    n = m ** 3
    w = float((m + 1) ** 2)  # 1/h^2 with h = 1/(m+1)

    def faces(k, axis):
        lo = np.empty_like(k)
        hi = np.empty_like(k)
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[axis] = slice(1, None)
        sl_hi[axis] = slice(0, -1)
        inner = _hmean(k[tuple(sl_lo)], k[tuple(sl_hi)])
        # face between node p and its lower neighbour / upper neighbour
        lo[tuple(sl_lo)] = inner
        hi[tuple(sl_hi)] = inner
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[axis] = 0
        last[axis] = -1
        lo[tuple(first)] = k[tuple(first)]   # boundary face: node's own coefficient
        hi[tuple(last)] = k[tuple(last)]
        return lo.reshape(n), hi.reshape(n)

    cxm, cxp = faces(kx, 2)
    cym, cyp = faces(ky, 1)
    czm, czp = faces(kz, 0)
    idx = np.arange(n, dtype=np.int64)
    i = idx % m
    j = (idx // m) % m
    k = idx // (m * m)
    diag = (((((cxm + cxp) + cym) + cyp) + czm) + czp) * w + shift
    vals = np.stack([-czm * w, -cym * w, -cxm * w, diag, -cxp * w, -cyp * w, -czp * w], axis=1)
    cols = np.stack([idx - m * m, idx - m, idx - 1, idx, idx + 1, idx + m, idx + m * m], axis=1)
    mask = np.stack([k > 0, j > 0, i > 0, np.ones(n, bool), i < m - 1, j < m - 1, k < m - 1], axis=1)
    return _compress(vals, cols, mask)


def diff3d(m: int, kind: str, s: float = 1000.0, seed: int = 0) -> CSR:
    """Diff3D coefficient laws of Section 4.1.1 (Eq. 4-1): const, ani, dis, rand."""
    shape = (m, m, m)
    if kind == "const":
        k = np.ones(shape)
        return fdm3d_7pt(k, k, k)
    if kind == "ani":      # kappa = diag(1, s, s)
        return fdm3d_7pt(np.ones(shape), np.full(shape, float(s)), np.full(shape, float(s)))
    if kind == "dis":      # kappa = s on [0.25, 0.75]^3, 1 elsewhere
        x = (np.arange(m) + 1.0) / (m + 1.0)
        inside = (x >= 0.25) & (x <= 0.75)
        cube = inside[:, None, None] & inside[None, :, None] & inside[None, None, :]
        k = np.where(cube, float(s), 1.0)
        return fdm3d_7pt(k, k, k)
    if kind == "rand":     # kappa = s^delta, delta iid U[0, 1] per node
        delta = uniform(seed, 11, m ** 3).reshape(shape)
        k = np.power(float(s), delta)
        return fdm3d_7pt(k, k, k)
    raise ValueError(kind)


def multiscale_core(m: int, s_in: float = 1e10, s_out: float = 1e2, seed: int = 0) -> CSR:
    """7-point diffusion whose coefficient is s^delta with delta iid U[0, 1] per node (the
    Diff3D-Rand law of Section 4.1.1), s = s_in on the central cube [0.25, 0.75]^3 (the region
    of the Diff3D-Dis law) and s = s_out elsewhere: a strongly multiscale core (multiscale
    strength, Eq. 4-5, up to s_in) inside a mildly multiscale rest."""
    x = (np.arange(m) + 1.0) / (m + 1.0)
    inside = (x >= 0.25) & (x <= 0.75)
    cube = inside[:, None, None] & inside[None, :, None] & inside[None, None, :]
    delta = uniform(seed, 61, m ** 3).reshape(m, m, m)
    k = np.power(np.where(cube, float(s_in), float(s_out)), delta)
    return fdm3d_7pt(k, k, k)


def diffusion_subcube(m: int = 128, sub: int = 8, lo: float = 1e-3, hi: float = 1e3,
                      dt: float = 1e-2, seed: int = 0) -> CSR:
    """7-point diffusion, coefficient log-uniform in [lo, hi], constant on sub^3 subcubes,
    harmonic-mean faces, diagonal shift 1/dt added to the 1/h^2-scaled operator."""
    nsub = (m + sub - 1) // sub
    e = uniform(seed, 21, nsub ** 3).reshape(nsub, nsub, nsub)
    ksub = np.power(10.0, math.log10(lo) + (math.log10(hi) - math.log10(lo)) * e)
    c = np.arange(m) // sub
    k = ksub[c[:, None, None], c[None, :, None], c[None, None, :]]
    return fdm3d_7pt(k, k, k, shift=1.0 / dt)


# ----------------------------------------------------------------------------------------
# Q1 finite elements (uniform grid, element size h), element-wise diagonal tensor
# ----------------------------------------------------------------------------------------
def _q1_1d(h: float):
    K = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    M = np.array([[2.0, 1.0], [1.0, 2.0]]) * (h / 6.0)
    return K, M


def fem3d_q1_27pt(kappa_e: np.ndarray, aniso=(1.0, 1.0, 1.0)) -> CSR:
    """27-point stencil of trilinear elements on (m+1)^3 elements, m^3 interior nodes.
    kappa_e is indexed [ez, ey, ex]; the element tensor is kappa_e * diag(aniso)."""
    me = kappa_e.shape[0]
    m = me - 1
    h = 1.0 / me
    K, M = _q1_1d(h)
    n = m ** 3
    # interior node (z, y, x) has full-grid index (z+1, y+1, x+1); element e spans nodes e, e+1
    Z, Y, X = np.meshgrid(np.arange(1, m + 1), np.arange(1, m + 1), np.arange(1, m + 1), indexing="ij")
    idx = np.arange(n, dtype=np.int64).reshape(m, m, m)
    vals, cols, masks = [], [], []
    ax, ay, az = aniso
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                acc = np.zeros((m, m, m))
                ez_list = [min(0, dz) - 0] if dz != 0 else [-1, 0]
                for oz in ([-1, 0] if dz == 0 else [min(0, dz)]):
                    for oy in ([-1, 0] if dy == 0 else [min(0, dy)]):
                        for ox in ([-1, 0] if dx == 0 else [min(0, dx)]):
                            # element index relative to the node: e = node + o
                            lpz, lpy, lpx = -oz, -oy, -ox            # local index of p in e
                            lqz, lqy, lqx = lpz + dz, lpy + dy, lpx + dx  # local index of q in e
                            fx = ax * K[lpx, lqx] * M[lpy, lqy] * M[lpz, lqz]
                            fy = ay * M[lpx, lqx] * K[lpy, lqy] * M[lpz, lqz]
                            fz = az * M[lpx, lqx] * M[lpy, lqy] * K[lpz, lqz]
                            ke = kappa_e[Z + oz, Y + oy, X + ox]
                            acc += ke * (fx + fy + fz)
                del ez_list
                zq, yq, xq = Z + dz, Y + dy, X + dx
                ok = (zq >= 1) & (zq <= m) & (yq >= 1) & (yq <= m) & (xq >= 1) & (xq <= m)
                vals.append(acc.reshape(n))
                cols.append((idx + dz * m * m + dy * m + dx).reshape(n))
                masks.append(ok.reshape(n))
    return _compress(np.stack(vals, 1), np.stack(cols, 1), np.stack(masks, 1))


def fdm2d_5pt(kn: np.ndarray) -> CSR:
    """2D 5-point node-based FDM, node coefficients kn[y, x], harmonic-mean faces."""
    m = kn.shape[0]
    n = m * m
    w = float((m + 1) ** 2)

    def faces(k, axis):
        lo = np.empty_like(k)
        hi = np.empty_like(k)
        if axis == 1:
            inner = _hmean(k[:, 1:], k[:, :-1])
            lo[:, 1:], hi[:, :-1] = inner, inner
            lo[:, 0], hi[:, -1] = k[:, 0], k[:, -1]
        else:
            inner = _hmean(k[1:, :], k[:-1, :])
            lo[1:, :], hi[:-1, :] = inner, inner
            lo[0, :], hi[-1, :] = k[0, :], k[-1, :]
        return lo.reshape(n), hi.reshape(n)

    cxm, cxp = faces(kn, 1)
    cym, cyp = faces(kn, 0)
    idx = np.arange(n, dtype=np.int64)
    i, j = idx % m, idx // m
    diag = (((cxm + cxp) + cym) + cyp) * w
    vals = np.stack([-cym * w, -cxm * w, diag, -cxp * w, -cyp * w], 1)
    cols = np.stack([idx - m, idx - 1, idx, idx + 1, idx + m], 1)
    mask = np.stack([j > 0, i > 0, np.ones(n, bool), i < m - 1, j < m - 1], 1)
    return _compress(vals, cols, mask)


def fem2d_q1_9pt(ke: np.ndarray) -> CSR:
    """9-point stencil of bilinear elements on (m+1)^2 elements, ke[ey, ex]."""
    me = ke.shape[0]
    m = me - 1
    h = 1.0 / me
    K, M = _q1_1d(h)
    n = m * m
    Y, X = np.meshgrid(np.arange(1, m + 1), np.arange(1, m + 1), indexing="ij")
    idx = np.arange(n, dtype=np.int64).reshape(m, m)
    vals, cols, masks = [], [], []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            acc = np.zeros((m, m))
            for oy in ([-1, 0] if dy == 0 else [min(0, dy)]):
                for ox in ([-1, 0] if dx == 0 else [min(0, dx)]):
                    lpy, lpx = -oy, -ox
                    lqy, lqx = lpy + dy, lpx + dx
                    f = K[lpx, lqx] * M[lpy, lqy] + M[lpx, lqx] * K[lpy, lqy]
                    acc += ke[Y + oy, X + ox] * f
            yq, xq = Y + dy, X + dx
            ok = (yq >= 1) & (yq <= m) & (xq >= 1) & (xq <= m)
            vals.append(acc.reshape(n))
            cols.append((idx + dy * m + dx).reshape(n))
            masks.append(ok.reshape(n))
    return _compress(np.stack(vals, 1), np.stack(cols, 1), np.stack(masks, 1))


# ----------------------------------------------------------------------------------------
# Block partitions
# ----------------------------------------------------------------------------------------
def diag_boost(A: CSR, pdiag: float) -> CSR:
    """Input of the diagonal-dominance experiment of Section 4.5.2: every diagonal entry grows by
    pdiag times the sum of the magnitudes of the row's off-diagonal entries."""
    val = np.array(A.val, dtype=np.float64, copy=True)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = A.colidx == rows
    off = np.zeros(A.n)
    np.add.at(off, rows[~diag], np.abs(val[~diag]))
    val[diag] += pdiag * off[rows[diag]]
    return CSR(A.n, A.rowptr, A.colidx, val)


def uniform_blocks(n: int, bs: int) -> np.ndarray:
    """Contiguous blocks of bs rows; the last block takes the ragged remainder."""
    bp = np.arange(0, n, bs, dtype=np.int64)
    return np.append(bp, n).astype(np.int32)


def material_blocks(material: np.ndarray, bmin: int = 16, bmax: int = 128) -> np.ndarray:
    """Walk rows in order; cut at every material change and every bmax rows; a piece
    shorter than bmin joins the previous block when the result stays <= bmax."""
    n = len(material)
    change = np.flatnonzero(material[1:] != material[:-1]) + 1
    run_starts = np.concatenate([[0], change])
    run_ends = np.concatenate([change, [n]])
    starts = []
    for a, b in zip(run_starts.tolist(), run_ends.tolist()):
        starts.extend(range(a, b, bmax))
    starts = np.array(starts, dtype=np.int64)
    ends = np.append(starts[1:], n)
    out = [0]
    for a, b in zip(starts.tolist(), ends.tolist()):
        if a == 0:
            out.append(b)
            continue
        prev_len = out[-1] - out[-2]
        if (b - a) < bmin and prev_len + (b - a) <= bmax:
            out[-1] = b
        else:
            out.append(b)
    return np.array(out, dtype=np.int32)


def voronoi_materials(m: int, nsites: int = 64, nmat: int = 5, seed: int = 0):
    """Per-node material id of a seeded Voronoi partition of (0,1)^3 (nearest site,
    lowest site index on ties) and per-site material U{0..nmat-1}."""
    sites = uniform(seed, 31, 3 * nsites).reshape(nsites, 3)
    site_mat = np.minimum((uniform(seed, 32, nsites) * nmat).astype(np.int64), nmat - 1)
    x = (np.arange(m) + 1.0) / (m + 1.0)
    mat = np.empty(m ** 3, dtype=np.int8)
    plane = np.stack(np.meshgrid(x, x, indexing="ij"), -1).reshape(-1, 2)  # (y, x)
    for kz in range(m):
        z = x[kz]
        d = ((plane[:, None, 1] - sites[None, :, 0]) ** 2 + (plane[:, None, 0] - sites[None, :, 1]) ** 2
             + (z - sites[None, :, 2]) ** 2)
        mat[kz * m * m:(kz + 1) * m * m] = site_mat[np.argmin(d, axis=1)]
    return mat


def solution(n: int, seed: int) -> np.ndarray:
    """Exact solution x* ~ U[-1, 1] (seeded)."""
    return 2.0 * uniform(seed, 1, n) - 1.0


# ----------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------
def make_problem(name: str, seed: int = 0, bs: int | None = None, m: int | None = None) -> Problem:
    """Named workloads; ``m`` shrinks a law to a smaller grid for tests.

    poisson2d      2D 5-point Poisson, integer stencil, 64x64, blocks of 8
    subcube3d      3D 7-point, coefficient log-uniform [1e-3, 1e3] on 8^3 subcubes,
                   shift 1/dt = 100, 128^3, blocks of 32 (or 64)
    aniso27        3D 27-point Q1, kappa_e ~ lognormal(0, 2), tensor diag(1, 1, 1e4),
                   160^3 interior nodes, blocks of 64
    voronoi3d      3D 7-point, 5 materials 10^{0,1.5,3,4.5,6} on 64 Voronoi cells,
                   256^3, uneven material-aligned blocks of 16..128
    diff3d-const / -ani / -dis / -rand   Section 4.1.1 laws at 128^3 (s = 1000)
    mscore3d       3D 7-point, Rand law with s = 1e10 on the central cube [0.25, 0.75]^3 and
                   s = 1e2 elsewhere, 128^3, blocks of 32 (the per-block selection workload)
    """
    meta = {}
    if name == "poisson2d":
        mm = m or 64
        A = poisson2d_5pt_int(mm)
        bp = uniform_blocks(A.n, bs or 8)
    elif name == "subcube3d":
        mm = m or 128
        A = diffusion_subcube(mm, 8, 1e-3, 1e3, 1e-2, seed)
        bp = uniform_blocks(A.n, bs or 32)
    elif name == "aniso27":
        mm = m or 160
        ke = np.exp(2.0 * normal(seed, 41, (mm + 1) ** 3)).reshape(mm + 1, mm + 1, mm + 1)
        A = fem3d_q1_27pt(ke, (1.0, 1.0, 1e4))
        bp = uniform_blocks(A.n, bs or 64)
    elif name == "voronoi3d":
        mm = m or 256
        mat = voronoi_materials(mm, 64, 5, seed)
        kmat = np.power(10.0, np.array([0.0, 1.5, 3.0, 4.5, 6.0]))
        k = kmat[mat].reshape(mm, mm, mm)
        A = fdm3d_7pt(k, k, k)
        bp = material_blocks(mat) if bs is None else uniform_blocks(A.n, bs)
        meta["material"] = mat
    elif name == "mscore3d":
        mm = m or 128
        A = multiscale_core(mm, 1e10, 1e2, seed)
        bp = uniform_blocks(A.n, bs or 32)
    elif name.startswith("diff3d-"):
        kind = name.split("-", 1)[1]
        mm = m or 128
        A = diff3d(mm, kind, 1000.0, seed)
        bp = uniform_blocks(A.n, bs or 32)
    else:
        raise ValueError(name)
    return Problem(name=name, A=A, block_ptr=bp, x_star=solution(A.n, seed), meta=meta)


def batch2d(count: int = 256, seed: int = 0, side_lo: int = 32, side_hi: int = 512,
            bs_choices=(16, 32)):
    """Independent 2D diffusion systems: side log-uniform in [side_lo, side_hi],
    5-point FDM or 9-point Q1 by draw, coefficient 10^U[-2, 2] per node/element."""
    out = []
    for s in range(count):
        u = uniform(seed, 51, 3, start=3 * s)
        mm = int(round(math.exp(math.log(side_lo) + (math.log(side_hi) - math.log(side_lo)) * u[0])))
        nine = u[1] >= 0.5
        bs = bs_choices[int(u[2] * len(bs_choices)) % len(bs_choices)]
        sub_seed = seed * 100003 + s
        if nine:
            ke = np.power(10.0, -2.0 + 4.0 * uniform(sub_seed, 52, (mm + 1) ** 2)).reshape(mm + 1, mm + 1)
            A = fem2d_q1_9pt(ke)
        else:
            kn = np.power(10.0, -2.0 + 4.0 * uniform(sub_seed, 53, mm * mm)).reshape(mm, mm)
            A = fdm2d_5pt(kn)
        out.append(Problem(name=f"batch2d[{s}]", A=A, block_ptr=uniform_blocks(A.n, bs),
                           x_star=solution(A.n, sub_seed), meta={"side": mm, "nine": bool(nine), "bs": bs}))
    return out
