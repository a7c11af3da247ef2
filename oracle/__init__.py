"""ctypes binding of the plain CPU FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the benchmark's
CPU-baseline leg. The product package never imports this module and shares no code with it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}
_parallel = False

FP64, FP32, BF16, FP16S = 0, 1, 2, 3
FMT_BYTES = {FP64: 8, FP32: 4, BF16: 2, FP16S: 2}
NFEAT = 12
POLICY_UNIFORM, POLICY_FMP, POLICY_HL, POLICY_LH = 0, 1, 2, 3


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction) into oracle/_build/liboracle.so, the
    single-threaded checker every test uses, or (parallel=True) liboracle_omp.so, the same
    source with OpenMP, used only to time the CPU baseline on all host cores."""
    out = _OUT_OMP if parallel else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        omp = ["-fopenmp"] if parallel else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", *omp,
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def use_parallel(on: bool) -> bool:
    """Route every following oracle call to the OpenMP build (on) or the single-threaded
    checker (off, the default). Only the benchmark's CPU-baseline timing turns it on; both
    builds give the same bits. Returns the previous setting."""
    global _parallel
    old = _parallel
    _parallel = bool(on)
    return old


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("status", C.c_int32),
                ("restarts", C.c_int32), ("low_applies", C.c_int32), ("high_applies", C.c_int32),
                ("relres", C.c_double), ("true_relres", C.c_double)]


def lib():
    with _lock:
        _lib = _libs.get(_parallel)
        if _lib is None:
            _lib = C.CDLL(build(parallel=_parallel))
            _libs[_parallel] = _lib
            P = C.c_void_p
            i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
            sig = {
                "orc_spmv": (None, [i32, P, P, P, P, P]),
                "orc_dot": (f64, [i64, P, P]),
                "orc_set_dot_order": (i32, [i32]),
                "orc_threads": (i32, []),
                "orc_residual": (None, [i32, P, P, P, P, P, P]),
                "orc_block_inverse": (i32, [i32, P, P, P, i32, P, P, P, P]),
                "orc_round_f32_bits": (C.c_uint32, [f64]),
                "orc_round_bf16_bits": (C.c_uint16, [f64]),
                "orc_round_f16_bits": (C.c_uint16, [f64]),
                "orc_decode_f32": (f64, [C.c_uint32]),
                "orc_decode_bf16": (f64, [C.c_uint16]),
                "orc_decode_f16": (f64, [C.c_uint16]),
                "orc_round_array": (None, [i32, i64, P, P]),
                "orc_block_scale": (C.c_float, [i32, i64, P]),
                "orc_pack": (None, [i32, P, P, P, P, P, P, P]),
                "orc_apply": (None, [i32, P, P, P, P, P, P, P, i32]),
                "orc_apply_fp64": (None, [i32, P, P, P, P, P]),
                "orc_pcg": (i32, [i32, P, P, P, i32, P, P, P, P, P, P, P, i32, f64, i32, i32,
                                  P, P, f64, i32, P, P, P]),
                "orc_multiscale": (None, [i32, P, P, P, P]),
                "orc_diag_boost": (None, [i32, P, P, P, f64]),
                "orc_features": (None, [i32, P, P, P, i32, P, P, P, P]),
                "orc_select_rule": (None, [i32, P, f64, P]),
                "orc_mlp_nparam": (i32, []),
                "orc_mlp_forward": (None, [i32, P, P, P]),
                "orc_mlp_loss_grad": (f64, [i32, P, P, P, P]),
                "orc_kt_dinv": (i32, [i32, P, P, P, P]),
                "orc_kt_apply": (i32, [i32, P, P, P, i32, P, i32, i32, i32, P, P]),
                "orc_pcg_kt": (i32, [i32, P, P, P, i32, P, i32, i32, i32, f64, i32, P, P, f64, i32, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(_lib, name)
                fn.restype = res
                fn.argtypes = args
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------------------------------
def spmv(A, x):
    x = _c(x, np.float64)
    y = np.empty(A.n)
    lib().orc_spmv(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), _p(x), _p(y))
    return y


def dot(a, b):
    a, b = _c(a, np.float64), _c(b, np.float64)
    return lib().orc_dot(len(a), _p(a), _p(b))


DOT_SEQUENTIAL, DOT_REVERSED, DOT_PAIRWISE, DOT_STRIDED, DOT_COMPENSATED = 0, 1, 2, 3, 4


def set_dot_order(order: int) -> int:
    """Summation order of every dot product and norm of the oracle's PCG (0 sequential, the
    default; 1 reversed; 2 pairwise; 3 1024 strided partials; 4 compensated). Returns the
    previous order. Process-wide: restore it after use."""
    return int(lib().orc_set_dot_order(int(order)))


def threads() -> int:
    """Threads the active build runs its loops on (1 for the single-threaded checker)."""
    return int(lib().orc_threads())


def residual(A, b, x):
    b, x = _c(b, np.float64), _c(x, np.float64)
    r = np.empty(A.n)
    lib().orc_residual(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), _p(b), _p(x), _p(r))
    return r


def dense_offsets(block_ptr):
    bs = np.diff(np.asarray(block_ptr, dtype=np.int64))
    off = np.zeros(len(bs) + 1, dtype=np.int64)
    np.cumsum(bs * bs, out=off[1:])
    return off


def block_inverse(A, block_ptr):
    """G (flat, row-major blocks at goff[b]), goff[nb+1], ||B_b||_1, number of singular blocks."""
    bp = _c(block_ptr, np.int32)
    goff = dense_offsets(bp)
    G = np.zeros(int(goff[-1]))
    n1 = np.zeros(len(bp) - 1)
    bad = lib().orc_block_inverse(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), len(bp) - 1, _p(bp),
                                  _p(goff), _p(G), _p(n1))
    return G, goff, n1, int(bad)


def block_of(G, goff, block_ptr, b):
    bs = int(block_ptr[b + 1] - block_ptr[b])
    return G[goff[b]:goff[b] + bs * bs].reshape(bs, bs)


def round_bits(fmt: int, x):
    x = _c(x, np.float64)
    dt = {FP32: np.uint32, BF16: np.uint16, FP16S: np.uint16}[fmt]
    out = np.empty(x.shape, dtype=dt)
    lib().orc_round_array(fmt, x.size, _p(x), _p(out))
    return out


def decode(fmt: int, bits):
    L = lib()
    f = {FP32: L.orc_decode_f32, BF16: L.orc_decode_bf16, FP16S: L.orc_decode_f16}[fmt]
    flat = np.asarray(bits).ravel()
    return np.array([f(int(v)) for v in flat]).reshape(np.shape(bits))


def pool_offsets(block_ptr, fmt):
    bs = np.diff(np.asarray(block_ptr, dtype=np.int64))
    nbytes = bs * bs * np.array([FMT_BYTES[int(f)] for f in fmt], dtype=np.int64)
    off = np.zeros(len(bs) + 1, dtype=np.int64)
    np.cumsum(nbytes, out=off[1:])
    return off


def pack(block_ptr, fmt, G, goff):
    """Round each block to its format: (pool bytes, qoff[nb+1], scale float32[nb])."""
    bp = _c(block_ptr, np.int32)
    fmt = _c(fmt, np.uint8)
    qoff = pool_offsets(bp, fmt)
    pool = np.zeros(int(qoff[-1]), dtype=np.uint8)
    scale = np.zeros(len(bp) - 1, dtype=np.float32)
    G = _c(G, np.float64)
    lib().orc_pack(len(bp) - 1, _p(bp), _p(fmt), _p(G), _p(_c(goff, np.int64)), _p(pool), _p(qoff), _p(scale))
    return pool, qoff, scale


def apply(block_ptr, fmt, pool, qoff, scale, r, mode=0):
    bp = _c(block_ptr, np.int32)
    r = _c(r, np.float64)
    z = np.empty_like(r)
    lib().orc_apply(len(bp) - 1, _p(bp), _p(_c(fmt, np.uint8)), _p(pool), _p(_c(qoff, np.int64)),
                    _p(_c(scale, np.float32)), _p(r), _p(z), mode)
    return z


def apply_fp64(block_ptr, G, goff, r):
    bp = _c(block_ptr, np.int32)
    r = _c(r, np.float64)
    z = np.empty_like(r)
    lib().orc_apply_fp64(len(bp) - 1, _p(bp), _p(G), _p(_c(goff, np.int64)), _p(r), _p(z))
    return z


class Preconditioner:
    """The FP64 inverse set G and (optionally) a low-precision packed set."""

    def __init__(self, A, block_ptr, fmt=None):
        self.block_ptr = _c(block_ptr, np.int32)
        self.G, self.goff, self.normB1, self.singular = block_inverse(A, self.block_ptr)
        self.fmt = None
        if fmt is not None:
            self.set_formats(fmt)

    @property
    def nb(self):
        return len(self.block_ptr) - 1

    def set_formats(self, fmt):
        if np.isscalar(fmt):
            fmt = np.full(self.nb, int(fmt), dtype=np.uint8)
        self.fmt = _c(fmt, np.uint8)
        self.pool, self.qoff, self.scale = pack(self.block_ptr, self.fmt, self.G, self.goff)


def pcg(A, P: Preconditioner, b, x0=None, tol=1e-10, maxit=1000, policy=POLICY_UNIFORM,
        adp_tol=10.0, mode=1, flexible=False):
    """Oracle PCG. Returns dict(x, iters, converged, status, relres, true_relres, hist, low_used).
    flexible: the Polak-Ribiere beta of flexible CG instead of rho_new / rho."""
    b = _c(b, np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    hist = np.full(maxit + 1, np.nan)
    low = np.zeros(maxit + 1, dtype=np.uint8)
    st = Stats()
    if policy != POLICY_UNIFORM and P.fmt is None:
        raise ValueError("policy needs a low-precision set")
    lib().orc_pcg(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), P.nb, _p(P.block_ptr), _p(P.G), _p(P.goff),
                  _p(P.fmt), _p(getattr(P, "pool", None)), _p(getattr(P, "qoff", None)),
                  _p(getattr(P, "scale", None)), policy, adp_tol, mode, int(bool(flexible)), _p(b), _p(x), tol, maxit,
                  _p(hist), _p(low), C.byref(st))
    k = st.iters
    return dict(x=x, iters=k, converged=bool(st.converged), status=st.status, relres=st.relres,
                true_relres=st.true_relres, restarts=st.restarts, hist=hist[:k + 1], low_used=low[:k + 1],
                low_applies=st.low_applies, high_applies=st.high_applies)


def kt_apply(A, block_ptr, k, t, r, prec=0):
    """z = M-hat^-1 r of BJAC(k, t) (Eq. 3-2 / 3-3); prec 0 binary64, 1 binary32 (Algorithm 3.1)."""
    r = _c(r, np.float64)
    bp = _c(block_ptr, np.int32)
    z = np.empty(A.n)
    rc = lib().orc_kt_apply(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), len(bp) - 1, _p(bp), k, t, prec, _p(r),
                            _p(z))
    if rc != 0:
        raise ValueError("a diagonal entry is not positive")
    return z


def pcg_kt(A, block_ptr, b, k=2, t=2, x0=None, tol=1e-10, maxit=1000, policy=POLICY_UNIFORM, adp_tol=10.0,
           flexible=False):
    """Oracle PCG with BJAC(k, t); policy as in pcg (the low set is the binary32 one)."""
    b = _c(b, np.float64)
    bp = _c(block_ptr, np.int32)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    hist = np.full(maxit + 1, np.nan)
    low = np.zeros(maxit + 1, dtype=np.uint8)
    st = Stats()
    lib().orc_pcg_kt(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), len(bp) - 1, _p(bp), k, t, policy, adp_tol,
                     int(bool(flexible)), _p(b), _p(x), tol, maxit, _p(hist), _p(low), C.byref(st))
    it = st.iters
    return dict(x=x, iters=it, converged=bool(st.converged), status=st.status, relres=st.relres,
                true_relres=st.true_relres, restarts=st.restarts, hist=hist[:it + 1], low_used=low[:it + 1],
                low_applies=st.low_applies, high_applies=st.high_applies)


def multiscale(A):
    tau = np.empty(A.n)
    lib().orc_multiscale(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), _p(tau))
    return tau


def diag_boost(A, pdiag):
    """Copy of A with a_ii += pdiag * sum_{j != i} |a_ij| (Section 4.5.2)."""
    from copy import copy
    B = copy(A)
    B.val = A.val.copy()
    lib().orc_diag_boost(A.n, _p(A.rowptr), _p(A.colidx), _p(B.val), pdiag)
    return B


def features(A, P: Preconditioner):
    feat = np.zeros((P.nb, NFEAT))
    lib().orc_features(A.n, _p(A.rowptr), _p(A.colidx), _p(A.val), P.nb, _p(P.block_ptr), _p(P.G),
                       _p(P.goff), _p(feat))
    return feat


def select_rule(feat, theta=0.1):
    feat = _c(feat, np.float64)
    out = np.zeros(len(feat), dtype=np.uint8)
    lib().orc_select_rule(len(feat), _p(feat), theta, _p(out))
    return out


def mlp_nparam():
    return lib().orc_mlp_nparam()


def mlp_forward(w, xin):
    w, xin = _c(w, np.float64), _c(xin, np.float64)
    out = np.zeros((len(xin), 3))
    lib().orc_mlp_forward(len(xin), _p(w), _p(xin), _p(out))
    return out


def mlp_loss_grad(w, xin, label):
    w, xin = _c(w, np.float64), _c(xin, np.float64)
    label = _c(label, np.int32)
    g = np.zeros(mlp_nparam())
    loss = lib().orc_mlp_loss_grad(len(xin), _p(w), _p(xin), _p(label), _p(g))
    return loss, g
