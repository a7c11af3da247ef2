"""Thin Python binding of the mpbjac C ABI (include/mpbjac.h).

Argument marshalling only: every step of the solver runs in the CUDA library. PyTorch
provides device memory and the current stream. There is no CPU fallback: if the library
or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

FP64, FP32, BF16, FP16S = 0, 1, 2, 3
FORMAT_NAMES = {FP64: "fp64", FP32: "fp32", BF16: "bf16", FP16S: "fp16s"}
SELECT_UNIFORM, SELECT_FIXED, SELECT_RULE, SELECT_MLP, SELECT_GIVEN, SELECT_KT = 0, 1, 2, 3, 4, 5
TEMPORAL_NONE, TEMPORAL_HL, TEMPORAL_LH = 0, 1, 2

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_NOT_SPD, ERR_CUDA, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_NO_MEMORY, ERR_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7)


class MpbjacError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mpbjac error {code}: {msg}")
        self.code = code


class bjac_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("val", C.c_void_p)]


class bjac_policy(C.Structure):
    _fields_ = [("select", C.c_int32), ("fixed_fmt", C.c_int32), ("temporal", C.c_int32),
                ("fp64_fallback", C.c_int32), ("adp_tol", C.c_double), ("theta", C.c_double),
                ("safety_theta", C.c_double), ("mlp_params", C.c_void_p), ("block_fmt", C.c_void_p),
                ("apply_variant", C.c_int32),
                ("graph_mode", C.c_int32), ("spmv_format", C.c_int32), ("kt_outer", C.c_int32),
                ("kt_inner", C.c_int32), ("flexible", C.c_int32), ("stream", C.c_void_p)]


class pcg_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("status", C.c_int32), ("restarts", C.c_int32),
                ("fallback_used", C.c_int32), ("low_applies", C.c_int32), ("high_applies", C.c_int32),
                ("graph_launches", C.c_int32), ("relres", C.c_double), ("true_relres", C.c_double),
                ("blocks_per_fmt", C.c_int32 * 4), ("setup_ms", C.c_float), ("solve_ms", C.c_float),
                ("kernel_launches", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load (building first if needed) the in-tree libmpbjac.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or os.environ.get("MPBJAC_REBUILD"):
                path = _build.build()
            L = C.CDLL(path)
            P, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            sigs = {
                "bjac_setup": (C.c_int, [C.POINTER(bjac_csr), P, i32, C.POINTER(bjac_policy), C.POINTER(P)]),
                "pcg_solve": (C.c_int, [P, P, P, f64, i32, C.POINTER(pcg_stats), P]),
                "bjac_destroy": (None, [P]),
                "bjac_last_error": (C.c_char_p, []),
                "bjac_spmv": (C.c_int, [C.POINTER(bjac_csr), P, P, P, P]),
                "bjac_residual": (C.c_int, [C.POINTER(bjac_csr), P, P, P, P, P]),
                "bjac_apply": (C.c_int, [P, i32, P, P, P]),
                "bjac_info": (C.c_int, [P, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]),
                "bjac_export": (C.c_int, [P, P, P, P, P, P, P]),
                "bjac_import_inverse": (C.c_int, [P, P]),
                "bjac_mlp_param_count": (i32, []),
                "pcg_profile": (C.c_int, [P, P, P, f64, i32, P, C.POINTER(i32)]),
                "bjac_apply_kernel": (C.c_int, [P, C.POINTER(i32), P]),
                "bjac_spmv_kernel": (C.c_int, [i32]),
                "bjac_l2_residency": (C.c_int, [i32]),
                "bjac_spmv_tuning": (C.c_int, [C.POINTER(bjac_csr), C.POINTER(i32), P]),
                "bjac_spmv_noalloc": (C.c_int, [C.POINTER(bjac_csr), P, P, P, P]),
                "bjac_batch_setup": (C.c_int, [i32, P, P, P, C.POINTER(bjac_policy), C.POINTER(P)]),
                "pcg_solve_batched": (C.c_int, [P, P, P, f64, i32, P]),
                "bjac_batch_info": (C.c_int, [P, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), P]),
                "bjac_batch_force_timeout": (C.c_int, [P, i32]),
                "bjac_batch_set_variant": (C.c_int, [P, i32]),
                "bjac_batch_destroy": (None, [P]),
                "bjac_mlp_grad": (C.c_int, [P, i32, P, P, i32, P, P, P]),
                "bjac_mlp_train": (C.c_int, [P, P, P, i32, i32, C.c_float, P, P]),
                "bjac_mlp_logits": (C.c_int, [P, i32, P, i32, P, P]),
                "bjac_handle_spmv": (C.c_int, [P, P, P, P]),
                "bjac_spmv_format": (C.c_int, [P, C.POINTER(i32), C.POINTER(i64), P]),
                "bjac_convert": (C.c_int, [P, P, P, i32, P]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, allow_positive: bool = False) -> int:
    if rc < 0 or (rc > 0 and not allow_positive):
        raise MpbjacError(rc, lib().bjac_last_error().decode())
    return rc


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("tensors must be contiguous CUDA tensors")


class DeviceCSR:
    """A CSR matrix resident on the GPU (int32 rowptr / colidx, float64 values)."""

    def __init__(self, A, device="cuda"):
        self.n = int(A.n)
        self.rowptr = torch.as_tensor(np.asarray(A.rowptr, dtype=np.int32)).to(device)
        self.colidx = torch.as_tensor(np.asarray(A.colidx, dtype=np.int32)).to(device)
        self.val = torch.as_tensor(np.asarray(A.val, dtype=np.float64)).to(device)
        self.nnz = int(self.colidx.numel())
        self.c = bjac_csr(self.n, self.nnz, self.rowptr.data_ptr(), self.colidx.data_ptr(), self.val.data_ptr())


def bjac_spmv(A: DeviceCSR, x, y, xy=None, stream=None):
    """y = A x (and xy[0] = x . y when a one-element float64 CUDA tensor xy is given)."""
    _require_cuda(x, y, xy)
    _check(lib().bjac_spmv(C.byref(A.c), _ptr(x), _ptr(y), _ptr(xy), _stream(stream)))


def bjac_spmv_noalloc(A: DeviceCSR, x, y, xy, stream=None):
    """y = A x and xy[0] = x . y without allocating any device memory (see include/mpbjac.h:
    for callers that cannot allocate while they run; shares one static buffer, so calls must
    not overlap on the GPU; at most 16,777,216 rows)."""
    _require_cuda(x, y, xy)
    _check(lib().bjac_spmv_noalloc(C.byref(A.c), _ptr(x), _ptr(y), _ptr(xy), _stream(stream)))


def bjac_l2_residency(keep: int) -> int:
    """Evict-last L2 policy for the PCG vectors in the solver loop (1, default) or plain
    accesses (0); returns the previous setting."""
    return _check(lib().bjac_l2_residency(int(keep)), allow_positive=True)


def bjac_spmv_kernel(variant: int) -> int:
    """0: timed choice (default), 1: TMA-staged tiles, 2: warp-cooperative, 5: a SELL-32 copy
    per standalone call (test mode). Returns the old value."""
    return _check(lib().bjac_spmv_kernel(int(variant)), allow_positive=True)


def bjac_spmv_tuning(A: DeviceCSR):
    """(kernel name in use for A, timed medians in ms for tma / warp)."""
    v = C.c_int32()
    ms = (C.c_float * 2)()
    _check(lib().bjac_spmv_tuning(C.byref(A.c), C.byref(v), ms))
    return {1: "tma", 2: "warp"}.get(v.value, "tma"), list(ms)


def bjac_residual(A: DeviceCSR, b, x, r, rr=None, stream=None):
    _require_cuda(b, x, r, rr)
    _check(lib().bjac_residual(C.byref(A.c), _ptr(b), _ptr(x), _ptr(r), _ptr(rr), _stream(stream)))


def make_policy(select=SELECT_FIXED, fixed_fmt=FP32, temporal=TEMPORAL_NONE, adp_tol=10.0, theta=0.1,
                safety_theta=0.5, fp64_fallback=False, mlp_params=None, block_fmt=None, apply_variant=0,
                graph_mode=0, spmv_format=0, kt_outer=2, kt_inner=2, flexible=False, stream=None):
    p = bjac_policy()
    p.select, p.fixed_fmt, p.temporal = select, fixed_fmt, temporal
    p.fp64_fallback = int(bool(fp64_fallback))
    p.adp_tol, p.theta, p.safety_theta = adp_tol, theta, safety_theta
    p.apply_variant = apply_variant
    p.graph_mode = graph_mode
    p.spmv_format = spmv_format
    p.kt_outer, p.kt_inner = kt_outer, kt_inner
    p.flexible = int(bool(flexible))
    p._mlp_keep = None
    if mlp_params is not None:
        arr = np.ascontiguousarray(mlp_params, dtype=np.float32)
        if arr.size != lib().bjac_mlp_param_count():
            raise ValueError("mlp_params has the wrong size")
        p._mlp_keep = arr
        p.mlp_params = arr.ctypes.data
    p._fmt_keep = None
    if block_fmt is not None:
        fa = np.ascontiguousarray(block_fmt, dtype=np.uint8)
        p._fmt_keep = fa
        p.block_fmt = fa.ctypes.data
    p.stream = _stream(stream)
    return p


class Handle:
    """Owns a bjac_handle (the preconditioner and the solver workspace)."""

    def __init__(self, A: DeviceCSR, block_ptr, policy: bjac_policy | None = None, **kw):
        self.A = A                          # the handle borrows A's device arrays
        self.block_ptr = np.ascontiguousarray(block_ptr, dtype=np.int32)
        self.policy = policy if policy is not None else make_policy(**kw)
        h = C.c_void_p()
        _check(lib().bjac_setup(C.byref(A.c), self.block_ptr.ctypes.data_as(C.c_void_p),
                                len(self.block_ptr) - 1, C.byref(self.policy), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().bjac_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nb(self):
        return len(self.block_ptr) - 1

    def solve(self, b, x, tol=1e-10, maxit=1000, hist=None):
        """pcg_solve; returns the stats as a dict. x holds x0 on entry."""
        _require_cuda(b, x, hist)
        st = pcg_stats()
        rc = lib().pcg_solve(self.h, _ptr(b), _ptr(x), tol, maxit, C.byref(st), _ptr(hist))
        if rc < 0 and rc != ERR_BREAKDOWN:
            _check(rc)
        return dict(status=rc, iters=st.iters, converged=bool(st.converged), restarts=st.restarts,
                    fallback_used=bool(st.fallback_used), low_applies=st.low_applies,
                    high_applies=st.high_applies, graph_launches=st.graph_launches, relres=st.relres,
                    true_relres=st.true_relres, blocks_per_fmt=list(st.blocks_per_fmt),
                    setup_ms=st.setup_ms, solve_ms=st.solve_ms, kernel_launches=st.kernel_launches)

    def profile(self, b, x, tol=1e-10, maxit=1000):
        """Per-kernel mean milliseconds of one PCG iteration (eager launches, CUDA events)."""
        _require_cuda(b, x)
        ms = (C.c_float * 4)()
        it = C.c_int32()
        _check(lib().pcg_profile(self.h, _ptr(b), _ptr(x), tol, maxit, ms, C.byref(it)))
        return dict(spmv=ms[0], update_r=ms[1], apply=ms[2], update_xp=ms[3], iters=it.value)

    def apply(self, r, z, set=1, rz=None):
        _require_cuda(r, z, rz)
        _check(lib().bjac_apply(self.h, set, _ptr(r), _ptr(z), _ptr(rz)))

    def spmv(self, x, y, xy=None):
        """y = A x (and xy[0] = x . y) in the layout the handle's PCG loop uses."""
        _require_cuda(x, y, xy)
        _check(lib().bjac_handle_spmv(self.h, _ptr(x), _ptr(y), _ptr(xy)))

    def spmv_format(self):
        """Layout of the loop SpMV: dict(format 'csr' | 'sell32' | 'sell32-prefetch', stored
        SELL-32 entries, timed ms of y = A x with the CSR and the two SELL-32 kernels)."""
        f, e = C.c_int32(), C.c_int64()
        ms = (C.c_float * 3)()
        _check(lib().bjac_spmv_format(self.h, C.byref(f), C.byref(e), ms))
        return dict(format={0: "csr", 1: "sell32", 2: "sell32-prefetch"}[f.value], entries=e.value, ms=list(ms))

    def apply_kernel(self):
        """(kernel name, autotuner timings in ms) of the low-precision apply."""
        k = C.c_int32()
        ms = (C.c_float * 4)()
        _check(lib().bjac_apply_kernel(self.h, C.byref(k), ms))
        return {0: "generic", 1: "tma", 2: "register", 3: "mixed"}[k.value], list(ms)

    def info(self):
        nb, pb, ge = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().bjac_info(self.h, C.byref(nb), C.byref(pb), C.byref(ge)))
        return nb.value, pb.value, ge.value

    def export(self):
        nb, pb, ge = self.info()
        fmt = np.zeros(nb, np.uint8)
        scale = np.zeros(nb, np.float32)
        qoff = np.zeros(nb + 1, np.int64)
        pool = np.zeros(max(pb, 1), np.uint8)
        G = np.zeros(max(ge, 1), np.float64)
        feat = np.zeros((nb, 12), np.float64)
        _check(lib().bjac_export(self.h, fmt.ctypes.data, scale.ctypes.data, qoff.ctypes.data, pool.ctypes.data,
                                 G.ctypes.data, feat.ctypes.data))
        return dict(fmt=fmt, scale=scale, qoff=qoff, pool=pool[:pb], G=G[:ge], feat=feat)

    def formats(self):
        """Format of every block (uint8[nb]) and nothing else."""
        nb, _, _ = self.info()
        fmt = np.zeros(nb, np.uint8)
        _check(lib().bjac_export(self.h, fmt.ctypes.data, None, None, None, None, None))
        return fmt

    def import_inverse(self, G):
        G = np.ascontiguousarray(G, dtype=np.float64)
        _check(lib().bjac_import_inverse(self.h, G.ctypes.data))


def bjac_setup(A: DeviceCSR, block_ptr, policy=None, **kw) -> Handle:
    return Handle(A, block_ptr, policy, **kw)


def pcg_solve(h: Handle, b, x, tol=1e-10, maxit=1000, hist=None):
    return h.solve(b, x, tol, maxit, hist)


def bjac_convert(x, stream=None):
    """(f, w): x (CUDA float64) rounded to binary32 by the library's integer routine, and f
    widened back to binary64 the same way."""
    _require_cuda(x)
    f = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    w = torch.empty(x.shape, dtype=torch.float64, device=x.device)
    _check(lib().bjac_convert(_ptr(x), _ptr(f), _ptr(w), x.numel(), _stream(stream)))
    return f, w


def bjac_mlp_param_count() -> int:
    return int(lib().bjac_mlp_param_count())


class Batch:
    """Many independent systems solved together (bjac_batch_setup / pcg_solve_batched)."""

    def __init__(self, As, block_ptrs, policy: bjac_policy | None = None, **kw):
        self.As = list(As)                       # DeviceCSR objects, borrowed during setup
        self.bps = [np.ascontiguousarray(bp, dtype=np.int32) for bp in block_ptrs]
        self.policy = policy if policy is not None else make_policy(**kw)
        ns = len(self.As)
        arr = (bjac_csr * ns)(*[a.c for a in self.As])
        ptrs = (C.c_void_p * ns)(*[bp.ctypes.data for bp in self.bps])
        nbs = (C.c_int32 * ns)(*[len(bp) - 1 for bp in self.bps])
        h = C.c_void_p()
        _check(lib().bjac_batch_setup(ns, C.cast(arr, C.c_void_p), C.cast(ptrs, C.c_void_p), C.cast(nbs, C.c_void_p),
                                      C.byref(self.policy), C.byref(h)))
        self.h = h
        self.nsys = ns

    def close(self):
        if getattr(self, "h", None):
            lib().bjac_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_variant(self, variant: int):
        """Force kernel variant 0..7 (32- and 64-row tiles at 2 / 4 / 6 CTAs per SM, then 128-row
        tiles at 4 / 6)."""
        _check(lib().bjac_batch_set_variant(self.h, int(variant)))

    def info(self):
        nt, tr, g = C.c_int32(), C.c_int32(), C.c_int32()
        ms = (C.c_float * 8)()
        _check(lib().bjac_batch_info(self.h, C.byref(nt), C.byref(tr), C.byref(g), ms))
        return dict(ntiles=nt.value, tile_rows=tr.value, grid=g.value, tune_ms=list(ms))

    def force_timeout(self, on: bool):
        """Test hook: the next solves' grid barriers time out (TIMEOUT, context usable)."""
        _check(lib().bjac_batch_force_timeout(self.h, int(bool(on))))

    def solve(self, bs, xs, tol=1e-10, maxit=5000):
        _require_cuda(*bs, *xs)
        ns = self.nsys
        bp = (C.c_void_p * ns)(*[b.data_ptr() for b in bs])
        xp = (C.c_void_p * ns)(*[x.data_ptr() for x in xs])
        st = (pcg_stats * ns)()
        rc = lib().pcg_solve_batched(self.h, C.cast(bp, C.c_void_p), C.cast(xp, C.c_void_p), tol, maxit,
                                     C.cast(st, C.c_void_p))
        if rc < 0 and rc != ERR_BREAKDOWN:
            _check(rc)
        return rc, [dict(iters=s.iters, converged=bool(s.converged), status=s.status, restarts=s.restarts,
                         relres=s.relres, true_relres=s.true_relres, solve_ms=s.solve_ms, setup_ms=s.setup_ms,
                         blocks_per_fmt=list(s.blocks_per_fmt))
                    for s in st]


def bjac_mlp_grad(params, feat, label, bf16_weights=True, tensor_cores=True, stream=None, mode=None):
    """(loss, gradient of the 5187 weights) of the selector on DEVICE feat (N x 12) / label (N).
    bfloat16 weights run on the tensor cores unless tensor_cores=False; binary32 weights on CUDA
    cores. `mode` passes the C mode (0, 1, 2) through unchanged."""
    _require_cuda(feat, label)
    pr = np.ascontiguousarray(params, dtype=np.float32)
    g = np.zeros(5187, np.float32)
    loss = C.c_float()
    if mode is None:
        mode = (1 if tensor_cores else 2) if bf16_weights else 0
    _check(lib().bjac_mlp_grad(pr.ctypes.data, int(mode), _ptr(feat), _ptr(label), feat.shape[0],
                               g.ctypes.data, C.byref(loss), _stream(stream)))
    return float(loss.value), g


def bjac_mlp_train(params, feat, label, epochs=300, lr=3e-3, stream=None):
    """Adam on the GPU; returns (new params, loss history)."""
    _require_cuda(feat, label)
    pr = np.array(params, dtype=np.float32, copy=True)
    hist = np.zeros(epochs, np.float32)
    _check(lib().bjac_mlp_train(pr.ctypes.data, _ptr(feat), _ptr(label), feat.shape[0], epochs, float(lr),
                                hist.ctypes.data, _stream(stream)))
    return pr, hist


def bjac_mlp_logits(params, feat, bf16_weights=True, tensor_cores=True, stream=None):
    """Selector logits (N x 3). bfloat16 weights run on the tensor cores (the forward pass the
    setup uses) unless tensor_cores=False; binary32 weights always run on CUDA cores."""
    _require_cuda(feat)
    pr = np.ascontiguousarray(params, dtype=np.float32)
    out = np.zeros((feat.shape[0], 3), np.float32)
    mode = (1 if tensor_cores else 2) if bf16_weights else 0
    _check(lib().bjac_mlp_logits(pr.ctypes.data, mode, _ptr(feat), feat.shape[0], out.ctypes.data, _stream(stream)))
    return out
