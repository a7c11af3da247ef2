"""Helpers shared by the GPU tests (the CUDA path through the C ABI, the oracle beside it)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2407_15973_gb300 import problems as PB


def need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    from paper_2407_15973_gb300 import binding
    binding.lib()
    return binding


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def spmv_tol(A, x):
    """1e-14 of max_i (|A||x|)_i: the stated SpMV tolerance."""
    absA = PB.CSR(A.n, A.rowptr, A.colidx, np.abs(A.val))
    return 1e-14 * np.max(O.spmv(absA, np.abs(x)))


def pool_block(pool, qoff, b, fmt, bs):
    raw = pool[qoff[b]:qoff[b] + bs * bs * {0: 8, 1: 4, 2: 2, 3: 2}[int(fmt)]]
    return raw


def csr_from_dense(D):
    import scipy.sparse as sp
    M = sp.csr_matrix(D)
    M.sort_indices()
    return PB.CSR(D.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
