// The inexact block Jacobi BJAC(k, t) of Eq. 3-2 / 3-3 (inner Jacobi sweeps inside the
// blocks, outer block-Jacobi sweeps on A), applied in binary64 or binary32.
#pragma once
#include "apply.cuh"
#include "common.cuh"
#include "sell.cuh"

namespace mpbjac {

struct KtSet {
    int n = 0, nb = 0, k = 2, t = 2;
    const int32_t *block_ptr = nullptr;   // [nb+1] device, borrowed from the handle
    int32_t *rblk = nullptr;              // [n] block of each row
    double *dinv64 = nullptr;             // [n] 1 / a_ii
    float *dinv32 = nullptr;              // [n] RN32(1 / a_ii) (low set only)
    float *val32 = nullptr;               // SELL-32 values rounded to binary32 (low set only)
    SellMat sell;                         // SELL-32 copy of A (owned here)
    double *w = nullptr, *y0 = nullptr, *y1 = nullptr;   // work vectors (n doubles each)
    double *zt = nullptr, *zt2 = nullptr;                // z, alternating between outer steps
};

// Build the set for A with contiguous blocks block_ptr (device, nb+1); lo: also the binary32
// copy. Returns NOT_SPD (with the row in *bad_row) when a diagonal entry is not positive.
int kt_build(const bjac_csr &A, const int32_t *d_block_ptr, int nb, int k, int t, bool lo, KtSet *out,
             int *bad_row, cudaStream_t st);
void kt_free(KtSet *K);

// z = M-hat^-1 r with the binary64 set (prec 0) or the binary32 set (prec 1), with r.z
// reduced through io.part / io.ticket and finished as the apply kernels do for `mode`
// (kApplyStandalone, kApplyInit, kApplyTemporal). With from_state, each kernel runs only if
// S->use_low equals prec (both precisions are then launched). *launches += kernels launched.
int launch_kt_apply(int mode, int prec, bool from_state, const KtSet &K, const ApplyIO &io, SolverState *S,
                    cudaStream_t st, int *launches);

}  // namespace mpbjac
