// Binary64 CSR SpMV (the working-precision q = A p of PCG, Section 3.2), its fused dot
// product, and the residual b - A x used for the initial and the true residual.
//
// One CTA of 256 threads owns a tile of 256 consecutive rows. The tile's nonzeros are
// contiguous in CSR order, so the CTA stages them chunk by chunk into shared memory with
// coalesced loads (values, and x gathered through the column indices); then each thread
// runs its own row's FMA chain in CSR order out of shared memory. Rows of any length work:
// a long row simply spans several chunks. CTAs walk tiles with a grid stride, so the rows
// in flight form one moving window and the gathered x entries stay in L2.
#include "common.cuh"

namespace mpbjac {

constexpr int kChunk = 2048;  // nonzeros staged per pass (2 x 16 KB of shared memory)

struct SpmvSmem {
    double v[kChunk];
    double x[kChunk];
    double red[kWarps];
};

// y_row = sum_k val[k] * x[colidx[k]] for this thread's row of tile r0 (0 if row >= n).
__device__ __forceinline__ double spmv_tile_row(int r0, int n, const int32_t *__restrict__ rowptr,
                                                const int32_t *__restrict__ colidx,
                                                const double *__restrict__ val,
                                                const double *__restrict__ x, SpmvSmem &sm) {
    const int row = r0 + (int)threadIdx.x;
    const int rend = min(r0 + kNT, n);
    const int lo = __ldg(rowptr + r0), hi = __ldg(rowptr + rend);
    int my_lo = hi, my_hi = hi;
    if (row < n) {
        my_lo = __ldg(rowptr + row);
        my_hi = __ldg(rowptr + row + 1);
    }
    double acc = 0.0;
    for (int c0 = lo; c0 < hi; c0 += kChunk) {
        const int c1 = min(c0 + kChunk, hi);
#pragma unroll 4
        for (int k = c0 + (int)threadIdx.x; k < c1; k += kNT) {
            const double v = __ldcs(val + k);
            const int c = __ldcs(colidx + k);
            sm.v[k - c0] = v;
            sm.x[k - c0] = __ldg(x + c);
        }
        __syncthreads();
        const int a = max(my_lo, c0), b = min(my_hi, c1);
        for (int k = a; k < b; ++k) acc = fma(sm.v[k - c0], sm.x[k - c0], acc);
        __syncthreads();
    }
    return acc;
}

// MODE 0: y = A x.   MODE 1: y = A x and *out = x . y.
// MODE 2: PCG step "q = A p; sigma = p.q; alpha = rho / sigma" (skips unless running).
template <int MODE>
__global__ void __launch_bounds__(kNT) k_spmv(int n, const int32_t *__restrict__ rowptr,
                                              const int32_t *__restrict__ colidx,
                                              const double *__restrict__ val,
                                              const double *__restrict__ x, double *__restrict__ y,
                                              double *part, unsigned int *ticket, double *out,
                                              SolverState *S) {
    __shared__ SpmvSmem sm;
    if (MODE == 2 && S->state != kRunning) return;
    const int ntiles = (n + kNT - 1) / kNT;
    double dot = 0.0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = t * kNT;
        const double acc = spmv_tile_row(r0, n, rowptr, colidx, val, x, sm);
        const int row = r0 + (int)threadIdx.x;
        if (row < n) {
            y[row] = acc;
            if (MODE != 0) dot = fma(acc, __ldg(x + row), dot);
        }
    }
    if (MODE == 0) return;
    const double bs = block_sum<kNT>(dot, sm.red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    if (!last_cta(ticket)) return;
    const double total = reduce_partials<kNT>(part, gridDim.x, 1, sm.red);
    if (threadIdx.x != 0) return;
    if (MODE == 1) {
        *out = total;
    } else {
        S->sigma = total;
        if (!finite_pos(total)) S->state = kBreakdownSigma;
        else S->alpha = S->rho / total;
    }
}

// r = b - A x with partial sums of r.r and b.b.
// MODE 0: *out = r.r.   MODE 1: PCG start (bnorm, relres, state, hist[iter]).
// MODE 2: true-residual check after the loop (true_relres; restart decision).
template <int MODE>
__global__ void __launch_bounds__(kNT) k_residual(int n, const int32_t *__restrict__ rowptr,
                                                  const int32_t *__restrict__ colidx,
                                                  const double *__restrict__ val,
                                                  const double *__restrict__ b,
                                                  const double *__restrict__ x, double *__restrict__ r,
                                                  double *part, unsigned int *ticket, double *out,
                                                  SolverState *S) {
    __shared__ SpmvSmem sm;
    const int ntiles = (n + kNT - 1) / kNT;
    double rr = 0.0, bb = 0.0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = t * kNT;
        const double acc = spmv_tile_row(r0, n, rowptr, colidx, val, x, sm);
        const int row = r0 + (int)threadIdx.x;
        if (row < n) {
            const double bi = b[row];
            const double ri = bi - acc;
            r[row] = ri;
            rr = fma(ri, ri, rr);
            bb = fma(bi, bi, bb);
        }
    }
    const double s1 = block_sum<kNT>(rr, sm.red);
    const double s2 = block_sum<kNT>(bb, sm.red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1;
        part[2 * blockIdx.x + 1] = s2;
    }
    if (!last_cta(ticket)) return;
    const double trr = reduce_partials<kNT>(part, gridDim.x, 2, sm.red);
    const double tbb = reduce_partials<kNT>(part + 1, gridDim.x, 2, sm.red);
    if (threadIdx.x != 0) return;
    if (MODE == 0) {
        *out = trr;
        return;
    }
    if (MODE == 1) {
        const double bnorm = sqrt(tbb);
        S->bnorm = bnorm;
        S->x_pending = 0;
        if (bnorm == 0.0) {
            S->relres = 0.0;
            S->true_relres = 0.0;
            S->state = kConverged;      // x is zeroed by the host
            return;
        }
        const double rel = sqrt(trr) / bnorm;
        S->relres = rel;
        S->true_relres = rel;
        if (S->hist) S->hist[S->iter] = rel;
        if (!(rel < 1.0e308)) S->state = kBreakdown;
        else if (rel <= S->tol) S->state = kConverged;
        else if (S->iter >= S->maxit) S->state = kMaxit;
        else S->state = kRunning;
        S->use_low = choose_low(S, rel);
        return;
    }
    // MODE 2: true residual after the recurrence met tol
    const double rel = S->bnorm > 0.0 ? sqrt(trr) / S->bnorm : 0.0;
    S->true_relres = rel;
    if (S->state == kConverged && rel > S->tol && S->iter < S->maxit && S->restarts < 8) {
        S->state = kRunning;          // restart from r = b - A x
        S->restarts += 1;
        S->relres = rel;
        S->use_low = choose_low(S, rel);
    }
}

// ----------------------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------------------
static int spmv_grid(int n) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_spmv<2>, kNT, 0) != cudaSuccess || v < 1) v = 1;
        per_sm = v;
    }
    const int ntiles = (n + kNT - 1) / kNT;
    int g = sm_count() * per_sm;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g > ntiles) g = ntiles;
    return g < 1 ? 1 : g;
}

int launch_spmv(const bjac_csr &A, const double *x, double *y, double *part, unsigned int *ticket,
                double *dot_out, SolverState *S, int mode, cudaStream_t st) {
    const int g = spmv_grid(A.n);
    if (mode == 0)
        k_spmv<0><<<g, kNT, 0, st>>>(A.n, A.rowptr, A.colidx, A.val, x, y, part, ticket, dot_out, S);
    else if (mode == 1)
        k_spmv<1><<<g, kNT, 0, st>>>(A.n, A.rowptr, A.colidx, A.val, x, y, part, ticket, dot_out, S);
    else
        k_spmv<2><<<g, kNT, 0, st>>>(A.n, A.rowptr, A.colidx, A.val, x, y, part, ticket, dot_out, S);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

int launch_residual(const bjac_csr &A, const double *b, const double *x, double *r, double *part,
                    unsigned int *ticket, double *rr_out, SolverState *S, int mode, cudaStream_t st) {
    const int g = spmv_grid(A.n);
    if (mode == 0)
        k_residual<0><<<g, kNT, 0, st>>>(A.n, A.rowptr, A.colidx, A.val, b, x, r, part, ticket, rr_out, S);
    else if (mode == 1)
        k_residual<1><<<g, kNT, 0, st>>>(A.n, A.rowptr, A.colidx, A.val, b, x, r, part, ticket, rr_out, S);
    else
        k_residual<2><<<g, kNT, 0, st>>>(A.n, A.rowptr, A.colidx, A.val, b, x, r, part, ticket, rr_out, S);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

}  // namespace mpbjac
