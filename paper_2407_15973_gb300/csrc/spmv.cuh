// SpMV kinds and their epilogues, shared by the CSR kernels and the sliced-ELLPACK kernel.
#pragma once
#include "common.cuh"

namespace mpbjac {

constexpr int kSpNT = 256;               // threads per CTA of the SpMV kernels

// the kinds of the PCG loop's SpMV
template <int KIND>
__host__ __device__ constexpr bool sp_loop() { return KIND == 2 || KIND == 3; }

enum SpmvKind {
    kSpY = 0,         // y = A x
    kSpYDot = 1,      // y = A x, *out = x . y
    kSpPcg = 2,       // PCG: q = A p and per-CTA partials of p . q (summed by loop_alpha)
    kSpPcgAlpha = 3,  // PCG: q = A p, sigma = p . q and alpha by the last CTA (for the generic apply)
    kResStandalone = 10,  // r = b - A x, *out = r . r
    kResStart = 11,       // PCG start: bnorm, relres, state
    kResCheck = 12,       // true residual after the loop; restart decision
};

// Final scalar step of an SpMV kind, run by one thread of the last CTA after the
// deterministic reduction: t1 = the fused dot product (or r.r), t2 = b.b (residual kinds).
template <int KIND>
__device__ __forceinline__ void spmv_finish(double t1, double t2, double *out, SolverState *S) {
    if (KIND == kSpYDot || KIND == kResStandalone) {
        *out = t1;
    } else if (KIND == kSpPcgAlpha) {
        S->x_pending = 0;      // set again once this iteration updates r
        S->sigma = t1;
        if (!finite_pos(t1)) S->state = kBreakdownSigma;
        else S->alpha = S->rho / t1;
    } else if (KIND == kResStart) {
        const double bnorm = sqrt(t2);
        S->bnorm = bnorm;
        S->x_pending = 0;
        if (bnorm == 0.0) {
            S->relres = 0.0;
            S->true_relres = 0.0;
            S->state = kConverged;      // x is zeroed by the host
            return;
        }
        const double rel = sqrt(t1) / bnorm;
        S->relres = rel;
        S->true_relres = rel;
        if (S->hist) S->hist[S->iter] = rel;
        if (!(rel < 1.0e308)) S->state = kBreakdown;
        else if (rel <= S->tol) S->state = kConverged;
        else if (S->iter >= S->maxit) S->state = kMaxit;
        else S->state = kRunning;
        S->use_low = choose_low(S, rel);
    } else {   // kResCheck
        const double rel = S->bnorm > 0.0 ? sqrt(t1) / S->bnorm : 0.0;
        S->true_relres = rel;
        S->x_pending = 0;
        if (S->state == kConverged && rel > S->tol && S->iter < S->maxit && S->restarts < 8) {
            S->state = kRunning;          // restart from r = b - A x
            S->restarts += 1;
            S->relres = rel;
            S->use_low = choose_low(S, rel);
        }
    }
}

}  // namespace mpbjac
