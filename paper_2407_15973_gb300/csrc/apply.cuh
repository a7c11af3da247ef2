// Declarations shared by the apply kernels and their callers.
#pragma once
#include "common.cuh"

namespace mpbjac {

enum ApplyMode {
    kApplyStandalone = 0,  // z = M^-1 r (set = io.set); optional r.z to io.out
    kApplyInit = 1,        // PCG start: z = M^-1 r, p = z, rho = r.z (set from S->use_low)
    kApplyTemporal = 2,    // PCG loop, aMP: set from S->use_low; beta = rho_new / rho
    kApplyFused = 3,       // PCG loop: r -= alpha q; z = M^-1 r; r.r, r.z; convergence; beta
    kApplySpec = 4,        // aMP loop: as kApplyFused with the set of the previous application;
                           // if this residual's relres picks the other set, S->redo is raised
                           // and rho / beta are left for the redo
    kApplyRedo = 5,        // aMP loop: only when S->redo: z = M^-1 r with S->use_low, rho, beta
};

struct ApplyIO {
    const double *r;       // residual in
    double *r_out;         // residual out (fused mode; may alias r)
    const double *q;       // A p (fused mode)
    double *z;
    double *p;             // init mode: p = z
    double *part;          // >= 2 * grid partial sums
    unsigned int *ticket;
    double *out;           // standalone: r.z (nullable)
    int *err;              // device error word (nullable)
    int set;               // 1 low-precision set, 0 binary64 set (standalone / fused)
    int only_set;          // -1: this launch serves both sets; else it serves only that set
    int flex;              // fused mode, register kernels: also sum q.z for the flexible-CG beta
    const double *spart;   // fused / speculative modes: the loop SpMV's partials of p.q (loop_alpha)
};

// ----------------------------------------------------------------------------------------
// epilogue shared by the apply kernels: the last CTA turns the partial sums into solver scalars
// ----------------------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void apply_finish(double rho, double rr, const ApplyIO &io, SolverState *S,
                                             int used_low, bool has_qz = false, double qz = 0.0) {
    if (MODE == kApplyStandalone) {
        if (io.out) *io.out = rho;
        return;
    }
    if (used_low) S->low_applies += 1;
    else S->high_applies += 1;
    if (MODE == kApplyInit) {
        S->rho = rho;
        if (!finite_pos(rho)) S->state = kBreakdown;
        return;
    }
    if (MODE == kApplyFused) {
        S->iter += 1;
        S->x_pending = 1;
        const double rel = sqrt(rr) / S->bnorm;
        S->relres = rel;
        S->rr = rr;
        if (S->hist) S->hist[S->iter] = rel;
        if (!(rel < 1.0e308)) { S->state = kBreakdown; return; }
        if (rel <= S->tol) { S->state = kConverged; return; }
        if (S->iter >= S->maxit) { S->state = kMaxit; return; }
    }
    // kApplyTemporal and kApplyFused (still running): beta = rho_new / rho_old. Flexible CG
    // takes beta = z_{k+1}^T (r_{k+1} - r_k) / rho_old = -alpha q.z_{k+1} / rho_old: here when the
    // kernel summed q.z (has_qz), else in a kernel of its own that reads rho_old from rho_prev.
    if (!finite_pos(rho)) { S->state = kBreakdown; return; }
    double beta = rho / S->rho;
    if (has_qz && S->flexible) beta = -S->alpha * qz / S->rho;
    if (!(fabs(beta) < 1.0e308)) { S->state = kBreakdown; return; }
    S->beta = beta;
    S->rho_prev = S->rho;
    S->rho = rho;
}

// aMP's speculative application and its redo (kApplySpec / kApplyRedo) for a low set of
// uniform 32-row blocks of one format and the binary64 set of the same blocks
bool spec_supported(const PSet &lo, const PSet &hi, int n);
int launch_apply_spec(int mode, const PSet &lo, const PSet &hi, const ApplyIO &io, SolverState *S, cudaStream_t st);

bool tma_supported(const PSet &P, int n);
int prepare_apply_tma(const PSet &P);   // set kernel attributes (call before any capture)
int launch_apply_tma(int mode, const PSet &P, const ApplyIO &io, SolverState *S, int n, cudaStream_t st);
bool reg_supported(const PSet &P, int n);
bool mix_supported(const PSet &P, int n);     // every block 32 rows: the mixed-format register kernel
int launch_apply_mix(int mode, const PSet &P, const ApplyIO &io, SolverState *S, cudaStream_t st);
int launch_apply_reg(int mode, const PSet &P, const ApplyIO &io, SolverState *S, cudaStream_t st);
int launch_apply_generic(int mode, const PSet &lo, const PSet &hi, const ApplyIO &io, SolverState *S,
                         cudaStream_t st);

bool spmv_forced_sell();                // bjac_spmv_kernel(5): standalone calls use a SELL-32 copy
int prepare_spmv(const bjac_csr &A);    // kernel attributes for A's SpMV variant (before any capture)
int launch_spmv(const bjac_csr &A, const double *x, double *y, double *part, unsigned int *ticket,
                double *dot_out, SolverState *S, int mode, cudaStream_t st);
int launch_residual(const bjac_csr &A, const double *b, const double *x, double *r, double *part,
                    unsigned int *ticket, double *rr_out, SolverState *S, int mode, cudaStream_t st);

}  // namespace mpbjac
