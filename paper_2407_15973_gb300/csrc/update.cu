// Vector kernels of the PCG loop (Section 3.2 recurrences): r -= alpha q with ||r|| for the
// aMP loop (Algorithms 3.2 / 3.3 read that relres), and x += alpha p, p = z + beta p.
#include "common.cuh"
#include "update.cuh"

namespace mpbjac {

// The flexible-beta dot product: half the CTAs of the plain vector kernels, so there are fewer
// per-CTA partial sums to add on the narrow FP64 pipe (each thread streams more pairs instead;
// measured in the PCG graph: 278 -> 252 ms for the 128^3 aMP(hl) flexible solve). The residual
// update of the aMP loop keeps the full grid, which measured faster there.
static int vec_grid_red(int n) {
    int g = sm_count() * 4;
    const int need = (n / 2 + kNT - 1) / kNT;
    if (g > need) g = need;
    if (g > kMaxGrid) g = kMaxGrid;
    return g < 1 ? 1 : g;
}

static int vec_grid2(int n) {
    int g = sm_count() * 8;
    const int need = (n / 2 + kNT - 1) / kNT;
    if (g > need) g = need;
    if (g > kMaxGrid) g = kMaxGrid;
    return g < 1 ? 1 : g;
}

// aMP loop: r -= alpha q, relres = ||r|| / ||b||, convergence test, precision for the next
// preconditioner application (Algorithms 3.2 / 3.3 read this relres). r, q: 16-byte aligned.
__global__ void __launch_bounds__(kNT) k_update_r(int n, const double *__restrict__ q, double *__restrict__ r,
                                                  double *part, const double *spart, SolverState *S) {
    pdl_enter();
    __shared__ double red[kNT];
    if (S->state != kRunning) return;
    double alpha;
    if (!loop_alpha(S, spart, alpha)) return;
    const uint64_t pol = vec_policy(S->l2_keep);
    double rr = 0.0;
    const int n2 = n >> 1;
    const double2 *q2 = reinterpret_cast<const double2 *>(q);
    double2 *r2 = reinterpret_cast<double2 *>(r);
#pragma unroll 2
    for (int i = blockIdx.x * kNT + threadIdx.x; i < n2; i += gridDim.x * kNT) {
        const double2 qv = ld_vec2(q2 + i, pol);
        double2 rv = ld_vec2(r2 + i, pol);
        rv.x = fma(-alpha, qv.x, rv.x);
        rv.y = fma(-alpha, qv.y, rv.y);
        st_vec2(r2 + i, rv, pol);
        rr = fma(rv.x, rv.x, rr);
        rr = fma(rv.y, rv.y, rr);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const double v = fma(-alpha, q[n - 1], r[n - 1]);
        r[n - 1] = v;
        rr = fma(v, v, rr);
    }
    const double v[1] = {rr};
    double bsum[1];
    cta_sum_to0<kNT, 1>(v, red, bsum);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum[0];
    if (!last_cta(&S->tickets[kTicketUpdR])) return;
    double tv[1];
    reduce_partials_to0<kNT, 1>(part, gridDim.x, 1, red, tv);
    if (threadIdx.x != 0) return;
    const double t = tv[0];
    S->iter += 1;
    S->x_pending = 1;
    S->rr = t;
    const double rel = sqrt(t) / S->bnorm;
    S->relres = rel;
    if (S->hist) S->hist[S->iter] = rel;
    if (!(rel < 1.0e308)) S->state = kBreakdown;
    else if (rel <= S->tol) S->state = kConverged;
    else if (S->iter >= S->maxit) S->state = kMaxit;
    S->use_low = choose_low(S, rel);
}

// x += alpha p (the update deferred from this iteration); p = z + beta p while running.
// The state it reads was final before this kernel started, so thread 0 of CTA 0 sets the
// graph's while-condition without any grid-wide step (x_pending is cleared by the next
// SpMV). z and p are 16-byte aligned (handle memory); x is the caller's vector and is checked.
// Each thread's first pair of p and x is loaded before the programmatic-launch wait: the only
// kernel that may still run then is this kernel's predecessor in the loop (an apply, the
// residual update or the flexible beta), and none of those writes p or x; the kernels that do
// (this kernel one iteration back, the initial apply) have completed. z is written by the
// predecessor and is read after the wait. S->x and S->l2_keep are set before the solve.
__global__ void __launch_bounds__(kNT) k_update_xp(int n, const double *__restrict__ z, double *__restrict__ p,
                                                   SolverState *S, cudaGraphConditionalHandle cond, int use_cond) {
    double *__restrict__ x = S->x;
    const uint64_t pol = vec_policy(S->l2_keep);
    const int gid = blockIdx.x * kNT + threadIdx.x, stride = gridDim.x * kNT;
    const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    const int n2 = n >> 1;
    const double2 *z2 = reinterpret_cast<const double2 *>(z);
    double2 *p2 = reinterpret_cast<double2 *>(p);
    double2 *x2 = reinterpret_cast<double2 *>(x);
    double2 p0 = make_double2(0.0, 0.0), x0 = make_double2(0.0, 0.0);
    if (vec && gid < n2) {
        p0 = ld_vec2(p2 + gid, pol);
        x0 = ld_vec2(x2 + gid, pol);
    }
    pdl_enter();
    const int xp = S->x_pending;
    const int run = S->state == kRunning;
    const double alpha = S->alpha, beta = S->beta;
    if ((xp | run) && vec) {
        if (gid < n2) {
            if (xp) st_vec2(x2 + gid, make_double2(fma(alpha, p0.x, x0.x), fma(alpha, p0.y, x0.y)), pol);
            if (run) {
                const double2 zv = ld_vec2(z2 + gid, pol);
                st_vec2(p2 + gid, make_double2(fma(beta, p0.x, zv.x), fma(beta, p0.y, zv.y)), pol);
            }
        }
#pragma unroll 2
        for (int i = gid + stride; i < n2; i += stride) {
            const double2 pv = ld_vec2(p2 + i, pol);
            if (xp) {
                double2 xv = ld_vec2(x2 + i, pol);
                xv.x = fma(alpha, pv.x, xv.x);
                xv.y = fma(alpha, pv.y, xv.y);
                st_vec2(x2 + i, xv, pol);
            }
            if (run) {
                const double2 zv = ld_vec2(z2 + i, pol);
                st_vec2(p2 + i, make_double2(fma(beta, pv.x, zv.x), fma(beta, pv.y, zv.y)), pol);
            }
        }
        if ((n & 1) && gid == 0) {
            const double pi = p[n - 1];
            if (xp) x[n - 1] = fma(alpha, pi, x[n - 1]);
            if (run) p[n - 1] = fma(beta, pi, z[n - 1]);
        }
    } else if (xp | run) {
        for (int i = gid; i < n; i += stride) {
            const double pi = p[i];
            if (xp) x[i] = fma(alpha, pi, x[i]);
            if (run) p[i] = fma(beta, pi, z[i]);
        }
    }
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, run ? 1u : 0u);
}

// Flexible (Polak-Ribiere) direction coefficient of flexible CG (Golub and Ye 1999, Notay 2000):
// beta_k = z_{k+1}^T (r_{k+1} - r_k) / rho_k. The loop has overwritten r_k, so the numerator is
// taken as -alpha_k (q_k . z_{k+1}), the same quantity by r_{k+1} = r_k - alpha_k q_k. Runs after
// the preconditioner application of a still-running iteration and replaces its beta.
__global__ void __launch_bounds__(kNT) k_flex_beta(int n, const double *__restrict__ q,
                                                   const double *__restrict__ z, double *part, SolverState *S) {
    pdl_enter();
    __shared__ double red[kNT];
    if (S->state != kRunning) return;
    const uint64_t pol = vec_policy(S->l2_keep);
    double s = 0.0;
    const int n2 = n >> 1;
    const double2 *q2 = reinterpret_cast<const double2 *>(q);
    const double2 *z2 = reinterpret_cast<const double2 *>(z);
#pragma unroll 2
    for (int i = blockIdx.x * kNT + threadIdx.x; i < n2; i += gridDim.x * kNT) {
        const double2 qv = ld_vec2(q2 + i, pol);
        const double2 zv = ld_vec2(z2 + i, pol);
        s = fma(qv.x, zv.x, s);
        s = fma(qv.y, zv.y, s);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) s = fma(q[n - 1], z[n - 1], s);
    const double v[1] = {s};
    double bsum[1];
    cta_sum_to0<kNT, 1>(v, red, bsum);
    if (threadIdx.x == 0) part[blockIdx.x] = bsum[0];
    if (!last_cta(&S->tickets[kTicketFlex])) return;
    double tv[1];
    reduce_partials_to0<kNT, 1>(part, gridDim.x, 1, red, tv);
    if (threadIdx.x != 0) return;
    const double t = tv[0];
    const double beta = -S->alpha * t / S->rho_prev;
    if (!(fabs(beta) < 1.0e308)) S->state = kBreakdown;
    else S->beta = beta;
}

int launch_flex_beta(int n, const double *q, const double *z, double *part, SolverState *S, cudaStream_t st) {
    MPB_CUDA(launch_kernel(k_flex_beta, vec_grid_red(n), kNT, 0, st, n, q, z, part, S));
    return MPBJAC_OK;
}

int launch_update_r(int n, const double *q, double *r, double *part, const double *spart, SolverState *S,
                    cudaStream_t st) {
    MPB_CUDA(launch_kernel(k_update_r, vec_grid2(n), kNT, 0, st, n, q, r, part, spart, S));
    return MPBJAC_OK;
}

int launch_update_xp(int n, const double *z, double *p, SolverState *S, cudaGraphConditionalHandle cond,
                     int use_cond, cudaStream_t st) {
    MPB_CUDA(launch_kernel(k_update_xp, vec_grid2(n), kNT, 0, st, n, z, p, S, cond, use_cond));
    return MPBJAC_OK;
}

}  // namespace mpbjac
