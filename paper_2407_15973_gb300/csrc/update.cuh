// Vector kernels of the PCG loop: the residual update of the aMP loop and the x / p update.
#pragma once
#include "common.cuh"

namespace mpbjac {

// aMP loop: alpha from the loop SpMV's partials (spart, loop_alpha), r -= alpha q with ||r||^2
// (grid reduction through part), relres, convergence, and the precision of the next
// preconditioner application.
int launch_update_r(int n, const double *q, double *r, double *part, const double *spart, SolverState *S,
                    cudaStream_t st);

// x += alpha p (deferred from this iteration) and p = z + beta p; sets the graph's loop
// condition when use_cond is 1.
int launch_update_xp(int n, const double *z, double *p, SolverState *S, cudaGraphConditionalHandle cond,
                     int use_cond, cudaStream_t st);

// Flexible CG: beta = z_{k+1}^T (r_{k+1} - r_k) / rho_k, evaluated as -alpha_k q_k^T z_{k+1} / rho_k
// (the residual recurrence r_{k+1} = r_k - alpha_k q_k), replacing the beta the apply set.
int launch_flex_beta(int n, const double *q, const double *z, double *part, SolverState *S, cudaStream_t st);

}  // namespace mpbjac
