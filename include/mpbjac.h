/*
 * mpbjac -- mixed-precision block-Jacobi preconditioned conjugate gradient on one GB300.
 *
 * C ABI. Every pointer is plain memory; which side (host or device) is stated per
 * argument. No function throws; each returns an int status (0 = success, < 0 = error,
 * > 0 = finished without meeting the tolerance) and leaves a thread-local message for
 * bjac_last_error(). Work is enqueued on the CUDA stream given in the policy or the call
 * (NULL = the legacy default stream); functions that return host data synchronise that
 * stream first, and say so.
 *
 * Method: arXiv 2407.15973, "Mixed Precision Block-Jacobi Preconditioner".
 *   BJAC            Eq. 3-1 with k = 1 and exact diagonal-block inverses (the special case
 *                   stated after Eq. 3-3): M^-1 = D_b^-1, D_b = diag{A_ii}.
 *   fMP-BJAC        Algorithm 3.1: r-hat = ConvertPrecision(r, p_l); z-hat = M^-1(p_l) r-hat;
 *                   z = ConvertPrecision(z-hat, p_w). Working precision p_w = binary64.
 *   aMP-BJAC(hl)    Algorithm 3.2: binary64 M^-1 while relres >= adp_tol, else fMP.
 *   aMP-BJAC(lh)    Algorithm 3.3: fMP while relres >= adp_tol, else binary64 M^-1.
 *   PCG             Section 3.2 (Hestenes-Stiefel CG), stopping rule of Section 4.2:
 *                   ||r_k||_2 / ||b||_2 <= tol with the recurrence residual, followed by a
 *                   true-residual check b - A x (Section 4.5.1).
 *   BJAC(k, t)      Eq. 3-2 / 3-3 with inner Jacobi sweeps (BJAC_SELECT_KT), the paper's
 *                   experimental configuration.
 * Beyond the paper (its exact blocks are the special case it names): per-block storage
 * formats FP32, BF16 and power-of-two-scaled FP16, chosen per block by a condition-number
 * rule or a learned selector; the flexible-CG direction coefficient (policy.flexible);
 * many independent systems in one persistent launch (bjac_batch_*).
 */
#ifndef MPBJAC_H
#define MPBJAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define MPBJAC_OK 0
#define MPBJAC_NOT_CONVERGED 1        /* maxit reached; x holds the last iterate        */
#define MPBJAC_ERR_INVALID_ARG (-1)   /* bad sizes / pointers / non-monotone offsets    */
#define MPBJAC_ERR_NOT_SPD (-2)       /* a diagonal block has a non-positive pivot      */
#define MPBJAC_ERR_CUDA (-3)          /* a CUDA runtime call failed                     */
#define MPBJAC_ERR_BREAKDOWN (-4)     /* PCG breakdown: p.Ap <= 0, r.z <= 0 or non-finite */
#define MPBJAC_ERR_TIMEOUT (-5)       /* a bounded device wait expired                  */
#define MPBJAC_ERR_NO_MEMORY (-6)     /* device allocation failed                       */
#define MPBJAC_ERR_UNSUPPORTED (-7)   /* option not available for these inputs          */

/* ---- storage formats of the block inverses ----------------------------------------- */
#define BJAC_FP64 0    /* binary64 (8 B per entry)                                          */
#define BJAC_FP32 1    /* binary32 (4 B)                                                    */
#define BJAC_BF16 2    /* bfloat16 (2 B) of G / s_b, s_b a per-block power of two          */
#define BJAC_FP16S 3   /* binary16 (2 B) of G / s_b, s_b = 2^(floor(log2 max|G_b|) - 14)     */

/* ---- how each block's format is chosen --------------------------------------------- */
#define BJAC_SELECT_UNIFORM 0   /* every block binary64 (the paper's uniform BJAC)          */
#define BJAC_SELECT_FIXED 1     /* every block policy.fixed_fmt (fMP-BJAC, Algorithm 3.1)   */
#define BJAC_SELECT_RULE 2      /* cheapest f with kappa_1(B_b) u_f <= theta                 */
#define BJAC_SELECT_MLP 3       /* learned 12-64-64-3 selector, then promoted until          */
                                /* kappa_1 u_f <= safety_theta                               */
#define BJAC_SELECT_GIVEN 4     /* every block the format policy.block_fmt[b] names          */
#define BJAC_SELECT_KT 5        /* the paper's inexact BJAC(k, t) of Eq. 3-2 / 3-3: no block   */
                                /* inverses; kt_inner Jacobi sweeps inside the blocks and      */
                                /* kt_outer block-Jacobi sweeps on A per application, blocks of */
                                /* any size (the paper: 32 blocks, k = t = 2); fixed_fmt FP32   */
                                /* keeps a binary32 set (fMP, aMP), FP64 only the binary64 one  */

/* ---- residual-driven switching (the paper's aMP-BJAC) ------------------------------- */
#define BJAC_TEMPORAL_NONE 0
#define BJAC_TEMPORAL_HL 1      /* Algorithm 3.2 */
#define BJAC_TEMPORAL_LH 2      /* Algorithm 3.3 */

/* Sparse matrix in CSR form. All three arrays are DEVICE pointers owned by the caller and
 * borrowed by every call (and by a handle for its whole life). rowptr has n+1 entries,
 * rowptr[0] = 0, rowptr[n] = nnz, non-decreasing; colidx[k] in [0, n). The matrix must
 * be symmetric positive definite for PCG (not checked beyond the block pivots). */
typedef struct bjac_csr {
    int32_t n;
    int32_t nnz;
    const int32_t *rowptr;
    const int32_t *colidx;
    const double *val;
} bjac_csr;

/* Preconditioner options. */
typedef struct bjac_policy {
    int32_t select;         /* BJAC_SELECT_*                                               */
    int32_t fixed_fmt;      /* BJAC_* format for BJAC_SELECT_FIXED                         */
    int32_t temporal;       /* BJAC_TEMPORAL_*; HL / LH keep the binary64 set as well      */
    int32_t fp64_fallback;  /* 1: if a mixed solve fails, re-solve with binary64 blocks    */
    double adp_tol;         /* aMP threshold on relres (paper defaults: 10 for hl, 1e-5 lh)*/
    double theta;           /* rule threshold on kappa_1 * u_f (0.1 if <= 0)               */
    double safety_theta;    /* MLP promotion threshold on kappa_1 * u_f (0.5 if <= 0)      */
    const float *mlp_params;/* HOST pointer, bjac_mlp_param_count() floats, for SELECT_MLP */
    const uint8_t *block_fmt;/* HOST pointer, nb formats, for SELECT_GIVEN                  */
    int32_t apply_variant;  /* low-precision apply kernel: 0 autotuned, 1 generic warp-per-
                               block, 2 TMA-staged, 3 register-direct (bs 32, one format),
                               4 register-direct for 32-row blocks of mixed formats           */
    int32_t graph_mode;     /* 0: each solve runs as one CUDA graph with a device-side while
                               loop (default); 1: the host enqueues the same kernels in
                               batches of 32 iterations and checks the state between batches */
    int32_t spmv_format;    /* matrix layout of the loop SpMV q = A p: 0 chosen at setup (a
                               SELL-32 copy is built when its padding stays under 1.5 nnz,
                               the CSR kernel and both SELL-32 kernels are timed once per
                               matrix shape and the fastest is kept), 1 the caller's CSR
                               arrays, 2 the SELL-32 copy, one slice at a time per warp, 3 the
                               SELL-32 copy with the next slice's first entries prefetched.
                               Every layout sums each row in CSR order: same result bits.  */
    int32_t kt_outer;       /* BJAC_SELECT_KT: outer sweeps k (0: 2)                        */
    int32_t kt_inner;       /* BJAC_SELECT_KT: inner Jacobi sweeps t (0: 2)                 */
    int32_t flexible;       /* 0: beta = rho_{k+1} / rho_k (standard PCG, as in the paper);
                               1: flexible CG (Golub-Ye 1999, Notay 2000), the Polak-Ribiere
                               beta = z_{k+1}^T (r_{k+1} - r_k) / rho_k, which keeps p_{k+1}
                               A-conjugate to p_k when the preconditioner changes between
                               iterations (aMP's switch) or is not exactly linear (a low-
                               precision apply); one more kernel per iteration. Not used by
                               the batched solver.                                          */
    void *stream;           /* cudaStream_t for setup and solves (NULL = default stream)   */
} bjac_policy;

/* Per-solve report (host struct, filled by pcg_solve, which synchronises the stream). */
typedef struct pcg_stats {
    int32_t iters;          /* SpMVs performed in the PCG loop                            */
    int32_t converged;      /* 1 if both the recurrence and the true residual meet tol    */
    int32_t status;         /* same value pcg_solve returns                               */
    int32_t restarts;       /* restarts from the true residual                            */
    int32_t fallback_used;  /* 1 if the binary64 fallback re-solve ran                    */
    int32_t low_applies;    /* preconditioner applications with the low-precision set     */
    int32_t high_applies;   /* ... with the binary64 set                                  */
    int32_t graph_launches; /* CUDA graph launches (one per restart)                       */
    double relres;          /* final recurrence ||r||/||b||                               */
    double true_relres;     /* final ||b - A x|| / ||b||                                  */
    int32_t blocks_per_fmt[4];
    float setup_ms;         /* time of bjac_setup (copied from the handle)                */
    float solve_ms;         /* device time of this solve (CUDA events on the stream)      */
    int32_t kernel_launches;/* kernels of this library the solve launched (the loop body's
                               copies that ran after convergence, which return at once,
                               included)                                                  */
} pcg_stats;

typedef struct bjac_handle bjac_handle;

/* Build the preconditioner of A for the contiguous row blocks
 *   block b = rows [block_ptr[b], block_ptr[b+1]),  b = 0 .. nb-1,
 * block_ptr is a HOST array of nb+1 int32 (block_ptr[0] = 0, block_ptr[nb] = n, every
 * block 1 .. 128 rows). Each block B_b = A[rows_b, rows_b] is inverted in binary64 on the
 * GPU (symmetric Gauss-Jordan sweep, SPD pivots checked), then rounded to its format.
 * *out receives a handle that owns all device memory it allocated; A stays borrowed.
 * Errors: INVALID_ARG, NOT_SPD (the handle is not created), CUDA, NO_MEMORY. */
int bjac_setup(const bjac_csr *A, const int32_t *block_ptr, int32_t nb, const bjac_policy *policy,
               bjac_handle **out);

/* Solve A x = b by PCG. b, x: DEVICE arrays of n doubles; x holds x0 on entry and the
 * solution on exit. tol: relative residual target; maxit: iteration cap (>= 0).
 * stats (HOST, nullable) is filled after a stream synchronisation. relres_hist (DEVICE,
 * nullable, maxit+1 doubles) receives relres after each iteration (index 0 = initial).
 * Returns OK, NOT_CONVERGED, BREAKDOWN, or an error code. */
int pcg_solve(bjac_handle *h, const double *b, double *x, double tol, int32_t maxit,
              pcg_stats *stats, double *relres_hist);

/* ---- batched solves: many independent systems in one persistent launch --------------- */
typedef struct bjac_batch bjac_batch;

/* Set up nsys independent systems A[s] (DEVICE CSR arrays, copied into one block-diagonal
 * matrix owned by the batch) with contiguous blocks block_ptr[s] (HOST, nb[s]+1 entries,
 * every block 1..32 rows). policy: select UNIFORM, FIXED, RULE or GIVEN (block_fmt then
 * names the format of every block of every system, systems in order; no aMP switching);
 * policy.stream is used for every call. The setup also times eight variants of the
 * persistent kernel (32- or 64-row work tiles with registers for 2, 4 or 6 CTAs per SM,
 * 128-row tiles for 4 or 6) on this batch (20 iterations each) and keeps the fastest.
 * Errors: INVALID_ARG, UNSUPPORTED (also for a row of more than 65535 entries), NOT_SPD,
 * CUDA, NO_MEMORY. */
int bjac_batch_setup(int32_t nsys, const bjac_csr *A, const int32_t *const *block_ptr, const int32_t *nb,
                     const bjac_policy *policy, bjac_batch **out);

/* Solve all systems of the batch by PCG at once: one cooperative persistent kernel,
 * captured once in a CUDA graph, in which every system has its own PCG scalars and stops at
 * its own convergence (recurrence relres <= tol, then a true-residual check with up to two
 * restarts). b[s], x[s]: DEVICE vectors of system s (x[s] holds x0 on entry). stats (HOST,
 * nullable, nsys entries). Returns OK if all converged, else the worst status (errors < 0
 * before NOT_CONVERGED); TIMEOUT if a grid barrier's bounded wait expired. Synchronises. */
int pcg_solve_batched(bjac_batch *h, const double *const *b, double *const *x, double tol, int32_t maxit,
                      pcg_stats *stats);

/* Work tiles, tile height chosen by the setup's timing, grid size and the timings of the
 * eight kernel variants (tune_ms[8]: 32-row tiles with registers for 2, 4, 6 CTAs per SM,
 * 64-row tiles likewise, then 128-row tiles for 4 and 6) of a batch. All outputs HOST and
 * nullable. */
int bjac_batch_info(const bjac_batch *h, int32_t *ntiles, int32_t *tile_rows, int32_t *grid, float *tune_ms);

/* Failure-path test hook: with on = 1, the grid barriers of the batch's next solves wait for
 * one CTA more than the grid holds, so every CTA's bounded wait (2 s of %globaltimer) expires,
 * the kernel leaves at that barrier and pcg_solve_batched returns TIMEOUT with the context
 * still usable; on = 0 restores normal solves. Nothing faults, traps or hangs. Returns
 * INVALID_ARG for a NULL batch or on outside {0, 1}. */
int bjac_batch_force_timeout(bjac_batch *h, int32_t on);

/* Use kernel variant `variant` (0..7, in the order of bjac_batch_info's tune_ms) for the
 * batch's next solves instead of the one the setup's timing chose; rebuilds the work tiles
 * when the tile height changes. Synchronises the batch's stream. Returns INVALID_ARG for a
 * NULL batch or a variant outside 0..7. Every variant gives a valid solve; they differ in
 * speed and in the grouping of the partial sums. */
int bjac_batch_set_variant(bjac_batch *h, int32_t variant);

void bjac_batch_destroy(bjac_batch *h);

/* Release everything the handle owns (synchronises its stream first). NULL is ignored. */
void bjac_destroy(bjac_handle *h);

/* Message of the last failing call on this thread ("" if none). */
const char *bjac_last_error(void);

/* ---- the steps of one PCG iteration, callable alone ---------------------------------- */

/* y = A x (DEVICE x, y; n doubles). If xy (DEVICE, nullable) is given, *xy = x . y is
 * written as well (deterministic two-stage reduction). For long rows the kernel stages tiles
 * with TMA copies under bounded waits; if one expires, *xy and the rows not reached are NaN. */
int bjac_spmv(const bjac_csr *A, const double *x, double *y, double *xy, void *stream);

/* Allocation-free y = A x and *xy = x . y, for callers that cannot allocate device memory
 * while they run (a fixed device-memory budget reserved up front, a hard memory cap, or code
 * that must not let cudaFree synchronise the device). The paper has no counterpart: this is a
 * deployment variant of bjac_spmv. Same arguments as bjac_spmv except that xy (DEVICE, one
 * double) is required. Instead of allocating scratch for the partial sums of the dot product
 * it uses a buffer in the library's static device memory: 65,536 partial-sum pairs (1 MiB),
 * which every GPU that loads the library holds until the process exits, so n is limited to
 * 16,777,216 rows (INVALID_ARG beyond, with a message naming the limit). The first call on a
 * device looks up that buffer's device address (cudaGetSymbolAddress, with the device
 * current); make that first call before any stream capture. Every call shares the one buffer
 * and finds there what the previous call left (the ticket counter is cleared each time):
 * calls that overlap on the GPU (other streams, other threads) race and must not be made.
 * Calls no cudaMalloc, cudaFree or allocating library routine. As in bjac_spmv, matrices with
 * long rows (mean > 8 nonzeros) stage their tiles with TMA copies whose waits are bounded: if
 * one expires, *xy and the rows the kernel did not reach are NaN (the call itself cannot tell). */
int bjac_spmv_noalloc(const bjac_csr *A, const double *x, double *y, double *xy, void *stream);

/* r = b - A x and, if rr (DEVICE, nullable) is given, *rr = r . r. */
int bjac_residual(const bjac_csr *A, const double *b, const double *x, double *r, double *rr,
                  void *stream);

/* z = M^-1 r with the handle's binary64 set (set = 0) or low-precision set (set = 1),
 * Algorithm 3.1 for the latter. r, z: DEVICE, n doubles. rz (DEVICE, nullable): r . z.
 * Uses the handle's stream. Error UNSUPPORTED if the requested set was not kept. */
int bjac_apply(bjac_handle *h, int32_t set, const double *r, double *z, double *rz);

/* The first min(maxit, 64) iterations of pcg_solve (no restart, no fallback), launched
 * kernel by kernel without the graph, back to back, with CUDA events around each kernel of
 * the loop body, to time them. ms (HOST, 4 floats) receives the mean device milliseconds
 * per iteration of: [0] q = A p with p.q, [1] r -= alpha q with ||r|| (aMP only, else 0),
 * [2] z = M^-1 r with r.z (fused with the r update outside aMP), [3] x += alpha p,
 * p = z + beta p. iters (HOST, nullable) receives the iterations averaged (those run before
 * convergence). x: DEVICE x0 in / iterate out. Synchronises the stream once. */
int pcg_profile(bjac_handle *h, const double *b, double *x, double tol, int32_t maxit, float *ms,
                int32_t *iters);

/* y = A x with the layout the handle's PCG loop uses (see bjac_policy.spmv_format), on the
 * handle's stream; *xy = x . y as well when xy (DEVICE, nullable) is given. x, y: DEVICE,
 * n doubles. Uses the handle's reduction scratch: not concurrent with a solve on the same
 * handle. */
int bjac_handle_spmv(bjac_handle *h, const double *x, double *y, double *xy);

/* ---- inspection (tests, tools) ------------------------------------------------------- */

/* The library's binary64 <-> binary32 conversions, element-wise over n entries: f[i] = x[i]
 * rounded to nearest even in binary32 (subnormals kept), w[i] = f[i] widened back. The apply
 * kernels convert r and z with these integer-only routines instead of the hardware
 * conversion (which would occupy the FP64 pipe); this entry lets a test compare them with
 * the hardware and with an independent rounding. x: DEVICE; f, w: DEVICE, nullable. */
int bjac_convert(const double *x, float *f, double *w, int32_t n, void *stream);

/* Layout of the loop SpMV (HOST outputs, each nullable): *format 0 = CSR arrays of the
 * caller, 1 = SELL-32 copy (slices of 32 rows padded to the slice's longest row, stored
 * column-major), 2 = the SELL-32 copy with prefetch; *entries = stored entries of the SELL-32
 * copy including padding (0 if none was kept); ms[3] = median times of one y = A x with the
 * CSR kernel and the two SELL-32 kernels when the setup timed them (else 0). */
int bjac_spmv_format(const bjac_handle *h, int32_t *format, int64_t *entries, float *ms);

/* Sizes: nb, bytes of the low-precision pool, entries of the binary64 pool (0 if not kept). */
int bjac_info(const bjac_handle *h, int32_t *nb, int64_t *pool_bytes, int64_t *g_entries);

/* Copy device state to HOST arrays (each nullable; synchronises the stream):
 * fmt[nb] (uint8), scale[nb] (float), qoff[nb+1] (int64 byte offsets of each block in the
 * pool), pool[pool_bytes], G[g_entries] (binary64 blocks, row-major, consecutive),
 * feat[nb*12] (double, computed on first request). */
int bjac_export(bjac_handle *h, uint8_t *fmt, float *scale, int64_t *qoff, uint8_t *pool,
                double *G, double *feat);

/* Replace the binary64 inverses by G (HOST, g_entries doubles, same layout as bjac_export)
 * and re-round every block to its current format. Lets a test feed identical inputs to
 * the GPU rounding and to an independent implementation. */
int bjac_import_inverse(bjac_handle *h, const double *G);

/* Kernel the handle uses for the low-precision apply (0 generic, 1 TMA-staged, 2
 * register-direct, 3 register-direct for mixed formats) and, when the autotuner ran, its
 * timings in ms (tune_ms[4], HOST, nullable; 0 for kernels not timed). */
int bjac_apply_kernel(const bjac_handle *h, int32_t *kind, float *tune_ms);

/* Process-wide choice of the SpMV kernel for matrices with short rows (mean <= 8 nonzeros):
 * 0 = timed once per matrix shape at setup and the faster kept (default), 1 = TMA-staged CTA
 * tiles, 2 = warp-cooperative, 5 = bjac_spmv and bjac_residual build a SELL-32 copy of A for
 * the call and run the SELL-32 kernel (a test mode: it allocates and synchronises; handles are
 * unaffected). Rows longer on average always use the TMA kernel with large stages. Returns
 * the previous setting, or INVALID_ARG (3 and 4 named kernels that no workload chose and are
 * no longer built). Not thread-safe. */
int bjac_spmv_kernel(int32_t variant);

/* Process-wide L2 residency of the PCG vectors in the solver loop: 1 (default) = the loop's
 * SpMV, apply and update kernels load and store r, z, p, q and x with an evict_last L2 policy
 * while the matrix and the block inverses stream with evict-first loads, so the vectors
 * (5 n doubles) stay in the L2 (129 MB) from one kernel to the next; 0 = plain vector accesses.
 * Applies to solves started afterwards; results are the same either way. Returns the previous
 * setting, or INVALID_ARG. Not thread-safe. */
int bjac_l2_residency(int32_t keep);

/* SpMV kernel that A's shape uses now (1 TMA-staged, 2 warp-cooperative) and, if the timing
 * ran for it, the two median times in ms (ms[2], HOST, nullable). */
int bjac_spmv_tuning(const bjac_csr *A, int32_t *variant, float *ms);

/* ---- the learned selector (training and inference on the GPU) ------------------------ */

/* Gradient of the mean softmax cross-entropy of the 12-64-64-3 selector over N samples.
 * params: HOST, bjac_mlp_param_count() floats (weights, then feature mean and standard
 * deviation used to standardise the inputs). feat: DEVICE N x 12 doubles (raw features as
 * bjac_export returns them); label: DEVICE N int32 classes (0 FP64, 1 FP32, 2 16-bit).
 * bf16_weights: 1 = the weights rounded to bfloat16 (as inference does) on the tensor cores
 * (tcgen05: layer 2's forward product, its back-propagation and its weight gradient as BF16
 * MMAs with FP32 accumulation, each binary32 activation or error entering as two bfloat16
 * parts), 2 = the same weights on CUDA cores, 0 = the binary32 values on CUDA cores.
 * grad: HOST, the first 5187 entries (weights only); loss: HOST. Returns
 * MPBJAC_ERR_INVALID_ARG for another bf16_weights value and MPBJAC_ERR_TIMEOUT when an MMA did
 * not complete within the bounded wait. */
int bjac_mlp_grad(const float *params, int32_t bf16_weights, const double *feat, const int32_t *label, int32_t N,
                  float *grad, float *loss, void *stream);

/* Full-batch Adam (beta 0.9 / 0.999) for `epochs` steps on the same loss with bfloat16
 * forward weights (the tensor-core gradient of bjac_mlp_grad mode 1) and binary32 masters;
 * params (HOST) is updated in place (the feature mean and deviation entries are left as
 * given). loss_hist: HOST, epochs floats, nullable; with it, an MMA timeout is reported as
 * MPBJAC_ERR_TIMEOUT. */
int bjac_mlp_train(float *params, const double *feat, const int32_t *label, int32_t N, int32_t epochs, float lr,
                   float *loss_hist, void *stream);

/* Logits (HOST, N x 3) of the selector for N feature rows (DEVICE). bf16_weights: 1 = weights
 * rounded to bfloat16 on the tensor cores (tcgen05; the forward pass bjac_setup's
 * BJAC_SELECT_MLP runs: the 64 x 64 layer as BF16 MMAs with FP32 accumulation, each hidden
 * value entering as two bfloat16 parts), 2 = the same weights on CUDA cores, 0 = binary32
 * weights on CUDA cores. Rows of a tile whose MMA did not complete in the bounded wait are NaN.
 * Returns MPBJAC_ERR_INVALID_ARG for another bf16_weights value. */
int bjac_mlp_logits(const float *params, int32_t bf16_weights, const double *feat, int32_t N, float *logits,
                    void *stream);

/* Number of floats of the selector's parameter vector:
 * W1[64][12] b1[64] W2[64][64] b2[64] W3[3][64] b3[3] mu[12] sd[12]. */
int32_t bjac_mlp_param_count(void);

#ifdef __cplusplus
}
#endif
#endif /* MPBJAC_H */
