/*
 * Plain CPU FP64 oracle for mixed-precision block-Jacobi PCG.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load this file. The product path never calls it and shares no code with it.
 *
 * Everything here is written for a reader checking it against the paper by eye: plain
 * loops, sequential sums in natural index order, binary64 arithmetic, no blocking, no
 * fusion. Build flags keep the compiler from contracting a*b+c into an FMA
 * (-ffp-contract=off), so every product and every sum is rounded once, in program order.
 *
 * Threads: the checker build (liboracle.so, used by every test) is single-threaded. A second
 * build of this same file with -fopenmp (liboracle_omp.so) serves only as the timed CPU
 * baseline: the `omp` pragmas below split loops whose iterations are independent (rows of
 * the SpMV, blocks of the inverse and the apply, entries of the vector updates) across
 * threads; every row, block and entry is computed exactly as in the serial loop and the dot
 * products stay sequential, so both builds give the same bits.
 *
 * Paper: "Mixed Precision Block-Jacobi Preconditioner: Algorithms, Performance Evaluation
 * and Feature Analysis" (arXiv 2407.15973).
 *
 * Sections:
 *   SpMV / dot          -- the working-precision operations of PCG (Section 3.2)
 *   block inverse       -- exact BJAC with k = 1, M^-1 = D_b^-1 (Eq. 3-1, special case
 *                          noted after Eq. 3-3), by LU with partial pivoting
 *   rounding            -- ConvertPrecision of Algorithm 3.1, written from the IEEE 754
 *                          binary32 / binary16 and bfloat16 bit layouts
 *   packing / apply     -- M^-1_bjac(p_l) applied to r-hat (Algorithm 3.1)
 *   PCG + policies      -- fMP (Algorithm 3.1), aMP(hl) (Algorithm 3.2), aMP(lh)
 *                          (Algorithm 3.3), convergence test of Section 4.2; optionally the
 *                          flexible-CG (Polak-Ribiere) direction coefficient
 *   multiscale / features / selection rule / MLP -- per-block quantities (Eq. 4-5,
 *                          Section 4.5.2) and the block-format selectors
 *   BJAC(k, t)          -- the inexact block Jacobi of Eq. 3-2 / 3-3 (inner Jacobi sweeps
 *                          inside the blocks, outer block-Jacobi sweeps), in binary64 or
 *                          binary32 (Algorithm 3.1), and PCG with it
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the loops below run on: 1 in the checker build, the OpenMP team size otherwise. */
int32_t orc_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORC_FP64 0
#define ORC_FP32 1
#define ORC_BF16 2
#define ORC_FP16S 3

/* ====================================================================================== */
/* SpMV and dot products (working precision p_w = binary64, Section 3.2)                  */
/* ====================================================================================== */

/* y = A x; row i sums val[k] * x[colidx[k]] for k = rowptr[i] .. rowptr[i+1]-1 in order. */
void orc_spmv(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
              const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[colidx[k]];
        y[i] = s;
    }
}

/* Summation order of orc_dot (and so of every dot product and norm in orc_pcg). Every order
 * rounds each product a_i * b_i once and adds the products in binary64; they differ only in
 * which partial sums are formed, so each is an equally valid evaluation of the definition.
 *   0  sequential from index 0 upward (the default; every pin and parity test uses it)
 *   1  sequential from index n-1 downward
 *   2  pairwise: the range is halved recursively, runs of <= 8 terms summed in order
 *   3  strided partials: 1024 running sums, sum p over the indices i = p (mod 1024) in
 *      increasing order, then the 1024 partials added pairwise (the shape of a grid-stride
 *      GPU reduction)
 *   4  compensated (Neumaier's variant of Kahan summation, Neumaier 1974): the running
 *      rounding error is carried and added at the end, nearly the exactly rounded sum
 * Only the spread test selects another order; the setting is process-wide. */
static int32_t g_dot_order = 0;

int32_t orc_set_dot_order(int32_t order) {
    int32_t old = g_dot_order;
    if (order >= 0 && order <= 4) g_dot_order = order;
    return old;
}

static double dot_pairwise(int64_t n, const double *a, const double *b) {
    if (n <= 8) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
        return s;
    }
    int64_t h = n / 2;
    return dot_pairwise(h, a, b) + dot_pairwise(n - h, a + h, b + h);
}

static double sum_pairwise(int64_t n, const double *v) {
    if (n <= 8) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += v[i];
        return s;
    }
    int64_t h = n / 2;
    return sum_pairwise(h, v) + sum_pairwise(n - h, v + h);
}

/* a . b in the order g_dot_order names (default: from index 0 upward). */
double orc_dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    if (g_dot_order == 1) {
        for (int64_t i = n - 1; i >= 0; --i) s += a[i] * b[i];
    } else if (g_dot_order == 2) {
        s = dot_pairwise(n, a, b);
    } else if (g_dot_order == 3) {
        double part[1024];
        for (int p = 0; p < 1024; ++p) part[p] = 0.0;
        for (int64_t i = 0; i < n; ++i) part[i % 1024] += a[i] * b[i];
        s = sum_pairwise(1024, part);
    } else if (g_dot_order == 4) {
        double c = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double t = a[i] * b[i];
            double u = s + t;
            if (fabs(s) >= fabs(t)) c += (s - u) + t;
            else c += (t - u) + s;
            s = u;
        }
        s += c;
    } else {
        for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    }
    return s;
}

/* r = b - A x (the "true" residual of Section 4.5.1: from the definition, not the recurrence). */
void orc_residual(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                  const double *b, const double *x, double *r) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[colidx[k]];
        r[i] = b[i] - s;
    }
}

/* ====================================================================================== */
/* Diagonal-block inverses: D_b = diag{A_ii} (Eq. 3-1); with k = 1 and exact inverses the  */
/* BJAC preconditioner is M^-1 = D_b^-1 (the special case stated after Eq. 3-3).            */
/* ====================================================================================== */

/* Dense copy of the diagonal block A[s:e, s:e] (columns outside the block are dropped). */
static void extract_block(const int32_t *rowptr, const int32_t *colidx, const double *val,
                          int32_t s, int32_t e, double *B) {
    int32_t bs = e - s;
    memset(B, 0, sizeof(double) * (size_t)bs * bs);
    for (int32_t i = s; i < e; ++i)
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int32_t j = colidx[k];
            if (j >= s && j < e) B[(size_t)(i - s) * bs + (j - s)] += val[k];
        }
}

/* Inverse of a dense bs x bs matrix by LU factorisation with partial (row) pivoting,
 * P B = L U, then solving L U x = P e_j for each identity column e_j.
 * Returns 0 on success, 1 if a pivot is exactly zero (singular block). */
static int lu_inverse(int32_t bs, const double *B, double *X, double *work, int32_t *perm) {
    double *LU = work;
    memcpy(LU, B, sizeof(double) * (size_t)bs * bs);
    for (int32_t i = 0; i < bs; ++i) perm[i] = i;
    for (int32_t k = 0; k < bs; ++k) {
        int32_t p = k;
        double best = fabs(LU[(size_t)k * bs + k]);
        for (int32_t i = k + 1; i < bs; ++i)
            if (fabs(LU[(size_t)i * bs + k]) > best) { best = fabs(LU[(size_t)i * bs + k]); p = i; }
        if (best == 0.0) return 1;
        if (p != k) {
            for (int32_t j = 0; j < bs; ++j) {
                double t = LU[(size_t)k * bs + j];
                LU[(size_t)k * bs + j] = LU[(size_t)p * bs + j];
                LU[(size_t)p * bs + j] = t;
            }
            int32_t t = perm[k]; perm[k] = perm[p]; perm[p] = t;
        }
        for (int32_t i = k + 1; i < bs; ++i) {
            double l = LU[(size_t)i * bs + k] / LU[(size_t)k * bs + k];
            LU[(size_t)i * bs + k] = l;
            for (int32_t j = k + 1; j < bs; ++j) LU[(size_t)i * bs + j] -= l * LU[(size_t)k * bs + j];
        }
    }
    double *y = work + (size_t)bs * bs;
    for (int32_t c = 0; c < bs; ++c) {
        /* forward: L y = P e_c (unit lower triangle) */
        for (int32_t i = 0; i < bs; ++i) {
            double s = (perm[i] == c) ? 1.0 : 0.0;
            for (int32_t j = 0; j < i; ++j) s -= LU[(size_t)i * bs + j] * y[j];
            y[i] = s;
        }
        /* backward: U x = y */
        for (int32_t i = bs - 1; i >= 0; --i) {
            double s = y[i];
            for (int32_t j = i + 1; j < bs; ++j) s -= LU[(size_t)i * bs + j] * X[(size_t)j * bs + c];
            X[(size_t)i * bs + c] = s / LU[(size_t)i * bs + i];
        }
    }
    return 0;
}

/* For every block b = [block_ptr[b], block_ptr[b+1]):  G_b = (B_b^-1 + B_b^-T) / 2, stored
 * row-major at G + goff[b]. normB1 (optional) receives ||B_b||_1 (max column sum).
 * Returns the number of singular blocks (their G is left zero). */
int32_t orc_block_inverse(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                          int32_t nb, const int32_t *block_ptr, const int64_t *goff, double *G,
                          double *normB1) {
    (void)n;
    int32_t maxbs = 0;
    for (int32_t b = 0; b < nb; ++b)
        if (block_ptr[b + 1] - block_ptr[b] > maxbs) maxbs = block_ptr[b + 1] - block_ptr[b];
    size_t m2 = (size_t)maxbs * maxbs;
    int32_t bad = 0;
#pragma omp parallel reduction(+ : bad)
    {
    double *B = malloc(sizeof(double) * m2);
    double *X = malloc(sizeof(double) * m2);
    double *work = malloc(sizeof(double) * (m2 + maxbs));
    int32_t *perm = malloc(sizeof(int32_t) * (maxbs > 0 ? maxbs : 1));
#pragma omp for schedule(dynamic, 64)
    for (int32_t b = 0; b < nb; ++b) {
        int32_t s = block_ptr[b], e = block_ptr[b + 1], bs = e - s;
        double *Gb = G + goff[b];
        extract_block(rowptr, colidx, val, s, e, B);
        if (normB1) {
            double mx = 0.0;
            for (int32_t j = 0; j < bs; ++j) {
                double c = 0.0;
                for (int32_t i = 0; i < bs; ++i) c += fabs(B[(size_t)i * bs + j]);
                if (c > mx) mx = c;
            }
            normB1[b] = mx;
        }
        if (lu_inverse(bs, B, X, work, perm)) {
            memset(Gb, 0, sizeof(double) * (size_t)bs * bs);
            ++bad;
            continue;
        }
        for (int32_t i = 0; i < bs; ++i)
            for (int32_t j = 0; j < bs; ++j)
                Gb[(size_t)i * bs + j] = 0.5 * (X[(size_t)i * bs + j] + X[(size_t)j * bs + i]);
    }
    free(B); free(X); free(work); free(perm);
    }
    return bad;
}

/* ====================================================================================== */
/* ConvertPrecision (Algorithm 3.1): round-to-nearest, ties-to-even, from binary64         */
/* directly to the target format (no intermediate format, so no double rounding).          */
/* A format has 1 sign bit, `ebits` exponent bits (bias 2^(ebits-1)-1) and `mbits` stored   */
/* fraction bits; subnormals are kept; overflow goes to infinity.                          */
/* ====================================================================================== */
static uint32_t round_bits(double x, int ebits, int mbits) {
    uint32_t sign = signbit(x) ? 1u : 0u;
    uint32_t expmask = (1u << ebits) - 1u;
    uint32_t sbit = sign << (ebits + mbits);
    if (isnan(x)) return sbit | (expmask << mbits) | (1u << (mbits - 1));
    double a = fabs(x);
    if (isinf(a)) return sbit | (expmask << mbits);
    if (a == 0.0) return sbit;
    int bias = (1 << (ebits - 1)) - 1;
    int e2;
    (void)frexp(a, &e2);              /* a = f 2^e2, f in [0.5, 1) */
    int E = e2 - 1;                   /* a in [2^E, 2^(E+1)) */
    if (E > bias) return sbit | (expmask << mbits);
    int et = E < 1 - bias ? 1 - bias : E;  /* exponent of the quantum's binade */
    double N = ldexp(a, mbits - et);  /* a / 2^(et - mbits): exact scaling */
    double I = floor(N);
    double frac = N - I;
    if (frac > 0.5 || (frac == 0.5 && fmod(I, 2.0) != 0.0)) I += 1.0;
    uint64_t q = (uint64_t)I;
    if (q == 0) return sbit;
    uint32_t field;
    uint64_t mant;
    if (q < (1ull << mbits)) {                 /* subnormal (only when et == 1 - bias) */
        field = 0; mant = q;
    } else if (q < (2ull << mbits)) {
        field = (uint32_t)(et + bias); mant = q - (1ull << mbits);
    } else {                                   /* rounding carried into the next binade */
        field = (uint32_t)(et + bias + 1); mant = 0;
    }
    if (field >= expmask) return sbit | (expmask << mbits);
    return sbit | (field << mbits) | (uint32_t)mant;
}

static double decode_bits(uint32_t bits, int ebits, int mbits) {
    uint32_t expmask = (1u << ebits) - 1u;
    int bias = (1 << (ebits - 1)) - 1;
    uint32_t sign = (bits >> (ebits + mbits)) & 1u;
    uint32_t field = (bits >> mbits) & expmask;
    uint32_t mant = bits & ((1u << mbits) - 1u);
    double v;
    if (field == expmask) v = mant ? NAN : INFINITY;
    else if (field == 0) v = ldexp((double)mant, 1 - bias - mbits);
    else v = ldexp((double)(mant | (1u << mbits)), (int)field - bias - mbits);
    return sign ? -v : v;
}

uint32_t orc_round_f32_bits(double x) { return round_bits(x, 8, 23); }
uint16_t orc_round_bf16_bits(double x) { return (uint16_t)round_bits(x, 8, 7); }
uint16_t orc_round_f16_bits(double x) { return (uint16_t)round_bits(x, 5, 10); }
double orc_decode_f32(uint32_t b) { return decode_bits(b, 8, 23); }
double orc_decode_bf16(uint16_t b) { return decode_bits(b, 8, 7); }
double orc_decode_f16(uint16_t b) { return decode_bits(b, 5, 10); }

void orc_round_array(int32_t fmt, int64_t count, const double *in, void *out) {
    for (int64_t i = 0; i < count; ++i) {
        if (fmt == ORC_FP32) ((uint32_t *)out)[i] = orc_round_f32_bits(in[i]);
        else if (fmt == ORC_BF16) ((uint16_t *)out)[i] = orc_round_bf16_bits(in[i]);
        else if (fmt == ORC_FP16S) ((uint16_t *)out)[i] = orc_round_f16_bits(in[i]);
        else ((double *)out)[i] = in[i];
    }
}

static float as_float(uint32_t bits) { float f; memcpy(&f, &bits, 4); return f; }

/* ====================================================================================== */
/* The low-precision preconditioner M^-1_bjac(p_l) (Algorithm 3.1 input).                  */
/* Block b is stored row-major in format fmt[b] at byte offset qoff[b] of `pool`, as       */
/* Q_b = RN_fmt(G_b / s_b). s_b = 1 for FP64 / FP32; for the 16-bit formats s_b is the     */
/* power of two 2^(floor(log2 max|G_b|) - 14), which puts max|Q_b| in [2^14, 2^15) and is   */
/* an exact scaling in binary64.                                                           */
/* ====================================================================================== */

float orc_block_scale(int32_t fmt, int64_t count, const double *Gb) {
    if (fmt == ORC_FP64 || fmt == ORC_FP32) return 1.0f;
    double mx = 0.0;
    for (int64_t i = 0; i < count; ++i) if (fabs(Gb[i]) > mx) mx = fabs(Gb[i]);
    if (mx == 0.0 || !isfinite(mx)) return 1.0f;
    int e2;
    (void)frexp(mx, &e2);
    return (float)ldexp(1.0, (e2 - 1) - 14);
}

void orc_pack(int32_t nb, const int32_t *block_ptr, const uint8_t *fmt, const double *G,
              const int64_t *goff, uint8_t *pool, const int64_t *qoff, float *scale) {
#pragma omp parallel for schedule(static)
    for (int32_t b = 0; b < nb; ++b) {
        int32_t bs = block_ptr[b + 1] - block_ptr[b];
        int64_t cnt = (int64_t)bs * bs;
        const double *Gb = G + goff[b];
        float s = orc_block_scale(fmt[b], cnt, Gb);
        scale[b] = s;
        uint8_t *dst = pool + qoff[b];
        for (int64_t i = 0; i < cnt; ++i) {
            double v = Gb[i] / (double)s;   /* power-of-two scaling: exact */
            if (fmt[b] == ORC_FP64) memcpy(dst + 8 * i, &v, 8);
            else if (fmt[b] == ORC_FP32) { uint32_t t = orc_round_f32_bits(v); memcpy(dst + 4 * i, &t, 4); }
            else if (fmt[b] == ORC_BF16) { uint16_t t = orc_round_bf16_bits(v); memcpy(dst + 2 * i, &t, 2); }
            else { uint16_t t = orc_round_f16_bits(v); memcpy(dst + 2 * i, &t, 2); }
        }
    }
}

/* Q_b[i][j] decoded exactly to binary64 (all formats embed exactly in binary64). */
static double q_entry(const uint8_t *blk, int f, int64_t idx) {
    if (f == ORC_FP64) { double v; memcpy(&v, blk + 8 * idx, 8); return v; }
    if (f == ORC_FP32) { uint32_t t; memcpy(&t, blk + 4 * idx, 4); return (double)as_float(t); }
    uint16_t t; memcpy(&t, blk + 2 * idx, 2);
    return f == ORC_BF16 ? orc_decode_bf16(t) : orc_decode_f16(t);
}

/* z = M^-1 r with the block-stored preconditioner (Algorithm 3.1).
 * FP64 blocks: z_b = Q_b r_b in binary64 (no conversion).
 * Low blocks:  r-hat = RN_fp32(r) (line "convert r to p_l"); z_b = s_b * Q_b r-hat.
 *   mode 0: the product is formed in binary64 from the exact decoded values (the ideal
 *           result of applying the stored low-precision operator);
 *   mode 1: "compute in p_l": each row is a binary32 dot product accumulated in natural
 *           order j = 0, 1, ... with fused multiply-add, acc = fmaf(Q_ij, r-hat_j, acc),
 *           multiplied by s_b in binary32 (a power of two), then widened to binary64. */
void orc_apply(int32_t nb, const int32_t *block_ptr, const uint8_t *fmt, const uint8_t *pool,
               const int64_t *qoff, const float *scale, const double *r, double *z, int32_t mode) {
    /* r-hat = ConvertPrecision(r, binary32), each entry rounded once */
    int32_t n = block_ptr[nb];
    float *rh = malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; ++i) rh[i] = as_float(orc_round_f32_bits(r[i]));
#pragma omp parallel for schedule(static)
    for (int32_t b = 0; b < nb; ++b) {
        int32_t s = block_ptr[b], bs = block_ptr[b + 1] - s;
        const uint8_t *blk = pool + qoff[b];
        int f = fmt[b];
        for (int32_t i = 0; i < bs; ++i) {
            if (f == ORC_FP64) {
                double acc = 0.0;
                for (int32_t j = 0; j < bs; ++j) acc += q_entry(blk, f, (int64_t)i * bs + j) * r[s + j];
                z[s + i] = acc;
            } else if (mode == 0) {
                double acc = 0.0;
                for (int32_t j = 0; j < bs; ++j) acc += q_entry(blk, f, (int64_t)i * bs + j) * (double)rh[s + j];
                z[s + i] = acc * (double)scale[b];
            } else {
                float acc = 0.0f;
                for (int32_t j = 0; j < bs; ++j) {
                    float q = (float)q_entry(blk, f, (int64_t)i * bs + j);
                    acc = fmaf(q, rh[s + j], acc);
                }
                z[s + i] = (double)(acc * scale[b]);
            }
        }
    }
    free(rh);
}

/* z = G r with the binary64 inverses (the uniform / high-precision preconditioner). */
void orc_apply_fp64(int32_t nb, const int32_t *block_ptr, const double *G, const int64_t *goff,
                    const double *r, double *z) {
#pragma omp parallel for schedule(static)
    for (int32_t b = 0; b < nb; ++b) {
        int32_t s = block_ptr[b], bs = block_ptr[b + 1] - s;
        const double *Gb = G + goff[b];
        for (int32_t i = 0; i < bs; ++i) {
            double acc = 0.0;
            for (int32_t j = 0; j < bs; ++j) acc += Gb[(size_t)i * bs + j] * r[s + j];
            z[s + i] = acc;
        }
    }
}

/* ====================================================================================== */
/* PCG (Hestenes-Stiefel) in binary64 with the (mixed-precision) BJAC preconditioner.      */
/* Stopping rule of Section 4.2: ||r_k||_2 / ||b||_2 <= tol, x0 given (zero in the paper). */
/* Preconditioner choice per application, from the relative residual of the residual     */
/* being preconditioned:                                                                  */
/*   policy 0  uniform: binary64 inverses G always                                         */
/*   policy 1  fMP (Algorithm 3.1): the stored low-precision set always                    */
/*   policy 2  aMP(hl) (Algorithm 3.2): G while relres >= adp_tol, else the low set        */
/*   policy 3  aMP(lh) (Algorithm 3.3): the low set while relres >= adp_tol, else G        */
/* After the recurrence meets tol, the true residual b - A x is formed; if it does not     */
/* meet tol, PCG restarts from it (r = b - A x, p = M^-1 r) while iterations remain.       */
/* Flexible (Polak-Ribiere) direction coefficient of flexible CG (G. H. Golub and Q. Ye, SIAM
 * J. Sci. Comput. 21, 1999; Y. Notay, SIAM J. Sci. Comput. 22, 2000):
 *     beta_k = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k),
 * in place of rho_{k+1} / rho_k. It keeps consecutive search directions A-conjugate when the
 * preconditioner changes between iterations (aMP's switch of Algorithms 3.2 / 3.3) or is not
 * exactly linear (a low-precision apply), and equals rho_{k+1} / rho_k for a fixed symmetric
 * preconditioner in exact arithmetic (z_{k+1}^T r_k = 0 there). */
static double flexible_beta(int32_t n, const double *z, const double *r, const double *r_prev, double rho) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += z[i] * (r[i] - r_prev[i]);
    return s / rho;
}

/* ====================================================================================== */
typedef struct {
    int32_t iters, converged, status, restarts, low_applies, high_applies;
    double relres, true_relres;
} orc_stats;

#define ORC_OK 0
#define ORC_BREAKDOWN -5
#define ORC_NOT_CONVERGED 1

typedef struct {
    int32_t nb;
    const int32_t *block_ptr;
    const double *G; const int64_t *goff;
    const uint8_t *fmt; const uint8_t *pool; const int64_t *qoff; const float *scale;
    int32_t policy; double adp_tol; int32_t mode;
} precond;

static int use_low(const precond *P, double relres) {
    switch (P->policy) {
        case 0: return 0;
        case 1: return 1;
        case 2: return !(relres >= P->adp_tol);
        default: return relres >= P->adp_tol;
    }
}

static void precondition(const precond *P, double relres, const double *r, double *z, orc_stats *st,
                         uint8_t *flag) {
    if (use_low(P, relres)) {
        orc_apply(P->nb, P->block_ptr, P->fmt, P->pool, P->qoff, P->scale, r, z, P->mode);
        st->low_applies++;
        if (flag) *flag = 1;
    } else {
        orc_apply_fp64(P->nb, P->block_ptr, P->G, P->goff, r, z);
        st->high_applies++;
        if (flag) *flag = 0;
    }
}

int32_t orc_pcg(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                int32_t nb, const int32_t *block_ptr, const double *G, const int64_t *goff,
                const uint8_t *fmt, const uint8_t *pool, const int64_t *qoff, const float *scale,
                int32_t policy, double adp_tol, int32_t mode, int32_t flexible,
                const double *b, double *x, double tol, int32_t maxit,
                double *hist, uint8_t *low_used, orc_stats *st) {
    precond P = {nb, block_ptr, G, goff, fmt, pool, qoff, scale, policy, adp_tol, mode};
    memset(st, 0, sizeof(*st));
    double *r = malloc(sizeof(double) * (size_t)n);
    double *z = malloc(sizeof(double) * (size_t)n);
    double *p = malloc(sizeof(double) * (size_t)n);
    double *q = malloc(sizeof(double) * (size_t)n);
    double *rp = malloc(sizeof(double) * (size_t)n);     /* r_k, kept for the flexible beta */
    double bnorm = sqrt(orc_dot(n, b, b));
    int32_t k = 0, status = ORC_OK;
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        st->converged = 1; st->relres = 0.0; st->true_relres = 0.0;
        goto done;
    }
    orc_residual(n, rowptr, colidx, val, b, x, r);
    double relres = sqrt(orc_dot(n, r, r)) / bnorm;
    st->true_relres = relres;
    if (hist) hist[0] = relres;
    for (;;) {                                   /* one pass per (re)start */
        if (relres <= tol) break;
        precondition(&P, relres, r, z, st, low_used ? &low_used[k] : NULL);
        double rho = orc_dot(n, r, z);
        if (!(rho > 0.0) || !isfinite(rho)) { status = ORC_BREAKDOWN; break; }
        #pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i) p[i] = z[i];
        while (k < maxit) {
            orc_spmv(n, rowptr, colidx, val, p, q);
            double sigma = orc_dot(n, p, q);
            if (!(sigma > 0.0) || !isfinite(sigma)) { status = ORC_BREAKDOWN; break; }
            double alpha = rho / sigma;
            #pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
            #pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < n; ++i) rp[i] = r[i];
            #pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
            ++k;
            relres = sqrt(orc_dot(n, r, r)) / bnorm;
            if (hist) hist[k] = relres;
            if (!isfinite(relres)) { status = ORC_BREAKDOWN; break; }
            if (relres <= tol) break;
            if (k >= maxit) break;
            precondition(&P, relres, r, z, st, low_used ? &low_used[k] : NULL);
            double rho_new = orc_dot(n, r, z);
            if (!(rho_new > 0.0) || !isfinite(rho_new)) { status = ORC_BREAKDOWN; break; }
            double beta = flexible ? flexible_beta(n, z, r, rp, rho) : rho_new / rho;
            if (!isfinite(beta)) { status = ORC_BREAKDOWN; break; }
            #pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
            rho = rho_new;
        }
        if (status != ORC_OK) break;
        /* true residual from the definition */
        orc_residual(n, rowptr, colidx, val, b, x, r);
        double tr = sqrt(orc_dot(n, r, r)) / bnorm;
        st->true_relres = tr;
        if (tr <= tol || k >= maxit || st->restarts >= 8) break;
        st->restarts++;
        relres = tr;
    }
    st->relres = relres;
    st->converged = (status == ORC_OK && relres <= tol && st->true_relres <= tol) ? 1 : 0;
    if (status == ORC_OK && !st->converged) status = ORC_NOT_CONVERGED;
done:
    st->iters = k;
    st->status = status;
    free(r); free(z); free(p); free(q); free(rp);
    return status;
}

/* ====================================================================================== */
/* Multiscale strength (Eq. 4-5): tau_i = max |a_ij| / min |a_ij| over nonzero            */
/* off-diagonal entries of row i. A row with no nonzero off-diagonal has tau_i = 1.        */
/* ====================================================================================== */
void orc_multiscale(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                    double *tau) {
    for (int32_t i = 0; i < n; ++i) {
        double mx = 0.0, mn = INFINITY;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colidx[k] == i || val[k] == 0.0) continue;
            double a = fabs(val[k]);
            if (a > mx) mx = a;
            if (a < mn) mn = a;
        }
        tau[i] = (mx > 0.0) ? mx / mn : 1.0;
    }
}

/* P_diag transform of Section 4.5.2: a_ii <- a_ii + P_diag * sum_{j != i} |a_ij| (in place). */
void orc_diag_boost(int32_t n, const int32_t *rowptr, const int32_t *colidx, double *val, double pdiag) {
    for (int32_t i = 0; i < n; ++i) {
        double off = 0.0;
        int32_t kd = -1;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colidx[k] == i) kd = k;
            else off += fabs(val[k]);
        }
        if (kd >= 0) val[kd] = val[kd] + pdiag * off;
    }
}

/* ====================================================================================== */
/* Per-block features (12 per block), the condition-number selection rule and the MLP.    */
/* These extend the paper: its Section 4.5 ties convergence delay to multiscale strength  */
/* (Eq. 4-5) and diagonal dominance (Section 4.5.2); the selectors use those and the       */
/* block condition number (Related Work, adaptive block-Jacobi precision by condition).   */
/* ====================================================================================== */
#define ORC_NFEAT 12
#define DOM_CAP 1e6

/* Feature vector of block b (binary64):
 *  0 log10 kappa_1(B) = log10(||B||_1 ||G||_1)        6 max_i log10 tau_i
 *  1 log10 ||B||_F                                    7 mean_i log10 tau_i
 *  2 min_i  d_i,  d_i = |a_ii| / sum_{j!=i}|a_ij|      8 log10(max|G| / min_{G!=0}|G|)
 *  3 mean_i d_i   (full rows; d_i capped at 1e6)       9 bs / 128
 *  4 min_i |a_ii| / max_i |a_ii|                      10 fraction of rows with |a_ii| > sum_{j!=i}|a_ij|
 *  5 sum_{i in b, j not in b} |a_ij| / sum_{i in b, all j} |a_ij|
 *                                                     11 mean_i (|a_ii| - sum_{j!=i}|a_ij|) / |a_ii|   */
void orc_features(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                  int32_t nb, const int32_t *block_ptr, const double *G, const int64_t *goff,
                  double *feat) {
    (void)n;
    for (int32_t b = 0; b < nb; ++b) {
        int32_t s = block_ptr[b], e = block_ptr[b + 1], bs = e - s;
        double *f = feat + (size_t)b * ORC_NFEAT;
        /* ||B||_1: max column sum of |B| inside the block */
        double *col = calloc((size_t)bs, sizeof(double));
        double fro = 0.0, dmin = INFINITY, dsum = 0.0, amin = INFINITY, amax = 0.0;
        double out_sum = 0.0, all_sum = 0.0, tmax = 0.0, tsum = 0.0, excess = 0.0;
        int32_t ndom = 0;
        for (int32_t i = s; i < e; ++i) {
            double diag = 0.0, off = 0.0, mx = 0.0, mn = INFINITY;
            for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                int32_t j = colidx[k];
                double a = fabs(val[k]);
                all_sum += a;
                if (j >= s && j < e) { col[j - s] += a; fro += val[k] * val[k]; }
                else out_sum += a;
                if (j == i) diag += a;
                else {
                    off += a;
                    if (val[k] != 0.0) { if (a > mx) mx = a; if (a < mn) mn = a; }
                }
            }
            double d = off > 0.0 ? diag / off : DOM_CAP;
            if (d > DOM_CAP) d = DOM_CAP;
            if (d < dmin) dmin = d;
            dsum += d;
            if (diag < amin) amin = diag;
            if (diag > amax) amax = diag;
            if (diag > off) ++ndom;
            excess += diag > 0.0 ? (diag - off) / diag : 0.0;
            double tau = mx > 0.0 ? mx / mn : 1.0;
            double lt = log10(tau);
            if (lt > tmax) tmax = lt;
            tsum += lt;
        }
        double n1B = 0.0;
        for (int32_t j = 0; j < bs; ++j) if (col[j] > n1B) n1B = col[j];
        free(col);
        const double *Gb = G + goff[b];
        double n1G = 0.0, gmax = 0.0, gmin = INFINITY;
        for (int32_t j = 0; j < bs; ++j) {
            double c = 0.0;
            for (int32_t i = 0; i < bs; ++i) {
                double a = fabs(Gb[(size_t)i * bs + j]);
                c += a;
                if (a > gmax) gmax = a;
                if (a > 0.0 && a < gmin) gmin = a;
            }
            if (c > n1G) n1G = c;
        }
        f[0] = log10(n1B * n1G);
        f[1] = 0.5 * log10(fro);
        f[2] = dmin;
        f[3] = dsum / bs;
        f[4] = amax > 0.0 ? amin / amax : 0.0;
        f[5] = all_sum > 0.0 ? out_sum / all_sum : 0.0;
        f[6] = tmax;
        f[7] = tsum / bs;
        f[8] = gmax > 0.0 ? log10(gmax / gmin) : 0.0;
        f[9] = bs / 128.0;
        f[10] = (double)ndom / bs;
        f[11] = excess / bs;
    }
}

/* Condition-number rule: the cheapest format f whose unit roundoff u_f satisfies
 * kappa_1(B) * u_f <= theta, trying in order
 *   FP16S (u = 2^-11; only if max|G| / min_{G!=0}|G| <= 2^29), BF16 (2^-8), FP32 (2^-24),
 * and FP64 otherwise. kappa_1 and the dynamic range come from features 0 and 8. */
void orc_select_rule(int32_t nb, const double *feat, double theta, uint8_t *fmt) {
    const double l2 = log10(2.0);
    for (int32_t b = 0; b < nb; ++b) {
        double lk = feat[(size_t)b * ORC_NFEAT + 0];
        double ldr = feat[(size_t)b * ORC_NFEAT + 8];
        double lt = log10(theta);
        uint8_t f;
        if (ldr <= 29 * l2 && lk - 11 * l2 <= lt) f = ORC_FP16S;
        else if (lk - 8 * l2 <= lt) f = ORC_BF16;
        else if (lk - 24 * l2 <= lt) f = ORC_FP32;
        else f = ORC_FP64;
        fmt[b] = f;
    }
}

/* ---- MLP 12 -> 64 -> 64 -> 3 (ReLU, softmax cross-entropy), binary64 --------------------
 * Parameter vector layout (row-major W[out][in]):
 *   W1[64][12], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]   (total 5187)
 * Input is standardised: xin_k = (feat_k - mu_k) / sd_k. Classes: 0 FP64, 1 FP32, 2 16-bit. */
#define H1 64
#define H2 64
#define NCLS 3
#define NPARAM (H1 * ORC_NFEAT + H1 + H2 * H1 + H2 + NCLS * H2 + NCLS)

int32_t orc_mlp_nparam(void) { return NPARAM; }

static void mlp_fwd_one(const double *w, const double *xin, double *h1, double *h2, double *logit) {
    const double *W1 = w, *b1 = W1 + H1 * ORC_NFEAT, *W2 = b1 + H1, *b2 = W2 + H2 * H1;
    const double *W3 = b2 + H2, *b3 = W3 + NCLS * H2;
    for (int o = 0; o < H1; ++o) {
        double s = b1[o];
        for (int i = 0; i < ORC_NFEAT; ++i) s += W1[o * ORC_NFEAT + i] * xin[i];
        h1[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < H2; ++o) {
        double s = b2[o];
        for (int i = 0; i < H1; ++i) s += W2[o * H1 + i] * h1[i];
        h2[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < NCLS; ++o) {
        double s = b3[o];
        for (int i = 0; i < H2; ++i) s += W3[o * H2 + i] * h2[i];
        logit[o] = s;
    }
}

/* Logits for m samples (feat already standardised into xin[m][12]). */
void orc_mlp_forward(int32_t m, const double *w, const double *xin, double *logits) {
    double h1[H1], h2[H2];
    for (int32_t s = 0; s < m; ++s) mlp_fwd_one(w, xin + (size_t)s * ORC_NFEAT, h1, h2, logits + (size_t)s * NCLS);
}

/* Mean softmax cross-entropy over m samples and its gradient with respect to w. */
double orc_mlp_loss_grad(int32_t m, const double *w, const double *xin, const int32_t *label, double *grad) {
    const double *W2 = w + H1 * ORC_NFEAT + H1, *W3 = W2 + H2 * H1 + H2;
    double *gW1 = grad, *gb1 = gW1 + H1 * ORC_NFEAT, *gW2 = gb1 + H1, *gb2 = gW2 + H2 * H1;
    double *gW3 = gb2 + H2, *gb3 = gW3 + NCLS * H2;
    memset(grad, 0, sizeof(double) * NPARAM);
    double loss = 0.0;
    double h1[H1], h2[H2], lg[NCLS], d3[NCLS], d2[H2], d1[H1];
    for (int32_t s = 0; s < m; ++s) {
        const double *x = xin + (size_t)s * ORC_NFEAT;
        mlp_fwd_one(w, x, h1, h2, lg);
        double mx = lg[0];
        for (int c = 1; c < NCLS; ++c) if (lg[c] > mx) mx = lg[c];
        double z = 0.0;
        for (int c = 0; c < NCLS; ++c) z += exp(lg[c] - mx);
        loss += -(lg[label[s]] - mx - log(z));
        for (int c = 0; c < NCLS; ++c) d3[c] = (exp(lg[c] - mx) / z - (c == label[s] ? 1.0 : 0.0)) / m;
        for (int c = 0; c < NCLS; ++c) {
            gb3[c] += d3[c];
            for (int i = 0; i < H2; ++i) gW3[c * H2 + i] += d3[c] * h2[i];
        }
        for (int i = 0; i < H2; ++i) {
            double sacc = 0.0;
            for (int c = 0; c < NCLS; ++c) sacc += W3[c * H2 + i] * d3[c];
            d2[i] = h2[i] > 0.0 ? sacc : 0.0;
        }
        for (int o = 0; o < H2; ++o) {
            gb2[o] += d2[o];
            for (int i = 0; i < H1; ++i) gW2[o * H1 + i] += d2[o] * h1[i];
        }
        for (int i = 0; i < H1; ++i) {
            double sacc = 0.0;
            for (int o = 0; o < H2; ++o) sacc += W2[o * H1 + i] * d2[o];
            d1[i] = h1[i] > 0.0 ? sacc : 0.0;
        }
        for (int o = 0; o < H1; ++o) {
            gb1[o] += d1[o];
            for (int i = 0; i < ORC_NFEAT; ++i) gW1[o * ORC_NFEAT + i] += d1[o] * x[i];
        }
    }
    return loss / m;
}

/* ====================================================================================== */
/* BJAC(k, t), Eq. 3-2 and Eq. 3-3. A_bd is the block-diagonal part of A (entries whose     */
/* row and column lie in the same block of block_ptr), D = diag(A):                        */
/*   D-hat^-1 w = sum_{i<t} (I - D^-1 A_bd)^i D^-1 w     (t Jacobi sweeps inside the blocks) */
/*   M-hat^-1 r = sum_{j<k} (I - D-hat^-1 A)^j D-hat^-1 r (k block-Jacobi sweeps)            */
/* Both sums are what the stationary iterations produce from a zero start, so they are      */
/* evaluated as                                                                            */
/*   z = 0; for j < k: { w = r - A z; y = 0; for i < t: y = y + D^-1 (w - A_bd y); z += y }  */
/* with, for every row, the product sum as one FMA chain in CSR order starting from 0, then  */
/* the difference, then y_i + dinv_i * u_i as one FMA.                                     */
/* prec 0: binary64 throughout. prec 1: Algorithm 3.1 with p_l = binary32: r-hat = RN32(r),   */
/* the values of A and dinv_i = RN32(1 / a_ii) (the reciprocal formed in binary64) stored in */
/* binary32, every operation in binary32, z widened exactly.                               */
/* ====================================================================================== */
static int32_t block_of_row(int32_t nb, const int32_t *block_ptr, int32_t i) {
    int32_t b = 0;
    while (b + 1 < nb && block_ptr[b + 1] <= i) ++b;
    return b;
}

/* dinv (binary64) from the diagonal; returns the first row without a positive diagonal, or -1 */
int32_t orc_kt_dinv(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, double *dinv) {
    for (int32_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (colidx[k] == i) d += val[k];
        if (!(d > 0.0)) return i;
        dinv[i] = 1.0 / d;
    }
    return -1;
}

static void kt_apply64(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, int32_t nb,
                       const int32_t *block_ptr, const int32_t *rblk, int32_t k, int32_t t, const double *dinv,
                       const double *r, double *z, double *w, double *y, double *y2) {
    for (int32_t i = 0; i < n; ++i) z[i] = 0.0;
    for (int32_t j = 0; j < k; ++j) {
        for (int32_t i = 0; i < n; ++i) {                      /* w = r - A z */
            double sum = 0.0;
            for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) sum = fma(val[e], z[colidx[e]], sum);
            w[i] = r[i] - sum;
        }
        for (int32_t i = 0; i < n; ++i) y[i] = 0.0;
        for (int32_t s = 0; s < t; ++s) {                      /* y = y + D^-1 (w - A_bd y) */
            for (int32_t i = 0; i < n; ++i) {
                const int32_t b = rblk[i];
                double sum = 0.0;
                for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    const int32_t c = colidx[e];
                    if (c >= block_ptr[b] && c < block_ptr[b + 1]) sum = fma(val[e], y[c], sum);
                }
                const double u = w[i] - sum;
                y2[i] = fma(dinv[i], u, y[i]);
            }
            for (int32_t i = 0; i < n; ++i) y[i] = y2[i];
        }
        for (int32_t i = 0; i < n; ++i) z[i] = z[i] + y[i];
    }
    (void)nb;
}

static void kt_apply32(int32_t n, const int32_t *rowptr, const int32_t *colidx, const float *val32, int32_t nb,
                       const int32_t *block_ptr, const int32_t *rblk, int32_t k, int32_t t, const float *dinv32,
                       const double *r, double *z, float *rh, float *zf, float *w, float *y, float *y2) {
    for (int32_t i = 0; i < n; ++i) rh[i] = as_float(orc_round_f32_bits(r[i]));
    for (int32_t i = 0; i < n; ++i) zf[i] = 0.0f;
    for (int32_t j = 0; j < k; ++j) {
        for (int32_t i = 0; i < n; ++i) {
            float sum = 0.0f;
            for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) sum = fmaf(val32[e], zf[colidx[e]], sum);
            w[i] = rh[i] - sum;
        }
        for (int32_t i = 0; i < n; ++i) y[i] = 0.0f;
        for (int32_t s = 0; s < t; ++s) {
            for (int32_t i = 0; i < n; ++i) {
                const int32_t b = rblk[i];
                float sum = 0.0f;
                for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    const int32_t c = colidx[e];
                    if (c >= block_ptr[b] && c < block_ptr[b + 1]) sum = fmaf(val32[e], y[c], sum);
                }
                const float u = w[i] - sum;
                y2[i] = fmaf(dinv32[i], u, y[i]);
            }
            for (int32_t i = 0; i < n; ++i) y[i] = y2[i];
        }
        for (int32_t i = 0; i < n; ++i) zf[i] = zf[i] + y[i];
    }
    for (int32_t i = 0; i < n; ++i) z[i] = (double)zf[i];
    (void)nb;
}

typedef struct {
    int32_t n, nb, k, t;
    const int32_t *rowptr, *colidx, *block_ptr;
    const double *val;
    int32_t *rblk;
    double *dinv, *w, *y, *y2;
    float *val32, *dinv32, *rh, *zf, *wf, *yf, *y2f;
} kt_state;

static int kt_init(kt_state *K, int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                   int32_t nb, const int32_t *block_ptr, int32_t k, int32_t t) {
    memset(K, 0, sizeof(*K));
    K->n = n; K->nb = nb; K->k = k; K->t = t;
    K->rowptr = rowptr; K->colidx = colidx; K->block_ptr = block_ptr; K->val = val;
    const int32_t nnz = rowptr[n];
    K->rblk = malloc(sizeof(int32_t) * (size_t)n);
    K->dinv = malloc(sizeof(double) * (size_t)n);
    K->w = malloc(sizeof(double) * (size_t)n);
    K->y = malloc(sizeof(double) * (size_t)n);
    K->y2 = malloc(sizeof(double) * (size_t)n);
    K->val32 = malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    K->dinv32 = malloc(sizeof(float) * (size_t)n);
    K->rh = malloc(sizeof(float) * (size_t)n);
    K->zf = malloc(sizeof(float) * (size_t)n);
    K->wf = malloc(sizeof(float) * (size_t)n);
    K->yf = malloc(sizeof(float) * (size_t)n);
    K->y2f = malloc(sizeof(float) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) K->rblk[i] = block_of_row(nb, block_ptr, i);
    if (orc_kt_dinv(n, rowptr, colidx, val, K->dinv) >= 0) return -1;
    for (int32_t i = 0; i < n; ++i) K->dinv32[i] = as_float(orc_round_f32_bits(K->dinv[i]));
    for (int32_t e = 0; e < nnz; ++e) K->val32[e] = as_float(orc_round_f32_bits(val[e]));
    return 0;
}

static void kt_free(kt_state *K) {
    void *ptrs[] = {K->rblk, K->dinv, K->w, K->y, K->y2, K->val32, K->dinv32, K->rh, K->zf, K->wf, K->yf, K->y2f};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
}

static void kt_apply(const kt_state *K, int32_t prec, const double *r, double *z) {
    if (prec == 0)
        kt_apply64(K->n, K->rowptr, K->colidx, K->val, K->nb, K->block_ptr, K->rblk, K->k, K->t, K->dinv, r, z,
                   K->w, K->y, K->y2);
    else
        kt_apply32(K->n, K->rowptr, K->colidx, K->val32, K->nb, K->block_ptr, K->rblk, K->k, K->t, K->dinv32, r, z,
                   K->rh, K->zf, K->wf, K->yf, K->y2f);
}

/* z = M-hat^-1 r; returns -1 if a diagonal entry is not positive */
int32_t orc_kt_apply(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, int32_t nb,
                     const int32_t *block_ptr, int32_t k, int32_t t, int32_t prec, const double *r, double *z) {
    kt_state K;
    if (kt_init(&K, n, rowptr, colidx, val, nb, block_ptr, k, t)) { kt_free(&K); return -1; }
    kt_apply(&K, prec, r, z);
    kt_free(&K);
    return 0;
}

/* PCG as orc_pcg with M-hat^-1 of BJAC(k, t): policy 0 binary64, 1 fMP (binary32), 2 hl, 3 lh */
int32_t orc_pcg_kt(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val, int32_t nb,
                   const int32_t *block_ptr, int32_t kk, int32_t tt, int32_t policy, double adp_tol,
                   int32_t flexible, const double *b, double *x, double tol, int32_t maxit, double *hist,
                   uint8_t *low_used, orc_stats *st) {
    memset(st, 0, sizeof(*st));
    kt_state K;
    if (kt_init(&K, n, rowptr, colidx, val, nb, block_ptr, kk, tt)) {
        kt_free(&K);
        st->status = ORC_BREAKDOWN;
        return ORC_BREAKDOWN;
    }
    precond P = {nb, block_ptr, NULL, NULL, NULL, NULL, NULL, NULL, policy, adp_tol, 1};
    double *r = malloc(sizeof(double) * (size_t)n);
    double *z = malloc(sizeof(double) * (size_t)n);
    double *p = malloc(sizeof(double) * (size_t)n);
    double *q = malloc(sizeof(double) * (size_t)n);
    double *rp = malloc(sizeof(double) * (size_t)n);
    double bnorm = sqrt(orc_dot(n, b, b));
    int32_t k = 0, status = ORC_OK;
#define KT_PRECONDITION(rel, flag)                                  \
    do {                                                            \
        const int lo_ = use_low(&P, (rel));                         \
        kt_apply(&K, lo_, r, z);                                    \
        if (lo_) st->low_applies++; else st->high_applies++;        \
        if (flag) *(flag) = (uint8_t)lo_;                           \
    } while (0)
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
        st->converged = 1; st->relres = 0.0; st->true_relres = 0.0;
        goto done;
    }
    orc_residual(n, rowptr, colidx, val, b, x, r);
    double relres = sqrt(orc_dot(n, r, r)) / bnorm;
    st->true_relres = relres;
    if (hist) hist[0] = relres;
    for (;;) {
        if (relres <= tol) break;
        KT_PRECONDITION(relres, low_used ? &low_used[k] : NULL);
        double rho = orc_dot(n, r, z);
        if (!(rho > 0.0) || !isfinite(rho)) { status = ORC_BREAKDOWN; break; }
        for (int32_t i = 0; i < n; ++i) p[i] = z[i];
        while (k < maxit) {
            orc_spmv(n, rowptr, colidx, val, p, q);
            double sigma = orc_dot(n, p, q);
            if (!(sigma > 0.0) || !isfinite(sigma)) { status = ORC_BREAKDOWN; break; }
            double alpha = rho / sigma;
            for (int32_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
            for (int32_t i = 0; i < n; ++i) rp[i] = r[i];
            for (int32_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
            ++k;
            relres = sqrt(orc_dot(n, r, r)) / bnorm;
            if (hist) hist[k] = relres;
            if (!isfinite(relres)) { status = ORC_BREAKDOWN; break; }
            if (relres <= tol) break;
            if (k >= maxit) break;
            KT_PRECONDITION(relres, low_used ? &low_used[k] : NULL);
            double rho_new = orc_dot(n, r, z);
            if (!(rho_new > 0.0) || !isfinite(rho_new)) { status = ORC_BREAKDOWN; break; }
            double beta = flexible ? flexible_beta(n, z, r, rp, rho) : rho_new / rho;
            if (!isfinite(beta)) { status = ORC_BREAKDOWN; break; }
            for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
            rho = rho_new;
        }
        if (status != ORC_OK) break;
        orc_residual(n, rowptr, colidx, val, b, x, r);
        double tr = sqrt(orc_dot(n, r, r)) / bnorm;
        st->true_relres = tr;
        if (tr <= tol || k >= maxit || st->restarts >= 8) break;
        st->restarts++;
        relres = tr;
    }
    st->relres = relres;
    st->converged = (status == ORC_OK && relres <= tol && st->true_relres <= tol) ? 1 : 0;
    if (status == ORC_OK && !st->converged) status = ORC_NOT_CONVERGED;
#undef KT_PRECONDITION
done:
    st->iters = k;
    st->status = status;
    free(r); free(z); free(p); free(q); free(rp);
    kt_free(&K);
    return status;
}
