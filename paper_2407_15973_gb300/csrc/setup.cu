// Preconditioner setup: for every diagonal block B_b = A[rows_b, rows_b] (Eq. 3-1, exact
// block inverses, the special case named after Eq. 3-3)
//   1. extract B_b from the CSR rows into shared memory (binary64), with per-row statistics
//      for the block features (multiscale strength of Eq. 4-5, diagonal dominance of
//      Section 4.5.2, off-block coupling);
//   2. invert it in place with the symmetric Gauss-Jordan sweep: pivot k maps
//        a_ij <- a_ij - a_ik a_kj / a_kk  (i, j != k),  a_ik <- a_ik / a_kk,  a_kk <- -1 / a_kk,
//      and after all pivots the array holds -B^-1. Only the upper triangle is updated
//      (bs^3 / 2 FMAs), which also makes G = B^-1 exactly symmetric. A pivot <= 0 means B
//      is not positive definite and is reported;
//   3. kappa_1(B) = ||B||_1 ||G||_1, the dynamic range of G, and the format choice;
//   4. ConvertPrecision of the inverse (Algorithm 3.1's M^-1(p_l)): Q = RN_f(G / s_b) with
//      s_b = 2^(floor(log2 max|G|) - 14) for the 16-bit formats (s_b = 1 otherwise).
// One CTA of 128 threads per block; the block (<= 128 x 128 doubles) lives in shared memory.
#include "common.cuh"
#include "setup.cuh"

#include <cfloat>

namespace mpbjac {

constexpr int kSetupNT = 128;
constexpr double kDomCap = 1.0e6;

__device__ __forceinline__ double bmax(double v, double *sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = sm[0];
#pragma unroll
    for (int i = 1; i < kSetupNT / 32; ++i) t = fmax(t, sm[i]);
    return t;
}
__device__ __forceinline__ double bmin(double v, double *sm) { return -bmax(-v, sm); }

// Round v (already divided by the block's scale) to format f and store entry idx.
__device__ __forceinline__ void store_fmt(uint8_t *out, int f, int idx, double v) {
    if (f == BJAC_FP64) reinterpret_cast<double *>(out)[idx] = v;
    else if (f == BJAC_FP32) reinterpret_cast<float *>(out)[idx] = __double2float_rn(v);
    else if (f == BJAC_BF16) reinterpret_cast<__nv_bfloat16 *>(out)[idx] = __double2bfloat16(v);
    else reinterpret_cast<__half *>(out)[idx] = __double2half(v);
}

// Condition-number rule: cheapest format whose unit roundoff u satisfies kappa_1 u <= theta;
// binary16 needs the block's dynamic range within 2^29, else bfloat16 is the 16-bit choice.
__device__ __forceinline__ int rule_format(double lk, double ldr, double theta) {
    const double l2 = 0.30102999566398120;  // log10(2)
    const double lt = log10(theta);
    if (ldr <= 29 * l2 && lk - 11 * l2 <= lt) return BJAC_FP16S;
    if (lk - 8 * l2 <= lt) return BJAC_BF16;
    if (lk - 24 * l2 <= lt) return BJAC_FP32;
    return BJAC_FP64;
}

__device__ __forceinline__ int scale_exp(double gmax) {
    return (gmax > 0.0 && gmax < DBL_MAX) ? ilogb(gmax) - 14 : 0;
}

__global__ void __launch_bounds__(kSetupNT) k_setup_blocks(SetupArgs a, int bs_max) {
    extern __shared__ __align__(16) double dsm[];
    double *sA = dsm;                                     // bs x bs (upper triangle used)
    double *sc = sA + bs_max * bs_max;                    // pivot column
    double *st = sc + bs_max;                             // pivot column / pivot
    uint16_t *tri = reinterpret_cast<uint16_t *>(st + bs_max);   // (i << 8 | j), i <= j
    __shared__ double red[kSetupNT / 32];

    const int b = blockIdx.x;
    const int s = a.block_ptr[b], e = a.block_ptr[b + 1], bs = e - s;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < bs * bs; idx += kSetupNT) sA[idx] = 0.0;
    // upper-triangle index table: row i occupies [i*bs - i(i-1)/2, +bs-i)
    for (int i = tid; i < bs; i += kSetupNT) {
        const int o = i * bs - (i * (i - 1)) / 2;
        for (int j = i; j < bs; ++j) tri[o + (j - i)] = (uint16_t)((i << 8) | j);
    }
    __syncthreads();

    // 1. extraction and per-row statistics (one thread per row; bs <= 128)
    double r_fro = 0.0, r_dmin = DBL_MAX, r_dsum = 0.0, r_amin = DBL_MAX, r_amax = 0.0;
    double r_out = 0.0, r_all = 0.0, r_tmax = 0.0, r_tsum = 0.0, r_ndom = 0.0, r_exc = 0.0;
    if (tid < bs) {
        const int i = s + tid;
        double diag = 0.0, off = 0.0, mx = 0.0, mn = DBL_MAX;
        for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
            const int j = a.colidx[k];
            const double v = a.val[k], av = fabs(v);
            r_all += av;
            if (j >= s && j < e) {
                sA[tid * bs + (j - s)] += v;
                r_fro = fma(v, v, r_fro);
            } else {
                r_out += av;
            }
            if (j == i) diag += av;
            else {
                off += av;
                if (v != 0.0) { mx = fmax(mx, av); mn = fmin(mn, av); }
            }
        }
        double d = off > 0.0 ? diag / off : kDomCap;
        if (d > kDomCap) d = kDomCap;
        r_dmin = d; r_dsum = d; r_amin = diag; r_amax = diag;
        r_ndom = diag > off ? 1.0 : 0.0;
        r_exc = diag > 0.0 ? (diag - off) / diag : 0.0;
        const double lt = log10(mx > 0.0 ? mx / mn : 1.0);
        r_tmax = lt; r_tsum = lt;
    }
    __syncthreads();
    // ||B||_1 (max column sum of |B|)
    double colsum = 0.0;
    if (tid < bs)
        for (int i = 0; i < bs; ++i) colsum += fabs(sA[i * bs + tid]);
    const double nB1 = bmax(colsum, red);

    // 2. symmetric Gauss-Jordan sweep over the upper triangle
    const int T = bs * (bs + 1) / 2;
    bool spd = true;
    for (int k = 0; k < bs; ++k) {
        const double d = sA[k * bs + k];
        if (!(d > 0.0)) { spd = false; break; }          // same value in every thread
        const double inv = 1.0 / d;
        if (tid < bs) {
            const double c = tid <= k ? sA[tid * bs + k] : sA[k * bs + tid];
            sc[tid] = c;
            st[tid] = c * inv;
        }
        __syncthreads();
        for (int t = tid; t < T; t += kSetupNT) {
            const int ij = tri[t];
            const int i = ij >> 8, j = ij & 255;
            if (i != k && j != k) sA[i * bs + j] = fma(-sc[i], st[j], sA[i * bs + j]);
        }
        if (tid < bs) {
            if (tid < k) sA[tid * bs + k] = st[tid];
            else if (tid > k) sA[k * bs + tid] = st[tid];
            else sA[k * bs + k] = -inv;
        }
        __syncthreads();
    }
    if (!spd) {
        if (tid == 0) {
            if (atomicCAS(a.status, 0, MPBJAC_ERR_NOT_SPD) == 0) a.status[1] = b;
            a.fmt[b] = BJAC_FP64;
            a.scale[b] = 1.0f;
        }
        return;
    }
    // G = -A (upper triangle mirrored)
    if (a.G) {
        double *Gb = a.G + a.goff[b];
        for (int idx = tid; idx < bs * bs; idx += kSetupNT) {
            const int i = idx / bs, j = idx - i * bs;
            Gb[idx] = -(i <= j ? sA[i * bs + j] : sA[j * bs + i]);
        }
    }
    // 3. ||G||_1, max |G|, min nonzero |G|
    double gcol = 0.0, gmx = 0.0, gmn = DBL_MAX;
    if (tid < bs) {
        for (int i = 0; i < bs; ++i) {
            const double v = fabs(i <= tid ? sA[i * bs + tid] : sA[tid * bs + i]);
            gcol += v;
            gmx = fmax(gmx, v);
            if (v > 0.0) gmn = fmin(gmn, v);
        }
    }
    const double nG1 = bmax(gcol, red);
    const double gmax = bmax(gmx, red);
    const double gmin = bmin(gmn, red);
    const double lk = log10(nB1 * nG1);
    const double ldr = gmax > 0.0 ? log10(gmax / gmin) : 0.0;
    if (a.feat) {
        const double fro = block_sum<kSetupNT>(r_fro, red);
        const double dmin = bmin(r_dmin, red);
        const double dsum = block_sum<kSetupNT>(r_dsum, red);
        const double amin = bmin(r_amin, red);
        const double amax = bmax(r_amax, red);
        const double osum = block_sum<kSetupNT>(r_out, red);
        const double asum = block_sum<kSetupNT>(r_all, red);
        const double tmax = bmax(r_tmax, red);
        const double tsum = block_sum<kSetupNT>(r_tsum, red);
        const double ndom = block_sum<kSetupNT>(r_ndom, red);
        const double exc = block_sum<kSetupNT>(r_exc, red);
        if (tid == 0) {
            double *f = a.feat + (size_t)b * 12;
            f[0] = lk;
            f[1] = 0.5 * log10(fro);
            f[2] = dmin;
            f[3] = dsum / bs;
            f[4] = amax > 0.0 ? amin / amax : 0.0;
            f[5] = asum > 0.0 ? osum / asum : 0.0;
            f[6] = tmax;
            f[7] = tsum / bs;
            f[8] = ldr;
            f[9] = bs / 128.0;
            f[10] = ndom / bs;
            f[11] = exc / bs;
        }
    }
    int f;
    if (a.select == BJAC_SELECT_UNIFORM) f = BJAC_FP64;
    else if (a.select == BJAC_SELECT_FIXED) f = a.fixed_fmt;
    else if (a.select == BJAC_SELECT_RULE) f = rule_format(lk, ldr, a.theta);
    else if (a.select == BJAC_SELECT_GIVEN) f = a.given[b];
    else f = BJAC_FP64;   // the learned selector decides in a later pass
    const int ex = (f == BJAC_BF16 || f == BJAC_FP16S) ? scale_exp(gmax) : 0;
    if (tid == 0) {
        a.kap[2 * b] = lk;
        a.kap[2 * b + 1] = ldr;
        a.fmt[b] = (uint8_t)f;
        a.scale[b] = (float)ldexp(1.0, ex);
    }
    // 4. round into the pool now when the offsets are already known
    if (a.pool) {
        uint8_t *out = a.pool + a.qoff[b];
        for (int idx = tid; idx < bs * bs; idx += kSetupNT) {
            const int i = idx / bs, j = idx - i * bs;
            const double g = -(i <= j ? sA[i * bs + j] : sA[j * bs + i]);
            store_fmt(out, f, idx, ldexp(g, -ex));
        }
    }
}

// Second pass: round every block of G to fmt[b] into the pool (scale from max |G_b|).
__global__ void __launch_bounds__(kSetupNT) k_pack(const int32_t *block_ptr, const int64_t *goff,
                                                   const double *G, const uint8_t *fmt, const int64_t *qoff,
                                                   uint8_t *pool, float *scale) {
    __shared__ double red[kSetupNT / 32];
    const int b = blockIdx.x;
    const int bs = block_ptr[b + 1] - block_ptr[b];
    const double *Gb = G + goff[b];
    double mx = 0.0;
    for (int idx = threadIdx.x; idx < bs * bs; idx += kSetupNT) mx = fmax(mx, fabs(Gb[idx]));
    const double gmax = bmax(mx, red);
    const int f = fmt[b];
    const int ex = (f == BJAC_BF16 || f == BJAC_FP16S) ? scale_exp(gmax) : 0;
    if (threadIdx.x == 0) scale[b] = (float)ldexp(1.0, ex);
    uint8_t *out = pool + qoff[b];
    for (int idx = threadIdx.x; idx < bs * bs; idx += kSetupNT) store_fmt(out, f, idx, ldexp(Gb[idx], -ex));
}

// Host launchers ---------------------------------------------------------------------------
size_t setup_smem_bytes(int bs_max) {
    const int T = bs_max * (bs_max + 1) / 2;
    return (size_t)bs_max * bs_max * 8 + 2 * (size_t)bs_max * 8 + (size_t)T * 2 + 16;
}

int launch_setup_blocks(const SetupArgs &a, int bs_max, cudaStream_t st) {
    const size_t smem = setup_smem_bytes(bs_max);
    MPB_CUDA(cudaFuncSetAttribute(k_setup_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_setup_blocks<<<a.nb, kSetupNT, smem, st>>>(a, bs_max);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

int launch_pack(int nb, const int32_t *block_ptr, const int64_t *goff, const double *G, const uint8_t *fmt,
                const int64_t *qoff, uint8_t *pool, float *scale, cudaStream_t st) {
    k_pack<<<nb, kSetupNT, 0, st>>>(block_ptr, goff, G, fmt, qoff, pool, scale);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

}  // namespace mpbjac
