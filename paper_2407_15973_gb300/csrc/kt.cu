// BJAC(k, t): the inexact block Jacobi of Eq. 3-2 / 3-3, the form the paper's experiments use
// (Section 4.2: 32 blocks, k = t = 2). A_bd is the block-diagonal part of A (entries whose row
// and column lie in the same block), D = diag(A). The two sums
//   D-hat^-1 w = sum_{i<t} (I - D^-1 A_bd)^i D^-1 w,    M-hat^-1 r = sum_{j<k} (I - D-hat^-1 A)^j D-hat^-1 r
// are what the stationary iterations produce from a zero start, so the apply runs
//   z = 0; for j < k: { w = r - A z; y = 0; for i < t: y = y + D^-1 (w - A_bd y); z = z + y }
// with every row's product sum one FMA chain in CSR order from 0, then the difference, then
// y_i + dinv_i u_i as one FMA; in binary64, or in binary32 for the low set (Algorithm 3.1:
// r-hat = RN32(r), A and dinv = RN32(1 / a_ii) stored in binary32, z widened exactly). The
// zero starts are taken as such (w = r-hat for j = 0, y = RN(dinv * w) for i = 0), which is
// bitwise what the general formulas give.
//
// One launch per sweep: the first sweep of an outer step also forms w (with one SpMV of A on
// z when j > 0), the others run one SpMV of A_bd on y. Every launch walks the SELL-32 copy of
// A (slices of 32 rows, column-major, one warp per slice); out-of-block entries are skipped
// by comparing the column with the row's block bounds. The last sweep widens z into the PCG
// vector and reduces r.z like the other apply kernels.
#include "apply.cuh"
#include "common.cuh"
#include "kt.cuh"
#include "spmv.cuh"

namespace mpbjac {

struct KtArgs {
    int n, nslices, nb;
    const int32_t *off, *col;
    const void *val;          // T[entries]
    const void *dinv;         // T[n]
    const int32_t *rblk, *block_ptr;
    const double *r;          // PCG residual (binary64)
    void *w;                  // T[n]
    const void *yin;          // T[n]
    void *yout;               // T[n]
    const void *zin;          // T[n], z of the apply after the previous outer step
    void *zout;               // T[n], z after this outer step (a different buffer)
    int prec, from_state;
    int outer;                // 1: this sweep forms w = r-hat - A z first (j > 0)
    int first;                // 1: this sweep is the first inner sweep (y = 0 before it)
    int acc;                  // 1: last inner sweep of an outer step: z = z + y
    int zero_z;               // 1: z is zero before this accumulation (j = 0)
    int final_;               // 1: last sweep of the apply: widen z, r.z
    ApplyIO io;
};

template <typename T> __device__ __forceinline__ T fma_t(T a, T b, T c);
template <> __device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> __device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <typename T> __device__ __forceinline__ T rhat(double r);
template <> __device__ __forceinline__ float rhat<float>(double r) { return f64_to_f32_rn(r); }
template <> __device__ __forceinline__ double rhat<double>(double r) { return r; }
template <typename T> __device__ __forceinline__ double widen(T v);
template <> __device__ __forceinline__ double widen<float>(float v) { return f32_to_f64(v); }
template <> __device__ __forceinline__ double widen<double>(double v) { return v; }

// U entries of this lane's row: loads, gathers, then the chain over the included entries
template <typename T, bool BD, int U>
__device__ __forceinline__ void kt_part(const T *__restrict__ pv, const int32_t *__restrict__ pc,
                                        const T *__restrict__ x, int blo, int bhi, T &acc) {
    T v[U], xv[U];
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        v[u] = pv[32 * u];
        c[u] = __ldcs(pc + 32 * u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const bool in = c[u] >= 0 && (!BD || (c[u] >= blo && c[u] < bhi));
        c[u] = in ? c[u] : -1;
        xv[u] = in ? __ldg(x + c[u]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (c[u] >= 0) acc = fma_t<T>(v[u], xv[u], acc);
}

template <typename T, bool BD>
__device__ __forceinline__ T kt_row_sum(const T *pv, const int32_t *pc, int len, const T *x, int blo, int bhi) {
    T acc = T(0);
    int j = 0;
    for (; j + 8 <= len; j += 8) kt_part<T, BD, 8>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc);
    switch (len - j) {
        case 1: kt_part<T, BD, 1>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc); break;
        case 2: kt_part<T, BD, 2>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc); break;
        case 3: kt_part<T, BD, 3>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc); break;
        case 4: kt_part<T, BD, 4>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc); break;
        case 5: kt_part<T, BD, 5>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc); break;
        case 6: kt_part<T, BD, 6>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc); break;
        case 7: kt_part<T, BD, 7>(pv + 32 * j, pc + 32 * j, x, blo, bhi, acc); break;
        default: break;
    }
    return acc;
}

constexpr int kKtSmemBlocks = 1024;      // block offsets kept in shared memory up to this many blocks

template <typename T, int MODE>
__global__ void __launch_bounds__(kSpNT) k_kt_sweep(KtArgs a, SolverState *S) {
    pdl_enter();
    constexpr int NW = kSpNT / 32;
    __shared__ double red[NW];
    __shared__ int32_t s_bp[kKtSmemBlocks + 1];
    const bool bp_smem = a.nb <= kKtSmemBlocks;
    if (!a.first && bp_smem) {
        for (int i = threadIdx.x; i <= a.nb; i += kSpNT) s_bp[i] = a.block_ptr[i];
        __syncthreads();
    }
    if (MODE != kApplyStandalone) {
        if (S->state != kRunning) return;
        if (a.from_state && S->use_low != a.prec) return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NW + warp, nw = gridDim.x * NW;
    const T *val = static_cast<const T *>(a.val);
    const T *dinv = static_cast<const T *>(a.dinv);
    T *w = static_cast<T *>(a.w);
    const T *yin = static_cast<const T *>(a.yin);
    T *yout = static_cast<T *>(a.yout);
    const T *zin = static_cast<const T *>(a.zin);
    T *zout = static_cast<T *>(a.zout);
    double rho = 0.0;
    for (int s = gw; s < a.nslices; s += nw) {
        const int row = (s << 5) + lane;
        const int o0 = __ldg(a.off + s);
        const int len = (__ldg(a.off + s + 1) - o0) >> 5;
        const T *pv = val + o0 + lane;
        const int32_t *pc = a.col + o0 + lane;
        T wi = T(0), yi = T(0);
        if (a.first) {
            // w = r-hat (j = 0) or r-hat - A z; then y = RN(dinv w) = y + dinv (w - A_bd y) at y = 0
            T sum = T(0);
            if (a.outer) sum = kt_row_sum<T, false>(pv, pc, len, zin, 0, 0);
            if (row < a.n) {
                wi = rhat<T>(a.r[row]) - sum;
                w[row] = wi;
                yi = fma_t<T>(dinv[row], wi - T(0), T(0));
            }
        } else {
            int blo = 0, bhi = 0;
            if (row < a.n) {
                if (bp_smem) {
                    // the row's block by bisection of the offsets in shared memory
                    int lo = 0, hi = a.nb;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s_bp[mid] <= row) lo = mid;
                        else hi = mid;
                    }
                    blo = s_bp[lo];
                    bhi = s_bp[lo + 1];
                } else {
                    const int b = a.rblk[row];
                    blo = __ldg(a.block_ptr + b);
                    bhi = __ldg(a.block_ptr + b + 1);
                }
            }
            const T sum = kt_row_sum<T, true>(pv, pc, len, yin, blo, bhi);
            if (row < a.n) yi = fma_t<T>(dinv[row], w[row] - sum, yin[row]);
        }
        if (row >= a.n) continue;
        yout[row] = yi;
        if (a.acc) {
            const T zi = (a.zero_z ? T(0) : zin[row]) + yi;
            if (!a.final_) {
                zout[row] = zi;
            } else {
                const double zd = widen<T>(zi);
                a.io.z[row] = zd;
                if (MODE == kApplyInit) a.io.p[row] = zd;
                rho = fma(a.r[row], zd, rho);
            }
        }
    }
    if (!a.final_) return;
    if (MODE == kApplyStandalone && a.io.out == nullptr) return;
    const double b1 = block_sum<kSpNT>(rho, red);
    if (threadIdx.x == 0) a.io.part[2 * blockIdx.x] = b1;
    if (!last_cta(a.io.ticket)) return;
    const double t1 = reduce_partials<kSpNT>(a.io.part, gridDim.x, 2, red);
    if (threadIdx.x == 0) apply_finish<MODE>(t1, 0.0, a.io, S, a.prec);
}

// ----------------------------------------------------------------------------------------
// setup
// ----------------------------------------------------------------------------------------
__global__ void k_kt_rows(int n, int nb, const int32_t *__restrict__ block_ptr, const int32_t *__restrict__ rowptr,
                          const int32_t *__restrict__ colidx, const double *__restrict__ val, int32_t *rblk,
                          double *dinv64, float *dinv32, int *bad) {
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        for (int i = block_ptr[b] + threadIdx.x; i < block_ptr[b + 1]; i += blockDim.x) {
            rblk[i] = b;
            double d = 0.0;
            for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (colidx[k] == i) d += val[k];
            if (!(d > 0.0)) {
                atomicMin(bad, i);
                d = 1.0;
            }
            const double inv = 1.0 / d;
            dinv64[i] = inv;
            if (dinv32) dinv32[i] = f64_to_f32_rn(inv);
        }
    }
}

__global__ void k_kt_round(long long count, const double *__restrict__ v, float *__restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = f64_to_f32_rn(v[e]);
}

void kt_free(KtSet *K) {
    void *ptrs[] = {K->rblk, K->dinv64, K->dinv32, K->val32, K->w, K->y0, K->y1, K->zt, K->zt2};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    sell_free(&K->sell);
    *K = KtSet{};
}

int kt_build(const bjac_csr &A, const int32_t *d_block_ptr, int nb, int k, int t, bool lo, KtSet *out,
             int *bad_row, cudaStream_t st) {
    kt_free(out);
    KtSet K;
    K.n = A.n;
    K.nb = nb;
    K.k = k;
    K.t = t;
    K.block_ptr = d_block_ptr;
    *bad_row = -1;
    auto fail_free = [&](int rc) {
        kt_free(&K);
        return rc;
    };
    const size_t n = (size_t)A.n;
    int *bad = nullptr;
    cudaError_t e = cudaMalloc(&K.rblk, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&K.dinv64, sizeof(double) * n);
    if (e == cudaSuccess && lo) e = cudaMalloc(&K.dinv32, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&K.w, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&K.y0, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&K.y1, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&K.zt, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&K.zt2, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
    if (e != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc (BJAC(k,t))"));
    const int init = INT32_MAX;
    e = cudaMemcpyAsync(bad, &init, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_kt_rows<<<std::min(nb, sm_count() * 8), 256, 0, st>>>(A.n, nb, d_block_ptr, A.rowptr, A.colidx, A.val,
                                                                 K.rblk, K.dinv64, K.dinv32, bad);
        e = cudaGetLastError();
    }
    int hbad = INT32_MAX;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(bad);
    if (e != cudaSuccess) return fail_free(cuda_fail(e, "BJAC(k,t) diagonal"));
    if (hbad != INT32_MAX) {
        *bad_row = hbad;
        return fail_free(fail(MPBJAC_ERR_NOT_SPD, "row " + std::to_string(hbad) + " has no positive diagonal entry"));
    }
    int rc = sell_build(A, 0.0, &K.sell, st);
    if (rc) return fail_free(rc);
    if (!K.sell.val) return fail_free(fail(MPBJAC_ERR_UNSUPPORTED, "A needs more than 2^31 stored SELL-32 entries"));
    if (lo) {
        e = cudaMalloc(&K.val32, sizeof(float) * (size_t)std::max(1ll, K.sell.entries));
        if (e != cudaSuccess) return fail_free(cuda_fail(e, "cudaMalloc (binary32 values)"));
        k_kt_round<<<sm_count() * 8, 256, 0, st>>>(K.sell.entries, K.sell.val, K.val32);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail_free(cuda_fail(e, "k_kt_round"));
    }
    *out = K;
    return MPBJAC_OK;
}

// ----------------------------------------------------------------------------------------
// apply
// ----------------------------------------------------------------------------------------
template <typename T, int MODE>
static int launch_sweep(const KtArgs &a, SolverState *S, cudaStream_t st) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_kt_sweep<T, MODE>, kSpNT, 0) != cudaSuccess || v < 1)
            v = 1;
        per_sm = v;
    }
    int g = sm_count() * per_sm;
    if (g > kMaxGrid) g = kMaxGrid;
    const int need = (a.nslices + kSpNT / 32 - 1) / (kSpNT / 32);
    if (g > need) g = need;
    if (g < 1) g = 1;
    MPB_CUDA(launch_kernel(k_kt_sweep<T, MODE>, g, kSpNT, 0, st, a, S));
    return MPBJAC_OK;
}

template <typename T>
static int launch_sweep_mode(int mode, const KtArgs &a, SolverState *S, cudaStream_t st) {
    switch (mode) {
        case kApplyStandalone: return launch_sweep<T, kApplyStandalone>(a, S, st);
        case kApplyInit: return launch_sweep<T, kApplyInit>(a, S, st);
        default: return launch_sweep<T, kApplyTemporal>(a, S, st);
    }
}

int launch_kt_apply(int mode, int prec, bool from_state, const KtSet &K, const ApplyIO &io, SolverState *S,
                    cudaStream_t st, int *launches) {
    if (prec == 1 && !K.val32) return fail(MPBJAC_ERR_UNSUPPORTED, "no binary32 BJAC(k,t) set");
    KtArgs a{};
    a.n = K.n;
    a.nb = K.nb;
    a.nslices = K.sell.nslices;
    a.off = K.sell.off;
    a.col = K.sell.col;
    a.val = prec ? static_cast<const void *>(K.val32) : static_cast<const void *>(K.sell.val);
    a.dinv = prec ? static_cast<const void *>(K.dinv32) : static_cast<const void *>(K.dinv64);
    a.rblk = K.rblk;
    a.block_ptr = K.block_ptr;
    a.r = io.r;
    a.w = K.w;
    a.prec = prec;
    a.from_state = from_state ? 1 : 0;
    a.io = io;
    void *ybuf[2] = {K.y0, K.y1};
    void *zbuf[2] = {K.zt, K.zt2};
    int cur = 0;
    for (int j = 0; j < K.k; ++j) {
        a.zin = zbuf[(j + 1) & 1];
        a.zout = zbuf[j & 1];
        for (int i = 0; i < K.t; ++i) {
            a.first = i == 0;
            a.outer = (i == 0 && j > 0) ? 1 : 0;
            a.yin = ybuf[cur];
            a.yout = ybuf[cur ^ 1];
            a.acc = i == K.t - 1;
            a.zero_z = j == 0;
            a.final_ = (j == K.k - 1 && i == K.t - 1) ? 1 : 0;
            const int rc = prec ? launch_sweep_mode<float>(mode, a, S, st) : launch_sweep_mode<double>(mode, a, S, st);
            if (rc) return rc;
            if (launches) *launches += 1;
            cur ^= 1;
        }
    }
    return MPBJAC_OK;
}

}  // namespace mpbjac
