// Sliced ELLPACK with slices of one warp (SELL-32): the loop SpMV q = A p of PCG
// (Section 3.2) on a copy of A laid out for coalesced loads.
//
// Slice s holds rows 32 s .. 32 s + 31, padded to the slice's longest row and stored
// column-major: entry j of row 32 s + i sits at off[s] + 32 j + i. The j-th value load of a
// warp is one aligned 256-byte segment and the j-th column load one 128-byte segment, with
// no staging through shared memory and a trip count that is the same for the whole warp.
// Padding entries carry column -1 and are skipped, so every lane runs exactly its own row's
// FMA chain in CSR order and y is bitwise the CSR kernels' result. Rows keep their order
// (no sorting by length), so no permutation of x or y is needed.
#include "common.cuh"
#include "sell.cuh"
#include "spmv.cuh"

namespace mpbjac {

// longest row of each slice (one warp per slice)
__global__ void k_sell_len(int n, int nslices, const int32_t *__restrict__ rowptr, int32_t *__restrict__ len) {
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nslices) return;
    const int row = (s << 5) + lane;
    const int l = row < n ? rowptr[row + 1] - rowptr[row] : 0;
    const int m = __reduce_max_sync(0xffffffffu, l);
    if (lane == 0) len[s] = m;
}

// off[s] = 32 * (len[0] + ... + len[s-1]) for s = 0..nslices with one CTA of 1024 threads
// (each scans a contiguous run; a Hillis-Steele scan joins the runs). info[0] = the total
// in 64 bits, info[1] = the longest slice. Offsets past 2^31 are clamped; the host then
// rejects the copy from info[0] before any of them is used.
__global__ void __launch_bounds__(1024) k_sell_scan(int nslices, const int32_t *__restrict__ len,
                                                    int32_t *__restrict__ off, long long *info) {
    __shared__ long long s_sum[1024];
    __shared__ int s_max[32];
    const int t = threadIdx.x;
    const int per = (nslices + 1023) / 1024;
    const int a = min(t * per, nslices), e = min(a + per, nslices);
    long long sum = 0;
    int mx = 0;
    for (int i = a; i < e; ++i) {
        sum += 32LL * len[i];
        mx = max(mx, len[i]);
    }
    s_sum[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long v = t >= o ? s_sum[t - o] : 0;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    long long run = s_sum[t] - sum;
    for (int i = a; i < e; ++i) {
        off[i] = (int32_t)min(run, (long long)INT32_MAX);
        run += 32LL * len[i];
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((t & 31) == 0) s_max[t >> 5] = mx;
    __syncthreads();
    if (t == 0) {
        int m = 0;
        for (int w = 0; w < 32; ++w) m = max(m, s_max[w]);
        const long long total = s_sum[1023];
        off[nslices] = (int32_t)min(total, (long long)INT32_MAX);
        info[0] = total;
        info[1] = m;
    }
}

// one warp per slice: copy the rows' entries column-major, pad with (0, -1)
__global__ void k_sell_fill(int n, int nslices, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                            const double *__restrict__ val, const int32_t *__restrict__ off, int32_t *__restrict__ scol,
                            double *__restrict__ sval) {
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nslices) return;
    const int o0 = off[s];
    const int len = (off[s + 1] - o0) >> 5;
    const int row = (s << 5) + lane;
    const int lo = row < n ? rowptr[row] : 0;
    const int rl = row < n ? rowptr[row + 1] - lo : 0;
    for (int j = 0; j < len; ++j) {
        const size_t k = (size_t)o0 + 32 * (size_t)j + lane;
        const bool in = j < rl;
        sval[k] = in ? val[lo + j] : 0.0;
        scol[k] = in ? colidx[lo + j] : -1;
    }
}

// U consecutive entries of this lane's row: all value and column loads first, then the x
// gathers, then the FMA chain (padding skipped)
template <int U>
__device__ __forceinline__ void sell_part(const double *__restrict__ pv, const int32_t *__restrict__ pc,
                                          const double *__restrict__ x, uint64_t pol, double &acc) {
    double vv[U], xv[U];
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        vv[u] = __ldcs(pv + 32 * u);
        cc[u] = __ldcs(pc + 32 * u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = cc[u] >= 0 ? ldg_vec(x + cc[u], pol) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (cc[u] >= 0) acc = fma(vv[u], xv[u], acc);
}

// gathers and FMA chain of U entries already loaded into registers
template <int U>
__device__ __forceinline__ void sell_fma(const double (&vv)[8], const int (&cc)[8], const double *__restrict__ x,
                                         uint64_t pol, double &acc) {
    double xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = cc[u] >= 0 ? ldg_vec(x + cc[u], pol) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (cc[u] >= 0) acc = fma(vv[u], xv[u], acc);
}

// the first (up to) 8 entries of every row of slice s, or nothing past the last slice
__device__ __forceinline__ void sell_head(int s, int nslices, int lane, const int32_t *__restrict__ off,
                                          const int32_t *__restrict__ col, const double *__restrict__ val,
                                          double (&vv)[8], int (&cc)[8], int &o0, int &len) {
    o0 = 0;
    len = 0;
    if (s < nslices) {
        o0 = __ldg(off + s);
        len = (__ldg(off + s + 1) - o0) >> 5;
    }
    const int cnt = len < 8 ? len : 8;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (u < cnt) {
            vv[u] = __ldcs(val + o0 + 32 * u + lane);
            cc[u] = __ldcs(col + o0 + 32 * u + lane);
        } else {
            vv[u] = 0.0;
            cc[u] = -1;
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(kSpNT, 6) k_spmv_sell(int n, int nslices, const int32_t *__restrict__ off,
                                                       const int32_t *__restrict__ col, const double *__restrict__ val,
                                                       const double *__restrict__ x, const double *__restrict__ b,
                                                       double *__restrict__ y, double *part, unsigned int *ticket,
                                                       double *out, SolverState *S) {
    constexpr int NW = kSpNT / 32;
    constexpr bool RES = KIND >= 10;
    __shared__ double red[2 * kSpNT];
    {
        // the warp's first slice of A (values, then columns) into L2 while the predecessor drains
        const int s0 = blockIdx.x * NW + (threadIdx.x >> 5), ln = threadIdx.x & 31;
        if (s0 < nslices) {
            const int o0 = __ldg(off + s0);
            const int len = (__ldg(off + s0 + 1) - o0) >> 5;
            const int nvl = 2 * len, ncl = len;          // 128-byte lines: 16 values, 32 columns
            for (int l = ln; l < nvl + ncl; l += 32) {
                if (l < nvl) prefetch_l2(val + o0 + 16 * l);
                else prefetch_l2(col + o0 + 32 * (l - nvl));
            }
        }
    }
    pdl_enter();
    if (sp_loop<KIND>()) {
        // the previous iteration's x update is done (stream order): clear its flag even when
        // this iteration does not run, so a loop body after convergence changes nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) S->x_pending = 0;
        if (S->state != kRunning) return;
    }
    const uint64_t pol = vec_policy(sp_loop<KIND>() ? S->l2_keep : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NW + warp, nw = gridDim.x * NW;
    double acc1 = 0.0, acc2 = 0.0;
    for (int s = gw; s < nslices; s += nw) {
        const int o0 = __ldg(off + s);
        const int len = (__ldg(off + s + 1) - o0) >> 5;      // the same in every lane
        const int row = (s << 5) + lane;
        double xr = 0.0, bi = 0.0;
        if (row < n) {
            if (RES) bi = b[row];
            else if (KIND != kSpY) xr = ldg_vec(x + row, pol);
        }
        const double *pv = val + o0 + lane;
        const int32_t *pc = col + o0 + lane;
        double acc = 0.0;
        int j = 0;
        for (; j + 8 <= len; j += 8) sell_part<8>(pv + 32 * j, pc + 32 * j, x, pol, acc);
        switch (len - j) {
            case 1: sell_part<1>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
            case 2: sell_part<2>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
            case 3: sell_part<3>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
            case 4: sell_part<4>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
            case 5: sell_part<5>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
            case 6: sell_part<6>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
            case 7: sell_part<7>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
            default: break;
        }
        if (row < n) {
            if (RES) {
                const double ri = bi - acc;
                st_vec(y + row, ri, pol);
                acc1 = fma(ri, ri, acc1);
                acc2 = fma(bi, bi, acc2);
            } else {
                st_vec(y + row, acc, pol);
                if (KIND != kSpY) acc1 = fma(acc, xr, acc1);
            }
        }
    }
    if (KIND == kSpY) return;
    double cs[2] = {0.0, 0.0};     // this CTA's partial sums (valid in thread 0)
    if (RES) {
        const double v[2] = {acc1, acc2};
        cta_sum_to0<kSpNT, 2>(v, red, cs);
    } else {
        const double v[1] = {acc1};
        double c1[1];
        cta_sum_to0<kSpNT, 1>(v, red, c1);
        cs[0] = c1[0];
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = cs[0];
        part[2 * blockIdx.x + 1] = cs[1];
    }
    if (KIND == kSpPcg) {     // the kernel that consumes alpha sums the partials (loop_alpha)
        if (blockIdx.x == 0)
            for (int c = gridDim.x + threadIdx.x; c < kMaxGrid; c += blockDim.x) part[2 * c] = 0.0;
        return;
    }
    if (!last_cta(ticket)) return;
    double t[2] = {0.0, 0.0};
    if (RES) {
        reduce_partials_to0<kSpNT, 2>(part, gridDim.x, 2, red, t);
    } else {
        double t1[1];
        reduce_partials_to0<kSpNT, 1>(part, gridDim.x, 2, red, t1);
        t[0] = t1[0];
    }
    if (threadIdx.x == 0) spmv_finish<KIND>(t[0], t[1], out, S);
}

// The same SpMV with the first chunk (up to 8 entries per row) of a warp's next slice loaded
// into registers while the current slice's x gathers and FMA chains run, so that every warp
// keeps two slices' loads in flight. Longer rows finish with unprefetched chunks of 8.
template <int KIND>
__global__ void __launch_bounds__(kSpNT, 3) k_spmv_sell_pf(int n, int nslices, const int32_t *__restrict__ off,
                                                          const int32_t *__restrict__ col,
                                                          const double *__restrict__ val,
                                                          const double *__restrict__ x, const double *__restrict__ b,
                                                          double *__restrict__ y, double *part, unsigned int *ticket,
                                                          double *out, SolverState *S) {
    constexpr int NW = kSpNT / 32;
    constexpr bool RES = KIND >= 10;
    __shared__ double red[2 * kSpNT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NW + warp, nw = gridDim.x * NW;
    double nv[8];
    int nc[8], n_o0, n_len;
    sell_head(gw, nslices, lane, off, col, val, nv, nc, n_o0, n_len);   // A only: before the wait
    pdl_enter();
    if (sp_loop<KIND>()) {
        // the previous iteration's x update is done (stream order): clear its flag even when
        // this iteration does not run, so a loop body after convergence changes nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) S->x_pending = 0;
        if (S->state != kRunning) return;
    }
    const uint64_t pol = vec_policy(sp_loop<KIND>() ? S->l2_keep : 0);
    double acc1 = 0.0, acc2 = 0.0;
    for (int s = gw; s < nslices; s += nw) {
        double cv[8];
        int cc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cv[u] = nv[u];
            cc[u] = nc[u];
        }
        const int o0 = n_o0, len = n_len;
        sell_head(s + nw, nslices, lane, off, col, val, nv, nc, n_o0, n_len);
        const int row = (s << 5) + lane;
        double xr = 0.0, bi = 0.0;
        if (row < n) {
            if (RES) bi = b[row];
            else if (KIND != kSpY) xr = ldg_vec(x + row, pol);
        }
        double acc = 0.0;
        switch (len < 8 ? len : 8) {
            case 1: sell_fma<1>(cv, cc, x, pol, acc); break;
            case 2: sell_fma<2>(cv, cc, x, pol, acc); break;
            case 3: sell_fma<3>(cv, cc, x, pol, acc); break;
            case 4: sell_fma<4>(cv, cc, x, pol, acc); break;
            case 5: sell_fma<5>(cv, cc, x, pol, acc); break;
            case 6: sell_fma<6>(cv, cc, x, pol, acc); break;
            case 7: sell_fma<7>(cv, cc, x, pol, acc); break;
            case 8: sell_fma<8>(cv, cc, x, pol, acc); break;
            default: break;
        }
        if (len > 8) {
            const double *pv = val + o0 + lane;
            const int32_t *pc = col + o0 + lane;
            int j = 8;
            for (; j + 8 <= len; j += 8) sell_part<8>(pv + 32 * j, pc + 32 * j, x, pol, acc);
            switch (len - j) {
                case 1: sell_part<1>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
                case 2: sell_part<2>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
                case 3: sell_part<3>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
                case 4: sell_part<4>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
                case 5: sell_part<5>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
                case 6: sell_part<6>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
                case 7: sell_part<7>(pv + 32 * j, pc + 32 * j, x, pol, acc); break;
                default: break;
            }
        }
        if (row < n) {
            if (RES) {
                const double ri = bi - acc;
                st_vec(y + row, ri, pol);
                acc1 = fma(ri, ri, acc1);
                acc2 = fma(bi, bi, acc2);
            } else {
                st_vec(y + row, acc, pol);
                if (KIND != kSpY) acc1 = fma(acc, xr, acc1);
            }
        }
    }
    if (KIND == kSpY) return;
    double cs[2] = {0.0, 0.0};     // this CTA's partial sums (valid in thread 0)
    if (RES) {
        const double v[2] = {acc1, acc2};
        cta_sum_to0<kSpNT, 2>(v, red, cs);
    } else {
        const double v[1] = {acc1};
        double c1[1];
        cta_sum_to0<kSpNT, 1>(v, red, c1);
        cs[0] = c1[0];
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = cs[0];
        part[2 * blockIdx.x + 1] = cs[1];
    }
    if (KIND == kSpPcg) {     // the kernel that consumes alpha sums the partials (loop_alpha)
        if (blockIdx.x == 0)
            for (int c = gridDim.x + threadIdx.x; c < kMaxGrid; c += blockDim.x) part[2 * c] = 0.0;
        return;
    }
    if (!last_cta(ticket)) return;
    double t[2] = {0.0, 0.0};
    if (RES) {
        reduce_partials_to0<kSpNT, 2>(part, gridDim.x, 2, red, t);
    } else {
        double t1[1];
        reduce_partials_to0<kSpNT, 1>(part, gridDim.x, 2, red, t1);
        t[0] = t1[0];
    }
    if (threadIdx.x == 0) spmv_finish<KIND>(t[0], t[1], out, S);
}

// ----------------------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------------------
void sell_free(SellMat *m) {
    if (m->off) cudaFree(m->off);
    if (m->col) cudaFree(m->col);
    if (m->val) cudaFree(m->val);
    *m = SellMat{};
}

int sell_build(const bjac_csr &A, double max_ratio, SellMat *out, cudaStream_t st) {
    sell_free(out);
    const int n = A.n;
    const int nslices = (n + 31) / 32;
    int32_t *off = nullptr, *len = nullptr;
    long long *info = nullptr;
    MPB_CUDA(cudaMalloc(&off, sizeof(int32_t) * ((size_t)nslices + 1)));
    cudaError_t e = cudaMalloc(&len, sizeof(int32_t) * (size_t)nslices + 2 * sizeof(long long) + 16);
    if (e != cudaSuccess) {
        cudaFree(off);
        return cuda_fail(e, "cudaMalloc");
    }
    info = reinterpret_cast<long long *>(reinterpret_cast<char *>(len) +
                                         ((sizeof(int32_t) * (size_t)nslices + 15) & ~(size_t)15));
    const int grid = (int)(((long long)nslices * 32 + 255) / 256);
    k_sell_len<<<grid, 256, 0, st>>>(n, nslices, A.rowptr, len);
    k_sell_scan<<<1, 1024, 0, st>>>(nslices, len, off, info);
    long long h_info[2] = {0, 0};
    e = cudaMemcpyAsync(h_info, info, sizeof(h_info), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(len);
    if (e != cudaSuccess) {
        cudaFree(off);
        return cuda_fail(e, "SELL-32 slice lengths");
    }
    const long long total = h_info[0];
    const bool too_big = total > (long long)INT32_MAX - 64;
    const bool too_padded = max_ratio > 0.0 && (double)total > max_ratio * (double)(A.nnz > 0 ? A.nnz : 1);
    if (too_big || too_padded) {
        cudaFree(off);
        return MPBJAC_OK;
    }
    SellMat m;
    m.n = n;
    m.nslices = nslices;
    m.off = off;
    m.entries = total;
    m.max_len = (int)h_info[1];
    const size_t cnt = total > 0 ? (size_t)total : 1;
    e = cudaMalloc(&m.col, sizeof(int32_t) * cnt);
    if (e == cudaSuccess) e = cudaMalloc(&m.val, sizeof(double) * cnt);
    if (e != cudaSuccess) {
        sell_free(&m);
        return cuda_fail(e, "cudaMalloc (SELL-32 copy)");
    }
    k_sell_fill<<<grid, 256, 0, st>>>(n, nslices, A.rowptr, A.colidx, A.val, m.off, m.col, m.val);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        sell_free(&m);
        return cuda_fail(e, "k_sell_fill");
    }
    *out = m;
    return MPBJAC_OK;
}

template <int KIND>
static int launch_sell_t(const SellMat &M, const double *x, const double *b, double *y, double *part,
                         unsigned int *ticket, double *out, SolverState *S, cudaStream_t st) {
    static int per_sm[2] = {0, 0};
    const int pf = M.kernel == 1;
    if (per_sm[pf] == 0) {
        int v = 0;
        cudaError_t e = pf ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_spmv_sell_pf<KIND>, kSpNT, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_spmv_sell<KIND>, kSpNT, 0);
        if (e != cudaSuccess || v < 1) v = 1;
        per_sm[pf] = v;
    }
    int g = sm_count() * per_sm[pf];
    if (g > kMaxGrid) g = kMaxGrid;
    const int need = (M.nslices + kSpNT / 32 - 1) / (kSpNT / 32);
    if (g > need) g = need;
    if (g < 1) g = 1;
    if (pf)
        MPB_CUDA(launch_kernel(k_spmv_sell_pf<KIND>, g, kSpNT, 0, st, M.n, M.nslices, (const int32_t *)M.off,
                               (const int32_t *)M.col, (const double *)M.val, x, b, y, part, ticket, out, S));
    else
        MPB_CUDA(launch_kernel(k_spmv_sell<KIND>, g, kSpNT, 0, st, M.n, M.nslices, (const int32_t *)M.off,
                               (const int32_t *)M.col, (const double *)M.val, x, b, y, part, ticket, out, S));
    return MPBJAC_OK;
}

int launch_spmv_sell(const SellMat &M, const double *x, const double *b, double *y, double *part,
                     unsigned int *ticket, double *out, SolverState *S, int kind, cudaStream_t st) {
    if (!M.val) return fail(MPBJAC_ERR_UNSUPPORTED, "no SELL-32 copy of A");
    switch (kind) {
        case kSpY: return launch_sell_t<kSpY>(M, x, b, y, part, ticket, out, S, st);
        case kSpYDot: return launch_sell_t<kSpYDot>(M, x, b, y, part, ticket, out, S, st);
        case kSpPcg: return launch_sell_t<kSpPcg>(M, x, b, y, part, ticket, out, S, st);
        case kSpPcgAlpha: return launch_sell_t<kSpPcgAlpha>(M, x, b, y, part, ticket, out, S, st);
        case kResStandalone: return launch_sell_t<kResStandalone>(M, x, b, y, part, ticket, out, S, st);
        case kResStart: return launch_sell_t<kResStart>(M, x, b, y, part, ticket, out, S, st);
        case kResCheck: return launch_sell_t<kResCheck>(M, x, b, y, part, ticket, out, S, st);
        default: return fail(MPBJAC_ERR_INVALID_ARG, "unknown SpMV kind");
    }
}

}  // namespace mpbjac
