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
// One CTA per block; the block (<= 128 x 128 doubles) lives in shared memory. Blocks are
// grouped by size (<= 32, <= 64, <= 128 rows) and each group runs with its own shared-memory
// size and CTA width (128, 256, 512 threads), so that small blocks are not held to the
// occupancy of the largest. Work that is not the sweep itself is kept off the (narrow)
// FP64 pipe of sm_103a: the pivot reciprocal is computed once per pivot, maxima and minima
// of non-negative values compare bit patterns as integers, the per-row statistics are
// reduced by one warp, and the rounding to the storage format is done in integer arithmetic.
#include "common.cuh"
#include "setup.cuh"

#include <algorithm>
#include <cfloat>
#include <vector>

namespace mpbjac {

constexpr double kDomCap = 1.0e6;
constexpr unsigned long long kSign = 0x8000000000000000ull;

__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ double neg(double v) {
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) ^ kSign));
}
__device__ __forceinline__ double absd(double v) {
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) & ~kSign));
}

// warp reductions (all lanes get the result): sum in binary64; max / min of NON-NEGATIVE
// values as integers (their bit patterns order like the values)
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ long long wmax_bits(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ long long wmin_bits(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Round-to-nearest-even of g * 2^-shift to a format with ebits exponent bits and mbits
// fraction bits (subnormals kept, overflow to infinity, NaN to a quiet NaN), from the
// binary64 bit layout in integer arithmetic. The scaling by 2^-shift is exact.
__device__ __forceinline__ uint32_t round_to_format(double g, int shift, int ebits, int mbits) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(g);
    const uint32_t sbit = (uint32_t)(u >> 63) << (ebits + mbits);
    const uint32_t emask = (1u << ebits) - 1u;
    const int E = (int)((u >> 52) & 0x7FF);
    const unsigned long long F = u & 0xFFFFFFFFFFFFFull;
    if (E == 0x7FF) return sbit | (emask << mbits) | (F ? (1u << (mbits - 1)) : 0u);
    unsigned long long M;
    int e;                                         // |g| = M 2^e
    if (E == 0) {
        if (F == 0) return sbit;
        M = F;
        e = -1074;
    } else {
        M = F | (1ull << 52);
        e = E - 1075;
    }
    e -= shift;
    const int bias = (1 << (ebits - 1)) - 1;
    const int emin = 1 - bias;
    const int p = 63 - __clzll((long long)M);     // leading bit of M
    const int E2 = p + e;                          // |v| in [2^E2, 2^(E2+1))
    int et = E2 < emin ? emin : E2;                // binade of the quantum
    const int sh = (et - mbits) - e;               // v / 2^(et - mbits) = M 2^-sh
    unsigned long long q;
    if (sh <= 0) {
        q = M << (-sh);                            // exact (fewer bits than the format holds)
    } else if (sh > 60) {
        q = 0;                                     // below half of the smallest quantum
    } else {
        q = M >> sh;
        const unsigned long long rem = M & ((1ull << sh) - 1ull);
        const unsigned long long half = 1ull << (sh - 1);
        q += (rem > half) | ((rem == half) & (q & 1ull));
    }
    if (q == 0) return sbit;
    if (q >= (2ull << mbits)) {                    // rounding carried into the next binade
        q >>= 1;
        et += 1;
    }
    uint32_t field, mant;
    if (q < (1ull << mbits)) {                     // subnormal (only when et == emin)
        field = 0;
        mant = (uint32_t)q;
    } else {
        field = (uint32_t)(et + bias);
        mant = (uint32_t)(q - (1ull << mbits));
    }
    if (field >= emask) return sbit | (emask << mbits);
    return sbit | (field << mbits) | mant;
}

// Round g / 2^shift to format f and store entry idx of a block.
__device__ __forceinline__ void store_fmt(uint8_t *out, int f, size_t idx, double g, int shift) {
    if (f == BJAC_FP64) reinterpret_cast<double *>(out)[idx] = g;
    else if (f == BJAC_FP32) reinterpret_cast<uint32_t *>(out)[idx] = round_to_format(g, 0, 8, 23);
    else if (f == BJAC_BF16) reinterpret_cast<uint16_t *>(out)[idx] = (uint16_t)round_to_format(g, shift, 8, 7);
    else reinterpret_cast<uint16_t *>(out)[idx] = (uint16_t)round_to_format(g, shift, 5, 10);
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

// per-row statistics kept in shared memory for the block features
enum RowStat { kRsFro = 0, kRsDom, kRsDiag, kRsOut, kRsAll, kRsTau, kRsNdom, kRsExc, kRsColB, kRsColG, kRsGmax,
               kRsGmin, kRsCount };

size_t setup_smem_bytes(int bs_max) {
    const int T = bs_max * (bs_max + 1) / 2;
    return (size_t)bs_max * bs_max * 8 + (2 + kRsCount) * (size_t)bs_max * 8 + (size_t)T * 2 + 16;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_setup_blocks(SetupArgs a, int bs_max, const int32_t *__restrict__ list) {
    extern __shared__ __align__(16) double dsm[];
    double *sA = dsm;                                     // bs x bs (upper triangle used)
    double *sc = sA + bs_max * bs_max;                    // pivot column
    double *st = sc + bs_max;                             // pivot column / pivot
    double *rs = st + bs_max;                             // kRsCount x bs_max row statistics
    uint16_t *tri = reinterpret_cast<uint16_t *>(rs + kRsCount * bs_max);   // (i << 8 | j), i <= j
    __shared__ double s_inv[2];
    __shared__ int s_ok[2];
    __shared__ int s_fmt, s_ex;

    const int b = list ? list[blockIdx.x] : blockIdx.x;
    const int s = a.block_ptr[b], e = a.block_ptr[b + 1], bs = e - s;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < bs * bs; idx += NT) sA[idx] = 0.0;
    // upper-triangle index table: row i occupies [i*bs - i(i-1)/2, +bs-i)
    for (int i = tid; i < bs; i += NT) {
        const int o = i * bs - (i * (i - 1)) / 2;
        for (int j = i; j < bs; ++j) tri[o + (j - i)] = (uint16_t)((i << 8) | j);
    }
    __syncthreads();

    // 1. extraction and per-row statistics (one thread per row; bs <= 128 <= NT)
    if (tid < bs) {
        const int i = s + tid;
        double fro = 0.0, all = 0.0, out = 0.0, diag = 0.0, off = 0.0;
        long long mx = 0, mn = 0x7FF0000000000000ll;      // |a_ij| bit patterns, j != i, nonzero
        for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
            const int j = a.colidx[k];
            const double v = a.val[k], av = absd(v);
            all += av;
            if (j >= s && j < e) {
                sA[tid * bs + (j - s)] += v;
                fro = fma(v, v, fro);
            } else {
                out += av;
            }
            if (j == i) {
                diag += av;
            } else {
                off += av;
                if (av != 0.0) {
                    const long long ab = dbits(av);
                    mx = ab > mx ? ab : mx;
                    mn = ab < mn ? ab : mn;
                }
            }
        }
        double d = off > 0.0 ? diag / off : kDomCap;
        if (d > kDomCap) d = kDomCap;
        rs[kRsFro * bs_max + tid] = fro;
        rs[kRsDom * bs_max + tid] = d;
        rs[kRsDiag * bs_max + tid] = diag;
        rs[kRsOut * bs_max + tid] = out;
        rs[kRsAll * bs_max + tid] = all;
        rs[kRsTau * bs_max + tid] = mx > 0 ? log10(__longlong_as_double(mx) / __longlong_as_double(mn)) : 0.0;
        rs[kRsNdom * bs_max + tid] = diag > off ? 1.0 : 0.0;
        rs[kRsExc * bs_max + tid] = diag > 0.0 ? (diag - off) / diag : 0.0;
    }
    __syncthreads();
    // column sums of |B| (||B||_1 is their maximum); the first pivot's reciprocal
    if (tid < bs) {
        double colsum = 0.0;
        for (int i = 0; i < bs; ++i) colsum += absd(sA[i * bs + tid]);
        rs[kRsColB * bs_max + tid] = colsum;
    }
    if (tid == 0) {
        const double d = sA[0];
        s_ok[0] = d > 0.0;
        s_inv[0] = 1.0 / d;
    }
    __syncthreads();

    // 2. symmetric Gauss-Jordan sweep over the upper triangle; the thread that updates the
    //    next pivot computes its reciprocal
    const int T = bs * (bs + 1) / 2;
    bool spd = true;
    for (int k = 0; k < bs; ++k) {
        if (!s_ok[k & 1]) { spd = false; break; }        // same value in every thread
        const double inv = s_inv[k & 1];
        if (tid < bs) {
            const double c = tid <= k ? sA[tid * bs + k] : sA[k * bs + tid];
            sc[tid] = c;
            st[tid] = c * inv;
        }
        __syncthreads();
        for (int t = tid; t < T; t += NT) {
            const int ij = tri[t];
            const int i = ij >> 8, j = ij & 255;
            if (i != k && j != k) {
                const double v = fma(-sc[i], st[j], sA[i * bs + j]);
                sA[i * bs + j] = v;
                if (i == k + 1 && j == k + 1) {
                    s_ok[(k + 1) & 1] = v > 0.0;
                    s_inv[(k + 1) & 1] = 1.0 / v;
                }
            }
        }
        if (tid < bs) {
            if (tid < k) sA[tid * bs + k] = st[tid];
            else if (tid > k) sA[k * bs + tid] = st[tid];
            else sA[k * bs + k] = neg(inv);
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
        for (int idx = tid; idx < bs * bs; idx += NT) {
            const int i = idx / bs, j = idx - i * bs;
            Gb[idx] = neg(i <= j ? sA[i * bs + j] : sA[j * bs + i]);
        }
    }
    // 3. column sums of |G|, max |G| and min nonzero |G| per column
    if (tid < bs) {
        double gcol = 0.0;
        long long gmx = 0, gmn = 0x7FF0000000000000ll;
        for (int i = 0; i < bs; ++i) {
            const double v = absd(i <= tid ? sA[i * bs + tid] : sA[tid * bs + i]);
            gcol += v;
            const long long vb = dbits(v);
            gmx = vb > gmx ? vb : gmx;
            if (vb > 0) gmn = vb < gmn ? vb : gmn;
        }
        rs[kRsColG * bs_max + tid] = gcol;
        rs[kRsGmax * bs_max + tid] = __longlong_as_double(gmx);
        rs[kRsGmin * bs_max + tid] = __longlong_as_double(gmn);
    }
    __syncthreads();
    // block totals by warp 0, then the features, the format and the scale by its lane 0
    if (tid < 32) {
        double fro = 0.0, dsum = 0.0, osum = 0.0, asum = 0.0, tsum = 0.0, ndom = 0.0, exc = 0.0;
        long long dmin = 0x7FF0000000000000ll, amin = 0x7FF0000000000000ll, amax = 0, tmax = 0;
        long long nb1 = 0, ng1 = 0, gmax = 0, gmin = 0x7FF0000000000000ll;
        for (int r = tid; r < bs; r += 32) {
            fro += rs[kRsFro * bs_max + r];
            dsum += rs[kRsDom * bs_max + r];
            osum += rs[kRsOut * bs_max + r];
            asum += rs[kRsAll * bs_max + r];
            tsum += rs[kRsTau * bs_max + r];
            ndom += rs[kRsNdom * bs_max + r];
            exc += rs[kRsExc * bs_max + r];
            const long long dm = dbits(rs[kRsDom * bs_max + r]), dg = dbits(rs[kRsDiag * bs_max + r]);
            const long long ta = dbits(rs[kRsTau * bs_max + r]);
            const long long cb = dbits(rs[kRsColB * bs_max + r]), cg = dbits(rs[kRsColG * bs_max + r]);
            const long long gx = dbits(rs[kRsGmax * bs_max + r]), gn = dbits(rs[kRsGmin * bs_max + r]);
            dmin = dm < dmin ? dm : dmin;
            amin = dg < amin ? dg : amin;
            amax = dg > amax ? dg : amax;
            tmax = ta > tmax ? ta : tmax;
            nb1 = cb > nb1 ? cb : nb1;
            ng1 = cg > ng1 ? cg : ng1;
            gmax = gx > gmax ? gx : gmax;
            gmin = gn < gmin ? gn : gmin;
        }
        fro = wsum(fro); dsum = wsum(dsum); osum = wsum(osum); asum = wsum(asum);
        tsum = wsum(tsum); ndom = wsum(ndom); exc = wsum(exc);
        dmin = wmin_bits(dmin); amin = wmin_bits(amin); amax = wmax_bits(amax); tmax = wmax_bits(tmax);
        nb1 = wmax_bits(nb1); ng1 = wmax_bits(ng1); gmax = wmax_bits(gmax); gmin = wmin_bits(gmin);
        if (tid == 0) {
            const double gmx = __longlong_as_double(gmax), gmn = __longlong_as_double(gmin);
            const double lk = log10(__longlong_as_double(nb1) * __longlong_as_double(ng1));
            const double ldr = gmx > 0.0 ? log10(gmx / gmn) : 0.0;
            if (a.feat) {
                double *f = a.feat + (size_t)b * 12;
                const double am = __longlong_as_double(amin), ax = __longlong_as_double(amax);
                f[0] = lk;
                f[1] = 0.5 * log10(fro);
                f[2] = __longlong_as_double(dmin);
                f[3] = dsum / bs;
                f[4] = ax > 0.0 ? am / ax : 0.0;
                f[5] = asum > 0.0 ? osum / asum : 0.0;
                f[6] = __longlong_as_double(tmax);
                f[7] = tsum / bs;
                f[8] = ldr;
                f[9] = bs / 128.0;
                f[10] = ndom / bs;
                f[11] = exc / bs;
            }
            int fm;
            if (a.select == BJAC_SELECT_UNIFORM) fm = BJAC_FP64;
            else if (a.select == BJAC_SELECT_FIXED) fm = a.fixed_fmt;
            else if (a.select == BJAC_SELECT_RULE) fm = rule_format(lk, ldr, a.theta);
            else if (a.select == BJAC_SELECT_GIVEN) fm = a.given[b];
            else fm = BJAC_FP64;   // the learned selector decides in a later pass
            const int ex = (fm == BJAC_BF16 || fm == BJAC_FP16S) ? scale_exp(gmx) : 0;
            a.kap[2 * b] = lk;
            a.kap[2 * b + 1] = ldr;
            a.fmt[b] = (uint8_t)fm;
            a.scale[b] = ldexpf(1.0f, ex);
            s_fmt = fm;
            s_ex = ex;
        }
    }
    // 4. round into the pool now when the offsets are already known
    if (a.pool) {
        __syncthreads();
        const int fm = s_fmt, ex = s_ex;
        uint8_t *out = a.pool + a.qoff[b];
        for (int idx = tid; idx < bs * bs; idx += NT) {
            const int i = idx / bs, j = idx - i * bs;
            store_fmt(out, fm, idx, neg(i <= j ? sA[i * bs + j] : sA[j * bs + i]), ex);
        }
    }
}

// Second pass: round every block of G to fmt[b] into the pool (scale from max |G_b|).
constexpr int kPackNT = 128;
__global__ void __launch_bounds__(kPackNT) k_pack(const int32_t *block_ptr, const int64_t *goff, const double *G,
                                                  const uint8_t *fmt, const int64_t *qoff, uint8_t *pool,
                                                  float *scale) {
    __shared__ long long red[kPackNT / 32];
    const int b = blockIdx.x;
    const int bs = block_ptr[b + 1] - block_ptr[b];
    const double *Gb = G + goff[b];
    long long mx = 0;
    for (int idx = threadIdx.x; idx < bs * bs; idx += kPackNT) {
        const long long v = dbits(absd(Gb[idx]));
        mx = v > mx ? v : mx;
    }
    mx = wmax_bits(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    for (int w = 0; w < kPackNT / 32; ++w) mx = red[w] > mx ? red[w] : mx;
    const double gmax = __longlong_as_double(mx);
    const int f = fmt[b];
    const int ex = (f == BJAC_BF16 || f == BJAC_FP16S) ? scale_exp(gmax) : 0;
    if (threadIdx.x == 0) scale[b] = ldexpf(1.0f, ex);
    uint8_t *out = pool + qoff[b];
    for (int idx = threadIdx.x; idx < bs * bs; idx += kPackNT) store_fmt(out, f, idx, Gb[idx], ex);
}

// Host launchers ---------------------------------------------------------------------------
template <int NT>
static int launch_class(const SetupArgs &a, int bs_max, const int32_t *list, int count, cudaStream_t st) {
    const size_t smem = setup_smem_bytes(bs_max);
    MPB_CUDA(cudaFuncSetAttribute(k_setup_blocks<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_setup_blocks<NT><<<count, NT, smem, st>>>(a, bs_max, list);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

static int launch_for(const SetupArgs &a, int bs_max, const int32_t *list, int count, cudaStream_t st) {
    if (count <= 0) return MPBJAC_OK;
    if (bs_max <= 32) return launch_class<128>(a, bs_max, list, count, st);
    if (bs_max <= 64) return launch_class<256>(a, bs_max, list, count, st);
    return launch_class<512>(a, bs_max, list, count, st);
}

int launch_setup_blocks(const SetupArgs &a, int bs_max, const int32_t *h_block_ptr, cudaStream_t st) {
    if (!h_block_ptr) return launch_for(a, bs_max, nullptr, a.nb, st);
    // group the blocks by size class; one class runs over all blocks without a list
    std::vector<int32_t> cls[3];
    int cmax[3] = {0, 0, 0};
    for (int b = 0; b < a.nb; ++b) {
        const int bs = h_block_ptr[b + 1] - h_block_ptr[b];
        const int c = bs <= 32 ? 0 : bs <= 64 ? 1 : 2;
        cls[c].push_back(b);
        cmax[c] = std::max(cmax[c], bs);
    }
    int used = 0;
    for (int c = 0; c < 3; ++c) used += !cls[c].empty();
    if (used <= 1) return launch_for(a, bs_max, nullptr, a.nb, st);
    int32_t *d_list = nullptr;
    MPB_CUDA(cudaMallocAsync((void **)&d_list, sizeof(int32_t) * (size_t)a.nb, st));
    size_t o = 0;
    int rc = MPBJAC_OK;
    for (int c = 2; c >= 0 && rc == MPBJAC_OK; --c) {      // largest blocks first
        if (cls[c].empty()) continue;
        cudaError_t e = cudaMemcpyAsync(d_list + o, cls[c].data(), sizeof(int32_t) * cls[c].size(),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy block list");
        else rc = launch_for(a, cmax[c], d_list + o, (int)cls[c].size(), st);
        o += cls[c].size();
    }
    // the host vectors must outlive the asynchronous copies
    const cudaError_t e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_list, st);
    if (rc) return rc;
    return e == cudaSuccess ? MPBJAC_OK : cuda_fail(e, "setup kernels");
}

int launch_pack(int nb, const int32_t *block_ptr, const int64_t *goff, const double *G, const uint8_t *fmt,
                const int64_t *qoff, uint8_t *pool, float *scale, cudaStream_t st) {
    k_pack<<<nb, kPackNT, 0, st>>>(block_ptr, goff, G, fmt, qoff, pool, scale);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

}  // namespace mpbjac
