// Block-Jacobi apply z = M^-1 r (Algorithm 3.1 for the low-precision set, Eq. 3-1 with
// exact block inverses for the binary64 set), with the dot product r.z fused, and, in the
// PCG loop, the residual recurrence r -= alpha q fused in front of it.
//
// Low-precision blocks: r-hat = RN_fp32(r) (ConvertPrecision to p_l), each output row is a
// binary32 FMA chain over the block's columns in natural order, then multiplied by the
// block's power-of-two scale in binary32 and widened to binary64 (ConvertPrecision to p_w).
// Every block is stored symmetric and row-major, so row j of a block is also its column j:
// lane i reads entry (j, i) while the warp sweeps j, which keeps every read coalesced and
// needs no cross-lane reduction.
//
// Two kernels:
//  * k_apply_generic: one warp per block, any block size 1..128, any mix of formats.
//  * k_apply_tma: all blocks of one size (32 or 64) and one low format. Persistent
//    CTAs stream groups of consecutive blocks (plus the matching slices of r and q)
//    through a ring of shared-memory stages filled by cp.async.bulk (TMA bulk copies)
//    that complete on mbarriers; every wait is bounded.
#include "common.cuh"
#include "apply.cuh"

namespace mpbjac {

// ----------------------------------------------------------------------------------------
// epilogue shared by both kernels: the last CTA turns the partial sums into solver scalars
// ----------------------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void apply_finish(double rho, double rr, const ApplyIO &io, SolverState *S,
                                             int used_low) {
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
    // kApplyTemporal and kApplyFused (still running): beta = rho_new / rho_old
    if (!finite_pos(rho)) { S->state = kBreakdown; return; }
    S->beta = rho / S->rho;
    S->rho = rho;
}

// ----------------------------------------------------------------------------------------
// generic: one warp per block
// ----------------------------------------------------------------------------------------
template <typename QT>
__device__ __forceinline__ float to_f32(QT v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename QT>
__device__ __forceinline__ float low_row(const QT *__restrict__ Q, const float *rh, int bs, int i) {
    float acc = 0.0f;
#pragma unroll 8
    for (int j = 0; j < bs; ++j) acc = fmaf(to_f32<QT>(__ldg(Q + (size_t)j * bs + i)), rh[j], acc);
    return acc;
}

template <int MODE>
__global__ void __launch_bounds__(kNT) k_apply_generic(PSet lo, PSet hi, ApplyIO io, SolverState *S) {
    __shared__ double s_r[kWarps][128];
    __shared__ float s_rh[kWarps][128];
    __shared__ double s_red[kWarps];
    int use_low = io.set;
    if (MODE != kApplyStandalone) {
        if (S->state != kRunning) return;
        if (MODE != kApplyFused) use_low = S->use_low;
        if (io.only_set >= 0 && io.only_set != use_low) return;
    }
    const PSet &P = use_low ? lo : hi;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;
    const double alpha = (MODE == kApplyFused) ? S->alpha : 0.0;
    double rho = 0.0, rr = 0.0;
    for (int b = gw; b < P.nb; b += nw) {
        const int s = __ldg(P.block_ptr + b), bs = __ldg(P.block_ptr + b + 1) - s;
        for (int i = lane; i < bs; i += 32) {
            double rv = io.r[s + i];
            if (MODE == kApplyFused) {
                rv = fma(-alpha, io.q[s + i], rv);
                io.r_out[s + i] = rv;
                rr = fma(rv, rv, rr);
            }
            s_r[warp][i] = rv;
            s_rh[warp][i] = __double2float_rn(rv);
        }
        __syncwarp();
        const int f = __ldg(P.fmt + b);
        const uint8_t *base = P.pool + __ldg(P.qoff + b);
        const float sc = __ldg(P.scale + b);
        for (int i = lane; i < bs; i += 32) {
            double zi;
            if (f == BJAC_FP64) {
                const double *G = reinterpret_cast<const double *>(base);
                double acc = 0.0;
#pragma unroll 4
                for (int j = 0; j < bs; ++j) acc = fma(__ldg(G + (size_t)j * bs + i), s_r[warp][j], acc);
                zi = acc;
            } else {
                float acc;
                if (f == BJAC_FP32) acc = low_row(reinterpret_cast<const float *>(base), s_rh[warp], bs, i);
                else if (f == BJAC_BF16) acc = low_row(reinterpret_cast<const __nv_bfloat16 *>(base), s_rh[warp], bs, i);
                else acc = low_row(reinterpret_cast<const __half *>(base), s_rh[warp], bs, i);
                zi = (double)(acc * sc);
            }
            io.z[s + i] = zi;
            if (MODE == kApplyInit) io.p[s + i] = zi;
            rho = fma(s_r[warp][i], zi, rho);
        }
        __syncwarp();
    }
    if (MODE == kApplyStandalone && io.out == nullptr) return;
    const double b1 = block_sum<kNT>(rho, s_red);
    const double b2 = block_sum<kNT>(rr, s_red);
    if (threadIdx.x == 0) {
        io.part[2 * blockIdx.x] = b1;
        io.part[2 * blockIdx.x + 1] = b2;
    }
    if (!last_cta(io.ticket)) return;
    const double t1 = reduce_partials<kNT>(io.part, gridDim.x, 2, s_red);
    const double t2 = reduce_partials<kNT>(io.part + 1, gridDim.x, 2, s_red);
    if (threadIdx.x == 0) apply_finish<MODE>(t1, t2, io, S, use_low);
}

// ----------------------------------------------------------------------------------------
// TMA-staged uniform kernel
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: gives up after ~1 s of device time or 2^26 polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (int it = 0; it < (1 << 26); ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((it & 255) == 255 && globaltimer_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

template <typename QT, int BS>
struct TmaGeom {
    static constexpr int kWPB = BS / 32;                     // warps per block
    static constexpr int kBPS = kWarps / kWPB;               // blocks per stage
    static constexpr int kRows = kBPS * BS;                  // rows per stage (= 256)
    static constexpr int kBlkBytes = BS * BS * (int)sizeof(QT);
    static constexpr int kQBytes = kBPS * kBlkBytes;
    static constexpr int kStageBytes = kQBytes + 2 * kRows * 8;   // Q blocks, r slice, q slice
    static constexpr int kBudget = 200 * 1024;
    static constexpr int kStages = (kBudget / kStageBytes) > 8 ? 8 : (kBudget / kStageBytes);
    static constexpr int kHeader = 128 + kRows * 4;               // barriers, r-hat
    static constexpr int kSmem = kHeader + kStages * kStageBytes;
};

template <typename QT, int BS, int MODE>
__global__ void __launch_bounds__(kNT, 1) k_apply_tma(PSet P, ApplyIO io, SolverState *S, int n) {
    using Geo = TmaGeom<QT, BS>;
    static_assert(Geo::kStages >= 2, "need at least two stages");
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    float *s_rh = reinterpret_cast<float *>(smem + 128);
    uint8_t *stages = smem + Geo::kHeader;
    __shared__ double s_red[kWarps];

    if (MODE != kApplyStandalone) {
        if (S->state != kRunning) return;
        if (MODE == kApplyTemporal || MODE == kApplyInit) {
            if (!S->use_low) return;     // the binary64 set runs in the generic kernel
        }
    }
    const int nb = P.nb;
    const int ngroups = (nb + Geo::kBPS - 1) / Geo::kBPS;
    const double alpha = (MODE == kApplyFused) ? S->alpha : 0.0;
    const bool with_q = (MODE == kApplyFused);

    auto issue = [&](int g, int s) {
        const int nblk = min(Geo::kBPS, nb - g * Geo::kBPS);
        const int rows = nblk * BS;
        const unsigned qbytes = (unsigned)(nblk * Geo::kBlkBytes);
        const unsigned vbytes = (unsigned)(rows * 8);
        uint8_t *dst = stages + (size_t)s * Geo::kStageBytes;
        mbar_expect_tx(&full[s], qbytes + vbytes * (with_q ? 2u : 1u));
        bulk_g2s(dst, P.pool + (size_t)g * Geo::kQBytes, qbytes, &full[s]);
        bulk_g2s(dst + Geo::kQBytes, io.r + (size_t)g * Geo::kRows, vbytes, &full[s]);
        if (with_q) bulk_g2s(dst + Geo::kQBytes + Geo::kRows * 8, io.q + (size_t)g * Geo::kRows, vbytes, &full[s]);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < Geo::kStages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < Geo::kStages; ++s) {
            const int g = blockIdx.x + s * gridDim.x;
            if (g < ngroups) issue(g, s);
        }
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bi = warp / Geo::kWPB, h = warp % Geo::kWPB;
    const int local_row = bi * BS + h * 32 + lane;      // row within the stage
    double rho = 0.0, rr = 0.0;
    bool timed_out = false;
    int it = 0;
    for (int g = blockIdx.x; g < ngroups; g += gridDim.x, ++it) {
        const int s = it % Geo::kStages;
        const unsigned phase = (unsigned)((it / Geo::kStages) & 1);
        const uint8_t *st = stages + (size_t)s * Geo::kStageBytes;
        const double *sr = reinterpret_cast<const double *>(st + Geo::kQBytes);
        const double *sq = reinterpret_cast<const double *>(st + Geo::kQBytes + Geo::kRows * 8);
        const int blk = g * Geo::kBPS + bi;
        const bool active = blk < nb;
        const int row = g * Geo::kRows + local_row;
        bool ok = mbar_wait_bounded(&full[s], phase);
        double rv = 0.0;
        if (ok && active) {
            rv = sr[local_row];
            if (MODE == kApplyFused) rv = fma(-alpha, sq[local_row], rv);
            s_rh[local_row] = __double2float_rn(rv);
        }
        timed_out = __syncthreads_or(!ok) != 0;
        if (timed_out) break;
        if (active) {
            const QT *Q = reinterpret_cast<const QT *>(st + (size_t)bi * Geo::kBlkBytes);
            const float4 *rh4 = reinterpret_cast<const float4 *>(s_rh + bi * BS);
            const int i = h * 32 + lane;
            float acc = 0.0f;
#pragma unroll
            for (int j4 = 0; j4 < BS / 4; ++j4) {
                const float4 r4 = rh4[j4];
                acc = fmaf(to_f32<QT>(Q[(4 * j4 + 0) * BS + i]), r4.x, acc);
                acc = fmaf(to_f32<QT>(Q[(4 * j4 + 1) * BS + i]), r4.y, acc);
                acc = fmaf(to_f32<QT>(Q[(4 * j4 + 2) * BS + i]), r4.z, acc);
                acc = fmaf(to_f32<QT>(Q[(4 * j4 + 3) * BS + i]), r4.w, acc);
            }
            const float sc = (sizeof(QT) == 2) ? __ldg(P.scale + blk) : 1.0f;
            const double zi = (double)(acc * sc);
            io.z[row] = zi;
            if (MODE == kApplyInit) io.p[row] = zi;
            if (MODE == kApplyFused) {
                io.r_out[row] = rv;
                rr = fma(rv, rv, rr);
            }
            rho = fma(rv, zi, rho);
        }
        __syncthreads();   // stage s and s_rh fully consumed
        if (threadIdx.x == 0) {
            const int g2 = g + Geo::kStages * gridDim.x;
            if (g2 < ngroups) issue(g2, s);
        }
    }
    if (timed_out) {
        // drain copies still in flight (bounded), record the failure, leave
        if (threadIdx.x == 0) {
            for (int k = 0; k < Geo::kStages; ++k) {
                const int itk = it + k;
                const int g = blockIdx.x + itk * gridDim.x;
                if (g < ngroups) (void)mbar_wait_bounded(&full[itk % Geo::kStages], (unsigned)((itk / Geo::kStages) & 1));
            }
            if (io.err) atomicExch(io.err, MPBJAC_ERR_TIMEOUT);
            if (MODE != kApplyStandalone) S->state = kBreakdown;
        }
        return;
    }
    (void)n;
    if (MODE == kApplyStandalone && io.out == nullptr) return;
    const double b1 = block_sum<kNT>(rho, s_red);
    const double b2 = block_sum<kNT>(rr, s_red);
    if (threadIdx.x == 0) {
        io.part[2 * blockIdx.x] = b1;
        io.part[2 * blockIdx.x + 1] = b2;
    }
    if (!last_cta(io.ticket)) return;
    const double t1 = reduce_partials<kNT>(io.part, gridDim.x, 2, s_red);
    const double t2 = reduce_partials<kNT>(io.part + 1, gridDim.x, 2, s_red);
    if (threadIdx.x == 0) apply_finish<MODE>(t1, t2, io, S, 1);
}

// ----------------------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------------------
static int generic_grid(int nb) {
    const int need = (nb + kWarps - 1) / kWarps;
    int g = sm_count() * 6;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g > need) g = need;
    return g < 1 ? 1 : g;
}

bool tma_supported(const PSet &P, int n) {
    if (P.ufmt < BJAC_FP32 || P.ufmt > BJAC_FP16S) return false;
    if (!(P.ubs == 32 || P.ubs == 64)) return false;
    if ((long long)P.ubs * P.nb != n) return false;
    return true;
}

// dry = true only raises the kernel's dynamic shared-memory limit (done at setup, so that
// no attribute call happens while a solve is being captured into a graph).
template <typename QT, int BS, int MODE>
static int launch_tma_t(const PSet &P, const ApplyIO &io, SolverState *S, int n, cudaStream_t st, bool dry) {
    using Geo = TmaGeom<QT, BS>;
    if (dry) {
        MPB_CUDA(cudaFuncSetAttribute(k_apply_tma<QT, BS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Geo::kSmem));
        return MPBJAC_OK;
    }
    const int ngroups = (P.nb + Geo::kBPS - 1) / Geo::kBPS;
    int g = sm_count();
    if (g > ngroups) g = ngroups;
    if (g < 1) g = 1;
    k_apply_tma<QT, BS, MODE><<<g, kNT, Geo::kSmem, st>>>(P, io, S, n);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

template <int MODE>
static int launch_tma_mode(const PSet &P, const ApplyIO &io, SolverState *S, int n, cudaStream_t st,
                           bool dry = false) {
    switch (P.ufmt * 1000 + P.ubs) {
        case BJAC_FP32 * 1000 + 32: return launch_tma_t<float, 32, MODE>(P, io, S, n, st, dry);
        case BJAC_FP32 * 1000 + 64: return launch_tma_t<float, 64, MODE>(P, io, S, n, st, dry);
        case BJAC_BF16 * 1000 + 32: return launch_tma_t<__nv_bfloat16, 32, MODE>(P, io, S, n, st, dry);
        case BJAC_BF16 * 1000 + 64: return launch_tma_t<__nv_bfloat16, 64, MODE>(P, io, S, n, st, dry);
        case BJAC_FP16S * 1000 + 32: return launch_tma_t<__half, 32, MODE>(P, io, S, n, st, dry);
        case BJAC_FP16S * 1000 + 64: return launch_tma_t<__half, 64, MODE>(P, io, S, n, st, dry);
        default: return fail(MPBJAC_ERR_UNSUPPORTED, "no TMA apply kernel for this format / block size");
    }
}

int prepare_apply_tma(const PSet &P) {
    ApplyIO io{};
    int rc = launch_tma_mode<kApplyStandalone>(P, io, nullptr, 0, nullptr, true);
    if (!rc) rc = launch_tma_mode<kApplyInit>(P, io, nullptr, 0, nullptr, true);
    if (!rc) rc = launch_tma_mode<kApplyTemporal>(P, io, nullptr, 0, nullptr, true);
    if (!rc) rc = launch_tma_mode<kApplyFused>(P, io, nullptr, 0, nullptr, true);
    return rc;
}

int launch_apply_tma(int mode, const PSet &P, const ApplyIO &io, SolverState *S, int n, cudaStream_t st) {
    switch (mode) {
        case kApplyStandalone: return launch_tma_mode<kApplyStandalone>(P, io, S, n, st);
        case kApplyInit: return launch_tma_mode<kApplyInit>(P, io, S, n, st);
        case kApplyTemporal: return launch_tma_mode<kApplyTemporal>(P, io, S, n, st);
        default: return launch_tma_mode<kApplyFused>(P, io, S, n, st);
    }
}

int launch_apply_generic(int mode, const PSet &lo, const PSet &hi, const ApplyIO &io, SolverState *S,
                         cudaStream_t st) {
    const int nb = (mode == kApplyStandalone || mode == kApplyFused) ? (io.set ? lo.nb : hi.nb)
                                                                      : (lo.nb > hi.nb ? lo.nb : hi.nb);
    const int g = generic_grid(nb);
    switch (mode) {
        case kApplyStandalone: k_apply_generic<kApplyStandalone><<<g, kNT, 0, st>>>(lo, hi, io, S); break;
        case kApplyInit: k_apply_generic<kApplyInit><<<g, kNT, 0, st>>>(lo, hi, io, S); break;
        case kApplyTemporal: k_apply_generic<kApplyTemporal><<<g, kNT, 0, st>>>(lo, hi, io, S); break;
        default: k_apply_generic<kApplyFused><<<g, kNT, 0, st>>>(lo, hi, io, S); break;
    }
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

}  // namespace mpbjac
