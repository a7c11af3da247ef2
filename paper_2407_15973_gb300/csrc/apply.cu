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
//  * k_apply_generic: one warp per block, any block size 1..128, any mix of formats; rows
//    that are 16-byte aligned are read with vector loads by the lane that owns them.
//  * k_apply_tma: all blocks of one size (32 or 64) and one low format. Persistent
//    CTAs stream groups of consecutive blocks (plus the matching slices of r and q)
//    through a ring of shared-memory stages filled by cp.async.bulk (TMA bulk copies)
//    that complete on mbarriers; every wait is bounded.
#include "common.cuh"
#include "apply.cuh"
#include "rows.cuh"
#include "tma.cuh"

namespace mpbjac {

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
__global__ void __launch_bounds__(kNT, 3) k_apply_generic(PSet lo, PSet hi, ApplyIO io, SolverState *S) {
    pdl_enter();
    __shared__ __align__(16) double s_r[kWarps][128];
    __shared__ __align__(16) float s_rh[kWarps][128];
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
    // alpha from the state: in front of this kernel the loop SpMV finishes p.q and alpha
    // itself (kSpPcgAlpha). Summing its partials here (loop_alpha) made this kernel 15 %
    // slower on binary32 / 16-bit sets of uneven blocks, for a reason not found.
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
            s_rh[warp][i] = f64_to_f32_rn(rv);
        }
        __syncwarp();
        const int f = __ldg(P.fmt + b);
        const uint8_t *base = P.pool + __ldg(P.qoff + b);
        const float sc = __ldg(P.scale + b);
        const int eb = f == BJAC_FP64 ? 8 : f == BJAC_FP32 ? 4 : 2;
        if (((bs * eb) & 15) == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0) {
            // rows are 16-byte aligned: lane-owns-row vector loads
            const int vpr = bs * eb / 16;
            const uint4 *Q4 = reinterpret_cast<const uint4 *>(base);
            for (int i = lane; i < bs; i += 32) {
                const uint4 *row = Q4 + (size_t)i * vpr;
                double zi;
                if (f == BJAC_FP64) {
                    zi = vec_row_f64(row, vpr, s_r[warp]);
                } else {
                    float acc;
                    if (f == BJAC_FP32) acc = vec_row_low<float>(row, vpr, s_rh[warp]);
                    else if (f == BJAC_BF16) acc = vec_row_low<__nv_bfloat16>(row, vpr, s_rh[warp]);
                    else acc = vec_row_low<__half>(row, vpr, s_rh[warp]);
                    zi = f32_to_f64(acc * sc);
                }
                io.z[s + i] = zi;
                if (MODE == kApplyInit) io.p[s + i] = zi;
                rho = fma(s_r[warp][i], zi, rho);
            }
            __syncwarp();
            continue;
        }
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
                zi = f32_to_f64(acc * sc);
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
// Each warp runs its own pipeline: a ring of kS shared-memory stages, each holding one
// block's inverse plus the block's slices of r (and q in the fused loop), filled by TMA
// bulk copies that lane 0 issues and that complete on the stage's mbarrier. Warps never
// wait for one another, so the only sync in the loop is __syncwarp.
template <typename QT, int BS>
struct TmaGeom {
    static constexpr int kQBytes = BS * BS * (int)sizeof(QT);
    static constexpr int kStageBytes = kQBytes + 2 * BS * 8;        // Q, r slice, q slice
    static constexpr int kBudget = 200 * 1024;
    static constexpr int kS = (kBudget / (3 * kStageBytes) >= 4) ? 3 : 2;
    static constexpr int kNWraw = kBudget / (kS * kStageBytes);
    static constexpr int kNW = kNWraw > 16 ? 16 : kNWraw;             // warps per CTA
    static constexpr int kThreads = kNW * 32;
    static constexpr int kBarBytes = ((kNW * kS * 8 + 127) / 128) * 128;
    static constexpr int kRhBytes = kNW * BS * 4;
    static constexpr int kHeader = kBarBytes + kRhBytes;
    static constexpr int kSmem = kHeader + kNW * kS * kStageBytes;
    static_assert(kNW >= 2, "stage too large");
    static_assert(kHeader % 16 == 0, "stage alignment");
};

template <typename QT, int BS, int MODE>
__global__ void __launch_bounds__(TmaGeom<QT, BS>::kThreads, 1) k_apply_tma(PSet P, ApplyIO io, SolverState *S,
                                                                            int n) {
    pdl_enter();
    using Geo = TmaGeom<QT, BS>;
    constexpr int RPL = BS / 32;     // rows per lane
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ double s_red[2][Geo::kNW];
    __shared__ int s_bad;

    if (MODE != kApplyStandalone) {
        if (S->state != kRunning) return;
        if (MODE == kApplyTemporal || MODE == kApplyInit) {
            if (!S->use_low) return;     // the binary64 set runs in the generic kernel
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem) + warp * Geo::kS;
    float *rh = reinterpret_cast<float *>(smem + Geo::kBarBytes) + warp * BS;
    uint8_t *stages = smem + Geo::kHeader + (size_t)warp * Geo::kS * Geo::kStageBytes;
    const int nb = P.nb;
    const int gw = blockIdx.x * Geo::kNW + warp, nw = gridDim.x * Geo::kNW;
    double alpha = 0.0;     // (before any copy is issued: a CTA may leave here)
    if (MODE == kApplyFused && !loop_alpha(S, io.spart, alpha)) return;
    const bool with_q = (MODE == kApplyFused);
    const unsigned vbytes = BS * 8;
    const unsigned tx = Geo::kQBytes + vbytes * (with_q ? 2u : 1u);

    auto issue = [&](int blk, int s) {
        uint8_t *dst = stages + (size_t)s * Geo::kStageBytes;
        mbar_expect_tx(&bars[s], tx);
        bulk_g2s(dst, P.pool + (size_t)blk * Geo::kQBytes, Geo::kQBytes, &bars[s]);
        bulk_g2s(dst + Geo::kQBytes, io.r + (size_t)blk * BS, vbytes, &bars[s]);
        if (with_q) bulk_g2s(dst + Geo::kQBytes + vbytes, io.q + (size_t)blk * BS, vbytes, &bars[s]);
    };

    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    if (lane == 0) {
        for (int s = 0; s < Geo::kS; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int s = 0; s < Geo::kS; ++s) {
            const int blk = gw + s * nw;
            if (blk < nb) issue(blk, s);
        }
    }
    __syncwarp();

    double rho = 0.0, rr = 0.0;
    bool ok = true;
    int it = 0;
    for (int blk = gw; blk < nb; blk += nw, ++it) {
        const int s = it % Geo::kS;
        const unsigned phase = (unsigned)((it / Geo::kS) & 1);
        const uint8_t *st = stages + (size_t)s * Geo::kStageBytes;
        const float sc = (sizeof(QT) == 2) ? __ldg(P.scale + blk) : 1.0f;   // issued before the wait
        ok = mbar_wait_bounded(&bars[s], phase);
        if (__any_sync(0xffffffffu, !ok)) { ok = false; break; }
        const double *sr = reinterpret_cast<const double *>(st + Geo::kQBytes);
        const double *sq = reinterpret_cast<const double *>(st + Geo::kQBytes + vbytes);
        double rv[RPL];
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
            const int i = h * 32 + lane;
            double v = sr[i];
            if (MODE == kApplyFused) v = fma(-alpha, sq[i], v);
            rv[h] = v;
            rh[i] = f64_to_f32_rn(v);
        }
        __syncwarp();
        const QT *Q = reinterpret_cast<const QT *>(st);
        const float4 *rh4 = reinterpret_cast<const float4 *>(rh);
        float acc[RPL];
#pragma unroll
        for (int h = 0; h < RPL; ++h) acc[h] = 0.0f;
#pragma unroll
        for (int j4 = 0; j4 < BS / 4; ++j4) {
            const float4 r4 = rh4[j4];
#pragma unroll
            for (int h = 0; h < RPL; ++h) {
                const int i = h * 32 + lane;
                acc[h] = fmaf(to_f32<QT>(Q[(4 * j4 + 0) * BS + i]), r4.x, acc[h]);
                acc[h] = fmaf(to_f32<QT>(Q[(4 * j4 + 1) * BS + i]), r4.y, acc[h]);
                acc[h] = fmaf(to_f32<QT>(Q[(4 * j4 + 2) * BS + i]), r4.z, acc[h]);
                acc[h] = fmaf(to_f32<QT>(Q[(4 * j4 + 3) * BS + i]), r4.w, acc[h]);
            }
        }
        __syncwarp();   // stage s and rh fully consumed by every lane
        if (lane == 0) {
            const int nxt = blk + Geo::kS * nw;
            if (nxt < nb) issue(nxt, s);
        }
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
            const size_t row = (size_t)blk * BS + h * 32 + lane;
            const double zi = f32_to_f64(acc[h] * sc);
            io.z[row] = zi;
            if (MODE == kApplyInit) io.p[row] = zi;
            if (MODE == kApplyFused) {
                io.r_out[row] = rv[h];
                rr = fma(rv[h], rv[h], rr);
            }
            rho = fma(rv[h], zi, rho);
        }
    }
    if (!ok) {
        // drain this warp's copies still in flight (bounded), then record the failure
        if (lane == 0) {
            for (int k = 0; k < Geo::kS; ++k) {
                const int itk = it + k;
                if (gw + itk * nw < nb) (void)mbar_wait_bounded(&bars[itk % Geo::kS], (unsigned)((itk / Geo::kS) & 1));
            }
            s_bad = 1;
        }
    }
    (void)n;
    // CTA reduction in fixed order (warp sums, then warps in index order)
    rho = warp_sum(rho);
    rr = warp_sum(rr);
    if (lane == 0) {
        s_red[0][warp] = rho;
        s_red[1][warp] = rr;
    }
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) {
            if (io.err) atomicExch(io.err, MPBJAC_ERR_TIMEOUT);
            if (MODE != kApplyStandalone) S->state = kBreakdown;
        }
        return;   // every thread of the CTA sees s_bad after the barrier
    }
    if (MODE == kApplyStandalone && io.out == nullptr) return;
    if (threadIdx.x == 0) {
        double b1 = 0.0, b2 = 0.0;
        for (int w = 0; w < Geo::kNW; ++w) {
            b1 += s_red[0][w];
            b2 += s_red[1][w];
        }
        io.part[2 * blockIdx.x] = b1;
        io.part[2 * blockIdx.x + 1] = b2;
    }
    if (!last_cta(io.ticket)) return;
    double t1 = 0.0, t2 = 0.0;
    if (threadIdx.x == 0) {
        for (int c = 0; c < (int)gridDim.x; ++c) {
            t1 += __ldcg(io.part + 2 * c);
            t2 += __ldcg(io.part + 2 * c + 1);
        }
        apply_finish<MODE>(t1, t2, io, S, 1);
    }
}

// ----------------------------------------------------------------------------------------
// register-direct uniform kernel: because every block is symmetric, row i of a block is also
// its column i, so lane i loads its own row with 16-byte loads (the whole block arrives in one
// round of coalesced-by-sector loads) and keeps it in registers; r-hat is shared through a
// small per-warp buffer. The next block's row, r and q are loaded before the current block is
// computed (two blocks in flight per warp). No TMA, no shared-memory copy of Q, no CTA sync.
// ----------------------------------------------------------------------------------------
template <typename QT, int BS, int MODE, bool FLEX = false>
__global__ void __launch_bounds__(kNT, sizeof(QT) == 2 ? 4 : 3) k_apply_reg(PSet P, ApplyIO io, SolverState *S) {
    using Geo = RegGeom<QT, BS>;
    constexpr int RPL = Geo::kRPL, VPR = Geo::kVPR, EPV = Geo::kEPV;
    __shared__ __align__(16) float s_rh[kWarps][BS];
    __shared__ double s_red[(MODE == kApplyFused && FLEX ? 3 : 2) * kNT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = P.nb;
    const int gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;
    const size_t blk_bytes = (size_t)BS * BS * sizeof(QT);

    uint4 qc[RPL][VPR], qn[RPL][VPR];
    double rc[RPL], rn[RPL], vc[RPL], vn[RPL];
    float sc_c = 1.0f, sc_n = 1.0f;
    // the inverse rows of a block (and its scale) do not change during a solve
    auto load_q = [&](int blk, uint4 (&qv)[RPL][VPR], float &sc) {
        const uint4 *base = reinterpret_cast<const uint4 *>(P.pool + (size_t)blk * blk_bytes);
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
#pragma unroll
            for (int v = 0; v < VPR; ++v) qv[h][v] = __ldcs(base + (size_t)(h * 32 + lane) * VPR + v);
        }
        if (sizeof(QT) == 2) sc = __ldg(P.scale + blk);
    };
    if (gw < nb) load_q(gw, qc, sc_c);       // before the wait: overlaps the predecessor's tail
    pdl_enter();
    if (MODE != kApplyStandalone) {
        if (S->state != kRunning) return;
        if (MODE == kApplyTemporal || MODE == kApplyInit) {
            if (!S->use_low) return;     // the binary64 set runs in the generic kernel
        }
    }
    const uint64_t pol = vec_policy(MODE != kApplyStandalone ? S->l2_keep : 0);
    auto load_v = [&](int blk, double (&rv)[RPL], double (&qq)[RPL]) {
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
            const int row = h * 32 + lane;
            rv[h] = ld_vec(io.r + (size_t)blk * BS + row, pol);
            if (MODE == kApplyFused) qq[h] = ld_vec(io.q + (size_t)blk * BS + row, pol);
        }
    };
    constexpr bool flex = MODE == kApplyFused && FLEX;
    double rho = 0.0, rr = 0.0, qz = 0.0;     // qz = q.z for the flexible beta
    if (gw < nb) load_v(gw, rc, vc);          // r and q do not depend on alpha: in flight meanwhile
    double alpha = 0.0;
    if (MODE == kApplyFused && !loop_alpha(S, io.spart, alpha)) return;
    for (int blk = gw; blk < nb; blk += nw) {
        const int nxt = blk + nw;
        if (nxt < nb) {
            load_q(nxt, qn, sc_n);
            load_v(nxt, rn, vn);
        }
        double rv[RPL];
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
            double v = rc[h];
            if (MODE == kApplyFused) v = fma(-alpha, vc[h], v);
            rv[h] = v;
            s_rh[warp][h * 32 + lane] = f64_to_f32_rn(v);
        }
        __syncwarp();
        const float4 *rh4 = reinterpret_cast<const float4 *>(s_rh[warp]);
        float acc[RPL];
#pragma unroll
        for (int h = 0; h < RPL; ++h) acc[h] = 0.0f;
#pragma unroll
        for (int v = 0; v < VPR; ++v) {
#pragma unroll
            for (int e4 = 0; e4 < EPV; e4 += 4) {
                const float4 r4 = rh4[(v * EPV + e4) >> 2];
#pragma unroll
                for (int h = 0; h < RPL; ++h) {
                    acc[h] = fmaf(vec_entry<QT>(qc[h][v], e4 + 0), r4.x, acc[h]);
                    acc[h] = fmaf(vec_entry<QT>(qc[h][v], e4 + 1), r4.y, acc[h]);
                    acc[h] = fmaf(vec_entry<QT>(qc[h][v], e4 + 2), r4.z, acc[h]);
                    acc[h] = fmaf(vec_entry<QT>(qc[h][v], e4 + 3), r4.w, acc[h]);
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
            const size_t row = (size_t)blk * BS + h * 32 + lane;
            const double zi = f32_to_f64(acc[h] * sc_c);
            st_vec(io.z + row, zi, pol);
            if (MODE == kApplyInit) st_vec(io.p + row, zi, pol);
            if (MODE == kApplyFused) {
                st_vec(io.r_out + row, rv[h], pol);
                rr = fma(rv[h], rv[h], rr);
                if (flex) qz = fma(vc[h], zi, qz);
            }
            rho = fma(rv[h], zi, rho);
        }
        // rotate the prefetched block into place
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
#pragma unroll
            for (int v = 0; v < VPR; ++v) qc[h][v] = qn[h][v];
            rc[h] = rn[h];
            vc[h] = vn[h];
        }
        sc_c = sc_n;
    }
    // rho, r.r and (flexible CG) q.z: partials in io.part with stride nv
    double b[3] = {0.0, 0.0, 0.0};
    if (flex) {
        const double v[3] = {rho, rr, qz};
        cta_sum_to0<kNT, 3>(v, s_red, b);
    } else {
        const double v[2] = {rho, rr};
        double b2[2];
        cta_sum_to0<kNT, 2>(v, s_red, b2);
        b[0] = b2[0];
        b[1] = b2[1];
    }
    if (MODE == kApplyStandalone && io.out == nullptr) return;
    const int nv = flex ? 3 : 2;
    if (threadIdx.x == 0)
        for (int k = 0; k < nv; ++k) io.part[nv * blockIdx.x + k] = b[k];
    if (!last_cta(io.ticket)) return;
    double t[3] = {0.0, 0.0, 0.0};
    if constexpr (flex) {
        reduce_partials_to0<kNT, 3>(io.part, gridDim.x, nv, s_red, t);
    } else {
        double t2[2];
        reduce_partials_to0<kNT, 2>(io.part, gridDim.x, nv, s_red, t2);
        t[0] = t2[0];
        t[1] = t2[1];
    }
    if (threadIdx.x == 0) apply_finish<MODE>(t[0], t[1], io, S, 1, flex, t[2]);
}

// ----------------------------------------------------------------------------------------
// register kernel for 32-row blocks of mixed formats (per-block rule or learned selection):
// one block per warp iteration, the block's format the same for the whole warp. Every lane
// issues all loads of its own row (row i of a symmetric block is its column i) before it
// touches r, so one memory round trip serves the block; binary64 blocks of such a set read
// their rows two vectors at a time. Same arithmetic, in the same order, as the other kernels.
// ----------------------------------------------------------------------------------------
template <typename QT>
__device__ __forceinline__ float mix_row(const uint4 (&q)[8], const float *rh) {
    constexpr int EPV = 16 / (int)sizeof(QT);
    constexpr int VPR = 32 / EPV;
    const float4 *rh4 = reinterpret_cast<const float4 *>(rh);
    float a = 0.0f;
#pragma unroll
    for (int v = 0; v < VPR; ++v) {
#pragma unroll
        for (int e4 = 0; e4 < EPV; e4 += 4) {
            const float4 r4 = rh4[(v * EPV + e4) >> 2];
            a = fmaf(vec_entry<QT>(q[v], e4 + 0), r4.x, a);
            a = fmaf(vec_entry<QT>(q[v], e4 + 1), r4.y, a);
            a = fmaf(vec_entry<QT>(q[v], e4 + 2), r4.z, a);
            a = fmaf(vec_entry<QT>(q[v], e4 + 3), r4.w, a);
        }
    }
    return a;
}

template <int MODE, bool FLEX = false>
__global__ void __launch_bounds__(kNT, 3) k_apply_mix32(PSet P, ApplyIO io, SolverState *S) {
    pdl_enter();
    __shared__ __align__(16) float s_rh[kWarps][32];
    __shared__ __align__(16) double s_r[kWarps][32];
    __shared__ double s_red[(MODE == kApplyFused && FLEX ? 3 : 2) * kNT];
    if (MODE != kApplyStandalone) {
        if (S->state != kRunning) return;
        if (MODE == kApplyTemporal || MODE == kApplyInit) {
            if (!S->use_low) return;     // the binary64 set runs in the generic kernel
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;
    double alpha = 0.0;
    if (MODE == kApplyFused && !loop_alpha(S, io.spart, alpha)) return;
    const uint64_t pol = vec_policy(MODE != kApplyStandalone ? S->l2_keep : 0);
    constexpr bool flex = MODE == kApplyFused && FLEX;
    double rho = 0.0, rr = 0.0, qz = 0.0;     // qz = q.z for the flexible beta
    for (int blk = gw; blk < P.nb; blk += nw) {
        const int f = __ldg(P.fmt + blk);
        const uint4 *base = reinterpret_cast<const uint4 *>(P.pool + __ldg(P.qoff + blk));
        const float sc = __ldg(P.scale + blk);
        const size_t row = (size_t)blk * 32 + lane;
        uint4 q[8];
        const int vpr = f == BJAC_FP32 ? 8 : 4;
        if (f != BJAC_FP64) {
#pragma unroll
            for (int v = 0; v < 8; ++v)
                if (v < vpr) q[v] = __ldcs(base + (size_t)lane * vpr + v);
        }
        double v = ld_vec(io.r + row, pol), qi = 0.0;
        if (MODE == kApplyFused) {
            qi = ld_vec(io.q + row, pol);
            v = fma(-alpha, qi, v);
        }
        s_r[warp][lane] = v;
        s_rh[warp][lane] = f64_to_f32_rn(v);
        __syncwarp();
        double zi;
        if (f == BJAC_FP64) {
            zi = vec_row_f64(base + (size_t)lane * 16, 16, s_r[warp]);
        } else {
            float acc;
            if (f == BJAC_FP32) acc = mix_row<float>(q, s_rh[warp]);
            else if (f == BJAC_BF16) acc = mix_row<__nv_bfloat16>(q, s_rh[warp]);
            else acc = mix_row<__half>(q, s_rh[warp]);
            zi = f32_to_f64(acc * sc);
        }
        st_vec(io.z + row, zi, pol);
        if (MODE == kApplyInit) st_vec(io.p + row, zi, pol);
        if (MODE == kApplyFused) {
            st_vec(io.r_out + row, v, pol);
            rr = fma(v, v, rr);
            if (flex) qz = fma(qi, zi, qz);
        }
        rho = fma(v, zi, rho);
        __syncwarp();
    }
    // rho, r.r and (flexible CG) q.z: partials in io.part with stride nv
    double b[3] = {0.0, 0.0, 0.0};
    if (flex) {
        const double v[3] = {rho, rr, qz};
        cta_sum_to0<kNT, 3>(v, s_red, b);
    } else {
        const double v[2] = {rho, rr};
        double b2[2];
        cta_sum_to0<kNT, 2>(v, s_red, b2);
        b[0] = b2[0];
        b[1] = b2[1];
    }
    if (MODE == kApplyStandalone && io.out == nullptr) return;
    const int nv = flex ? 3 : 2;
    if (threadIdx.x == 0)
        for (int k = 0; k < nv; ++k) io.part[nv * blockIdx.x + k] = b[k];
    if (!last_cta(io.ticket)) return;
    double t[3] = {0.0, 0.0, 0.0};
    if constexpr (flex) {
        reduce_partials_to0<kNT, 3>(io.part, gridDim.x, nv, s_red, t);
    } else {
        double t2[2];
        reduce_partials_to0<kNT, 2>(io.part, gridDim.x, nv, s_red, t2);
        t[0] = t2[0];
        t[1] = t2[1];
    }
    if (threadIdx.x == 0) apply_finish<MODE>(t[0], t[1], io, S, 1, flex, t[2]);
}

// ----------------------------------------------------------------------------------------
// aMP (Algorithms 3.2 / 3.3) without a separate residual-update kernel. The set of an
// application depends on the relres of the residual it preconditions, which is known only
// after a grid-wide sum; so the application after iteration k is made speculatively with the
// set of the previous application (the choice changes a few times per solve at most), fused
// with r -= alpha q as in fMP, and the last CTA compares that set with the one the exact
// relres picks. If they agree, rho and beta are committed; if not, S->redo is raised and the
// kApplyRedo launch that follows applies the right set to the updated r (the speculative z
// and rho are discarded). A committed application is the same arithmetic, in the same order,
// as in the separate kernels. Blocks of 32 rows: the low set of one format (lane i keeps its
// row of the next block in registers, as in k_apply_reg), the binary64 set by 16-byte pairs.
// ----------------------------------------------------------------------------------------
template <typename QT, int MODE, bool FLEX>
__global__ void __launch_bounds__(kNT, sizeof(QT) == 2 ? 4 : 3) k_apply_spec(PSet lo, PSet hi, ApplyIO io,
                                                                            SolverState *S) {
    pdl_enter();
    using Geo = RegGeom<QT, 32>;
    constexpr int VPR = Geo::kVPR, EPV = Geo::kEPV;
    constexpr int NV = FLEX ? 3 : 2;
    constexpr bool SPEC = MODE == kApplySpec;
    __shared__ __align__(16) float s_rh[kWarps][32];
    __shared__ __align__(16) double s_r[kWarps][32];
    __shared__ double s_red[3 * kNT];
    if (S->state != kRunning) return;
    if (!SPEC && !S->redo) return;
    const int use_low = S->use_low;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = lo.nb;
    const int gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;
    double alpha = 0.0;
    if (SPEC && !loop_alpha(S, io.spart, alpha)) return;
    const uint64_t pol = vec_policy(S->l2_keep);
    const double *__restrict__ q = io.q;
    double *__restrict__ r = io.r_out;
    double *__restrict__ z = io.z;
    double rho = 0.0, rr = 0.0, qz = 0.0;
    if (use_low) {
        const size_t blk_bytes = (size_t)32 * 32 * sizeof(QT);
        uint4 qc[VPR], qn[VPR];
        double rc = 0.0, rn = 0.0, vc = 0.0, vn = 0.0;
        float sc_c = 1.0f, sc_n = 1.0f;
        auto load = [&](int blk, uint4 (&qv)[VPR], double &rv, double &qq, float &sc) {
            const uint4 *base = reinterpret_cast<const uint4 *>(lo.pool + (size_t)blk * blk_bytes);
#pragma unroll
            for (int v = 0; v < VPR; ++v) qv[v] = __ldcs(base + (size_t)lane * VPR + v);
            const size_t row = (size_t)blk * 32 + lane;
            rv = ld_vec(r + row, pol);
            if (SPEC || FLEX) qq = ld_vec(q + row, pol);
            if (sizeof(QT) == 2) sc = __ldg(lo.scale + blk);
        };
        if (gw < nb) load(gw, qc, rc, vc, sc_c);
        for (int blk = gw; blk < nb; blk += nw) {
            const int nxt = blk + nw;
            if (nxt < nb) load(nxt, qn, rn, vn, sc_n);
            const double v = SPEC ? fma(-alpha, vc, rc) : rc;
            s_rh[warp][lane] = f64_to_f32_rn(v);
            __syncwarp();
            const float4 *rh4 = reinterpret_cast<const float4 *>(s_rh[warp]);
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < VPR; ++k) {
#pragma unroll
                for (int e4 = 0; e4 < EPV; e4 += 4) {
                    const float4 r4 = rh4[(k * EPV + e4) >> 2];
                    acc = fmaf(vec_entry<QT>(qc[k], e4 + 0), r4.x, acc);
                    acc = fmaf(vec_entry<QT>(qc[k], e4 + 1), r4.y, acc);
                    acc = fmaf(vec_entry<QT>(qc[k], e4 + 2), r4.z, acc);
                    acc = fmaf(vec_entry<QT>(qc[k], e4 + 3), r4.w, acc);
                }
            }
            __syncwarp();
            const size_t row = (size_t)blk * 32 + lane;
            const double zi = f32_to_f64(acc * sc_c);
            st_vec(z + row, zi, pol);
            if (SPEC) {
                st_vec(r + row, v, pol);
                rr = fma(v, v, rr);
            }
            if (FLEX) qz = fma(vc, zi, qz);
            rho = fma(v, zi, rho);
#pragma unroll
            for (int k = 0; k < VPR; ++k) qc[k] = qn[k];
            rc = rn;
            vc = vn;
            sc_c = sc_n;
        }
    } else {
        for (int blk = gw; blk < nb; blk += nw) {
            const size_t row = (size_t)blk * 32 + lane;
            double v = ld_vec(r + row, pol), qi = 0.0;
            if (SPEC || FLEX) qi = ld_vec(q + row, pol);
            if (SPEC) v = fma(-alpha, qi, v);
            s_r[warp][lane] = v;
            __syncwarp();
            const uint4 *base = reinterpret_cast<const uint4 *>(hi.pool + __ldg(hi.qoff + blk));
            const double zi = vec_row_f64(base + (size_t)lane * 16, 16, s_r[warp]);
            __syncwarp();
            st_vec(z + row, zi, pol);
            if (SPEC) {
                st_vec(r + row, v, pol);
                rr = fma(v, v, rr);
            }
            if (FLEX) qz = fma(qi, zi, qz);
            rho = fma(v, zi, rho);
        }
    }
    double b[3] = {0.0, 0.0, 0.0};
    if (FLEX) {
        const double v3[3] = {rho, rr, qz};
        cta_sum_to0<kNT, 3>(v3, s_red, b);
    } else {
        const double v2[2] = {rho, rr};
        double b2[2];
        cta_sum_to0<kNT, 2>(v2, s_red, b2);
        b[0] = b2[0];
        b[1] = b2[1];
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NV; ++k) io.part[NV * blockIdx.x + k] = b[k];
    if (!last_cta(io.ticket)) return;
    double tv[NV];
    reduce_partials_to0<kNT, NV>(io.part, gridDim.x, NV, s_red, tv);
    if (threadIdx.x != 0) return;
    const double t_rho = tv[0], t_rr = SPEC ? tv[1] : 0.0, t_qz = FLEX ? tv[NV - 1] : 0.0;
    if (SPEC) {
        // the recurrence residual of this iteration: relres, convergence, the set it picks
        S->iter += 1;
        S->x_pending = 1;
        const double rel = sqrt(t_rr) / S->bnorm;
        S->relres = rel;
        S->rr = t_rr;
        if (S->hist) S->hist[S->iter] = rel;
        if (!(rel < 1.0e308)) { S->state = kBreakdown; return; }
        if (rel <= S->tol) { S->state = kConverged; return; }
        if (S->iter >= S->maxit) { S->state = kMaxit; return; }
        const int want = choose_low(S, rel);
        if (want != use_low) {
            S->use_low = want;
            S->redo = 1;
            return;
        }
    } else {
        S->redo = 0;
    }
    if (use_low) S->low_applies += 1;
    else S->high_applies += 1;
    if (!finite_pos(t_rho)) { S->state = kBreakdown; return; }
    double beta = t_rho / S->rho;
    if (FLEX && S->flexible) beta = -S->alpha * t_qz / S->rho;
    if (!(fabs(beta) < 1.0e308)) { S->state = kBreakdown; return; }
    S->beta = beta;
    S->rho_prev = S->rho;
    S->rho = t_rho;
}

// ----------------------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------------------
// resident CTAs of the generic kernel (one wave), at most the blocks' warps
template <int MODE>
static int generic_grid(int nb) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_generic<MODE>, kNT, 0) != cudaSuccess || v < 1)
            v = 1;
        per_sm = v;
    }
    const int need = (nb + kWarps - 1) / kWarps;
    int g = sm_count() * per_sm;
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
    int g = sm_count();
    const int need = (P.nb + Geo::kNW - 1) / Geo::kNW;
    if (g > need) g = need;
    if (g < 1) g = 1;
    MPB_CUDA(launch_kernel(k_apply_tma<QT, BS, MODE>, g, Geo::kThreads, Geo::kSmem, st, P, io, S, n));
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

template <typename QT, int BS, int MODE, bool FLEX = false>
static int launch_reg_t(const PSet &P, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_reg<QT, BS, MODE, FLEX>, kNT, 0) != cudaSuccess || v < 1)
            v = 1;
        per_sm = v;
    }
    int g = sm_count() * per_sm;
    const int need = (P.nb + kWarps - 1) / kWarps;
    if (g > need) g = need;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g < 1) g = 1;
    MPB_CUDA(launch_kernel(k_apply_reg<QT, BS, MODE, FLEX>, g, kNT, 0, st, P, io, S));
    return MPBJAC_OK;
}

template <int MODE, bool FLEX = false>
static int launch_reg_mode(const PSet &P, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    switch (P.ufmt * 1000 + P.ubs) {
        case BJAC_FP32 * 1000 + 32: return launch_reg_t<float, 32, MODE, FLEX>(P, io, S, st);
        case BJAC_BF16 * 1000 + 32: return launch_reg_t<__nv_bfloat16, 32, MODE, FLEX>(P, io, S, st);
        case BJAC_FP16S * 1000 + 32: return launch_reg_t<__half, 32, MODE, FLEX>(P, io, S, st);
        default: return fail(MPBJAC_ERR_UNSUPPORTED, "no register apply kernel for this format / block size");
    }
}

template <int MODE, bool FLEX = false>
static int launch_mix_t(const PSet &P, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_mix32<MODE, FLEX>, kNT, 0) != cudaSuccess || v < 1)
            v = 1;
        per_sm = v;
    }
    int g = sm_count() * per_sm;
    const int need = (P.nb + kWarps - 1) / kWarps;
    if (g > need) g = need;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g < 1) g = 1;
    MPB_CUDA(launch_kernel(k_apply_mix32<MODE, FLEX>, g, kNT, 0, st, P, io, S));
    return MPBJAC_OK;
}

bool mix_supported(const PSet &P, int n) { return P.ubs == 32 && (long long)P.nb * 32 == n; }

template <typename QT, int MODE, bool FLEX>
static int launch_spec_t(const PSet &lo, const PSet &hi, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_spec<QT, MODE, FLEX>, kNT, 0) != cudaSuccess ||
            v < 1)
            v = 1;
        per_sm = v;
    }
    int g = sm_count() * per_sm;
    const int need = (lo.nb + kWarps - 1) / kWarps;
    if (g > need) g = need;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g < 1) g = 1;
    MPB_CUDA(launch_kernel(k_apply_spec<QT, MODE, FLEX>, g, kNT, 0, st, lo, hi, io, S));
    return MPBJAC_OK;
}

template <int MODE, bool FLEX>
static int launch_spec_mode(const PSet &lo, const PSet &hi, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    switch (lo.ufmt) {
        case BJAC_FP32: return launch_spec_t<float, MODE, FLEX>(lo, hi, io, S, st);
        case BJAC_BF16: return launch_spec_t<__nv_bfloat16, MODE, FLEX>(lo, hi, io, S, st);
        case BJAC_FP16S: return launch_spec_t<__half, MODE, FLEX>(lo, hi, io, S, st);
        default: return fail(MPBJAC_ERR_UNSUPPORTED, "no speculative aMP apply kernel for this format");
    }
}

bool spec_supported(const PSet &lo, const PSet &hi, int n) {
    return reg_supported(lo, n) && hi.ufmt == BJAC_FP64 && hi.ubs == 32 && (long long)hi.nb * 32 == n;
}

int launch_apply_spec(int mode, const PSet &lo, const PSet &hi, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    if (mode == kApplySpec)
        return io.flex ? launch_spec_mode<kApplySpec, true>(lo, hi, io, S, st)
                       : launch_spec_mode<kApplySpec, false>(lo, hi, io, S, st);
    if (mode == kApplyRedo)
        return io.flex ? launch_spec_mode<kApplyRedo, true>(lo, hi, io, S, st)
                       : launch_spec_mode<kApplyRedo, false>(lo, hi, io, S, st);
    return fail(MPBJAC_ERR_INVALID_ARG, "launch_apply_spec takes kApplySpec or kApplyRedo");
}

int launch_apply_mix(int mode, const PSet &P, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    switch (mode) {
        case kApplyStandalone: return launch_mix_t<kApplyStandalone>(P, io, S, st);
        case kApplyInit: return launch_mix_t<kApplyInit>(P, io, S, st);
        case kApplyTemporal: return launch_mix_t<kApplyTemporal>(P, io, S, st);
        default:
            return io.flex ? launch_mix_t<kApplyFused, true>(P, io, S, st) : launch_mix_t<kApplyFused>(P, io, S, st);
    }
}

bool reg_supported(const PSet &P, int n) {
    return tma_supported(P, n) && P.ubs == 32;
}

int launch_apply_reg(int mode, const PSet &P, const ApplyIO &io, SolverState *S, cudaStream_t st) {
    switch (mode) {
        case kApplyStandalone: return launch_reg_mode<kApplyStandalone>(P, io, S, st);
        case kApplyInit: return launch_reg_mode<kApplyInit>(P, io, S, st);
        case kApplyTemporal: return launch_reg_mode<kApplyTemporal>(P, io, S, st);
        default:
            return io.flex ? launch_reg_mode<kApplyFused, true>(P, io, S, st) : launch_reg_mode<kApplyFused>(P, io, S, st);
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
    switch (mode) {
        case kApplyStandalone:
            MPB_CUDA(launch_kernel(k_apply_generic<kApplyStandalone>, generic_grid<kApplyStandalone>(nb), kNT, 0, st,
                                   lo, hi, io, S));
            break;
        case kApplyInit:
            MPB_CUDA(launch_kernel(k_apply_generic<kApplyInit>, generic_grid<kApplyInit>(nb), kNT, 0, st, lo, hi, io,
                                   S));
            break;
        case kApplyTemporal:
            MPB_CUDA(launch_kernel(k_apply_generic<kApplyTemporal>, generic_grid<kApplyTemporal>(nb), kNT, 0, st, lo,
                                   hi, io, S));
            break;
        default:
            MPB_CUDA(launch_kernel(k_apply_generic<kApplyFused>, generic_grid<kApplyFused>(nb), kNT, 0, st, lo, hi,
                                   io, S));
            break;
    }
    return MPBJAC_OK;
}

}  // namespace mpbjac
