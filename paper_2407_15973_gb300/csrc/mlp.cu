// Learned per-block format selector (an extension of the paper's Section 4.5 feature
// analysis: block features -> storage format), evaluated on the tensor cores.
//
// One CTA of 128 threads takes tiles of 128 blocks (one sample per thread and per TMEM lane):
//   layer 1 (12 -> 64, ReLU)  CUDA cores, binary32 FMA chains, weights rounded to bfloat16;
//   layer 2 (64 -> 64)        tcgen05 MMA, M = 128 samples, N = 64, K = 64, FP32 accumulators
//                             in TMEM. The weights are bfloat16 already; each hidden value h1
//                             is split into bfloat16 parts hi = bf16(h1), lo = bf16(h1 - hi), and
//                             the two products hi W2^T + lo W2^T are accumulated, so h1 enters
//                             with about 16 significant bits instead of 8 (relative error of
//                             the split <= 2^-17) and the logits stay within binary32 rounding
//                             of the CUDA-core forward pass;
//   bias, ReLU, layer 3 (64 -> 3) and the class -> format choice: CUDA cores, after a TMEM load.
#include "common.cuh"
#include "mlp.cuh"
#include "tc.cuh"

namespace mpbjac {

constexpr int kTcM = 128;                 // samples per tile = TMEM lanes
constexpr int kTcNT = 128;                // one thread per sample
constexpr uint32_t kTcCols = 64;          // TMEM columns: layer 2's 64 FP32 outputs
constexpr uint32_t kLbo = 128, kSbo = kH1 * 16;

struct MlpTcSmem {
    alignas(1024) uint16_t a_hi[kTcM * kH1];   // A operands: h1 split, core-matrix layout
    alignas(1024) uint16_t a_lo[kTcM * kH1];
    alignas(1024) uint16_t w2[kH2 * kH1];      // B operand: W2 (row = output, K = input)
    float w1t[kFeat][kH1];
    float b1[kH1], b2[kH2], w3[kCls][kH2], b3[kCls];
    float mu[kFeat], sd[kFeat];
    uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// class -> storage format: 16-bit is binary16 when the dynamic range fits, else bfloat16; then
// promote until kappa_1 * u_f <= safety_theta (never demotes). lk, ldr: log10 kappa_1 and
// log10 of the dynamic range.
__device__ __forceinline__ uint8_t format_of_class(int cls, double lk, double ldr, double safety) {
    const double l2 = 0.30102999566398120;
    int f = cls == 0 ? BJAC_FP64 : cls == 1 ? BJAC_FP32 : (ldr <= 29 * l2 ? BJAC_FP16S : BJAC_BF16);
    const double ls = log10(safety);
    if (f == BJAC_FP16S && lk - 11 * l2 > ls) f = BJAC_FP32;
    if (f == BJAC_BF16 && lk - 8 * l2 > ls) f = BJAC_FP32;
    if (f == BJAC_FP32 && lk - 24 * l2 > ls) f = BJAC_FP64;
    return (uint8_t)f;
}

// SELECT: fmt[b] for every block; else logits[3 b + c]. A tile whose MMA does not complete
// within the bounded wait, and every later tile of that CTA, is marked (fmt 0xFF, NaN logits).
template <bool SELECT>
__global__ void __launch_bounds__(kTcNT) k_mlp_tc(const float *params, int nb, const double *feat, const double *kap,
                                                   double safety, uint8_t *fmt, float *logits) {
    __shared__ MlpTcSmem s;
    const int t = threadIdx.x, warp = t >> 5;
    for (int e = t; e < kH2 * kH1; e += kTcNT)
        s.w2[tc::core_off(e / kH1, e % kH1, kH1) >> 1] = bf16_bits(params[kOffW2 + e]);
    for (int e = t; e < kH1 * kFeat; e += kTcNT) s.w1t[e % kFeat][e / kFeat] = bf16r(params[kOffW1 + e]);
    for (int e = t; e < kCls * kH2; e += kTcNT) s.w3[e / kH2][e % kH2] = bf16r(params[kOffW3 + e]);
    if (t < kH1) s.b1[t] = bf16r(params[kOffB1 + t]);
    if (t < kH2) s.b2[t] = bf16r(params[kOffB2 + t]);
    if (t < kCls) s.b3[t] = bf16r(params[kOffB3 + t]);
    if (t < kFeat) {
        s.mu[t] = params[kOffMu + t];
        s.sd[t] = params[kOffSd + t];
    }
    if (t == 0) {
        mbar_init(&s.bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&s.tmem, kTcCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = s.tmem;
    const uint32_t a_hi = smem_u32(s.a_hi), a_lo = smem_u32(s.a_lo), bw = smem_u32(s.w2);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, kH2);
    const int ntiles = (int)(((long long)nb + kTcM - 1) / kTcM);
    unsigned phase = 0;
    int tile = blockIdx.x;
    bool failed = false;
    for (; tile < ntiles; tile += gridDim.x) {
        const long long b = (long long)tile * kTcM + t;
        float x[kFeat];
#pragma unroll
        for (int k = 0; k < kFeat; ++k)
            x[k] = b < nb ? (float)((feat[(size_t)b * kFeat + k] - (double)s.mu[k]) / (double)s.sd[k]) : 0.0f;
        // layer 1, eight hidden units (one K chunk of the A operands) at a time
#pragma unroll 1
        for (int j = 0; j < kH1 / 8; ++j) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float hv[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int o = 8 * j + e + q;
                    float a = s.b1[o];
#pragma unroll
                    for (int k = 0; k < kFeat; ++k) a = fmaf(s.w1t[k][o], x[k], a);
                    hv[q] = fmaxf(a, 0.0f);
                }
                const uint16_t h0 = bf16_bits(hv[0]), h1 = bf16_bits(hv[1]);
                const float r0 = hv[0] - __bfloat162float(__ushort_as_bfloat16(h0));   // exact
                const float r1 = hv[1] - __bfloat162float(__ushort_as_bfloat16(h1));
                hi[e >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                lo[e >> 1] = (uint32_t)bf16_bits(r0) | ((uint32_t)bf16_bits(r1) << 16);
            }
            const uint32_t off = tc::core_off(t, 8 * j, kH1);
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(s.a_hi) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(s.a_lo) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        tc::fence_proxy_async();   // the A stores (and, on the first tile, W2) -> tensor core
        tc::fence_before_sync();   // the previous tile's TMEM loads are done before the next MMA
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kH1 / 16; ++kk)
                tc::mma_bf16(tm, tc::sdesc(a_hi + 256 * kk, kLbo, kSbo), tc::sdesc(bw + 256 * kk, kLbo, kSbo), idesc,
                             kk > 0);
#pragma unroll
            for (int kk = 0; kk < kH1 / 16; ++kk)
                tc::mma_bf16(tm, tc::sdesc(a_lo + 256 * kk, kLbo, kSbo), tc::sdesc(bw + 256 * kk, kLbo, kSbo), idesc, 1);
            tc::commit(&s.bar);
        }
        const bool ok = mbar_wait_bounded(&s.bar, phase);
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        float acc0[32], acc1[32];    // this thread's TMEM lane: layer-2 outputs 0..31, 32..63
        tc::ld_32cols(tm + ((uint32_t)(32 * warp) << 16), acc0);
        tc::ld_32cols(tm + ((uint32_t)(32 * warp) << 16) + 32, acc1);
        float lg[kCls];
#pragma unroll
        for (int c = 0; c < kCls; ++c) {
            float v = 0.0f;
#pragma unroll
            for (int o = 0; o < kH2; ++o) {
                const float h2 = fmaxf((o < 32 ? acc0[o] : acc1[o - 32]) + s.b2[o], 0.0f);
                v = fmaf(s.w3[c][o], h2, v);
            }
            lg[c] = v + s.b3[c];
        }
        if (b < nb) {
            if (SELECT) {
                int cls = 0;
                for (int c = 1; c < kCls; ++c)
                    if (lg[c] > lg[cls]) cls = c;
                fmt[b] = format_of_class(cls, kap[2 * b], kap[2 * b + 1], safety);
            } else {
#pragma unroll
                for (int c = 0; c < kCls; ++c) logits[(size_t)b * kCls + c] = lg[c];
            }
        }
    }
    if (failed) {
        // the MMAs of this tile may still be running: wait for them (bounded) before TMEM is
        // freed, and mark this tile and the CTA's later ones as not evaluated
        if (t == 0) (void)mbar_wait_bounded(&s.bar, phase);
        for (; tile < ntiles; tile += gridDim.x) {
            const long long b = (long long)tile * kTcM + t;
            if (b >= nb) continue;
            if (SELECT) fmt[b] = 0xFF;
            else
                for (int c = 0; c < kCls; ++c) logits[(size_t)b * kCls + c] = __int_as_float(0x7fc00000);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, kTcCols);
}

static int mlp_tc_grid(int nb) {
    long long g = ((long long)nb + kTcM - 1) / kTcM;
    if (g > sm_count() * 4) g = sm_count() * 4;
    return g < 1 ? 1 : (int)g;
}

int launch_mlp_select(const float *params, int nb, const double *feat, const double *kap, double safety_theta,
                      uint8_t *fmt, cudaStream_t st) {
    float *dp = nullptr;
    MPB_CUDA(cudaMallocAsync((void **)&dp, sizeof(float) * kMlpParams, st));
    MPB_CUDA(cudaMemcpyAsync(dp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
    k_mlp_tc<true><<<mlp_tc_grid(nb), kTcNT, 0, st>>>(dp, nb, feat, kap, safety_theta, fmt, nullptr);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(dp, st);
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_tc");
    return MPBJAC_OK;
}

int launch_mlp_logits_tc(const float *dparams, int n, const double *feat, float *logits, cudaStream_t st) {
    k_mlp_tc<false><<<mlp_tc_grid(n), kTcNT, 0, st>>>(dparams, n, feat, nullptr, 1.0, nullptr, logits);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

}  // namespace mpbjac
