// Gradient of the per-block selector's softmax cross-entropy on the tensor cores (tcgen05),
// for the bfloat16 weights that inference uses (the binary32-weight gradient stays on CUDA
// cores in mlp_train.cu).
//
// One CTA of 128 threads per SM takes tiles of 128 samples (one sample per thread and per TMEM
// lane). The three 64 x 64 products of layer 2 run as BF16 x BF16 -> FP32 MMAs (M = 128):
//   forward        c  = h1 W2^T            A = h1 [s][i],  B = W2 [o][i]       TMEM cols   0.. 63
//   back-prop      d1 = d2 W2              A = d2 [s][o],  B = W2^T [i][o]     TMEM cols  64..127
//   weight grad    gW2 += d2^T h1          A = d2^T [o][s] (rows 64..127 zero),
//                                          B = h1^T [i][s], K = the tile's samples,
//                                          accumulated over the CTA's tiles    TMEM cols 128..191
// Binary32 operands (h1, d2) enter as two bfloat16 parts (hi = bf16(v), lo = bf16(v - hi));
// the weight gradient takes hi.hi + hi.lo + lo.hi. Everything else (layers 1 and 3, softmax,
// the masks, the bias and W1 / W3 gradients) runs on CUDA cores; the sums over a tile's samples
// are column sums in sample order through shared memory, so the result does not depend on
// timing. Each CTA writes one partial gradient; k_mlp_reduce_adam adds them in CTA order.
#include "common.cuh"
#include "mlp.cuh"
#include "tc.cuh"

namespace mpbjac {

constexpr int kGM = 128;                           // samples per tile = TMEM lanes
constexpr int kGNT = 128;
constexpr uint32_t kGCols = 256;                   // TMEM columns (three 64-column products)
constexpr int kNG = kMlpWeights - kH2 * kH1;       // gradient entries outside W2 (1,091)
constexpr int kStageW = 80;                        // row stride of the per-sample staging buffer

struct GradSmem {
    alignas(1024) uint16_t w2[kH2 * kH1];          // forward B: W2 [o][i], K = i
    alignas(1024) uint16_t w2t[kH1 * kH2];         // back-prop B: W2^T [i][o], K = o
    alignas(1024) uint16_t a_hi[kGM * kH1];        // A: h1 [s][i] (forward), then d2 [s][o]
    alignas(1024) uint16_t a_lo[kGM * kH1];
    alignas(1024) uint16_t d2t_hi[128 * kGM];      // weight-gradient A: d2^T [o][s]
    alignas(1024) uint16_t d2t_lo[128 * kGM];
    alignas(1024) uint16_t h1t_hi[kH1 * kGM];      // weight-gradient B: h1^T [i][s]
    alignas(1024) uint16_t h1t_lo[kH1 * kGM];
    float stage[kGM * kStageW];                    // per-sample vectors for the column sums
    float gacc[kNG];                               // this CTA's gradient outside W2 (grad_index)
    float w1t[kFeat][kH1];
    float b1[kH1], b2[kH2], w3[kCls][kH2], b3[kCls];
    float mu[kFeat], sd[kFeat];
    double loss[kGM];
    uint64_t bar;
    uint32_t tmem;
};

// position in the parameter vector of gacc entry j: W1 and b1 first, then b2, W3 and b3
__host__ __device__ constexpr int grad_index(int j) { return j < kOffW2 ? j : j + kH2 * kH1; }

__device__ __forceinline__ uint16_t g_bf16(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float g_bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ void g_split(float v, uint16_t &hi, uint16_t &lo) {
    hi = g_bf16(v);
    lo = g_bf16(v - __bfloat162float(__ushort_as_bfloat16(hi)));     // the difference is exact
}
__device__ __forceinline__ void g_store2(uint16_t *base, uint32_t off_bytes, uint16_t v) {
    *reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(base) + off_bytes) = v;
}

// d2 of one sample from its staged row (h2 in 0..63, d3 in 64..66): (h2 > 0) W3^T d3, the
// FMA chain over the classes in order
__device__ __forceinline__ float g_d2(const GradSmem &s, const float *row, int o) {
    float dv = 0.0f;
#pragma unroll
    for (int c = 0; c < kCls; ++c) dv = fmaf(s.w3[c][o], row[kH2 + c], dv);
    return row[o] > 0.0f ? dv : 0.0f;
}

// partial[blockIdx.x][kMlpWeights] and loss_part[blockIdx.x]: this CTA's gradient and loss
// sums. A CTA whose MMA does not complete within the bounded wait writes NaN for both.
__global__ void __launch_bounds__(kGNT, 1) k_mlp_grad_tc(const float *params, const double *feat,
                                                         const int32_t *label, int N, float *partial,
                                                         double *loss_part) {
    extern __shared__ __align__(1024) uint8_t g_raw[];
    GradSmem &s = *reinterpret_cast<GradSmem *>(g_raw);
    const int t = threadIdx.x, warp = t >> 5;
    for (int e = t; e < kH2 * kH1; e += kGNT) {
        const int o = e / kH1, i = e % kH1;
        const uint16_t w = g_bf16(params[kOffW2 + e]);
        s.w2[tc::core_off(o, i, kH1) >> 1] = w;
        s.w2t[tc::core_off(i, o, kH2) >> 1] = w;
    }
    for (int e = t; e < kH1 * kFeat; e += kGNT) s.w1t[e % kFeat][e / kFeat] = g_bf16r(params[kOffW1 + e]);
    for (int e = t; e < kCls * kH2; e += kGNT) s.w3[e / kH2][e % kH2] = g_bf16r(params[kOffW3 + e]);
    if (t < kH1) s.b1[t] = g_bf16r(params[kOffB1 + t]);
    if (t < kH2) s.b2[t] = g_bf16r(params[kOffB2 + t]);
    if (t < kCls) s.b3[t] = g_bf16r(params[kOffB3 + t]);
    if (t < kFeat) {
        s.mu[t] = params[kOffMu + t];
        s.sd[t] = params[kOffSd + t];
    }
    for (int e = t; e < kNG; e += kGNT) s.gacc[e] = 0.0f;
    // rows 64..127 of the weight-gradient A stay zero (rows 0..63 are rewritten every tile)
    for (int e = t; e < 128 * kGM / 8; e += kGNT) {
        reinterpret_cast<uint4 *>(s.d2t_hi)[e] = make_uint4(0u, 0u, 0u, 0u);
        reinterpret_cast<uint4 *>(s.d2t_lo)[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (t == 0) {
        mbar_init(&s.bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&s.tmem, kGCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = s.tmem, tlane = (uint32_t)(32 * warp) << 16;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 64);
    constexpr uint32_t kLbo = 128, kSbo64 = kH1 * 16, kSbo128 = kGM * 16;
    const uint32_t sa_hi = smem_u32(s.a_hi), sa_lo = smem_u32(s.a_lo), sw2 = smem_u32(s.w2), sw2t = smem_u32(s.w2t);
    const uint32_t sdt_hi = smem_u32(s.d2t_hi), sdt_lo = smem_u32(s.d2t_lo);
    const uint32_t sht_hi = smem_u32(s.h1t_hi), sht_lo = smem_u32(s.h1t_lo);
    const float inv_n = 1.0f / (float)N;
    const int ntiles = (N + kGM - 1) / kGM;
    unsigned phase = 0;
    bool failed = false, first_w = true;
    double loss_cta = 0.0;
    float *st = s.stage + (size_t)t * kStageW;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int smp = tile * kGM + t;
        const bool valid = smp < N;
        float x[kFeat];
#pragma unroll
        for (int k = 0; k < kFeat; ++k)
            x[k] = valid ? (float)((feat[(size_t)smp * kFeat + k] - (double)s.mu[k]) / (double)s.sd[k]) : 0.0f;
        // layer 1 (binary32 FMA chains, bias first, as the CUDA-core kernel); h1 in two parts into
        // the forward A ([s][i]) and the weight-gradient B ([i][s]); the ReLU mask as bits
        uint64_t m1 = 0;
#pragma unroll 1
        for (int j = 0; j < kH1 / 8; ++j) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                uint16_t ph[2], pl[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int o = 8 * j + e + q;
                    float a = s.b1[o];
#pragma unroll
                    for (int k = 0; k < kFeat; ++k) a = fmaf(s.w1t[k][o], x[k], a);
                    const float h = fmaxf(a, 0.0f);
                    if (h > 0.0f) m1 |= 1ull << o;
                    g_split(h, ph[q], pl[q]);
                    g_store2(s.h1t_hi, tc::core_off(o, t, kGM), ph[q]);
                    g_store2(s.h1t_lo, tc::core_off(o, t, kGM), pl[q]);
                }
                hi[e >> 1] = (uint32_t)ph[0] | ((uint32_t)ph[1] << 16);
                lo[e >> 1] = (uint32_t)pl[0] | ((uint32_t)pl[1] << 16);
            }
            const uint32_t off = tc::core_off(t, 8 * j, kH1);
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(s.a_hi) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(s.a_lo) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        // forward product c = h1 W2^T
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kH1 / 16; ++kk)
                tc::mma_bf16(tm, tc::sdesc(sa_hi + 256 * kk, kLbo, kSbo64), tc::sdesc(sw2 + 256 * kk, kLbo, kSbo64), idesc,
                             kk > 0);
#pragma unroll
            for (int kk = 0; kk < kH1 / 16; ++kk)
                tc::mma_bf16(tm, tc::sdesc(sa_lo + 256 * kk, kLbo, kSbo64), tc::sdesc(sw2 + 256 * kk, kLbo, kSbo64), idesc, 1);
            tc::commit(&s.bar);
        }
        if (!__syncthreads_and(mbar_wait_bounded(&s.bar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // h2 = relu(c + b2) into this sample's staging row
        {
            float c0[32];
            tc::ld_32cols(tm + tlane, c0);
#pragma unroll
            for (int o = 0; o < 32; ++o) st[o] = fmaxf(c0[o] + s.b2[o], 0.0f);
            tc::ld_32cols(tm + tlane + 32, c0);
#pragma unroll
            for (int o = 0; o < 32; ++o) st[32 + o] = fmaxf(c0[o] + s.b2[32 + o], 0.0f);
        }
        // layer 3 and the softmax cross-entropy: d3 = (softmax - onehot) / N
        float lg[kCls];
#pragma unroll
        for (int c = 0; c < kCls; ++c) {
            float v = 0.0f;
#pragma unroll 8
            for (int o = 0; o < kH2; ++o) v = fmaf(s.w3[c][o], st[o], v);
            lg[c] = v + s.b3[c];
        }
        const int y = valid ? label[smp] : 0;
        float mx = lg[0];
#pragma unroll
        for (int c = 1; c < kCls; ++c) mx = fmaxf(mx, lg[c]);
        float ex[kCls], z = 0.0f;
#pragma unroll
        for (int c = 0; c < kCls; ++c) {
            ex[c] = expf(lg[c] - mx);
            z += ex[c];
        }
#pragma unroll
        for (int c = 0; c < kCls; ++c) st[kH2 + c] = valid ? (ex[c] / z - (c == y ? 1.0f : 0.0f)) * inv_n : 0.0f;
        s.loss[t] = valid ? -(double)(lg[y] - mx - logf(z)) : 0.0;
        // d2 into the back-prop A ([s][o]; the forward has consumed h1) and the weight-gradient
        // A ([o][s])
#pragma unroll 1
        for (int j = 0; j < kH2 / 8; ++j) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                uint16_t ph[2], pl[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int o = 8 * j + e + q;
                    g_split(g_d2(s, st, o), ph[q], pl[q]);
                    g_store2(s.d2t_hi, tc::core_off(o, t, kGM), ph[q]);
                    g_store2(s.d2t_lo, tc::core_off(o, t, kGM), pl[q]);
                }
                hi[e >> 1] = (uint32_t)ph[0] | ((uint32_t)ph[1] << 16);
                lo[e >> 1] = (uint32_t)pl[0] | ((uint32_t)pl[1] << 16);
            }
            const uint32_t off = tc::core_off(t, 8 * j, kH2);
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(s.a_hi) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(s.a_lo) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();     // the forward product's TMEM loads are done
        __syncthreads();
        // back-prop d1 = d2 W2 and the weight gradient gW2 += d2^T h1 (hi.hi + hi.lo + lo.hi)
        if (t == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kH2 / 16; ++kk)
                tc::mma_bf16(tm + 64, tc::sdesc(sa_hi + 256 * kk, kLbo, kSbo64), tc::sdesc(sw2t + 256 * kk, kLbo, kSbo64),
                             idesc, kk > 0);
#pragma unroll
            for (int kk = 0; kk < kH2 / 16; ++kk)
                tc::mma_bf16(tm + 64, tc::sdesc(sa_lo + 256 * kk, kLbo, kSbo64), tc::sdesc(sw2t + 256 * kk, kLbo, kSbo64),
                             idesc, 1);
#pragma unroll
            for (int kk = 0; kk < kGM / 16; ++kk)
                tc::mma_bf16(tm + 128, tc::sdesc(sdt_hi + 256 * kk, kLbo, kSbo128),
                             tc::sdesc(sht_hi + 256 * kk, kLbo, kSbo128), idesc, (first_w && kk == 0) ? 0u : 1u);
#pragma unroll
            for (int kk = 0; kk < kGM / 16; ++kk)
                tc::mma_bf16(tm + 128, tc::sdesc(sdt_hi + 256 * kk, kLbo, kSbo128),
                             tc::sdesc(sht_lo + 256 * kk, kLbo, kSbo128), idesc, 1);
#pragma unroll
            for (int kk = 0; kk < kGM / 16; ++kk)
                tc::mma_bf16(tm + 128, tc::sdesc(sdt_lo + 256 * kk, kLbo, kSbo128),
                             tc::sdesc(sht_hi + 256 * kk, kLbo, kSbo128), idesc, 1);
            tc::commit(&s.bar);
        }
        first_w = false;
        // while the tensor core runs: W3 and b3 sums over the tile's samples, in sample order
        for (int q = t; q < kCls * kH2 + kCls; q += kGNT) {
            float acc = 0.0f;
            if (q < kCls * kH2) {
                const int c = q / kH2, o = q % kH2;
                for (int r = 0; r < kGM; ++r) acc = fmaf(s.stage[r * kStageW + kH2 + c], s.stage[r * kStageW + o], acc);
            } else {
                for (int r = 0; r < kGM; ++r) acc += s.stage[r * kStageW + kH2 + (q - kCls * kH2)];
            }
            s.gacc[kH1 * kFeat + kH1 + kH2 + q] += acc;     // W3 then b3 (after W1, b1, b2)
        }
        if (t == 0)
            for (int r = 0; r < kGM; ++r) loss_cta += s.loss[r];
        if (!__syncthreads_and(mbar_wait_bounded(&s.bar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // b2: the sum of d2 (recomputed from this sample's row, which nobody reads any more)
        {
            float d2[kH2];
#pragma unroll
            for (int o = 0; o < kH2; ++o) d2[o] = g_d2(s, st, o);
#pragma unroll
            for (int o = 0; o < kH2; ++o) st[o] = d2[o];
        }
        __syncthreads();
        if (t < kH2) {
            float acc = 0.0f;
            for (int r = 0; r < kGM; ++r) acc += s.stage[r * kStageW + t];
            s.gacc[kH1 * kFeat + kH1 + t] += acc;
        }
        __syncthreads();
        // d1 from TMEM, masked by h1 > 0, and x: then the b1 and W1 sums
        {
            float e0[32];
            tc::ld_32cols(tm + tlane + 64, e0);
#pragma unroll
            for (int i = 0; i < 32; ++i) st[i] = (((m1 >> i) & 1ull) && valid) ? e0[i] : 0.0f;
            tc::ld_32cols(tm + tlane + 96, e0);
#pragma unroll
            for (int i = 0; i < 32; ++i) st[32 + i] = (((m1 >> (32 + i)) & 1ull) && valid) ? e0[i] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kFeat; ++k) st[kH1 + k] = x[k];
        __syncthreads();
        for (int q = t; q < kH1 * kFeat + kH1; q += kGNT) {
            float acc = 0.0f;
            if (q < kH1 * kFeat) {
                const int i = q / kFeat, k = q % kFeat;
                for (int r = 0; r < kGM; ++r) acc = fmaf(s.stage[r * kStageW + i], s.stage[r * kStageW + kH1 + k], acc);
            } else {
                for (int r = 0; r < kGM; ++r) acc += s.stage[r * kStageW + (q - kH1 * kFeat)];
            }
            s.gacc[q] += acc;
        }
        // (the next tile's first barrier follows its layer 1, before the staging rows change)
    }
    float *out = partial + (size_t)blockIdx.x * kMlpWeights;
    if (failed) {
        // the MMAs in flight must finish (bounded) before TMEM is freed; the gradient is NaN
        if (t == 0) (void)mbar_wait_bounded(&s.bar, phase);
        for (int e = t; e < kMlpWeights; e += kGNT) out[e] = __int_as_float(0x7fc00000);
        if (t == 0) loss_part[blockIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
        __syncthreads();
        for (int q = t; q < kNG; q += kGNT) out[grad_index(q)] = s.gacc[q];
        if (warp < 2) {     // rows o = 0..63 of gW2 live in TMEM lanes 0..63
            float g0[32];
            float *row = out + kOffW2 + (size_t)t * kH1;
            tc::ld_32cols(tm + tlane + 128, g0);
#pragma unroll
            for (int i = 0; i < 32; ++i) row[i] = first_w ? 0.0f : g0[i];
            tc::ld_32cols(tm + tlane + 160, g0);
#pragma unroll
            for (int i = 0; i < 32; ++i) row[32 + i] = first_w ? 0.0f : g0[i];
        }
        if (t == 0) loss_part[blockIdx.x] = loss_cta;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, kGCols);
}

int mlp_grad_tc_grid(int N) {
    int g = (N + kGM - 1) / kGM;
    if (g > sm_count()) g = sm_count();
    return g < 1 ? 1 : g;
}

int launch_mlp_grad_tc(const float *dparams, const double *feat, const int32_t *label, int N, float *partial,
                       double *loss_part, int grid, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        MPB_CUDA(cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)));
        attr = true;
    }
    k_mlp_grad_tc<<<grid, kGNT, sizeof(GradSmem), st>>>(dparams, feat, label, N, partial, loss_part);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

}  // namespace mpbjac
