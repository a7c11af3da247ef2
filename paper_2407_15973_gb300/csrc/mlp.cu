// Learned per-block format selector (an extension of the paper's Section 4.5 feature
// analysis: block features -> storage format). Inference reads BF16-rounded weights and
// accumulates in binary32; one warp evaluates one block's 12 features.
#include "common.cuh"
#include "mlp.cuh"

namespace mpbjac {

constexpr int kMlpNT = 256;

struct MlpSmem {
    float w1t[kFeat][kH1];   // transposed: [in][out], conflict-free across lanes
    float b1[kH1];
    float w2t[kH1][kH2];
    float b2[kH2];
    float w3[kCls][kH2];
    float b3[kCls];
    float mu[kFeat], sd[kFeat];
};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ void load_weights(MlpSmem &m, const float *p, int bf16_weights) {
    for (int t = threadIdx.x; t < kH1 * kFeat; t += blockDim.x) {
        const int o = t / kFeat, k = t % kFeat;
        const float v = p[kOffW1 + t];
        m.w1t[k][o] = bf16_weights ? bf16r(v) : v;
    }
    for (int t = threadIdx.x; t < kH2 * kH1; t += blockDim.x) {
        const int o = t / kH1, i = t % kH1;
        const float v = p[kOffW2 + t];
        m.w2t[i][o] = bf16_weights ? bf16r(v) : v;
    }
    for (int t = threadIdx.x; t < kCls * kH2; t += blockDim.x) {
        const float v = p[kOffW3 + t];
        m.w3[t / kH2][t % kH2] = bf16_weights ? bf16r(v) : v;
    }
    for (int t = threadIdx.x; t < kH1; t += blockDim.x) m.b1[t] = bf16_weights ? bf16r(p[kOffB1 + t]) : p[kOffB1 + t];
    for (int t = threadIdx.x; t < kH2; t += blockDim.x) m.b2[t] = bf16_weights ? bf16r(p[kOffB2 + t]) : p[kOffB2 + t];
    for (int t = threadIdx.x; t < kCls; t += blockDim.x) m.b3[t] = bf16_weights ? bf16r(p[kOffB3 + t]) : p[kOffB3 + t];
    for (int t = threadIdx.x; t < kFeat; t += blockDim.x) {
        m.mu[t] = p[kOffMu + t];
        m.sd[t] = p[kOffSd + t];
    }
}

// Forward pass of one sample by one warp. x: standardised features (lane k < 12 holds x_k).
// Returns logits in every lane; h1/h2 (two units per lane: lane, lane + 32) optional.
__device__ __forceinline__ void mlp_forward_warp(const MlpSmem &m, float xk, float lg[kCls], float *h1o = nullptr,
                                                 float *h2o = nullptr) {
    const int lane = threadIdx.x & 31;
    float a0 = m.b1[lane], a1 = m.b1[lane + 32];
#pragma unroll
    for (int k = 0; k < kFeat; ++k) {
        const float xv = __shfl_sync(0xffffffffu, xk, k);
        a0 = fmaf(m.w1t[k][lane], xv, a0);
        a1 = fmaf(m.w1t[k][lane + 32], xv, a1);
    }
    const float h10 = fmaxf(a0, 0.0f), h11 = fmaxf(a1, 0.0f);
    float c0 = m.b2[lane], c1 = m.b2[lane + 32];
#pragma unroll 8
    for (int i = 0; i < kH1; ++i) {
        const float hv = __shfl_sync(0xffffffffu, i < 32 ? h10 : h11, i & 31);
        c0 = fmaf(m.w2t[i][lane], hv, c0);
        c1 = fmaf(m.w2t[i][lane + 32], hv, c1);
    }
    const float h20 = fmaxf(c0, 0.0f), h21 = fmaxf(c1, 0.0f);
#pragma unroll
    for (int c = 0; c < kCls; ++c) {
        float v = fmaf(m.w3[c][lane], h20, m.w3[c][lane + 32] * h21);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        lg[c] = v + m.b3[c];
    }
    if (h1o) { h1o[0] = h10; h1o[1] = h11; }
    if (h2o) { h2o[0] = h20; h2o[1] = h21; }
}

__device__ __forceinline__ float standardise(const MlpSmem &m, const double *f, int lane) {
    return lane < kFeat ? (float)((f[lane] - (double)m.mu[lane]) / (double)m.sd[lane]) : 0.0f;
}

__global__ void __launch_bounds__(kMlpNT) k_mlp_select(const float *params, int nb, const double *feat,
                                                       const double *kap, double safety, uint8_t *fmt) {
    __shared__ MlpSmem m;
    load_weights(m, params, 1);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * kMlpNT + threadIdx.x) >> 5, nw = (gridDim.x * kMlpNT) >> 5;
    const double l2 = 0.30102999566398120;
    for (int b = gw; b < nb; b += nw) {
        const float xk = standardise(m, feat + (size_t)b * kFeat, lane);
        float lg[kCls];
        mlp_forward_warp(m, xk, lg);
        if (lane == 0) {
            int cls = 0;
            for (int c = 1; c < kCls; ++c)
                if (lg[c] > lg[cls]) cls = c;
            const double lk = kap[2 * b], ldr = kap[2 * b + 1];
            // class -> format; 16-bit is binary16 when the dynamic range fits, else bfloat16
            int f = cls == 0 ? BJAC_FP64 : cls == 1 ? BJAC_FP32 : (ldr <= 29 * l2 ? BJAC_FP16S : BJAC_BF16);
            const double ls = log10(safety);
            // safety: promote until kappa_1 * u_f <= safety_theta (never demotes)
            if (f == BJAC_FP16S && lk - 11 * l2 > ls) f = BJAC_FP32;
            if (f == BJAC_BF16 && lk - 8 * l2 > ls) f = BJAC_FP32;
            if (f == BJAC_FP32 && lk - 24 * l2 > ls) f = BJAC_FP64;
            fmt[b] = (uint8_t)f;
        }
    }
}

int launch_mlp_select(const float *params, int nb, const double *feat, const double *kap, double safety_theta,
                      uint8_t *fmt, cudaStream_t st) {
    float *dp = nullptr;
    MPB_CUDA(cudaMallocAsync((void **)&dp, sizeof(float) * kMlpParams, st));
    MPB_CUDA(cudaMemcpyAsync(dp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
    int g = (nb + kMlpNT / 32 - 1) / (kMlpNT / 32);
    if (g > sm_count() * 4) g = sm_count() * 4;
    if (g < 1) g = 1;
    k_mlp_select<<<g, kMlpNT, 0, st>>>(dp, nb, feat, kap, safety_theta, fmt);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(dp, st);
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_select");
    return MPBJAC_OK;
}

}  // namespace mpbjac
