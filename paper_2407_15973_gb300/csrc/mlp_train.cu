// Training of the per-block format selector on the GPU: forward and backward passes of the
// 12-64-64-3 ReLU MLP with a softmax cross-entropy loss, full-batch Adam on binary32 master
// weights. The forward pass reads weights rounded to bfloat16 (the weights inference uses)
// or the binary32 masters (bf16_weights = 0); gradients are taken with respect to the
// weights actually used and applied to the masters.
//
// The bfloat16-weight gradient runs on the tensor cores (mlp_grad_tc.cu); the kernel below
// serves the binary32 weights and, for comparison, the bfloat16 weights on CUDA cores.
//
// Determinism: one warp handles samples gw, gw + nw, ... in a fixed order and accumulates
// their gradient in its own shared-memory slice (each lane owns distinct entries, so no
// atomics); the slices are written out and summed over warps in index order.
#include <vector>

#include "common.cuh"
#include "mlp.cuh"

namespace mpbjac {

constexpr int kTrainWarps = 4;
constexpr int kTrainNT = kTrainWarps * 32;

struct TrainW {
    float w1t[kFeat][kH1];
    float b1[kH1];
    float w2t[kH1][kH2];
    float b2[kH2];
    float w3[kCls][kH2];
    float b3[kCls];
    float mu[kFeat], sd[kFeat];
};

__device__ __forceinline__ float maybe_bf16(float v, int bf16) { return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v; }

// partial[w][kMlpWeights] receives warp w's gradient sum; loss_part[w] its loss sum
__global__ void __launch_bounds__(kTrainNT) k_mlp_grad(const float *params, int bf16, const double *feat,
                                                       const int32_t *label, int N, float *partial,
                                                       double *loss_part) {
    __shared__ TrainW m;
    extern __shared__ float gsm[];                      // kTrainWarps * kMlpWeights
    for (int t = threadIdx.x; t < kH1 * kFeat; t += kTrainNT) m.w1t[t % kFeat][t / kFeat] = maybe_bf16(params[kOffW1 + t], bf16);
    for (int t = threadIdx.x; t < kH2 * kH1; t += kTrainNT) m.w2t[t % kH1][t / kH1] = maybe_bf16(params[kOffW2 + t], bf16);
    for (int t = threadIdx.x; t < kCls * kH2; t += kTrainNT) m.w3[t / kH2][t % kH2] = maybe_bf16(params[kOffW3 + t], bf16);
    for (int t = threadIdx.x; t < kH1; t += kTrainNT) m.b1[t] = maybe_bf16(params[kOffB1 + t], bf16);
    for (int t = threadIdx.x; t < kH2; t += kTrainNT) m.b2[t] = maybe_bf16(params[kOffB2 + t], bf16);
    for (int t = threadIdx.x; t < kCls; t += kTrainNT) m.b3[t] = maybe_bf16(params[kOffB3 + t], bf16);
    for (int t = threadIdx.x; t < kFeat; t += kTrainNT) {
        m.mu[t] = params[kOffMu + t];
        m.sd[t] = params[kOffSd + t];
    }
    for (int t = threadIdx.x; t < kTrainWarps * kMlpWeights; t += kTrainNT) gsm[t] = 0.0f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kTrainWarps + warp, nw = gridDim.x * kTrainWarps;
    float *g = gsm + warp * kMlpWeights;
    float *gW1 = g + kOffW1, *gb1 = g + kOffB1, *gW2 = g + kOffW2, *gb2 = g + kOffB2, *gW3 = g + kOffW3,
          *gb3 = g + kOffB3;
    const float inv_n = 1.0f / (float)N;
    double loss = 0.0;
    for (long long s = gw; s < N; s += nw) {
        const float xk = lane < kFeat ? (float)((feat[(size_t)s * kFeat + lane] - (double)m.mu[lane]) / (double)m.sd[lane])
                                      : 0.0f;
        // forward: two hidden units per lane (o = lane, lane + 32)
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
        float lg[kCls];
#pragma unroll
        for (int c = 0; c < kCls; ++c) {
            float v = fmaf(m.w3[c][lane], h20, m.w3[c][lane + 32] * h21);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            lg[c] = v + m.b3[c];
        }
        // softmax cross-entropy: d3 = (softmax - onehot) / N
        const int y = label[s];
        float mx = lg[0];
#pragma unroll
        for (int c = 1; c < kCls; ++c) mx = fmaxf(mx, lg[c]);
        float e[kCls], z = 0.0f;
#pragma unroll
        for (int c = 0; c < kCls; ++c) {
            e[c] = expf(lg[c] - mx);
            z += e[c];
        }
        if (lane == 0) loss += -(double)(lg[y] - mx - logf(z));
        float d3[kCls];
#pragma unroll
        for (int c = 0; c < kCls; ++c) d3[c] = (e[c] / z - (c == y ? 1.0f : 0.0f)) * inv_n;
        // layer 3 gradients and back-propagation to h2
        float d20 = 0.0f, d21 = 0.0f;
#pragma unroll
        for (int c = 0; c < kCls; ++c) {
            gW3[c * kH2 + lane] += d3[c] * h20;
            gW3[c * kH2 + lane + 32] += d3[c] * h21;
            d20 = fmaf(m.w3[c][lane], d3[c], d20);
            d21 = fmaf(m.w3[c][lane + 32], d3[c], d21);
        }
        if (lane < kCls) gb3[lane] += d3[lane];
        d20 = h20 > 0.0f ? d20 : 0.0f;
        d21 = h21 > 0.0f ? d21 : 0.0f;
        // layer 2: gW2[o][i] += d2[o] h1[i]; d1[i] = sum_o W2[o][i] d2[o]
        gb2[lane] += d20;
        gb2[lane + 32] += d21;
        float e0 = 0.0f, e1 = 0.0f;    // d1 for i = lane, lane + 32
#pragma unroll 4
        for (int i = 0; i < kH1; ++i) {
            const float hv = __shfl_sync(0xffffffffu, i < 32 ? h10 : h11, i & 31);
            gW2[lane * kH1 + i] += d20 * hv;
            gW2[(lane + 32) * kH1 + i] += d21 * hv;
        }
#pragma unroll 4
        for (int o = 0; o < kH2; ++o) {
            const float dv = __shfl_sync(0xffffffffu, o < 32 ? d20 : d21, o & 31);
            e0 = fmaf(m.w2t[lane][o], dv, e0);
            e1 = fmaf(m.w2t[lane + 32][o], dv, e1);
        }
        e0 = h10 > 0.0f ? e0 : 0.0f;
        e1 = h11 > 0.0f ? e1 : 0.0f;
        gb1[lane] += e0;
        gb1[lane + 32] += e1;
#pragma unroll
        for (int k = 0; k < kFeat; ++k) {
            const float xv = __shfl_sync(0xffffffffu, xk, k);
            gW1[lane * kFeat + k] += e0 * xv;
            gW1[(lane + 32) * kFeat + k] += e1 * xv;
        }
    }
    __syncwarp();
    float *out = partial + (size_t)gw * kMlpWeights;
    for (int j = lane; j < kMlpWeights; j += 32) out[j] = g[j];
    if (lane == 0) loss_part[gw] = loss;
}

// grad[j] = sum over warps (index order); optional Adam step on the masters
__global__ void k_mlp_reduce_adam(const float *partial, int nwarps, float *grad, float *params, float *m1, float *m2,
                                  float lr, float b1, float b2, float eps, int step, int do_step) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kMlpWeights) return;
    float gsum = 0.0f;
    for (int w = 0; w < nwarps; ++w) gsum += partial[(size_t)w * kMlpWeights + j];
    grad[j] = gsum;
    if (!do_step) return;
    const float a = b1 * m1[j] + (1.0f - b1) * gsum;
    const float v = b2 * m2[j] + (1.0f - b2) * gsum * gsum;
    m1[j] = a;
    m2[j] = v;
    const float ah = a / (1.0f - powf(b1, (float)step));
    const float vh = v / (1.0f - powf(b2, (float)step));
    params[j] -= lr * ah / (sqrtf(vh) + eps);
}

static int grad_launch(int N) {
    long long g = ((long long)N + kTrainWarps - 1) / kTrainWarps;
    const int cap = sm_count() * 4;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// partial gradients (kMlpWeights floats each) that the gradient pass of `mode` writes
static int grad_parts(int mode, int N) { return mode == 1 ? mlp_grad_tc_grid(N) : grad_launch(N) * kTrainWarps; }

// one gradient pass: mode 0 binary32 weights, 1 bfloat16 weights on the tensor cores, 2 bfloat16
// weights on CUDA cores; dpart / dloss hold grad_parts(mode, N) entries
static int grad_pass(int mode, const float *dp, const double *feat, const int32_t *label, int N, float *dpart,
                     double *dloss, cudaStream_t st) {
    if (mode == 1) return launch_mlp_grad_tc(dp, feat, label, N, dpart, dloss, mlp_grad_tc_grid(N), st);
    static bool attr = false;
    const size_t smem = sizeof(float) * kTrainWarps * kMlpWeights;
    if (!attr) {
        MPB_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    k_mlp_grad<<<grad_launch(N), kTrainNT, smem, st>>>(dp, mode ? 1 : 0, feat, label, N, dpart, dloss);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

}  // namespace mpbjac

using namespace mpbjac;

extern "C" int bjac_mlp_grad(const float *params, int32_t bf16_weights, const double *feat, const int32_t *label,
                             int32_t N, float *grad, float *loss, void *stream) {
    if (!params || !feat || !label || !grad || N < 1 || bf16_weights < 0 || bf16_weights > 2)
        return fail(MPBJAC_ERR_INVALID_ARG, "bad MLP gradient arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int nparts = grad_parts(bf16_weights, N);
    float *dp = nullptr, *dpart = nullptr, *dgrad = nullptr;
    double *dloss = nullptr;
    MPB_CUDA(cudaMallocAsync((void **)&dp, sizeof(float) * kMlpParams, st));
    MPB_CUDA(cudaMallocAsync((void **)&dpart, sizeof(float) * (size_t)nparts * kMlpWeights, st));
    MPB_CUDA(cudaMallocAsync((void **)&dgrad, sizeof(float) * kMlpWeights, st));
    MPB_CUDA(cudaMallocAsync((void **)&dloss, sizeof(double) * nparts, st));
    MPB_CUDA(cudaMemcpyAsync(dp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
    int rc = grad_pass(bf16_weights, dp, feat, label, N, dpart, dloss, st);
    if (rc != MPBJAC_OK) return rc;
    k_mlp_reduce_adam<<<(kMlpWeights + 255) / 256, 256, 0, st>>>(dpart, nparts, dgrad, nullptr, nullptr, nullptr, 0, 0, 0,
                                                                 0, 0, 0);
    MPB_CUDA(cudaGetLastError());
    std::vector<double> hl(nparts);
    MPB_CUDA(cudaMemcpyAsync(grad, dgrad, sizeof(float) * kMlpWeights, cudaMemcpyDeviceToHost, st));
    MPB_CUDA(cudaMemcpyAsync(hl.data(), dloss, sizeof(double) * nparts, cudaMemcpyDeviceToHost, st));
    MPB_CUDA(cudaStreamSynchronize(st));
    double l = 0.0;
    for (double v : hl) l += v;
    if (loss) *loss = (float)(l / N);
    cudaFreeAsync(dp, st);
    cudaFreeAsync(dpart, st);
    cudaFreeAsync(dgrad, st);
    cudaFreeAsync(dloss, st);
    MPB_CUDA(cudaStreamSynchronize(st));
    if (l != l) return fail(MPBJAC_ERR_TIMEOUT, "MLP gradient MMA did not complete");
    return MPBJAC_OK;
}

extern "C" int bjac_mlp_train(float *params, const double *feat, const int32_t *label, int32_t N, int32_t epochs,
                              float lr, float *loss_hist, void *stream) {
    if (!params || !feat || !label || N < 1 || epochs < 1 || !(lr > 0.0f))
        return fail(MPBJAC_ERR_INVALID_ARG, "bad MLP training arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int nwarps = grad_parts(1, N);
    float *dp = nullptr, *dpart = nullptr, *dgrad = nullptr, *m1 = nullptr, *m2 = nullptr;
    double *dloss = nullptr;
    MPB_CUDA(cudaMallocAsync((void **)&dp, sizeof(float) * kMlpParams, st));
    MPB_CUDA(cudaMallocAsync((void **)&dpart, sizeof(float) * (size_t)nwarps * kMlpWeights, st));
    MPB_CUDA(cudaMallocAsync((void **)&dgrad, sizeof(float) * kMlpWeights, st));
    MPB_CUDA(cudaMallocAsync((void **)&m1, sizeof(float) * kMlpWeights, st));
    MPB_CUDA(cudaMallocAsync((void **)&m2, sizeof(float) * kMlpWeights, st));
    MPB_CUDA(cudaMallocAsync((void **)&dloss, sizeof(double) * nwarps, st));
    MPB_CUDA(cudaMemcpyAsync(dp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
    MPB_CUDA(cudaMemsetAsync(m1, 0, sizeof(float) * kMlpWeights, st));
    MPB_CUDA(cudaMemsetAsync(m2, 0, sizeof(float) * kMlpWeights, st));
    std::vector<double> hl(nwarps);
    for (int ep = 1; ep <= epochs; ++ep) {
        const int rc = grad_pass(1, dp, feat, label, N, dpart, dloss, st);
        if (rc != MPBJAC_OK) return rc;
        k_mlp_reduce_adam<<<(kMlpWeights + 255) / 256, 256, 0, st>>>(dpart, nwarps, dgrad, dp, m1, m2, lr, 0.9f, 0.999f,
                                                                     1e-8f, ep, 1);
        MPB_CUDA(cudaGetLastError());
        if (loss_hist) {
            MPB_CUDA(cudaMemcpyAsync(hl.data(), dloss, sizeof(double) * nwarps, cudaMemcpyDeviceToHost, st));
            MPB_CUDA(cudaStreamSynchronize(st));
            double l = 0.0;
            for (double v : hl) l += v;
            loss_hist[ep - 1] = (float)(l / N);
            if (l != l) return fail(MPBJAC_ERR_TIMEOUT, "MLP gradient MMA did not complete");
        }
    }
    MPB_CUDA(cudaMemcpyAsync(params, dp, sizeof(float) * kMlpWeights, cudaMemcpyDeviceToHost, st));
    MPB_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(dp, st);
    cudaFreeAsync(dpart, st);
    cudaFreeAsync(dgrad, st);
    cudaFreeAsync(m1, st);
    cudaFreeAsync(m2, st);
    cudaFreeAsync(dloss, st);
    MPB_CUDA(cudaStreamSynchronize(st));
    return MPBJAC_OK;
}

// Logits of the selector for N feature rows on CUDA cores (binary32 or bfloat16-rounded weights);
// the tensor-core forward pass is in mlp.cu.
__global__ void k_mlp_logits(const float *params, int bf16, const double *feat, int N, float *out) {
    __shared__ TrainW m;
    for (int t = threadIdx.x; t < kH1 * kFeat; t += blockDim.x) m.w1t[t % kFeat][t / kFeat] = maybe_bf16(params[kOffW1 + t], bf16);
    for (int t = threadIdx.x; t < kH2 * kH1; t += blockDim.x) m.w2t[t % kH1][t / kH1] = maybe_bf16(params[kOffW2 + t], bf16);
    for (int t = threadIdx.x; t < kCls * kH2; t += blockDim.x) m.w3[t / kH2][t % kH2] = maybe_bf16(params[kOffW3 + t], bf16);
    for (int t = threadIdx.x; t < kH1; t += blockDim.x) m.b1[t] = maybe_bf16(params[kOffB1 + t], bf16);
    for (int t = threadIdx.x; t < kH2; t += blockDim.x) m.b2[t] = maybe_bf16(params[kOffB2 + t], bf16);
    for (int t = threadIdx.x; t < kCls; t += blockDim.x) m.b3[t] = maybe_bf16(params[kOffB3 + t], bf16);
    for (int t = threadIdx.x; t < kFeat; t += blockDim.x) {
        m.mu[t] = params[kOffMu + t];
        m.sd[t] = params[kOffSd + t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (long long s = gw; s < N; s += nw) {
        const float xk = lane < kFeat ? (float)((feat[(size_t)s * kFeat + lane] - (double)m.mu[lane]) / (double)m.sd[lane])
                                      : 0.0f;
        float a0 = m.b1[lane], a1 = m.b1[lane + 32];
        for (int k = 0; k < kFeat; ++k) {
            const float xv = __shfl_sync(0xffffffffu, xk, k);
            a0 = fmaf(m.w1t[k][lane], xv, a0);
            a1 = fmaf(m.w1t[k][lane + 32], xv, a1);
        }
        const float h10 = fmaxf(a0, 0.0f), h11 = fmaxf(a1, 0.0f);
        float c0 = m.b2[lane], c1 = m.b2[lane + 32];
        for (int i = 0; i < kH1; ++i) {
            const float hv = __shfl_sync(0xffffffffu, i < 32 ? h10 : h11, i & 31);
            c0 = fmaf(m.w2t[i][lane], hv, c0);
            c1 = fmaf(m.w2t[i][lane + 32], hv, c1);
        }
        const float h20 = fmaxf(c0, 0.0f), h21 = fmaxf(c1, 0.0f);
        for (int c = 0; c < kCls; ++c) {
            float v = fmaf(m.w3[c][lane], h20, m.w3[c][lane + 32] * h21);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) out[(size_t)s * kCls + c] = v + m.b3[c];
        }
    }
}

extern "C" int bjac_mlp_logits(const float *params, int32_t bf16_weights, const double *feat, int32_t N, float *logits,
                               void *stream) {
    if (!params || !feat || !logits || N < 1 || bf16_weights < 0 || bf16_weights > 2)
        return fail(MPBJAC_ERR_INVALID_ARG, "bad MLP inference arguments");
    cudaStream_t st = (cudaStream_t)stream;
    float *dp = nullptr, *dout = nullptr;
    MPB_CUDA(cudaMallocAsync((void **)&dp, sizeof(float) * kMlpParams, st));
    MPB_CUDA(cudaMallocAsync((void **)&dout, sizeof(float) * (size_t)N * kCls, st));
    MPB_CUDA(cudaMemcpyAsync(dp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
    if (bf16_weights == 1) {
        const int rc = launch_mlp_logits_tc(dp, N, feat, dout, st);
        if (rc != MPBJAC_OK) return rc;
    } else {
        long long g = ((long long)N + 7) / 8;
        if (g > sm_count() * 4) g = sm_count() * 4;
        k_mlp_logits<<<(int)g, 256, 0, st>>>(dp, bf16_weights ? 1 : 0, feat, N, dout);
        MPB_CUDA(cudaGetLastError());
    }
    MPB_CUDA(cudaMemcpyAsync(logits, dout, sizeof(float) * (size_t)N * kCls, cudaMemcpyDeviceToHost, st));
    MPB_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(dp, st);
    cudaFreeAsync(dout, st);
    MPB_CUDA(cudaStreamSynchronize(st));
    return MPBJAC_OK;
}
