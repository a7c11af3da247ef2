// Gradient of the per-block selector's softmax cross-entropy on the tensor cores (tcgen05),
// for the bfloat16 weights that inference uses (the binary32-weight gradient stays on CUDA
// cores in mlp_train.cu).
//
// One CTA of 128 threads per SM takes tiles of 128 samples (one sample per thread and per TMEM
// lane). Every product of the backward pass with a 64-wide side runs as BF16 x BF16 -> FP32 MMAs
// with M = 128 (D = A B^T, both operands K-major):
//   forward      c   = h1 W2^T          A = h1 [s][i]                B = W2 [o][i]       TMEM   0.. 63
//   back-prop    d1  = d2 W2            A = d2 [s][o]                B = W2^T [i][o]     TMEM  64..127
//   W2, b2       gW2 += d2^T [h1 | 1]   A = T (rows 0..63 = d2^T)    B = [h1^T; 1] (N 80) TMEM 128..207
//   W3           gW3 += h2^T d3         A = T (rows 64..127 = h2^T)  B = d3^T (N 16)     TMEM 208..223
//   W1, b1       gW1 += e^T [x | 1]     A = T (rows 0..63 = e^T)     B = [x^T; 1] (N 16) TMEM 224..239
// where T is one 128 x 128 operand [row][sample] (K = the tile's samples): its rows 0..63 hold
// d2^T and later e^T (the layer-1 error, masked by h1 > 0), its rows 64..127 h2^T. An MMA over
// all 128 rows of T fills the TMEM lanes of the other half with products nobody reads. A row of
// ones in B turns the same MMA into the bias gradient (column 64 of gW2 is gb2, column 12 of
// gW1 is gb1). The weight gradients accumulate in TMEM over all of a CTA's tiles.
// Binary32 operands enter as two bfloat16 parts (hi = bf16(v), lo = bf16(v - hi)); products of
// two such operands take hi.hi + hi.lo + lo.hi, the forward and back-propagation (W2 exact in
// bfloat16) hi + lo. Layers 1 and 3, the softmax and the masks run on CUDA cores; gb3 and the
// loss are per-thread sums added in thread order at the end, so the result does not depend on
// timing. Each CTA writes one partial gradient; k_mlp_reduce_adam adds them in CTA order.
#include "common.cuh"
#include "mlp.cuh"
#include "tc.cuh"

namespace mpbjac {

constexpr int kGM = 128;                           // samples per tile = TMEM lanes
constexpr int kGNT = 128;
constexpr uint32_t kGCols = 256;                   // TMEM columns
constexpr int kSW = 65;                            // staging row stride (floats): conflict-free columns
constexpr int kNB2 = 80;                           // rows of [h1^T; 1] (N of the gW2 product)
constexpr int kNX = 16;                            // rows of [x^T; 1] and of d3^T
constexpr uint32_t kColFwd = 0, kColBack = 64, kColW2 = 128, kColW3 = 208, kColW1 = 224;

struct GradSmem {
    alignas(1024) uint16_t w2[kH2 * kH1];          // forward B: W2 [o][i], K = i
    alignas(1024) uint16_t w2t[kH1 * kH2];         // back-prop B: W2^T [i][o], K = o
    alignas(1024) uint16_t a_hi[kGM * kH1];        // A: h1 [s][i] (forward), then d2 [s][o]
    alignas(1024) uint16_t a_lo[kGM * kH1];
    alignas(1024) uint16_t t_hi[128 * kGM];        // T [row][s]: d2^T / e^T (0..63), h2^T (64..127)
    alignas(1024) uint16_t t_lo[128 * kGM];
    alignas(1024) uint16_t h1t_hi[kNB2 * kGM];     // [h1^T; ones; zeros] [i][s]
    alignas(1024) uint16_t h1t_lo[kNB2 * kGM];
    alignas(1024) uint16_t d3t_hi[kNX * kGM];      // [d3^T; zeros] [c][s]
    alignas(1024) uint16_t d3t_lo[kNX * kGM];
    alignas(1024) uint16_t xt_hi[2][kNX * kGM];    // [x^T; ones; zeros] [k][s], one per tile parity
    alignas(1024) uint16_t xt_lo[2][kNX * kGM];
    float stage[kGM * kSW];                        // [s][f]: a 64-wide operand before its transpose
    float w1t[kFeat][kH1];
    float b1[kH1], b2[kH2], w3[kCls][kH2], b3[kCls];
    float mu[kFeat], sd[kFeat];
    float gb3[kGM][kCls];
    double loss[kGM];
    uint64_t bar;
    uint32_t tmem;
};
static_assert(sizeof(GradSmem) <= 227 * 1024, "one CTA's dynamic shared memory");

__device__ __forceinline__ uint16_t g_bf16(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float g_bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ void g_split(float v, uint16_t &hi, uint16_t &lo) {
    hi = g_bf16(v);
    lo = g_bf16(v - __bfloat162float(__ushort_as_bfloat16(hi)));     // the difference is exact
}
__device__ __forceinline__ void g_store2(uint16_t *base, uint32_t off_bytes, uint16_t v) {
    *reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(base) + off_bytes) = v;
}
__device__ __forceinline__ void g_store16(uint16_t *base, uint32_t off_bytes, uint4 v) {
    *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(base) + off_bytes) = v;
}

// rows row0 .. row0 + 63 of a K-major [row][sample] operand from the staging buffer [s][f]: item
// (f, g) packs samples 8g .. 8g + 7 of row f into one 16-byte core-matrix row, hi and lo parts.
// A warp reads 32 consecutive f of one sample (stride kSW = 65: 32 different banks).
__device__ __forceinline__ void emit_t64(const float *stage, uint16_t *hi, uint16_t *lo, int row0, int t) {
#pragma unroll 2
    for (int m = 0; m < 8; ++m) {
        const int q = t + kGNT * m;
        const int f = q & 63, g = q >> 6;
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            uint16_t h0, l0, h1, l1;
            g_split(stage[(8 * g + j) * kSW + f], h0, l0);
            g_split(stage[(8 * g + j + 1) * kSW + f], h1, l1);
            h[j >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            l[j >> 1] = (uint32_t)l0 | ((uint32_t)l1 << 16);
        }
        const uint32_t off = tc::core_off(row0 + f, 8 * g, kGM);
        g_store16(hi, off, make_uint4(h[0], h[1], h[2], h[3]));
        g_store16(lo, off, make_uint4(l[0], l[1], l[2], l[3]));
    }
}

// the three products hi.hi + hi.lo + lo.hi of a K = 128 (samples) weight gradient, N rows of B
// (the loops stay rolled: unrolled, the compiler keeps every descriptor of every call live
// across the whole tile)
__device__ __forceinline__ void mma_sample_k(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                             uint32_t idesc, bool first) {
    constexpr uint32_t kLbo = 128, kSbo = kGM * 16;
#pragma unroll 1
    for (int kk = 0; kk < kGM / 16; ++kk)
        tc::mma_bf16(d, tc::sdesc(a_hi + 256 * kk, kLbo, kSbo), tc::sdesc(b_hi + 256 * kk, kLbo, kSbo), idesc,
                     (first && kk == 0) ? 0u : 1u);
#pragma unroll 1
    for (int kk = 0; kk < kGM / 16; ++kk)
        tc::mma_bf16(d, tc::sdesc(a_hi + 256 * kk, kLbo, kSbo), tc::sdesc(b_lo + 256 * kk, kLbo, kSbo), idesc, 1);
#pragma unroll 1
    for (int kk = 0; kk < kGM / 16; ++kk)
        tc::mma_bf16(d, tc::sdesc(a_lo + 256 * kk, kLbo, kSbo), tc::sdesc(b_hi + 256 * kk, kLbo, kSbo), idesc, 1);
}

// D = A B^T for K = 64 (A [s][*] in two parts, B exact in bfloat16), N = 64
__device__ __forceinline__ void mma_k64(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b) {
    constexpr uint32_t kLbo = 128, kSbo = kH1 * 16;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 64);
#pragma unroll 1
    for (int kk = 0; kk < kH1 / 16; ++kk)
        tc::mma_bf16(d, tc::sdesc(a_hi + 256 * kk, kLbo, kSbo), tc::sdesc(b + 256 * kk, kLbo, kSbo), idesc, kk > 0);
#pragma unroll 1
    for (int kk = 0; kk < kH1 / 16; ++kk)
        tc::mma_bf16(d, tc::sdesc(a_lo + 256 * kk, kLbo, kSbo), tc::sdesc(b + 256 * kk, kLbo, kSbo), idesc, 1);
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
        g_store2(s.w2, tc::core_off(o, i, kH1), w);
        g_store2(s.w2t, tc::core_off(i, o, kH2), w);
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
    // the constant rows: ones in row 64 of [h1^T; 1] and row 12 of [x^T; 1], zeros below them and
    // in rows 3..15 of d3^T (the lo parts of the ones are zero)
    {
        const uint16_t one = g_bf16(1.0f);
        for (int e = t; e < (kNB2 - kH1) * kGM; e += kGNT) {
            const int r = kH1 + e / kGM, c = e % kGM;
            g_store2(s.h1t_hi, tc::core_off(r, c, kGM), r == kH1 ? one : (uint16_t)0);
            g_store2(s.h1t_lo, tc::core_off(r, c, kGM), 0);
        }
        for (int e = t; e < (kNX - kFeat) * kGM; e += kGNT) {
            const int r = kFeat + e / kGM, c = e % kGM;
            for (int b = 0; b < 2; ++b) {
                g_store2(s.xt_hi[b], tc::core_off(r, c, kGM), r == kFeat ? one : (uint16_t)0);
                g_store2(s.xt_lo[b], tc::core_off(r, c, kGM), 0);
            }
        }
        for (int e = t; e < (kNX - kCls) * kGM; e += kGNT) {
            const int r = kCls + e / kGM, c = e % kGM;
            g_store2(s.d3t_hi, tc::core_off(r, c, kGM), 0);
            g_store2(s.d3t_lo, tc::core_off(r, c, kGM), 0);
        }
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
    const uint32_t sa_hi = smem_u32(s.a_hi), sa_lo = smem_u32(s.a_lo), sw2 = smem_u32(s.w2), sw2t = smem_u32(s.w2t);
    const uint32_t st_hi = smem_u32(s.t_hi), st_lo = smem_u32(s.t_lo);
    const uint32_t sh_hi = smem_u32(s.h1t_hi), sh_lo = smem_u32(s.h1t_lo);
    const uint32_t sd_hi = smem_u32(s.d3t_hi), sd_lo = smem_u32(s.d3t_lo);
    const float inv_n = 1.0f / (float)N;
    const int ntiles = (int)(((long long)N + kGM - 1) / kGM);
    unsigned phase = 0;
    bool failed = false, first = true;
    double loss_t = 0.0;                       // this thread's samples, in tile order
    float gb3_t[kCls] = {0.0f, 0.0f, 0.0f};
    float *row = s.stage + (size_t)t * kSW;    // this sample's staging row
    int par = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, par ^= 1) {
        const long long smp = (long long)tile * kGM + t;
        const bool valid = smp < N;
        float x[kFeat];
#pragma unroll
        for (int k = 0; k < kFeat; ++k) {
            x[k] = valid ? (float)((feat[(size_t)smp * kFeat + k] - (double)s.mu[k]) / (double)s.sd[k]) : 0.0f;
            uint16_t xh, xl;
            g_split(x[k], xh, xl);
            g_store2(s.xt_hi[par], tc::core_off(k, t, kGM), xh);
            g_store2(s.xt_lo[par], tc::core_off(k, t, kGM), xl);
        }
        // layer 1 (binary32 FMA chains, bias first, as the CUDA-core kernel) into the staging row
        // and from there into the forward A ([s][i]); the ReLU mask as bits
        uint64_t m1 = 0;
#pragma unroll 4
        for (int o = 0; o < kH1; ++o) {
            float a = s.b1[o];
#pragma unroll
            for (int k = 0; k < kFeat; ++k) a = fmaf(s.w1t[k][o], x[k], a);
            const float h = fmaxf(a, 0.0f);
            if (h > 0.0f) m1 |= 1ull << o;
            row[o] = h;
        }
#pragma unroll 1
        for (int j = 0; j < kH1 / 8; ++j) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                uint16_t h0, l0, h1, l1;
                g_split(row[8 * j + e], h0, l0);
                g_split(row[8 * j + e + 1], h1, l1);
                hi[e >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                lo[e >> 1] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
            const uint32_t off = tc::core_off(t, 8 * j, kH1);
            g_store16(s.a_hi, off, make_uint4(hi[0], hi[1], hi[2], hi[3]));
            g_store16(s.a_lo, off, make_uint4(lo[0], lo[1], lo[2], lo[3]));
        }
        __syncthreads();
        emit_t64(s.stage, s.h1t_hi, s.h1t_lo, 0, t);     // h1^T into rows 0..63 of [h1^T; 1]
        // forward product c = h1 W2^T
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            mma_k64(tm + kColFwd, sa_hi, sa_lo, sw2);
            tc::commit(&s.bar);
        }
        if (!__syncthreads_and(mbar_wait_bounded(&s.bar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // h2 = relu(c + b2) into the staging row, its mask, and layer 3 (FMA chains over o)
        uint64_t m2 = 0;
        float lg[kCls] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float c0[32];
            tc::ld_32cols(tm + tlane + kColFwd + 32 * half, c0);
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int o = 32 * half + u;
                const float h = fmaxf(c0[u] + s.b2[o], 0.0f);
                if (h > 0.0f) m2 |= 1ull << o;
                row[o] = h;
#pragma unroll
                for (int c = 0; c < kCls; ++c) lg[c] = fmaf(s.w3[c][o], h, lg[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < kCls; ++c) lg[c] += s.b3[c];
        // softmax cross-entropy: d3 = (softmax - onehot) / N
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
        float d3[kCls];
#pragma unroll
        for (int c = 0; c < kCls; ++c) {
            d3[c] = valid ? (ex[c] / z - (c == y ? 1.0f : 0.0f)) * inv_n : 0.0f;
            gb3_t[c] += d3[c];
            uint16_t dh, dl;
            g_split(d3[c], dh, dl);
            g_store2(s.d3t_hi, tc::core_off(c, t, kGM), dh);
            g_store2(s.d3t_lo, tc::core_off(c, t, kGM), dl);
        }
        if (valid) loss_t += -(double)(lg[y] - mx - logf(z));
        __syncthreads();
        emit_t64(s.stage, s.t_hi, s.t_lo, kH1, t);       // h2^T into rows 64..127 of T
        // d2 = (h2 > 0) W3^T d3 (FMA chains over the classes) into the staging row, once the
        // h2^T transpose has read it, and from there into the back-prop A ([s][o]; the forward
        // has consumed h1)
        __syncthreads();
#pragma unroll 8
        for (int o = 0; o < kH2; ++o) {
            float v = 0.0f;
#pragma unroll
            for (int c = 0; c < kCls; ++c) v = fmaf(s.w3[c][o], d3[c], v);
            row[o] = ((m2 >> o) & 1ull) ? v : 0.0f;
        }
#pragma unroll 1
        for (int j = 0; j < kH2 / 8; ++j) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                uint16_t h0, l0, h1, l1;
                g_split(row[8 * j + e], h0, l0);
                g_split(row[8 * j + e + 1], h1, l1);
                hi[e >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                lo[e >> 1] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
            const uint32_t off = tc::core_off(t, 8 * j, kH2);
            g_store16(s.a_hi, off, make_uint4(hi[0], hi[1], hi[2], hi[3]));
            g_store16(s.a_lo, off, make_uint4(lo[0], lo[1], lo[2], lo[3]));
        }
        __syncthreads();
        emit_t64(s.stage, s.t_hi, s.t_lo, 0, t);         // d2^T into rows 0..63 of T
        tc::fence_proxy_async();
        tc::fence_before_sync();                         // the forward product's TMEM loads are done
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            mma_k64(tm + kColBack, sa_hi, sa_lo, sw2t);
            mma_sample_k(tm + kColW2, st_hi, st_lo, sh_hi, sh_lo, tc::idesc_bf16_f32(128, kNB2), first);
            mma_sample_k(tm + kColW3, st_hi, st_lo, sd_hi, sd_lo, tc::idesc_bf16_f32(128, kNX), first);
            tc::commit(&s.bar);
        }
        if (!__syncthreads_and(mbar_wait_bounded(&s.bar, phase))) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // e = d1 masked by h1 > 0 (and by the sample's validity) into the staging row
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float e0[32];
            tc::ld_32cols(tm + tlane + kColBack + 32 * half, e0);
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int i = 32 * half + u;
                row[i] = (((m1 >> i) & 1ull) && valid) ? e0[u] : 0.0f;
            }
        }
        __syncthreads();
        emit_t64(s.stage, s.t_hi, s.t_lo, 0, t);         // e^T into rows 0..63 of T
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            mma_sample_k(tm + kColW1, st_hi, st_lo, smem_u32(s.xt_hi[par]), smem_u32(s.xt_lo[par]),
                         tc::idesc_bf16_f32(128, kNX), first);
        }
        first = false;
        // this product completes under the next tile's commit (or the one after the loop); the
        // next tile writes only the other [x^T; 1] buffer before that commit
    }
    if (!failed && !first) {
        if (t == 0) tc::commit(&s.bar);
        if (!__syncthreads_and(mbar_wait_bounded(&s.bar, phase))) failed = true;
        else phase ^= 1u;
        tc::fence_after_sync();
    }
    float *out = partial + (size_t)blockIdx.x * kMlpWeights;
    if (failed) {
        // the MMAs in flight must finish (bounded) before TMEM is freed; the gradient is NaN
        if (t == 0) (void)mbar_wait_bounded(&s.bar, phase);
        for (int e = t; e < kMlpWeights; e += kGNT) out[e] = __int_as_float(0x7fc00000);
        if (t == 0) loss_part[blockIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
        s.loss[t] = loss_t;
#pragma unroll
        for (int c = 0; c < kCls; ++c) s.gb3[t][c] = gb3_t[c];
        if (warp < 2) {
            // lanes 0..63: rows o of gW2 (columns 0..63) and gb2 (column 64); rows i of gW1
            // (columns 0..11) and gb1 (column 12)
            float v[32];
            const int o = t;
            if (first) {
                for (int i = 0; i < kH1; ++i) out[kOffW2 + o * kH1 + i] = 0.0f;
                out[kOffB2 + o] = 0.0f;
                for (int k = 0; k < kFeat; ++k) out[kOffW1 + o * kFeat + k] = 0.0f;
                out[kOffB1 + o] = 0.0f;
            } else {
                tc::ld_32cols(tm + tlane + kColW2, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) out[kOffW2 + o * kH1 + i] = v[i];
                tc::ld_32cols(tm + tlane + kColW2 + 32, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) out[kOffW2 + o * kH1 + 32 + i] = v[i];
                tc::ld_32cols(tm + tlane + kColW2 + 64, v);
                out[kOffB2 + o] = v[0];
                tc::ld_32cols(tm + tlane + kColW1, v);
#pragma unroll
                for (int k = 0; k < kFeat; ++k) out[kOffW1 + o * kFeat + k] = v[k];
                out[kOffB1 + o] = v[kFeat];
            }
        } else {
            // lanes 64..127: gW3[c][o] for o = lane - 64 (columns 0..2)
            float v[32];
            const int o = t - kH1;
            if (!first) tc::ld_32cols(tm + tlane + kColW3, v);
#pragma unroll
            for (int c = 0; c < kCls; ++c) out[kOffW3 + c * kH2 + o] = first ? 0.0f : v[c];
        }
        __syncthreads();
        if (t < kCls) {
            float acc = 0.0f;
            for (int r = 0; r < kGM; ++r) acc += s.gb3[r][t];
            out[kOffB3 + t] = acc;
        }
        if (t == kCls) {
            double acc = 0.0;
            for (int r = 0; r < kGM; ++r) acc += s.loss[r];
            loss_part[blockIdx.x] = acc;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, kGCols);
}

int mlp_grad_tc_grid(int N) {
    long long g = ((long long)N + kGM - 1) / kGM;
    if (g > sm_count()) g = sm_count();
    return g < 1 ? 1 : (int)g;
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
