// Shared device helpers and host-side declarations of the mpbjac library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>

#include "mpbjac.h"

namespace mpbjac {

// ----------------------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define MPB_CUDA(call)                                                    \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::mpbjac::cuda_fail(e_, #call);     \
    } while (0)

// ----------------------------------------------------------------------------------------
// launch geometry
// ----------------------------------------------------------------------------------------
constexpr int kNT = 256;                 // threads per CTA of the streaming kernels
constexpr int kWarps = kNT / 32;
constexpr int kMaxGrid = 152 * 8;        // upper bound on CTAs of any reducing kernel
int sm_count();

// ----------------------------------------------------------------------------------------
// programmatic dependent launch: a loop kernel launched with the programmatic attribute may
// be scheduled while its predecessor in the stream is still draining. It waits here until
// that predecessor has completed and its writes are visible, before touching any global
// memory, and at once lets its own successor be scheduled (the successor waits the same
// way). Both instructions are no-ops for a kernel launched without the attribute. Before the
// wait a kernel may read only what no kernel of the solve writes (the matrix, the block
// inverses): the predecessor may still be running.
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// bring one 128-byte line into L2 (no register result; a hint the memory system may drop)
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ----------------------------------------------------------------------------------------
// L2 residency. The PCG vectors (r, z, p, q, x: n doubles each) are read again by the next
// kernel of the same iteration, while the matrix and the block inverses are streamed once per
// iteration (their loads use ld.global.cs, evict-first). With keep set, the loop kernels give
// their vector loads and stores an evict_last policy so that the streams evict each other
// rather than the vectors; without it the policy is evict_normal (a plain access).
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t vec_policy(int keep) {
    uint64_t p;
    if (keep) asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double ld_vec(const double *a, uint64_t pol) {
    double v;
    asm("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ldg_vec(const double *a, uint64_t pol) {     // read-only in the kernel
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_vec2(const double2 *a, uint64_t pol) {
    double2 v;
    asm("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_vec(double *a, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_vec2(double2 *a, double2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(a), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
}

// Host: whether launches made by this thread now carry the programmatic attribute (set
// around the PCG loop body only).
bool pdl_on();
void pdl_set(bool on);

template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                                 Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    if (pdl_on()) {
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ----------------------------------------------------------------------------------------
// solver state shared by the kernels of one PCG loop (device memory, one per handle)
// ----------------------------------------------------------------------------------------
enum SolverStateCode : int32_t {
    kRunning = 0,
    kConverged = 1,
    kMaxit = 2,
    kBreakdown = 3,        // r.z <= 0 or non-finite scalars after the x/r update
    kBreakdownSigma = 4,   // p.Ap <= 0 before the x/r update of this iteration
    kTimeout = 5,          // a bounded wait of a loop kernel expired (a TMA copy did not land)
};

struct SolverState {
    // configuration, written by the host before each solve
    double tol;
    double adp_tol;
    double *x;             // solution vector (device)
    double *hist;          // relres history (device, nullable)
    int32_t maxit;
    int32_t temporal;      // BJAC_TEMPORAL_*
    int32_t low_default;   // set used when temporal == NONE: 1 low, 0 binary64
    int32_t l2_keep;       // PCG vectors accessed with an evict_last L2 policy (vec_policy)
    // dynamic state
    double bnorm;
    double rho, sigma, alpha, beta, rr, relres, true_relres;
    double rho_prev;       // rho of the previous application (the flexible beta's denominator)
    int32_t iter, state, use_low, x_pending;
    int32_t low_applies, high_applies, restarts;
    int32_t flexible;      // flexible-CG beta (set by the host for the solve)
    int32_t redo;          // aMP: the speculative application used the other set; apply again
    int32_t pad_;
    unsigned int tickets[8];
};

enum Ticket { kTicketSpmv = 0, kTicketUpdR = 1, kTicketApply = 2, kTicketUpdXP = 3, kTicketRes = 4,
              kTicketInit = 5, kTicketFlex = 6 };

__device__ __forceinline__ int choose_low(const SolverState *S, double relres) {
    if (S->temporal == BJAC_TEMPORAL_HL) return !(relres >= S->adp_tol);   // Algorithm 3.2
    if (S->temporal == BJAC_TEMPORAL_LH) return relres >= S->adp_tol;      // Algorithm 3.3
    return S->low_default;
}

// ----------------------------------------------------------------------------------------
// a preconditioner set: nb blocks, each stored row-major in its own format in a byte pool
// ----------------------------------------------------------------------------------------
struct PSet {
    const int32_t *block_ptr;  // [nb+1]
    const uint8_t *fmt;        // [nb]
    const float *scale;        // [nb]
    const int64_t *qoff;       // [nb+1] byte offsets into pool
    const uint8_t *pool;
    int32_t nb;
    int32_t ubs;               // common block size if every block has it (else 0)
    int32_t ufmt;              // common format (else -1)
    int32_t pad;
};

// ----------------------------------------------------------------------------------------
// deterministic reductions
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA in a fixed order; result valid in every thread. sm: >= NT/32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sm) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) t += sm[i];
    return t;
}

// Sums over the CTA of NV per-thread values, valid in thread 0 only (the per-CTA partials of
// a grid reduction). The values pass through shared memory and warp 0 adds them: NT/32 adds
// per lane in a fixed order, then one warp tree per value. That is about a sixth of the FP64
// instructions of a tree in every warp, and the FP64 pipe is a co-bound of the loop kernels.
// sm: NV * NT doubles.
template <int NT, int NV>
__device__ __forceinline__ void cta_sum_to0(const double (&v)[NV], double *sm, double (&out)[NV]) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k * NT + threadIdx.x] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = 0.0;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = sm[k * NT + threadIdx.x];
#pragma unroll
            for (int i = 1; i < NT / 32; ++i) s += sm[k * NT + threadIdx.x + 32 * i];
            out[k] = warp_sum(s);
        }
    }
}

// Every CTA publishes its partials (written by thread 0), then the last CTA to arrive
// (ticket) sees them all. Only thread 0 fences: it wrote the partials and takes the ticket.
// Returns true in every thread of that last CTA. The ticket counter is reset there.
__device__ __forceinline__ bool last_cta(unsigned int *ticket) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0) *ticket = 0u;
    }
    return s_last != 0;
}

// Sum of part[0..count) (written by other CTAs) in fixed order, by a whole CTA.
template <int NT>
__device__ __forceinline__ double reduce_partials(const double *part, int count, int stride, double *sm) {
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += NT) v += __ldcg(part + (size_t)i * stride);
    return block_sum<NT>(v, sm);
}

// The sums over i < count of part[i * stride + k], k < NV (per-CTA partials written by other
// CTAs), in a fixed order, valid in thread 0 only: each thread adds every NT-th partial in
// turn, then warp 0 adds the NT per-thread sums (cta_sum_to0) and ends in one butterfly. On
// the 2-lane FP64 pipe that is about 36 FP64 warp instructions per value, against about 128
// for reduce_partials (a butterfly in every warp, then every thread adding the warp sums); the
// last CTA of a loop kernel runs it while the next kernel waits. sm: NV * NT doubles.
template <int NT, int NV>
__device__ __forceinline__ void reduce_partials_to0(const double *part, int count, int stride, double *sm,
                                                    double (&out)[NV]) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = threadIdx.x < count ? __ldcg(part + (size_t)threadIdx.x * stride + k) : 0.0;
    for (int i = threadIdx.x + NT; i < count; i += NT)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __ldcg(part + (size_t)i * stride + k);
    cta_sum_to0<NT, NV>(v, sm, out);
}

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && v < 1.0e308; }

// The loop SpMV leaves one partial sum of p.q per CTA (stride 2, at kSpPartOff in the part
// buffer; its CTA 0 zeroes the slots up to kMaxGrid that no CTA wrote) and no final
// reduction: the kernel that consumes alpha sums them itself, in every CTA, in one fixed order
// whatever the CTA's size: 256 lanes, lane v adding slots v, v + 256, ... in turn (the zero
// slots come last and change nothing); then one warp, lane l adding the sums of lanes
// l, l + 32, ..., l + 224 in turn, and a butterfly over the warp. On sm_103a the FP64 pipe
// does 2 lanes per clock per SM, so every FP64 instruction of a warp counts: this order takes
// about 42 of them per CTA, against 88 when each group of 32 lanes ends in its own butterfly.
// Every CTA gets the same sigma and alpha = rho / sigma; CTA 0 records them in S. When sigma is
// not a positive finite number, every CTA returns false and CTA 0 records the breakdown, so all
// of them leave before any ticket. Every thread of the CTA must call it.
constexpr int kSpPartOff = 3 * kMaxGrid;
__device__ __forceinline__ bool loop_alpha(SolverState *S, const double *spart, double &alpha) {
    __shared__ double s_lane[256];
    __shared__ double s_alpha;
    __shared__ int s_ok;
    static_assert(kMaxGrid >= 256, "every lane has a first slot");
    const double rho = threadIdx.x == 0 ? S->rho : 0.0;
    for (int v = threadIdx.x; v < 256; v += blockDim.x) {
        double a = __ldg(spart + 2 * v);       // written by the previous kernel: read-only here
#pragma unroll
        for (int k = 1; k < (kMaxGrid + 255) / 256; ++k) {
            const int c = v + 256 * k;
            if (c < kMaxGrid) a += __ldg(spart + 2 * c);
        }
        s_lane[v] = a;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double t = s_lane[lane];
#pragma unroll
        for (int j = 1; j < 8; ++j) t += s_lane[lane + 32 * j];
        t = warp_sum(t);
        if (lane == 0) {
            const bool ok = finite_pos(t);
            const double a = ok ? rho / t : 0.0;
            s_ok = ok;
            s_alpha = a;
            if (blockIdx.x == 0) {
                S->sigma = t;
                if (ok) S->alpha = a;
                else S->state = kBreakdownSigma;
            }
        }
    }
    __syncthreads();
    alpha = s_alpha;
    return s_ok != 0;
}


}  // namespace mpbjac

namespace mpbjac {

// ----------------------------------------------------------------------------------------
// binary64 <-> binary32 conversions done with integer operations only, so that they take no
// slot of the (narrow) FP64 pipe of sm_103a. Written from the IEEE 754 bit layouts:
//   binary64 = sign | 11-bit exponent (bias 1023) | 52-bit fraction
//   binary32 = sign | 8-bit exponent (bias 127)   | 23-bit fraction
// Every input class is handled (zeros, subnormal results, overflow, infinities, NaN);
// finite results are round-to-nearest-even with subnormals kept, i.e. the correctly
// rounded value. A NaN stays a quiet NaN that keeps the top payload bits.
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ float f64_to_f32_rn(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned int sign = (unsigned int)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7FF);
    const unsigned long long frac = u & 0xFFFFFFFFFFFFFull;
    unsigned int r;
    if (e == 0x7FF) {                                   // infinity or NaN
        r = 0x7F800000u | (frac ? (0x400000u | (unsigned int)(frac >> 29)) : 0u);
    } else if (e > 1023 + 127) {                        // beyond the binary32 range: infinity
        r = 0x7F800000u;
    } else if (e >= 1023 - 126) {                       // normal binary32 result
        r = ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)(frac >> 29);
        const unsigned int rem = (unsigned int)(frac & 0x1FFFFFFFu);   // the 29 dropped bits
        const unsigned int half = 0x10000000u;
        r += (rem > half) | ((rem == half) & (r & 1u));               // carry may reach the exponent
    } else if (e == 0) {                                // binary64 zero or subnormal: below 2^-1022
        r = 0u;
    } else {
        // binary32 subnormal or zero: |d| = M 2^(e - 1075) with M = 2^52 + frac, i.e.
        // M 2^-(926 - e) units of 2^-149; shift by 926 - e > 29 and round to nearest even
        const int sh = 926 - e;
        if (sh > 54) {
            r = 0u;                                     // below half of 2^-149
        } else {
            const unsigned long long M = frac | (1ull << 52);
            const unsigned long long q = M >> sh;
            const unsigned long long rem = M & ((1ull << sh) - 1ull);
            const unsigned long long half = 1ull << (sh - 1);
            r = (unsigned int)q + (unsigned int)((rem > half) | ((rem == half) & (q & 1ull)));
        }
    }
    return __uint_as_float(sign | r);
}

__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned int e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    unsigned long long bits;
    if (e == 0xFFu) {                                   // infinity or NaN (payload kept)
        bits = 0x7FF0000000000000ull | ((unsigned long long)m << 29);
    } else if (e != 0u) {                               // normal
        bits = ((unsigned long long)(e + 1023u - 127u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0u) {                               // zero
        bits = 0ull;
    } else {                                            // subnormal m 2^-149: normalise
        const int p = 31 - __clz((int)m);               // leading bit, 0..22
        bits = ((unsigned long long)(p - 149 + 1023) << 52) |
               (((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
    }
    return __longlong_as_double((long long)(sign | bits));
}

}  // namespace mpbjac
