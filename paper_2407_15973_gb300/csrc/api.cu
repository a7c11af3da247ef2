// C ABI of mpbjac: handle lifecycle, setup orchestration, the PCG driver (one CUDA graph
// with a device-side while loop per solve), and the single-step entry points.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "apply.cuh"
#include "common.cuh"
#include "kt.cuh"
#include "mlp.cuh"
#include "sell.cuh"
#include "setup.cuh"
#include "spmv.cuh"
#include "update.cuh"

namespace mpbjac {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? MPBJAC_ERR_NO_MEMORY : MPBJAC_ERR_CUDA;
}

int sm_count() {
    static int v = 0;
    if (v == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    }
    return v;
}

static int fmt_bytes(int f) { return f == BJAC_FP64 ? 8 : f == BJAC_FP32 ? 4 : 2; }

// kernels that can apply the low-precision set (the binary64 set always uses the generic one)
enum ApplyKind { kApplyKindGeneric = 0, kApplyKindTma = 1, kApplyKindReg = 2, kApplyKindMix = 3 };

// ----------------------------------------------------------------------------------------
// vector kernels of the PCG loop
// ----------------------------------------------------------------------------------------
static int vec_grid(int n) {
    int g = sm_count() * 4;
    const int need = (n + kNT - 1) / kNT;
    if (g > need) g = need;
    if (g > kMaxGrid) g = kMaxGrid;
    return g < 1 ? 1 : g;
}


// element-wise f = RNE binary32 of x and w = f widened back, both by the integer routines the
// apply kernels use
__global__ void k_convert(int n, const double *__restrict__ x, float *__restrict__ f, double *__restrict__ w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float v = f64_to_f32_rn(x[i]);
        if (f) f[i] = v;
        if (w) w[i] = f32_to_f64(v);
    }
}

__global__ void k_zero_if_zero_rhs(int n, SolverState *S) {
    if (S->bnorm != 0.0) return;
    double *x = S->x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

__global__ void k_validate_csr(int n, int nnz, const int32_t *rowptr, const int32_t *colidx, int *status) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (tid == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) atomicCAS(status, 0, MPBJAC_ERR_INVALID_ARG);
    for (int i = tid; i < n; i += stride)
        if (rowptr[i + 1] < rowptr[i]) atomicCAS(status, 0, MPBJAC_ERR_INVALID_ARG);
    for (int k = tid; k < nnz; k += stride) {
        const int c = colidx[k];
        if (c < 0 || c >= n) atomicCAS(status, 0, MPBJAC_ERR_INVALID_ARG);
    }
}

}  // namespace mpbjac

using namespace mpbjac;

// ------------------------------------------------------------------------------------------
// handle
// ------------------------------------------------------------------------------------------
struct bjac_handle {
    bjac_csr A{};
    bjac_policy pol{};
    cudaStream_t stream = nullptr;
    int n = 0, nb = 0, bs_max = 0, ubs = 0;
    std::vector<int32_t> h_block_ptr;
    std::vector<int64_t> h_goff, h_qoff;
    int32_t *d_block_ptr = nullptr;
    int64_t *d_goff = nullptr;
    double *d_G = nullptr;
    uint8_t *d_fmt_hi = nullptr;
    float *d_scale_hi = nullptr;
    int64_t *d_qoff_hi = nullptr;
    uint8_t *d_fmt = nullptr;
    float *d_scale = nullptr;
    int64_t *d_qoff = nullptr;
    uint8_t *d_pool = nullptr;
    int64_t pool_bytes = 0;
    double *d_feat = nullptr;
    double *d_kap = nullptr;
    int *d_status = nullptr;
    bool have_lo = false, have_hi = false;
    PSet lo{}, hi{};
    // solve workspace
    double *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_x0 = nullptr;
    double *d_part = nullptr;
    SolverState *d_S = nullptr;
    SolverState *h_S = nullptr;   // pinned mirror
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    float setup_ms = 0.0f;
    int32_t blocks_per_fmt[4] = {0, 0, 0, 0};
    int apply_kind = kApplyKindGeneric;   // kernel used for the low-precision set
    float tune_ms[4] = {0, 0, 0, 0};      // autotuner timings (generic, TMA, register, mixed register)
    SellMat sell{};                       // SELL-32 copy of A (val NULL if not kept)
    int use_sell = 0;                     // loop SpMV on the SELL-32 copy
    float spmv_ms[3] = {0, 0, 0};         // timed y = A x: CSR, SELL-32, SELL-32 with prefetch
    int body_launches[2] = {0, 0};        // kernels in one body of each solve graph
    KtSet kt;                             // BJAC(k, t) of Eq. 3-2 / 3-3 (select KT)
    long long launches = 0;               // kernels launched by the last solve
};

static void free_handle(bjac_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < 2; ++i) {
        if (h->exec[i]) cudaGraphExecDestroy(h->exec[i]);
        if (h->graph[i]) cudaGraphDestroy(h->graph[i]);
    }
    void *ptrs[] = {h->d_block_ptr, h->d_goff, h->d_G, h->d_fmt_hi, h->d_scale_hi, h->d_qoff_hi, h->d_fmt,
                    h->d_scale, h->d_qoff, h->d_pool, h->d_feat, h->d_kap, h->d_status, h->d_r, h->d_z,
                    h->d_p, h->d_q, h->d_x0, h->d_part, h->d_S};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    sell_free(&h->sell);
    kt_free(&h->kt);
    if (h->h_S) cudaFreeHost(h->h_S);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

template <typename T>
static int dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    MPB_CUDA(cudaMalloc((void **)p, count * sizeof(T)));
    return MPBJAC_OK;
}

#define MPB_TRY(expr)                 \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != MPBJAC_OK) {       \
            free_handle(h);           \
            return rc_;               \
        }                             \
    } while (0)

static int check_csr_host(const bjac_csr *A) {
    if (!A) return fail(MPBJAC_ERR_INVALID_ARG, "A is NULL");
    if (A->n <= 0) return fail(MPBJAC_ERR_INVALID_ARG, "n must be positive");
    if (A->nnz < 0) return fail(MPBJAC_ERR_INVALID_ARG, "nnz must be non-negative");
    if (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->val)))
        return fail(MPBJAC_ERR_INVALID_ARG, "CSR pointers must be non-NULL");
    return MPBJAC_OK;
}

static PSet make_pset(const bjac_handle *h, const uint8_t *fmt, const float *scale, const int64_t *qoff,
                      const uint8_t *pool, int ufmt) {
    PSet P;
    P.block_ptr = h->d_block_ptr;
    P.fmt = fmt;
    P.scale = scale;
    P.qoff = qoff;
    P.pool = pool;
    P.nb = h->nb;
    P.ubs = h->ubs;
    P.ufmt = ufmt;
    P.pad = 0;
    return P;
}

// Autotuner for the low-precision apply: when the set is uniform (one block size, one
// format) every applicable kernel is timed on this very set (standalone launches on the
// handle's stream, CUDA events, best of three after one warm-up) and the fastest is kept.
// policy.apply_variant forces a kernel instead (1 generic, 2 TMA-staged, 3 register).
// Results are cached per (format, block size, block count) for the life of the process.
struct TuneKey {
    int fmt, bs, nb;
    bool operator==(const TuneKey &o) const { return fmt == o.fmt && bs == o.bs && nb == o.nb; }
};
struct TuneResult {
    int kind;
    float ms[4];
};
static std::vector<std::pair<TuneKey, TuneResult>> g_tune_cache;

static int choose_apply_kind(bjac_handle *h) {
    const bool tma_ok = tma_supported(h->lo, h->n);
    const bool reg_ok = reg_supported(h->lo, h->n);
    const bool mix_ok = mix_supported(h->lo, h->n);
    const int v = h->pol.apply_variant;
    if (v == 4) { h->apply_kind = mix_ok ? kApplyKindMix : kApplyKindGeneric; return MPBJAC_OK; }
    if (v == 1 || (!tma_ok && !mix_ok)) { h->apply_kind = kApplyKindGeneric; return MPBJAC_OK; }
    if (v == 2) { h->apply_kind = tma_ok ? kApplyKindTma : kApplyKindGeneric; return MPBJAC_OK; }
    if (v == 3) { h->apply_kind = reg_ok ? kApplyKindReg : tma_ok ? kApplyKindTma : kApplyKindGeneric; return MPBJAC_OK; }
    // blocks of 32 rows in several formats: the mixed register kernel, without timing (it beat
    // the generic kernel on every such set timed); on uniform 32-row sets the generic kernel is
    // not timed either (it lost to both the register and the TMA kernel every time: 49 against
    // 29 and 33 us for the BF16 set of the 128^3 workload), the other two are
    if (mix_ok && h->lo.ufmt < 0) { h->apply_kind = kApplyKindMix; return MPBJAC_OK; }
    const TuneKey key{h->lo.ufmt, h->lo.ubs, h->nb};
    for (auto &e : g_tune_cache)
        if (e.first == key) {
            h->apply_kind = e.second.kind;
            for (int i = 0; i < 4; ++i) h->tune_ms[i] = e.second.ms[i];
            return MPBJAC_OK;
        }
    cudaStream_t st = h->stream;
    double *r = nullptr, *z = nullptr, *part = nullptr;
    unsigned int *ticket = nullptr;
    MPB_CUDA(cudaMalloc(&r, sizeof(double) * h->n));
    MPB_CUDA(cudaMalloc(&z, sizeof(double) * h->n));
    MPB_CUDA(cudaMalloc(&part, sizeof(double) * 3 * kMaxGrid + 64));
    ticket = reinterpret_cast<unsigned int *>(part + 3 * kMaxGrid);
    MPB_CUDA(cudaMemsetAsync(r, 0, sizeof(double) * h->n, st));
    MPB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
    ApplyIO io{};
    io.r = r;
    io.z = z;
    io.part = part;
    io.ticket = ticket;
    io.set = 1;
    io.only_set = -1;
    cudaEvent_t e0, e1;
    MPB_CUDA(cudaEventCreate(&e0));
    MPB_CUDA(cudaEventCreate(&e1));
    // interleaved rounds over the candidate kernels, median of 7 after a warm-up round
    constexpr int kRounds = 8;
    float t[4][kRounds] = {};
    auto usable = [&](int k) {
        return (k == kApplyKindGeneric && !reg_ok) || (k == kApplyKindTma && tma_ok) || (k == kApplyKindReg && reg_ok) ||
               (k == kApplyKindMix && mix_ok && !reg_ok);
    };
    for (int rep = 0; rep < kRounds; ++rep) {
        for (int k = 0; k < 4; ++k) {
            if (!usable(k)) continue;
            MPB_CUDA(cudaEventRecord(e0, st));
            int rc = k == kApplyKindGeneric ? launch_apply_generic(kApplyStandalone, h->lo, h->lo, io, nullptr, st)
                     : k == kApplyKindTma   ? launch_apply_tma(kApplyStandalone, h->lo, io, nullptr, h->n, st)
                     : k == kApplyKindReg   ? launch_apply_reg(kApplyStandalone, h->lo, io, nullptr, st)
                                            : launch_apply_mix(kApplyStandalone, h->lo, io, nullptr, st);
            if (rc) return rc;
            MPB_CUDA(cudaEventRecord(e1, st));
            MPB_CUDA(cudaEventSynchronize(e1));
            cudaEventElapsedTime(&t[k][rep], e0, e1);
        }
    }
    float best = 1e30f;
    int best_kind = reg_ok ? kApplyKindReg : kApplyKindGeneric;
    for (int k = 0; k < 4; ++k) {
        if (!usable(k)) continue;
        std::sort(t[k] + 1, t[k] + kRounds);
        const float med = t[k][1 + (kRounds - 1) / 2];
        h->tune_ms[k] = med;
        if (med < best) { best = med; best_kind = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(r);
    cudaFree(z);
    cudaFree(part);
    h->apply_kind = best_kind;
    g_tune_cache.push_back({key, TuneResult{best_kind, {h->tune_ms[0], h->tune_ms[1], h->tune_ms[2], h->tune_ms[3]}}});
    return MPBJAC_OK;
}

// Layout of the loop SpMV. policy.spmv_format 1 keeps the caller's CSR arrays, 2 always
// builds the SELL-32 copy (one slice at a time per warp) and 3 the same copy with the next
// slice's head prefetched. By default the copy is built when its padding stays under 1.5 nnz
// and y = A x is timed with the CSR kernel and both SELL-32 kernels (interleaved rounds on a
// nonzero x, median of 7 after a warm-up round, on the handle's stream); the fastest is
// kept (the prefetching one only when 3 % faster than the better of the others), and the
// decision is cached per (n, nnz) for the life of the process. All give the same result
// bits.
struct SpFmtTune {
    int n, nnz, choice;       // 0 CSR, 1 SELL-32, 2 SELL-32 with prefetch
    float ms[3];
};
static std::vector<SpFmtTune> g_spfmt_cache;

static int choose_spmv_format(bjac_handle *h) {
    const int f = h->pol.spmv_format;
    cudaStream_t st = h->stream;
    h->use_sell = 0;
    if (f == 1) return MPBJAC_OK;
    if (f == 0) {
        for (const SpFmtTune &t : g_spfmt_cache)
            if (t.n == h->A.n && t.nnz == h->A.nnz) {
                for (int i = 0; i < 3; ++i) h->spmv_ms[i] = t.ms[i];
                if (t.choice == 0) return MPBJAC_OK;
                int rc = sell_build(h->A, 1.5, &h->sell, st);
                if (rc) return rc;
                h->use_sell = h->sell.val != nullptr;
                h->sell.kernel = t.choice - 1;
                return MPBJAC_OK;
            }
    }
    int rc = sell_build(h->A, f >= 2 ? 0.0 : 1.5, &h->sell, st);
    if (rc) return rc;
    if (!h->sell.val) {
        if (f >= 2) return fail(MPBJAC_ERR_UNSUPPORTED, "A needs more than 2^31 stored SELL-32 entries");
        g_spfmt_cache.push_back({h->A.n, h->A.nnz, 0, {0.0f, 0.0f, 0.0f}});
        return MPBJAC_OK;
    }
    if (f >= 2) {
        h->use_sell = 1;
        h->sell.kernel = f - 2;
        return MPBJAC_OK;
    }
    double *x = h->d_p, *y = h->d_q;
    MPB_CUDA(cudaMemsetAsync(x, 0x3F, sizeof(double) * h->n, st));     // every entry about 4.8e-4
    cudaEvent_t e0, e1;
    MPB_CUDA(cudaEventCreate(&e0));
    MPB_CUDA(cudaEventCreate(&e1));
    constexpr int kRounds = 8;
    float t[3][kRounds] = {};
    for (int rep = 0; rep < kRounds; ++rep) {
        for (int k = 0; k < 3; ++k) {
            MPB_CUDA(cudaEventRecord(e0, st));
            if (k == 0) {
                rc = launch_spmv(h->A, x, y, nullptr, nullptr, nullptr, nullptr, 0, st);
            } else {
                h->sell.kernel = k - 1;
                rc = launch_spmv_sell(h->sell, x, nullptr, y, nullptr, nullptr, nullptr, nullptr, kSpY, st);
            }
            if (rc) return rc;
            MPB_CUDA(cudaEventRecord(e1, st));
            MPB_CUDA(cudaEventSynchronize(e1));
            cudaEventElapsedTime(&t[k][rep], e0, e1);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int k = 0; k < 3; ++k) {
        std::sort(t[k] + 1, t[k] + kRounds);
        h->spmv_ms[k] = t[k][1 + (kRounds - 1) / 2];
    }
    // the prefetching kernel holds more registers: keep it only when clearly faster
    int best = h->spmv_ms[1] < h->spmv_ms[0] ? 1 : 0;
    if (h->spmv_ms[2] < 0.97f * h->spmv_ms[best]) best = 2;
    h->use_sell = best > 0;
    if (best > 0) h->sell.kernel = best - 1;
    else sell_free(&h->sell);
    g_spfmt_cache.push_back({h->A.n, h->A.nnz, best, {h->spmv_ms[0], h->spmv_ms[1], h->spmv_ms[2]}});
    return MPBJAC_OK;
}

// the loop SpMV in the handle's layout: q = A p and per-CTA partials of p.q, which the next
// kernel sums into alpha (loop_alpha); or, when the next kernel is the generic apply
// (finish_alpha), with sigma and alpha finished by the SpMV's last CTA
static int launch_loop_spmv(const bjac_handle *h, cudaStream_t st, bool finish_alpha) {
    unsigned int *ticket = &h->d_S->tickets[kTicketSpmv];
    double *spart = h->d_part + kSpPartOff;
    if (h->use_sell)
        return launch_spmv_sell(h->sell, h->d_p, nullptr, h->d_q, spart, ticket, nullptr, h->d_S,
                                finish_alpha ? kSpPcgAlpha : kSpPcg, st);
    return launch_spmv(h->A, h->d_p, h->d_q, spart, ticket, nullptr, h->d_S, finish_alpha ? 3 : 2, st);
}

extern "C" {

const char *bjac_last_error(void) { return g_err.c_str(); }

int32_t bjac_mlp_param_count(void) { return kMlpParams; }

int bjac_setup(const bjac_csr *A, const int32_t *block_ptr, int32_t nb, const bjac_policy *policy,
               bjac_handle **out) {
    if (!out) return fail(MPBJAC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_csr_host(A);
    if (rc) return rc;
    if (!policy) return fail(MPBJAC_ERR_INVALID_ARG, "policy is NULL");
    if (!block_ptr || nb < 1) return fail(MPBJAC_ERR_INVALID_ARG, "need nb >= 1 blocks");
    if (block_ptr[0] != 0 || block_ptr[nb] != A->n)
        return fail(MPBJAC_ERR_INVALID_ARG, "block_ptr must start at 0 and end at n");
    const bjac_policy &P = *policy;
    if (P.select < BJAC_SELECT_UNIFORM || P.select > BJAC_SELECT_KT)
        return fail(MPBJAC_ERR_INVALID_ARG, "unknown select");
    const bool kt = P.select == BJAC_SELECT_KT;
    int bs_max = 0, ubs = block_ptr[1] - block_ptr[0];
    for (int b = 0; b < nb; ++b) {
        const int bs = block_ptr[b + 1] - block_ptr[b];
        if (bs < 1 || (!kt && bs > 128)) return fail(MPBJAC_ERR_INVALID_ARG, "every block needs 1..128 rows");
        bs_max = std::max(bs_max, bs);
        if (bs != ubs) ubs = 0;
    }
    if (kt) {
        if (P.fixed_fmt != BJAC_FP64 && P.fixed_fmt != BJAC_FP32)
            return fail(MPBJAC_ERR_INVALID_ARG, "BJAC(k,t) takes fixed_fmt FP64 or FP32");
        if (P.temporal != BJAC_TEMPORAL_NONE && P.fixed_fmt != BJAC_FP32)
            return fail(MPBJAC_ERR_INVALID_ARG, "aMP switching needs the binary32 BJAC(k,t) set");
        if (P.kt_outer < 0 || P.kt_inner < 0 || P.kt_outer > 64 || P.kt_inner > 64)
            return fail(MPBJAC_ERR_INVALID_ARG, "kt_outer and kt_inner must be 0..64 (0: 2)");
    }
    if (P.select == BJAC_SELECT_GIVEN) {
        if (!P.block_fmt) return fail(MPBJAC_ERR_INVALID_ARG, "SELECT_GIVEN needs block_fmt");
        for (int b = 0; b < nb; ++b)
            if (P.block_fmt[b] > BJAC_FP16S) return fail(MPBJAC_ERR_INVALID_ARG, "block_fmt entries must be 0..3");
    }
    if (P.select == BJAC_SELECT_FIXED && (P.fixed_fmt < BJAC_FP64 || P.fixed_fmt > BJAC_FP16S))
        return fail(MPBJAC_ERR_INVALID_ARG, "unknown fixed_fmt");
    if (P.temporal < BJAC_TEMPORAL_NONE || P.temporal > BJAC_TEMPORAL_LH)
        return fail(MPBJAC_ERR_INVALID_ARG, "unknown temporal policy");
    if (P.select == BJAC_SELECT_MLP && !P.mlp_params)
        return fail(MPBJAC_ERR_INVALID_ARG, "SELECT_MLP needs mlp_params");
    if (P.temporal != BJAC_TEMPORAL_NONE && P.select == BJAC_SELECT_UNIFORM)
        return fail(MPBJAC_ERR_INVALID_ARG, "aMP switching needs a low-precision set");
    if (P.spmv_format < 0 || P.spmv_format > 3) return fail(MPBJAC_ERR_INVALID_ARG, "spmv_format must be 0..3");
    if (P.flexible != 0 && P.flexible != 1) return fail(MPBJAC_ERR_INVALID_ARG, "flexible must be 0 or 1");

    bjac_handle *h = new bjac_handle();
    h->A = *A;
    h->pol = P;
    if (h->pol.theta <= 0.0) h->pol.theta = 0.1;
    if (h->pol.safety_theta <= 0.0) h->pol.safety_theta = 0.5;
    h->pol.mlp_params = nullptr;   // not retained
    h->pol.block_fmt = nullptr;
    h->stream = (cudaStream_t)P.stream;
    h->n = A->n;
    h->nb = nb;
    h->bs_max = bs_max;
    h->ubs = ubs;
    h->h_block_ptr.assign(block_ptr, block_ptr + nb + 1);
    cudaStream_t st = h->stream;
    MPB_TRY(cudaEventCreate(&h->ev0) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "cudaEventCreate"));
    MPB_TRY(cudaEventCreate(&h->ev1) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "cudaEventCreate"));
    if (cudaEventRecord(h->ev0, st) != cudaSuccess) { free_handle(h); return cuda_fail(cudaGetLastError(), "event"); }

    if (kt) {
        // BJAC(k, t) of Eq. 3-2 / 3-3: no block inverses; diag(A), block ids and the SELL-32 copy
        h->h_goff.assign(nb + 1, 0);
        h->have_hi = true;
        h->have_lo = P.fixed_fmt == BJAC_FP32;
        h->blocks_per_fmt[h->have_lo ? BJAC_FP32 : BJAC_FP64] = nb;
        MPB_TRY(dalloc(&h->d_block_ptr, nb + 1));
        MPB_TRY(dalloc(&h->d_status, 2));
        MPB_TRY(cudaMemcpyAsync(h->d_block_ptr, block_ptr, sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, st) ==
                        cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "copy block_ptr"));
        MPB_TRY(cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) == cudaSuccess
                    ? 0 : cuda_fail(cudaGetLastError(), "memset"));
        k_validate_csr<<<std::max(1, std::min(sm_count() * 4, (A->nnz + 255) / 256)), 256, 0, st>>>(
            A->n, A->nnz, A->rowptr, A->colidx, h->d_status);
        int vstat[2] = {0, 0};
        MPB_TRY(cudaMemcpyAsync(vstat, h->d_status, sizeof(vstat), cudaMemcpyDeviceToHost, st) == cudaSuccess
                    ? 0 : cuda_fail(cudaGetLastError(), "copy status"));
        MPB_TRY(cudaStreamSynchronize(st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "validate csr"));
        if (vstat[0] != 0) {
            free_handle(h);
            return fail(MPBJAC_ERR_INVALID_ARG, "CSR arrays are inconsistent (rowptr not monotone / column out of range)");
        }
        int bad = -1;
        MPB_TRY(kt_build(*A, h->d_block_ptr, nb, P.kt_outer > 0 ? P.kt_outer : 2, P.kt_inner > 0 ? P.kt_inner : 2,
                         h->have_lo, &h->kt, &bad, st));
        MPB_TRY(prepare_spmv(*A));
    } else {
    // geometry
        h->h_goff.resize(nb + 1);
        h->h_goff[0] = 0;
        for (int b = 0; b < nb; ++b) {
            const int64_t bs = block_ptr[b + 1] - block_ptr[b];
            h->h_goff[b + 1] = h->h_goff[b] + bs * bs;
        }
        const bool fixed_now = P.select == BJAC_SELECT_FIXED || P.select == BJAC_SELECT_UNIFORM ||
                               P.select == BJAC_SELECT_GIVEN;
        h->have_hi = P.select == BJAC_SELECT_UNIFORM || P.temporal != BJAC_TEMPORAL_NONE || P.fp64_fallback ||
                     !fixed_now;
        h->have_lo = P.select != BJAC_SELECT_UNIFORM;

        MPB_TRY(dalloc(&h->d_block_ptr, nb + 1));
        MPB_TRY(dalloc(&h->d_goff, nb + 1));
        MPB_TRY(dalloc(&h->d_status, 2));
        MPB_TRY(dalloc(&h->d_fmt, nb));
        MPB_TRY(dalloc(&h->d_scale, nb));
        MPB_TRY(dalloc(&h->d_qoff, nb + 1));
        MPB_TRY(dalloc(&h->d_kap, 2 * (size_t)nb));
        MPB_TRY(dalloc(&h->d_feat, 12 * (size_t)nb));
        if (h->have_hi) MPB_TRY(dalloc(&h->d_G, (size_t)h->h_goff[nb]));
        MPB_TRY(cudaMemcpyAsync(h->d_block_ptr, block_ptr, sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, st) ==
                        cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "copy block_ptr"));
        MPB_TRY(cudaMemcpyAsync(h->d_goff, h->h_goff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, st) ==
                        cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "copy goff"));
        MPB_TRY(cudaMemsetAsync(h->d_status, 0, 2 * sizeof(int), st) == cudaSuccess ? 0
                                                                                    : cuda_fail(cudaGetLastError(), "memset"));
        k_validate_csr<<<std::max(1, std::min(sm_count() * 4, (A->nnz + 255) / 256)), 256, 0, st>>>(
            A->n, A->nnz, A->rowptr, A->colidx, h->d_status);
        int hstat[2] = {0, 0};
        MPB_TRY(cudaMemcpyAsync(hstat, h->d_status, sizeof(hstat), cudaMemcpyDeviceToHost, st) == cudaSuccess
                    ? 0 : cuda_fail(cudaGetLastError(), "copy status"));
        MPB_TRY(cudaStreamSynchronize(st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "validate csr"));
        if (hstat[0] != 0) {
            free_handle(h);
            return fail(MPBJAC_ERR_INVALID_ARG, "CSR arrays are inconsistent (rowptr not monotone / column out of range)");
        }

        // low-precision pool offsets known now for fixed formats
        int fixed_fmt = P.select == BJAC_SELECT_UNIFORM ? BJAC_FP64 : P.fixed_fmt;
        auto set_qoff = [&](const std::vector<uint8_t> &fmts) {
            h->h_qoff.assign(nb + 1, 0);
            for (int b = 0; b < nb; ++b) {
                const int64_t bs = block_ptr[b + 1] - block_ptr[b];
                int64_t bytes = bs * bs * fmt_bytes(fmts.empty() ? fixed_fmt : fmts[b]);
                bytes = (bytes + 15) & ~int64_t(15);
                h->h_qoff[b + 1] = h->h_qoff[b] + bytes;
            }
            h->pool_bytes = h->h_qoff[nb];
        };
        SetupArgs a{};
        a.n = A->n;
        a.rowptr = A->rowptr;
        a.colidx = A->colidx;
        a.val = A->val;
        a.block_ptr = h->d_block_ptr;
        a.nb = nb;
        a.goff = h->d_goff;
        a.G = h->d_G;
        a.select = P.select;
        a.fixed_fmt = fixed_fmt;
        a.theta = h->pol.theta;
        a.fmt = h->d_fmt;
        a.scale = h->d_scale;
        a.feat = h->d_feat;
        a.kap = h->d_kap;
        a.status = h->d_status;
        if (h->have_lo && fixed_now) {
            if (P.select == BJAC_SELECT_GIVEN) {
                std::vector<uint8_t> given(P.block_fmt, P.block_fmt + nb);
                set_qoff(given);
                MPB_TRY(cudaMemcpyAsync(h->d_fmt, P.block_fmt, nb, cudaMemcpyHostToDevice, st) == cudaSuccess
                            ? 0 : cuda_fail(cudaGetLastError(), "copy block_fmt"));
                a.given = h->d_fmt;
            } else {
                set_qoff({});
            }
            MPB_TRY(dalloc(&h->d_pool, (size_t)h->pool_bytes));
            MPB_TRY(cudaMemcpyAsync(h->d_qoff, h->h_qoff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice,
                                    st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "copy qoff"));
            a.qoff = h->d_qoff;
            a.pool = h->d_pool;
        }
        MPB_TRY(prepare_spmv(*A));
        MPB_TRY(launch_setup_blocks(a, bs_max, h->h_block_ptr.data(), st));
        if (P.select == BJAC_SELECT_MLP) {
            MPB_TRY(launch_mlp_select(P.mlp_params, nb, h->d_feat, h->d_kap, h->pol.safety_theta, h->d_fmt, st));
        }
        std::vector<uint8_t> hfmt(nb);
        MPB_TRY(cudaMemcpyAsync(hfmt.data(), h->d_fmt, nb, cudaMemcpyDeviceToHost, st) == cudaSuccess
                    ? 0 : cuda_fail(cudaGetLastError(), "copy fmt"));
        MPB_TRY(cudaMemcpyAsync(hstat, h->d_status, sizeof(hstat), cudaMemcpyDeviceToHost, st) == cudaSuccess
                    ? 0 : cuda_fail(cudaGetLastError(), "copy status"));
        MPB_TRY(cudaStreamSynchronize(st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "setup kernel"));
        if (hstat[0] != 0) {
            free_handle(h);
            return fail(MPBJAC_ERR_NOT_SPD, "diagonal block " + std::to_string(hstat[1]) +
                                                " has a non-positive pivot (not positive definite)");
        }
        if (P.select == BJAC_SELECT_MLP) {
            for (int b = 0; b < nb; ++b)
                if (hfmt[b] > BJAC_FP16S) {
                    free_handle(h);
                    return fail(MPBJAC_ERR_TIMEOUT, "the selector's tensor-core MMA did not complete (block " +
                                                        std::to_string(b) + ")");
                }
        }
        if (h->have_lo && !fixed_now) {     // per-block formats: compact pool, second pass
            set_qoff(hfmt);
            MPB_TRY(dalloc(&h->d_pool, (size_t)h->pool_bytes));
            MPB_TRY(cudaMemcpyAsync(h->d_qoff, h->h_qoff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice,
                                    st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "copy qoff"));
            MPB_TRY(launch_pack(nb, h->d_block_ptr, h->d_goff, h->d_G, h->d_fmt, h->d_qoff, h->d_pool, h->d_scale, st));
        }
        int ufmt = -1;
        if (h->have_lo) {
            ufmt = hfmt[0];
            for (int b = 0; b < nb; ++b) {
                h->blocks_per_fmt[hfmt[b] & 3] += 1;
                if (hfmt[b] != ufmt) ufmt = -1;
            }
            h->lo = make_pset(h, h->d_fmt, h->d_scale, h->d_qoff, h->d_pool, ufmt);
            if (tma_supported(h->lo, h->n)) MPB_TRY(prepare_apply_tma(h->lo));
            MPB_TRY(choose_apply_kind(h));
        } else {
            h->blocks_per_fmt[BJAC_FP64] = nb;
        }
        if (h->have_hi) {
            std::vector<int64_t> qhi(nb + 1);
            for (int b = 0; b <= nb; ++b) qhi[b] = h->h_goff[b] * 8;
            std::vector<float> ones(nb, 1.0f);
            MPB_TRY(dalloc(&h->d_fmt_hi, nb));
            MPB_TRY(dalloc(&h->d_scale_hi, nb));
            MPB_TRY(dalloc(&h->d_qoff_hi, nb + 1));
            MPB_TRY(cudaMemsetAsync(h->d_fmt_hi, 0, nb, st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "memset"));
            MPB_TRY(cudaMemcpyAsync(h->d_scale_hi, ones.data(), sizeof(float) * nb, cudaMemcpyHostToDevice, st) ==
                            cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "copy"));
            MPB_TRY(cudaMemcpyAsync(h->d_qoff_hi, qhi.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, st) ==
                            cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "copy"));
            h->hi = make_pset(h, h->d_fmt_hi, h->d_scale_hi, h->d_qoff_hi, reinterpret_cast<uint8_t *>(h->d_G),
                              BJAC_FP64);
        }
    }
    // solve workspace
    const size_t n = (size_t)A->n;
    MPB_TRY(dalloc(&h->d_r, n));
    MPB_TRY(dalloc(&h->d_z, n));
    MPB_TRY(dalloc(&h->d_p, n));
    MPB_TRY(dalloc(&h->d_q, n));
    // up to 3 partial sums per CTA of the apply, then the loop SpMV's (stride 2) at kSpPartOff
    MPB_TRY(dalloc(&h->d_part, (size_t)kSpPartOff + 2 * (size_t)kMaxGrid));
    MPB_TRY(dalloc(&h->d_S, 1));
    if (P.fp64_fallback) MPB_TRY(dalloc(&h->d_x0, n));
    MPB_TRY(cudaMallocHost((void **)&h->h_S, sizeof(SolverState)) == cudaSuccess
                ? 0 : cuda_fail(cudaGetLastError(), "cudaMallocHost"));
    memset(h->h_S, 0, sizeof(SolverState));
    MPB_TRY(cudaMemsetAsync(h->d_S, 0, sizeof(SolverState), st) == cudaSuccess
                ? 0 : cuda_fail(cudaGetLastError(), "memset"));
    MPB_TRY(choose_spmv_format(h));
    MPB_TRY(cudaEventRecord(h->ev1, st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "event"));
    MPB_TRY(cudaStreamSynchronize(st) == cudaSuccess ? 0 : cuda_fail(cudaGetLastError(), "setup"));
    cudaEventElapsedTime(&h->setup_ms, h->ev0, h->ev1);
    *out = h;
    return MPBJAC_OK;
}

void bjac_destroy(bjac_handle *h) { free_handle(h); }

}  // extern "C"

// ------------------------------------------------------------------------------------------
// PCG driver
// ------------------------------------------------------------------------------------------
static ApplyIO base_io(bjac_handle *h) {
    ApplyIO io{};
    io.r = h->d_r;
    io.r_out = h->d_r;
    io.q = h->d_q;
    io.z = h->d_z;
    io.p = h->d_p;
    io.part = h->d_part;
    io.spart = h->d_part + kSpPartOff;
    io.ticket = &h->d_S->tickets[kTicketApply];
    io.out = nullptr;
    io.err = nullptr;
    io.set = 1;
    io.only_set = -1;
    return io;
}

// Apply for the init / aMP modes: the set is read on the device (S->use_low). The
// binary64 set always goes to the generic kernel; the low set to the TMA kernel when it
// fits one, each launch returning at once when the other set is selected.
static bool lo_uses_tma(const bjac_handle *h) { return h->have_lo && h->apply_kind != kApplyKindGeneric; }

// launch the low-precision set's specialised kernel (TMA-staged or register-direct)
static int launch_lo_special(const bjac_handle *h, int mode, const ApplyIO &io, cudaStream_t st) {
    if (h->apply_kind == kApplyKindReg) return launch_apply_reg(mode, h->lo, io, h->d_S, st);
    if (h->apply_kind == kApplyKindMix) return launch_apply_mix(mode, h->lo, io, h->d_S, st);
    return launch_apply_tma(mode, h->lo, io, h->d_S, h->n, st);
}

static int launch_apply_select(bjac_handle *h, int mode, cudaStream_t st, bool low_only, bool high_only) {
    ApplyIO io = base_io(h);
    const bool lo_tma = lo_uses_tma(h);
    PSet lo = h->have_lo ? h->lo : h->hi;
    PSet hi = h->have_hi ? h->hi : h->lo;
    if (lo_tma && !high_only) {
        int rc = launch_lo_special(h, mode, io, st);
        if (rc) return rc;
        if (low_only) return MPBJAC_OK;
        io.only_set = 0;
        return launch_apply_generic(mode, lo, hi, io, h->d_S, st);
    }
    io.only_set = low_only ? 1 : (high_only ? 0 : -1);
    return launch_apply_generic(mode, lo, hi, io, h->d_S, st);
}


#define MPB_TRY_RC(expr)          \
    do {                          \
        const int rc_ = (expr);   \
        if (rc_) return rc_;      \
    } while (0)

// The first preconditioner application of a (re)start: z = M^-1 r, p = z, rho = r.z.
static int launch_init_apply(bjac_handle *h, bool temporal, bool low_only, bool high_only, cudaStream_t st,
                             long long *launches) {
    if (h->pol.select == BJAC_SELECT_KT) {
        ApplyIO io = base_io(h);
        int n = 0;
        if (temporal) {
            MPB_TRY_RC(launch_kt_apply(kApplyInit, 1, true, h->kt, io, h->d_S, st, &n));
            MPB_TRY_RC(launch_kt_apply(kApplyInit, 0, true, h->kt, io, h->d_S, st, &n));
        } else {
            MPB_TRY_RC(launch_kt_apply(kApplyInit, low_only ? 1 : 0, false, h->kt, io, h->d_S, st, &n));
        }
        *launches += n;
        return MPBJAC_OK;
    }
    MPB_TRY_RC(launch_apply_select(h, kApplyInit, st, low_only, high_only));
    *launches += (lo_uses_tma(h) && !high_only && !low_only) ? 2 : 1;
    return MPBJAC_OK;
}

// Iterations per body of the device-side while loop. After convergence the remaining copies
// of the body return at once; the loop condition is evaluated once per body.
constexpr int kBodyIters = 4;

// launches made by this thread carry the programmatic attribute while on
namespace mpbjac {
static thread_local bool t_pdl = false;
bool pdl_on() { return t_pdl; }
void pdl_set(bool on) { t_pdl = on; }
}  // namespace mpbjac
struct PdlOff {
    ~PdlOff() { pdl_set(false); }
};

// aMP runs as a speculative application plus a redo (k_apply_spec) when both sets are uniform
// 32-row blocks (the low one of one format) and no other apply kernel is forced; otherwise the
// residual update, the application and the flexible beta are separate kernels.
static bool amp_spec(const bjac_handle *h) {
    if (h->pol.select == BJAC_SELECT_KT || !h->have_lo || !h->have_hi) return false;
    if (h->pol.apply_variant != 0 && h->pol.apply_variant != 3) return false;
    return spec_supported(h->lo, h->hi, h->n);
}

// One PCG iteration: captured into the body of a device-side while loop, or launched
// eagerly by the profiler with an event between kernels (ev != nullptr: ev[0..4]).
// pdl_first: the SpMV may overlap its predecessor kernel (programmatic launch; the later
// kernels of the iteration always may, unless events sit between them). set_cond: this
// copy's x/p update sets the while-loop condition. *launches += kernels launched.
static int capture_body(bjac_handle *h, int which, cudaStream_t cs, cudaGraphConditionalHandle cond,
                        cudaEvent_t *ev, bool pdl_first, bool set_cond, int *launches) {
    PdlOff pdl_guard;
    const bool temporal = (which == 0) && h->pol.temporal != BJAC_TEMPORAL_NONE;
    const bool use_low = (which == 0) && h->have_lo;
    const bool pdl = ev == nullptr;
    const bool kt = h->pol.select == BJAC_SELECT_KT;
    if (ev) MPB_CUDA(cudaEventRecord(ev[0], cs));
    pdl_set(pdl && pdl_first);
    const bool generic_next = !kt && !temporal && !(use_low && lo_uses_tma(h));
    int rc = launch_loop_spmv(h, cs, generic_next);
    if (rc) return rc;
    *launches += 1;
    pdl_set(pdl);
    if (ev) MPB_CUDA(cudaEventRecord(ev[1], cs));
    if (kt) {
        // r -= alpha q and the convergence test first, then the sweeps of the set in use
        MPB_TRY_RC(launch_update_r(h->n, h->d_q, h->d_r, h->d_part, h->d_part + kSpPartOff, h->d_S, cs));
        *launches += 1;
        if (ev) MPB_CUDA(cudaEventRecord(ev[2], cs));
        ApplyIO io = base_io(h);
        if (temporal) {
            MPB_TRY_RC(launch_kt_apply(kApplyTemporal, 1, true, h->kt, io, h->d_S, cs, launches));
            MPB_TRY_RC(launch_kt_apply(kApplyTemporal, 0, true, h->kt, io, h->d_S, cs, launches));
        } else {
            MPB_TRY_RC(launch_kt_apply(kApplyTemporal, use_low ? 1 : 0, false, h->kt, io, h->d_S, cs, launches));
        }
    } else if (temporal && amp_spec(h)) {
        // speculative application with the previous set, fused with r -= alpha q, then the
        // redo that runs only when this residual's relres picked the other set
        if (ev) MPB_CUDA(cudaEventRecord(ev[2], cs));
        ApplyIO io = base_io(h);
        io.flex = h->pol.flexible;
        MPB_TRY_RC(launch_apply_spec(kApplySpec, h->lo, h->hi, io, h->d_S, cs));
        MPB_TRY_RC(launch_apply_spec(kApplyRedo, h->lo, h->hi, io, h->d_S, cs));
        *launches += 2;
    } else if (temporal) {
        MPB_TRY_RC(launch_update_r(h->n, h->d_q, h->d_r, h->d_part, h->d_part + kSpPartOff, h->d_S, cs));
        if (ev) MPB_CUDA(cudaEventRecord(ev[2], cs));
        rc = launch_apply_select(h, kApplyTemporal, cs, false, false);
        if (rc) return rc;
        *launches += lo_uses_tma(h) ? 3 : 2;
    } else {
        if (ev) MPB_CUDA(cudaEventRecord(ev[2], cs));
        ApplyIO io = base_io(h);
        io.set = use_low ? 1 : 0;
        io.flex = h->pol.flexible;
        if (use_low && lo_uses_tma(h)) rc = launch_lo_special(h, kApplyFused, io, cs);
        else rc = launch_apply_generic(kApplyFused, use_low ? h->lo : h->hi, h->have_hi ? h->hi : h->lo, io,
                                       h->d_S, cs);
        if (rc) return rc;
        *launches += 1;
    }
    // the fused register kernels sum q.z themselves and finish the flexible beta
    const bool flex_fused = (!kt && !temporal && use_low && lo_uses_tma(h) &&
                             (h->apply_kind == kApplyKindReg || h->apply_kind == kApplyKindMix)) ||
                            (temporal && amp_spec(h));
    if (h->pol.flexible && !flex_fused) {
        MPB_TRY_RC(launch_flex_beta(h->n, h->d_q, h->d_z, h->d_part, h->d_S, cs));
        *launches += 1;
    }
    if (ev) MPB_CUDA(cudaEventRecord(ev[3], cs));
    MPB_TRY_RC(launch_update_xp(h->n, h->d_z, h->d_p, h->d_S, cond, set_cond ? 1 : 0, cs));
    *launches += 1;
    if (ev) MPB_CUDA(cudaEventRecord(ev[4], cs));
    return MPBJAC_OK;
}

static int build_graph(bjac_handle *h, int which) {
    cudaGraph_t g = nullptr;
    MPB_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cudaGraphConditionalHandleCreate"); }
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cudaGraphAddNode(while)"); }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cudaStreamCreate"); }
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); cudaGraphDestroy(g); return cuda_fail(e, "BeginCaptureToGraph"); }
    int rc = MPBJAC_OK, body_launches = 0;
    for (int k = 0; k < kBodyIters && rc == MPBJAC_OK; ++k)
        rc = capture_body(h, which, cs, cond, nullptr, k > 0, k == kBodyIters - 1, &body_launches);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (rc || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return rc ? rc : cuda_fail(e, "EndCapture");
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cudaGraphInstantiate"); }
    h->graph[which] = g;
    h->exec[which] = ex;
    h->body_launches[which] = body_launches;
    return MPBJAC_OK;
}

// Process-wide: loop kernels give the PCG vectors an evict_last L2 policy (bjac_l2_residency).
static int g_l2_keep = 1;

// One full solve with preconditioner selection `which` (0 = policy, 1 = binary64 fallback).
static int run_solve(bjac_handle *h, int which, const double *b, double *x, double tol, int maxit, double *hist,
                     int *graph_launches) {
    cudaStream_t st = h->stream;
    SolverState &hs = *h->h_S;
    memset(&hs, 0, sizeof(SolverState));
    hs.tol = tol;
    hs.adp_tol = h->pol.adp_tol;
    hs.x = x;
    hs.hist = hist;
    hs.maxit = maxit;
    hs.temporal = which == 0 ? h->pol.temporal : BJAC_TEMPORAL_NONE;
    hs.low_default = (which == 0 && h->have_lo) ? 1 : 0;
    hs.l2_keep = g_l2_keep;
    hs.flexible = h->pol.flexible;
    MPB_CUDA(cudaMemcpyAsync(h->d_S, &hs, sizeof(SolverState), cudaMemcpyHostToDevice, st));
    int rc = launch_residual(h->A, b, x, h->d_r, h->d_part, &h->d_S->tickets[kTicketRes], nullptr, h->d_S, 1, st);
    if (rc) return rc;
    k_zero_if_zero_rhs<<<vec_grid(h->n), kNT, 0, st>>>(h->n, h->d_S);
    h->launches += 2;
    const bool eager = h->pol.graph_mode == 1;
    if (!eager && !h->exec[which]) {
        rc = build_graph(h, which);
        if (rc) return rc;
    }
    int iter_before = 0;
    for (int pass = 0; pass < 9; ++pass) {
        const bool temporal = hs.temporal != BJAC_TEMPORAL_NONE;
        const bool low_only = !temporal && hs.low_default == 1, high_only = !temporal && hs.low_default == 0;
        rc = launch_init_apply(h, temporal, low_only, high_only, st, &h->launches);
        if (rc) return rc;
        if (eager) {
            // the same loop body, enqueued from the host in batches of 32 iterations; once the
            // state leaves "running" every kernel returns at once
            int32_t state = kRunning;
            int n_launch = 0;
            while (state == kRunning) {
                for (int k = 0; k < 32; ++k) {
                    rc = capture_body(h, which, st, cudaGraphConditionalHandle{}, nullptr, true, false, &n_launch);
                    if (rc) return rc;
                }
                MPB_CUDA(cudaMemcpyAsync(&state, &h->d_S->state, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                MPB_CUDA(cudaStreamSynchronize(st));
            }
            h->launches += n_launch;
        } else {
            MPB_CUDA(cudaGraphLaunch(h->exec[which], st));
            *graph_launches += 1;
        }
        rc = launch_residual(h->A, b, x, h->d_r, h->d_part, &h->d_S->tickets[kTicketRes], nullptr, h->d_S, 2, st);
        if (rc) return rc;
        h->launches += 1;
        MPB_CUDA(cudaMemcpyAsync(&hs, h->d_S, sizeof(SolverState), cudaMemcpyDeviceToHost, st));
        MPB_CUDA(cudaStreamSynchronize(st));
        if (!eager) {
            // the body runs at least once per graph launch, then until a body ends with the
            // state no longer running
            const int ran = hs.iter - iter_before;
            const int bodies = ran > 0 ? (ran + kBodyIters - 1) / kBodyIters : 1;
            h->launches += (long long)bodies * h->body_launches[which];
        }
        iter_before = hs.iter;
        if (hs.state != kRunning) break;      // no restart requested
    }
    return MPBJAC_OK;
}

extern "C" int pcg_solve(bjac_handle *h, const double *b, double *x, double tol, int32_t maxit, pcg_stats *stats,
                         double *relres_hist) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "handle is NULL");
    if (!b || !x) return fail(MPBJAC_ERR_INVALID_ARG, "b and x must be device pointers");
    if (maxit < 0 || !(tol >= 0.0)) return fail(MPBJAC_ERR_INVALID_ARG, "need maxit >= 0 and tol >= 0");
    cudaStream_t st = h->stream;
    MPB_CUDA(cudaEventRecord(h->ev0, st));
    if (h->d_x0) MPB_CUDA(cudaMemcpyAsync(h->d_x0, x, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
    int launches = 0;
    h->launches = 0;
    int rc = run_solve(h, 0, b, x, tol, maxit, relres_hist, &launches);
    if (rc) return rc;
    SolverState res = *h->h_S;
    int fallback = 0;
    auto status_of = [&](const SolverState &s) {
        if (s.state == kTimeout) return MPBJAC_ERR_TIMEOUT;
        if (s.state == kBreakdown || s.state == kBreakdownSigma) return MPBJAC_ERR_BREAKDOWN;
        if (s.state == kConverged && s.true_relres <= tol) return MPBJAC_OK;
        return MPBJAC_NOT_CONVERGED;
    };
    int status = status_of(res);
    if (status != MPBJAC_OK && status != MPBJAC_ERR_TIMEOUT && h->pol.fp64_fallback && h->have_lo && h->have_hi) {
        MPB_CUDA(cudaMemcpyAsync(x, h->d_x0, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
        rc = run_solve(h, 1, b, x, tol, maxit, relres_hist, &launches);
        if (rc) return rc;
        const int lo_ap = res.low_applies;
        res = *h->h_S;
        res.low_applies += lo_ap;
        status = status_of(res);
        fallback = 1;
    }
    MPB_CUDA(cudaEventRecord(h->ev1, st));
    MPB_CUDA(cudaEventSynchronize(h->ev1));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->iters = res.iter;
        stats->converged = status == MPBJAC_OK;
        stats->status = status;
        stats->restarts = res.restarts;
        stats->fallback_used = fallback;
        stats->low_applies = res.low_applies;
        stats->high_applies = res.high_applies;
        stats->graph_launches = launches;
        stats->kernel_launches = h->launches > INT32_MAX ? INT32_MAX : (int32_t)h->launches;
        stats->relres = res.relres;
        stats->true_relres = res.true_relres;
        for (int i = 0; i < 4; ++i) stats->blocks_per_fmt[i] = h->blocks_per_fmt[i];
        stats->setup_ms = h->setup_ms;
        cudaEventElapsedTime(&stats->solve_ms, h->ev0, h->ev1);
    }
    if (status == MPBJAC_ERR_TIMEOUT) set_error("a bounded wait of a loop kernel expired (a TMA copy did not land)");
    if (status == MPBJAC_ERR_BREAKDOWN) set_error("PCG breakdown (p.Ap <= 0 or r.z <= 0 or non-finite)");
    else if (status == MPBJAC_NOT_CONVERGED) set_error("maximum number of iterations reached");
    return status;
}

// ------------------------------------------------------------------------------------------
// single steps
// ------------------------------------------------------------------------------------------
// standalone SpMV kinds on a SELL-32 copy built for this call alone (bjac_spmv_kernel(5),
// for tests of the layout on any matrix); synchronises the stream before freeing the copy
static int sell_once(const bjac_csr &A, int kind, const double *x, const double *b, double *y, double *part,
                     unsigned int *ticket, double *out, cudaStream_t st) {
    SellMat m;
    int rc = sell_build(A, 0.0, &m, st);
    if (rc) return rc;
    if (!m.val) return fail(MPBJAC_ERR_UNSUPPORTED, "A needs more than 2^31 stored SELL-32 entries");
    rc = launch_spmv_sell(m, x, b, y, part, ticket, out, nullptr, kind, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    sell_free(&m);
    if (rc) return rc;
    return e == cudaSuccess ? MPBJAC_OK : cuda_fail(e, "SELL-32 SpMV");
}

extern "C" int bjac_spmv(const bjac_csr *A, const double *x, double *y, double *xy, void *stream) {
    int rc = check_csr_host(A);
    if (rc) return rc;
    if (!x || !y) return fail(MPBJAC_ERR_INVALID_ARG, "x and y must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    rc = prepare_spmv(*A);
    if (rc) return rc;
    const bool sell = spmv_forced_sell();
    if (!xy) {
        if (sell) return sell_once(*A, kSpY, x, nullptr, y, nullptr, nullptr, nullptr, st);
        return launch_spmv(*A, x, y, nullptr, nullptr, nullptr, nullptr, 0, st);
    }
    // scratch for the deterministic reduction: partial sums and a ticket counter
    void *scratch = nullptr;
    const size_t bytes = sizeof(double) * kMaxGrid + 256;
    MPB_CUDA(cudaMallocAsync(&scratch, bytes, st));
    double *part = static_cast<double *>(scratch);
    unsigned int *ticket = reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + sizeof(double) * kMaxGrid);
    MPB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
    rc = sell ? sell_once(*A, kSpYDot, x, nullptr, y, part, ticket, xy, st)
              : launch_spmv(*A, x, y, part, ticket, xy, nullptr, 1, st);
    cudaFreeAsync(scratch, st);
    return rc;
}

extern "C" int bjac_residual(const bjac_csr *A, const double *b, const double *x, double *r, double *rr,
                             void *stream) {
    int rc = check_csr_host(A);
    if (rc) return rc;
    if (!b || !x || !r) return fail(MPBJAC_ERR_INVALID_ARG, "b, x and r must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    rc = prepare_spmv(*A);
    if (rc) return rc;
    void *scratch = nullptr;
    const size_t bytes = sizeof(double) * 2 * kMaxGrid + 256;
    MPB_CUDA(cudaMallocAsync(&scratch, bytes, st));
    double *part = static_cast<double *>(scratch);
    unsigned int *ticket =
        reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + sizeof(double) * 2 * kMaxGrid);
    double *dummy = reinterpret_cast<double *>(static_cast<char *>(scratch) + sizeof(double) * 2 * kMaxGrid + 64);
    MPB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
    rc = spmv_forced_sell() ? sell_once(*A, kResStandalone, x, b, r, part, ticket, rr ? rr : dummy, st)
                            : launch_residual(*A, b, x, r, part, ticket, rr ? rr : dummy, nullptr, 0, st);
    cudaFreeAsync(scratch, st);
    return rc;
}

extern "C" int bjac_apply(bjac_handle *h, int32_t set, const double *r, double *z, double *rz) {
    if (!h || !r || !z) return fail(MPBJAC_ERR_INVALID_ARG, "handle, r and z must be non-NULL");
    if (set != 0 && set != 1) return fail(MPBJAC_ERR_INVALID_ARG, "set must be 0 or 1");
    if ((set == 1 && !h->have_lo) || (set == 0 && !h->have_hi))
        return fail(MPBJAC_ERR_UNSUPPORTED, "requested preconditioner set was not kept");
    ApplyIO io = base_io(h);
    io.r = r;
    io.r_out = nullptr;
    io.q = nullptr;
    io.z = z;
    io.p = nullptr;
    io.out = rz;
    io.set = set;
    if (h->pol.select == BJAC_SELECT_KT) return launch_kt_apply(kApplyStandalone, set, false, h->kt, io, nullptr,
                                                                h->stream, nullptr);
    // bulk copies need 16-byte aligned sources
    const bool aligned = (reinterpret_cast<uintptr_t>(r) & 15) == 0;
    if (set == 1 && lo_uses_tma(h) && (aligned || h->apply_kind >= kApplyKindReg)) {
        if (h->apply_kind == kApplyKindReg) return launch_apply_reg(kApplyStandalone, h->lo, io, nullptr, h->stream);
        if (h->apply_kind == kApplyKindMix) return launch_apply_mix(kApplyStandalone, h->lo, io, nullptr, h->stream);
        return launch_apply_tma(kApplyStandalone, h->lo, io, nullptr, h->n, h->stream);
    }
    return launch_apply_generic(kApplyStandalone, h->have_lo ? h->lo : h->hi, h->have_hi ? h->hi : h->lo, io,
                                nullptr, h->stream);
}

extern "C" int bjac_l2_residency(int32_t keep) {
    if (keep != 0 && keep != 1) return fail(MPBJAC_ERR_INVALID_ARG, "keep must be 0 or 1");
    const int old = g_l2_keep;
    g_l2_keep = keep;
    return old;
}

extern "C" int bjac_handle_spmv(bjac_handle *h, const double *x, double *y, double *xy) {
    if (!h || !x || !y) return fail(MPBJAC_ERR_INVALID_ARG, "handle, x and y must be non-NULL");
    unsigned int *ticket = &h->d_S->tickets[kTicketSpmv];
    const int mode = xy ? 1 : 0;
    if (h->use_sell)
        return launch_spmv_sell(h->sell, x, nullptr, y, h->d_part, ticket, xy, nullptr, mode ? kSpYDot : kSpY,
                                h->stream);
    return launch_spmv(h->A, x, y, h->d_part, ticket, xy, nullptr, mode, h->stream);
}

extern "C" int bjac_convert(const double *x, float *f, double *w, int32_t n, void *stream) {
    if (n < 0 || (n > 0 && !x)) return fail(MPBJAC_ERR_INVALID_ARG, "need n >= 0 and x");
    if (n == 0) return MPBJAC_OK;
    k_convert<<<vec_grid(n), kNT, 0, (cudaStream_t)stream>>>(n, x, f, w);
    MPB_CUDA(cudaGetLastError());
    return MPBJAC_OK;
}

extern "C" int bjac_spmv_format(const bjac_handle *h, int32_t *format, int64_t *entries, float *ms) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "handle is NULL");
    if (format) *format = h->use_sell ? 1 + h->sell.kernel : 0;
    if (entries) *entries = h->use_sell ? h->sell.entries : 0;
    if (ms)
        for (int i = 0; i < 3; ++i) ms[i] = h->spmv_ms[i];
    return MPBJAC_OK;
}

extern "C" int bjac_info(const bjac_handle *h, int32_t *nb, int64_t *pool_bytes, int64_t *g_entries) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "handle is NULL");
    if (nb) *nb = h->nb;
    if (pool_bytes) *pool_bytes = h->have_lo ? h->pool_bytes : 0;
    if (g_entries) *g_entries = h->have_hi ? h->h_goff[h->nb] : 0;
    return MPBJAC_OK;
}

extern "C" int bjac_export(bjac_handle *h, uint8_t *fmt, float *scale, int64_t *qoff, uint8_t *pool, double *G,
                           double *feat) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "handle is NULL");
    if (h->pol.select == BJAC_SELECT_KT) return fail(MPBJAC_ERR_UNSUPPORTED, "BJAC(k,t) keeps no block inverses");
    cudaStream_t st = h->stream;
    const int nb = h->nb;
    if (fmt) MPB_CUDA(cudaMemcpyAsync(fmt, h->have_lo ? h->d_fmt : h->d_fmt_hi, nb, cudaMemcpyDeviceToHost, st));
    if (scale)
        MPB_CUDA(cudaMemcpyAsync(scale, h->have_lo ? h->d_scale : h->d_scale_hi, sizeof(float) * nb,
                                 cudaMemcpyDeviceToHost, st));
    if (qoff && h->have_lo) memcpy(qoff, h->h_qoff.data(), sizeof(int64_t) * (nb + 1));
    if (pool && h->have_lo)
        MPB_CUDA(cudaMemcpyAsync(pool, h->d_pool, (size_t)h->pool_bytes, cudaMemcpyDeviceToHost, st));
    if (G && h->have_hi)
        MPB_CUDA(cudaMemcpyAsync(G, h->d_G, sizeof(double) * (size_t)h->h_goff[nb], cudaMemcpyDeviceToHost, st));
    if (feat) MPB_CUDA(cudaMemcpyAsync(feat, h->d_feat, sizeof(double) * 12 * (size_t)nb, cudaMemcpyDeviceToHost, st));
    MPB_CUDA(cudaStreamSynchronize(st));
    return MPBJAC_OK;
}

extern "C" int bjac_import_inverse(bjac_handle *h, const double *G) {
    if (!h || !G) return fail(MPBJAC_ERR_INVALID_ARG, "handle and G must be non-NULL");
    if (h->pol.select == BJAC_SELECT_KT) return fail(MPBJAC_ERR_UNSUPPORTED, "BJAC(k,t) keeps no block inverses");
    if (!h->have_hi) return fail(MPBJAC_ERR_UNSUPPORTED, "this handle keeps no binary64 set");
    cudaStream_t st = h->stream;
    MPB_CUDA(cudaMemcpyAsync(h->d_G, G, sizeof(double) * (size_t)h->h_goff[h->nb], cudaMemcpyHostToDevice, st));
    if (h->have_lo) {
        int rc = launch_pack(h->nb, h->d_block_ptr, h->d_goff, h->d_G, h->d_fmt, h->d_qoff, h->d_pool, h->d_scale, st);
        if (rc) return rc;
    }
    MPB_CUDA(cudaStreamSynchronize(st));
    return MPBJAC_OK;
}

// Eager (graph-free) run of up to min(maxit, 64) iterations of the same PCG loop, all
// enqueued back to back with CUDA events around every kernel of the loop body and one
// synchronisation at the end (so no host latency lands inside a timed interval). Iterations
// after convergence, whose kernels return at once, are left out of the averages.
// ms[0..3]: mean device time per iteration of the SpMV step, the residual-update step (aMP
// only; 0 otherwise), the preconditioner apply step, and the x/p update step.
extern "C" int pcg_profile(bjac_handle *h, const double *b, double *x, double tol, int32_t maxit, float *ms,
                           int32_t *iters) {
    if (!h || !b || !x || !ms) return fail(MPBJAC_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = h->stream;
    SolverState &hs = *h->h_S;
    memset(&hs, 0, sizeof(SolverState));
    hs.tol = tol;
    hs.adp_tol = h->pol.adp_tol;
    hs.x = x;
    hs.maxit = maxit;
    hs.temporal = h->pol.temporal;
    hs.low_default = h->have_lo ? 1 : 0;
    hs.l2_keep = g_l2_keep;
    hs.flexible = h->pol.flexible;
    MPB_CUDA(cudaMemcpyAsync(h->d_S, &hs, sizeof(SolverState), cudaMemcpyHostToDevice, st));
    int rc = launch_residual(h->A, b, x, h->d_r, h->d_part, &h->d_S->tickets[kTicketRes], nullptr, h->d_S, 1, st);
    if (rc) return rc;
    const bool temporal = hs.temporal != BJAC_TEMPORAL_NONE;
    long long init_launches = 0;
    rc = launch_init_apply(h, temporal, !temporal && hs.low_default == 1, !temporal && hs.low_default == 0, st,
                           &init_launches);
    if (rc) return rc;
    const int cap = maxit < 64 ? maxit : 64;
    std::vector<cudaEvent_t> ev((size_t)cap * 5);
    for (auto &e : ev) MPB_CUDA(cudaEventCreate(&e));
    int n_launch = 0;
    for (int k = 0; k < cap && rc == 0; ++k)
        rc = capture_body(h, 0, st, cudaGraphConditionalHandle{}, &ev[(size_t)k * 5], false, false, &n_launch);
    if (rc == 0) MPB_CUDA(cudaMemcpyAsync(&hs, h->d_S, sizeof(SolverState), cudaMemcpyDeviceToHost, st));
    if (rc == 0) MPB_CUDA(cudaStreamSynchronize(st));
    const int ran = rc == 0 ? (hs.iter < cap ? hs.iter : cap) : 0;
    double acc[4] = {0, 0, 0, 0};
    for (int k = 0; k < ran; ++k) {
        for (int i = 0; i < 4; ++i) {
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[(size_t)k * 5 + i], ev[(size_t)k * 5 + i + 1]);
            acc[i] += t;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc) return rc;
    for (int i = 0; i < 4; ++i) ms[i] = ran ? (float)(acc[i] / ran) : 0.0f;
    if (iters) *iters = ran;
    return MPBJAC_OK;
}

extern "C" int bjac_apply_kernel(const bjac_handle *h, int32_t *kind, float *tune_ms) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "handle is NULL");
    if (kind) *kind = h->apply_kind;
    if (tune_ms)
        for (int i = 0; i < 4; ++i) tune_ms[i] = h->tune_ms[i];
    return MPBJAC_OK;
}
