// Allocation-free SpMV with its dot product.
//
// Some callers cannot allocate device memory while they run: a solver embedded in a larger
// simulation that reserved its whole device-memory budget up front, code running under a
// hard memory cap, or code that must not call cudaMalloc / cudaFree because cudaFree
// synchronises the whole device and would break the overlap they depend on. The ordinary
// bjac_spmv allocates (stream-ordered) scratch for the partial sums of x . y on every call;
// this variant reduces through a fixed buffer that lives in the library's own static device
// memory instead, and allocates nothing.
#include <mutex>

#include "apply.cuh"
#include "common.cuh"

namespace mpbjac {

int launch_spmv_dot_grid(const bjac_csr &A, const double *x, double *y, double *part, unsigned int *ticket,
                         double *out, cudaStream_t st, int max_ctas);

// One partial pair per CTA, one CTA per 256 rows: 65,536 CTAs cover n <= 16,777,216 rows.
// 1 MiB of partial sums plus the ticket counter; every GPU that loads the library holds it
// until the process exits.
constexpr int kNoAllocCtas = 65536;
constexpr long long kNoAllocMaxRows = (long long)kNoAllocCtas * 256;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocCtas + 32];

// Device address of g_noalloc_scratch, looked up once per device (with that device current).
static int scratch_address(double **out) {
    static std::mutex mu;
    static double *addr[64] = {};
    int dev = 0;
    MPB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(MPBJAC_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        addr[dev] = static_cast<double *>(p);
    }
    *out = addr[dev];
    return MPBJAC_OK;
}

}  // namespace mpbjac

extern "C" int bjac_spmv_noalloc(const bjac_csr *A, const double *x, double *y, double *xy, void *stream) {
    using namespace mpbjac;
    if (!A) return fail(MPBJAC_ERR_INVALID_ARG, "A is NULL");
    if (A->n <= 0 || A->nnz < 0) return fail(MPBJAC_ERR_INVALID_ARG, "need n > 0 and nnz >= 0");
    if (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->val)))
        return fail(MPBJAC_ERR_INVALID_ARG, "CSR pointers must be non-NULL");
    if (!x || !y || !xy) return fail(MPBJAC_ERR_INVALID_ARG, "x, y and xy must be device pointers");
    if ((long long)A->n > kNoAllocMaxRows)
        return fail(MPBJAC_ERR_INVALID_ARG, "bjac_spmv_noalloc handles at most 16,777,216 rows "
                                            "(the fixed scratch buffer holds 65,536 partial sums); use bjac_spmv");
    double *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + 2 * kNoAllocCtas);
    // the buffer keeps whatever the previous call left; the ticket must start at zero
    MPB_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
    return launch_spmv_dot_grid(*A, x, y, scratch, ticket, xy, st, kNoAllocCtas);
}
