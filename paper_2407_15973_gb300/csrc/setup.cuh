// Declarations of the setup kernels.
#pragma once
#include "common.cuh"

namespace mpbjac {

struct SetupArgs {
    int n;
    const int32_t *rowptr;
    const int32_t *colidx;
    const double *val;
    const int32_t *block_ptr;
    int nb;
    const int64_t *goff;     // element offset of block b in G
    double *G;               // binary64 inverses (nullable: not kept)
    int select;              // BJAC_SELECT_*
    int fixed_fmt;
    double theta;
    uint8_t *fmt;            // [nb] out
    float *scale;            // [nb] out
    const int64_t *qoff;     // byte offsets into pool (used only when pool != nullptr)
    uint8_t *pool;           // nullable: round in a later pass
    double *feat;            // [nb * 12] (nullable)
    double *kap;             // [2 nb]: log10 kappa_1, log10 dynamic range of G
    int *status;             // [2]: first error code, its block
    const uint8_t *given;    // [nb] formats for BJAC_SELECT_GIVEN (device), else nullptr
};

size_t setup_smem_bytes(int bs_max);
// h_block_ptr (HOST, nullable): block sizes for grouping the blocks by size class.
int launch_setup_blocks(const SetupArgs &a, int bs_max, const int32_t *h_block_ptr, cudaStream_t st);
int launch_pack(int nb, const int32_t *block_ptr, const int64_t *goff, const double *G, const uint8_t *fmt,
                const int64_t *qoff, uint8_t *pool, float *scale, cudaStream_t st);

}  // namespace mpbjac
