// Sliced-ELLPACK (SELL-32) copy of a CSR matrix, owned by a handle, and its SpMV.
#pragma once
#include "common.cuh"

namespace mpbjac {

struct SellMat {
    int n = 0;
    int nslices = 0;              // ceil(n / 32); slice s holds rows 32 s .. 32 s + 31
    int32_t *off = nullptr;       // [nslices + 1] first stored entry of each slice (multiple of 32)
    int32_t *col = nullptr;       // [entries] column index, -1 for padding
    double *val = nullptr;        // [entries] value, 0 for padding
    long long entries = 0;        // stored entries including the padding
    int max_len = 0;              // longest row
    int kernel = 0;               // 0: one slice at a time per warp; 1: next slice's head prefetched
};

// Build the copy of A on the stream (reads the CSR once, writes 12 bytes per stored entry).
// If the padded copy would hold more than max_ratio * nnz entries (max_ratio > 0) or more
// than 2^31 - 64 entries, nothing is kept and out->val stays NULL. Synchronises the stream.
int sell_build(const bjac_csr &A, double max_ratio, SellMat *out, cudaStream_t st);
void sell_free(SellMat *m);

// The same kinds as the CSR SpMV (SpmvKind), with bitwise the same y: each row is summed
// as an FMA chain in CSR order.
int launch_spmv_sell(const SellMat &M, const double *x, const double *b, double *y, double *part,
                     unsigned int *ticket, double *out, SolverState *S, int kind, cudaStream_t st);

}  // namespace mpbjac
