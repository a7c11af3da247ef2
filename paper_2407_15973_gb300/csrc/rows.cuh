// Row kernels shared by the block-apply kernels: lane i reads row i of a symmetric block
// (which is also its column i) with 16-byte loads and runs its FMA chain over the columns in
// natural order.
#pragma once
#include "common.cuh"

namespace mpbjac {

template <typename QT, int BS>
struct RegGeom {
    static constexpr int kRPL = BS / 32;                       // rows per lane
    static constexpr int kVPR = BS * (int)sizeof(QT) / 16;     // 16-byte vectors per row
    static constexpr int kEPV = 16 / (int)sizeof(QT);          // entries per vector
};

template <typename QT>
__device__ __forceinline__ float vec_entry(const uint4 &v, int e);
template <> __device__ __forceinline__ float vec_entry<float>(const uint4 &v, int e) {
    const unsigned w = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
    return __uint_as_float(w);
}
template <> __device__ __forceinline__ float vec_entry<__nv_bfloat16>(const uint4 &v, int e) {
    const unsigned w = (e >> 1) == 0 ? v.x : (e >> 1) == 1 ? v.y : (e >> 1) == 2 ? v.z : v.w;
    return __uint_as_float((e & 1) ? (w & 0xFFFF0000u) : (w << 16));     // bfloat16 -> binary32 is exact
}
template <> __device__ __forceinline__ float vec_entry<__half>(const uint4 &v, int e) {
    const unsigned w = (e >> 1) == 0 ? v.x : (e >> 1) == 1 ? v.y : (e >> 1) == 2 ? v.z : v.w;
    return __half2float(__ushort_as_half((unsigned short)((e & 1) ? (w >> 16) : (w & 0xFFFFu))));
}

// one output row of a low-precision block: row = this row's 16-byte vectors, rh = r-hat
template <typename QT>
__device__ __forceinline__ float vec_row_low(const uint4 *__restrict__ row, int vpr, const float *rh) {
    constexpr int EPV = 16 / (int)sizeof(QT);
    const float4 *rh4 = reinterpret_cast<const float4 *>(rh);
    float a = 0.0f;
    for (int v0 = 0; v0 < vpr; v0 += 2) {
        uint4 q[2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (v0 + u < vpr) q[u] = __ldg(row + v0 + u);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (v0 + u < vpr) {
#pragma unroll
                for (int e4 = 0; e4 < EPV; e4 += 4) {
                    const float4 r4 = rh4[((v0 + u) * EPV + e4) >> 2];
                    a = fmaf(vec_entry<QT>(q[u], e4 + 0), r4.x, a);
                    a = fmaf(vec_entry<QT>(q[u], e4 + 1), r4.y, a);
                    a = fmaf(vec_entry<QT>(q[u], e4 + 2), r4.z, a);
                    a = fmaf(vec_entry<QT>(q[u], e4 + 3), r4.w, a);
                }
            }
        }
    }
    return a;
}

// one output row of a binary64 block
__device__ __forceinline__ double vec_row_f64(const uint4 *__restrict__ row, int vpr, const double *r) {
    const double2 *r2 = reinterpret_cast<const double2 *>(r);
    double a = 0.0;
    for (int v0 = 0; v0 < vpr; v0 += 2) {
        uint4 q[2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (v0 + u < vpr) q[u] = __ldg(row + v0 + u);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (v0 + u < vpr) {
                const double2 rr = r2[v0 + u];
                a = fma(__hiloint2double((int)q[u].y, (int)q[u].x), rr.x, a);
                a = fma(__hiloint2double((int)q[u].w, (int)q[u].z), rr.y, a);
            }
        }
    }
    return a;
}

}  // namespace mpbjac
