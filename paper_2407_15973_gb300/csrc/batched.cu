// Batched PCG: many independent systems of uneven size solved together in ONE persistent,
// cooperative kernel launch (captured in a CUDA graph). The systems' CSR matrices are
// concatenated into one block-diagonal matrix (global row / column numbering) and their
// diagonal blocks into one block list, so the setup kernels of the single-system path build
// the preconditioner unchanged. Every system keeps its own PCG scalars (alpha, beta, rho,
// relres, iteration count, state) and converges on its own; the rows of finished systems are
// skipped.
//
// Work is cut into tiles of TR rows that never cross a system (nor a diagonal block). Each
// tile's rows are also stored as 32-row slices in sliced-ELLPACK form (column-major, padded
// to the slice's longest row, padding column -1), so the SpMV's loads are coalesced and each
// row keeps its FMA chain in CSR order. Per iteration the kernel runs five phases separated
// by grid barriers, over a list of the tiles whose system is still running (rebuilt after
// every iteration, so finished systems cost nothing):
//   A  q = A p on the listed tiles, per-tile partial of p.q
//   B  per system: sigma = sum of its tiles' partials (fixed order), alpha = rho / sigma
//   C  r -= alpha q, z = M^-1 r (Algorithm 3.1 for low blocks), per-tile partials r.r, r.z
//   D  per system: relres, convergence / maxit, beta = rho' / rho
//   E  x += alpha p, p = z + beta p
// Grid barriers spin on a generation counter with a time bound; a timeout sets an error
// word and every CTA leaves at its next barrier, so a stall can never hang the GPU.
// Data one CTA writes and another reads later in the same launch (vectors gathered by the
// SpMV, per-system scalars) is read with L1-bypassing loads; a tile is always handled by
// the same warp, so its own rows need no such care.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "apply.cuh"
#include "common.cuh"
#include "rows.cuh"
#include "setup.cuh"
#include "tma.cuh"

namespace mpbjac {

struct BatchDev {
    int n_tot, nsys, ntiles;
    int32_t slot_eb;             // bytes per entry of a block's pool slot (8: room for any format)
    const int32_t *rowptr, *colidx;
    const double *val;
    const int32_t *block_ptr;
    const uint8_t *fmt;
    const float *scale;
    const int64_t *qoff;
    const uint8_t *pool;
    const int32_t *tile_row;     // [ntiles+1] first row of each tile
    const int32_t *tile_sys;     // [ntiles] owning system
    const int32_t *tile_blk;     // [ntiles] first block of each tile
    const int32_t *sys_tile;     // [nsys+1] first tile of each system
    const int4 *tinfo;           // [2 * ntiles] per tile: r0, r1, system, first block, common
                                 // block size (0 if mixed), first stored entry, slice lengths
    const int32_t *soff;         // [ntiles * TR/32 + 1] first stored entry of each 32-row slice
    const int32_t *scol;         // sliced-ELLPACK column indices (-1: padding)
    const double *sval;          // sliced-ELLPACK values
    int32_t *alist;              // [2 * ntiles] two lists of the running systems' tiles (any order)
    int32_t *nlist;              // [2] their lengths; the lists are used alternately
    const double *b;
    double *x, *r, *z, *p, *q;
    double *part;                // [2 * ntiles]
    // per-system state
    double *bnorm, *rho, *alpha, *beta, *relres, *true_relres;
    int32_t *iter, *state, *xpend, *restarts;
    double tol;
    int32_t maxit;
    // barrier and control
    unsigned int *bar_count, *bar_gen;
    int32_t *err, *active;
    int32_t *changed;            // a system left the running state this iteration: rebuild the list
    int32_t bar_extra;           // arrivals a barrier waits for beyond the grid (0; 1 = forced timeout)
};

__device__ __forceinline__ bool grid_barrier(const BatchDev &d) {
    __shared__ int s_ok;     // thread 0's decision, so that the whole CTA leaves or stays together
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = d.bar_gen;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(d.bar_count, 1u);
        if (arrived == gridDim.x - 1 + (unsigned int)d.bar_extra) {
            *d.bar_count = 0u;
            __threadfence();
            atomicAdd(d.bar_gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            int polls = 0;
            while (*gen == g) {
                if (((++polls) & 1023) == 0 && globaltimer_ns() - t0 > 2000000000ull) {
                    atomicExch(d.err, MPBJAC_ERR_TIMEOUT);
                    break;
                }
                if (*((volatile int32_t *)d.err) != 0) break;
            }
        }
        __threadfence();
        s_ok = *((volatile int32_t *)d.err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// a tile's description, read with two 16-byte loads: rows [r0, r1), system, first block,
// common block size (0 if mixed), the first stored entry of its first 32-row slice and the
// stored lengths of its (up to four) slices as 16-bit fields (slice k's entries follow slice
// k-1's: 32 x length each)
struct TileInfo {
    int r0, r1, sys, blk0, ubs, so0, len01, len23;
};
__device__ __forceinline__ int slice_len(const TileInfo &ti, int h) {
    const int w = h < 2 ? ti.len01 : ti.len23;
    return (h & 1) ? (int)((unsigned)w >> 16) : (w & 0xFFFF);
}

__device__ __forceinline__ TileInfo load_tile(const BatchDev &d, int t) {
    const int4 a = __ldg(d.tinfo + 2 * t), b = __ldg(d.tinfo + 2 * t + 1);
    return TileInfo{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}

// U entries of one sliced-ELLPACK row (U = the slice's stored length, or a chunk of it: the
// same in every lane): loads, then gathers, then the FMA chain in order (padding skipped)
template <int U>
__device__ __forceinline__ void ell_part(const double *__restrict__ pv, const int32_t *__restrict__ pc,
                                         const double *xin, double &acc) {
    double v[U], xv[U];
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        v[u] = __ldcs(pv + 32 * u);
        c[u] = __ldcs(pc + 32 * u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldcg(xin + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
}

// a slice row of stored length len: chunks of 8, then the exact remainder, so that no FMA is
// issued for entries past the slice's length
__device__ __forceinline__ void ell_row(const double *__restrict__ pv, const int32_t *__restrict__ pc, int len,
                                        const double *xin, double &acc) {
    int j = 0;
    for (; j + 8 <= len; j += 8) ell_part<8>(pv + 32 * j, pc + 32 * j, xin, acc);
    switch (len - j) {
        case 1: ell_part<1>(pv + 32 * j, pc + 32 * j, xin, acc); break;
        case 2: ell_part<2>(pv + 32 * j, pc + 32 * j, xin, acc); break;
        case 3: ell_part<3>(pv + 32 * j, pc + 32 * j, xin, acc); break;
        case 4: ell_part<4>(pv + 32 * j, pc + 32 * j, xin, acc); break;
        case 5: ell_part<5>(pv + 32 * j, pc + 32 * j, xin, acc); break;
        case 6: ell_part<6>(pv + 32 * j, pc + 32 * j, xin, acc); break;
        case 7: ell_part<7>(pv + 32 * j, pc + 32 * j, xin, acc); break;
        default: break;
    }
}

// q or r rows of a tile: each lane owns one row of each of the tile's 32-row slices
template <int TR>
__device__ __forceinline__ void tile_spmv(const BatchDev &d, const TileInfo &ti, const double *xin, int mode,
                                          double &part_a, double &part_b) {
    // mode 0: q = A p, part_a += p.q ; mode 1: r = b - A x, part_a += r.r, part_b += b.b
    const int lane = threadIdx.x & 31;
    int o0 = ti.so0;
#pragma unroll 1
    for (int h = 0; h < TR / 32; ++h) {
        if (ti.r0 + h * 32 >= ti.r1) break;              // same in every lane
        const int row = ti.r0 + h * 32 + lane;
        const int len = slice_len(ti, h);
        const double *pv = d.sval + o0 + lane;
        const int32_t *pc = d.scol + o0 + lane;
        o0 += 32 * len;
        // this row's p (mode 0) or b (mode 1), loaded before the gathers: after the store of q
        // the compiler could not move the load ahead of it
        const double own = row < ti.r1 ? (mode == 0 ? __ldcg(xin + row) : d.b[row]) : 0.0;
        double acc = 0.0;
        ell_row(pv, pc, len, xin, acc);
        if (row >= ti.r1) continue;
        if (mode == 0) {
            d.q[row] = acc;
            part_a = fma(acc, own, part_a);
        } else {
            const double bi = own;
            const double ri = bi - acc;
            d.r[row] = ri;
            part_a = fma(ri, ri, part_a);
            part_b = fma(bi, bi, part_b);
        }
    }
}

// z = M^-1 r on a tile (blocks lie inside tiles). mode 0: plain (with p = z when init);
// mode 1: r -= alpha q first. part_a += r.z, part_b += r.r.
template <int TR, int FMT>
__device__ __forceinline__ void tile_apply(const BatchDev &d, const TileInfo &ti, double alpha, int fused, int init,
                                           float *s_rh, double *s_r, double &part_a, double &part_b) {
    const int lane = threadIdx.x & 31;
    const int r0 = ti.r0, r1 = ti.r1;
    // blocks of one size: their pool slots are consecutive, so one offset (loaded with the r
    // and q rows) places them all
    const long long q0 = ti.ubs > 0 ? __ldg(d.qoff + ti.blk0) : 0;
    const long long slot = ((long long)ti.ubs * ti.ubs * d.slot_eb + 15) & ~15ll;
    double rv[TR / 32], qv[TR / 32];     // every r (and q) row of the tile in one round trip
#pragma unroll
    for (int h = 0; h < TR / 32; ++h) {
        const int row = r0 + h * 32 + lane;
        rv[h] = row < r1 ? d.r[row] : 0.0;
        qv[h] = (fused && row < r1) ? d.q[row] : 0.0;
    }
#pragma unroll
    for (int h = 0; h < TR / 32; ++h) {
        const int row = r0 + h * 32 + lane;
        if (row < r1) {
            double v = rv[h];
            if (fused) {
                v = fma(-alpha, qv[h], v);
                d.r[row] = v;
                part_b = fma(v, v, part_b);
            }
            s_r[h * 32 + lane] = v;
            s_rh[h * 32 + lane] = f64_to_f32_rn(v);
        }
    }
    __syncwarp();
    // z of every row of the tile, stored after the loop so that the loads of the later slices'
    // inverse rows need not wait behind the earlier slices' stores
    double zv[TR / 32];
#pragma unroll
    for (int h = 0; h < TR / 32; ++h) {
        const int row = r0 + h * 32 + lane;
        zv[h] = 0.0;
        if (row < r1) {
            // this row's block: arithmetic when the tile's blocks share one size
            int bk, bs0, bs;
            const uint8_t *base;
            if (ti.ubs > 0) {
                const int k = (row - r0) / ti.ubs;
                bk = ti.blk0 + k;
                bs = ti.ubs;
                bs0 = r0 + k * bs;
                base = d.pool + q0 + k * slot;
            } else {
                bk = ti.blk0;
                while (d.block_ptr[bk + 1] <= row) ++bk;
                bs0 = d.block_ptr[bk];
                bs = d.block_ptr[bk + 1] - bs0;
                base = d.pool + d.qoff[bk];
            }
            const int i = row - bs0, off = bs0 - r0;
            const int f = FMT >= 0 ? FMT : d.fmt[bk];      // a batch of one format knows it at compile time
            const int eb = f == BJAC_FP64 ? 8 : f == BJAC_FP32 ? 4 : 2;
            double zi;
            if (((bs * eb) & 15) == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0 && (off & 3) == 0) {
                // 16-byte aligned rows and r slices: the lane reads its own row with vector loads
                const int vpr = bs * eb / 16;
                const uint4 *rowq = reinterpret_cast<const uint4 *>(base) + (size_t)i * vpr;
                if (f == BJAC_FP64) {
                    zi = vec_row_f64(rowq, vpr, s_r + off);
                } else {
                    float acc;
                    if (f == BJAC_FP32) acc = vec_row_low<float>(rowq, vpr, s_rh + off);
                    else if (f == BJAC_BF16) acc = vec_row_low<__nv_bfloat16>(rowq, vpr, s_rh + off);
                    else acc = vec_row_low<__half>(rowq, vpr, s_rh + off);
                    zi = f32_to_f64(acc * d.scale[bk]);
                }
            } else if (f == BJAC_FP64) {
                const double *G = reinterpret_cast<const double *>(base);
                double acc = 0.0;
                for (int j = 0; j < bs; ++j) acc = fma(G[(size_t)j * bs + i], s_r[off + j], acc);
                zi = acc;
            } else {
                float acc = 0.0f;
                if (f == BJAC_FP32) {
                    const float *Q = reinterpret_cast<const float *>(base);
                    for (int j = 0; j < bs; ++j) acc = fmaf(Q[(size_t)j * bs + i], s_rh[off + j], acc);
                } else if (f == BJAC_BF16) {
                    const __nv_bfloat16 *Q = reinterpret_cast<const __nv_bfloat16 *>(base);
                    for (int j = 0; j < bs; ++j) acc = fmaf(__bfloat162float(Q[(size_t)j * bs + i]), s_rh[off + j], acc);
                } else {
                    const __half *Q = reinterpret_cast<const __half *>(base);
                    for (int j = 0; j < bs; ++j) acc = fmaf(__half2float(Q[(size_t)j * bs + i]), s_rh[off + j], acc);
                }
                zi = f32_to_f64(acc * d.scale[bk]);
            }
            zv[h] = zi;
            part_a = fma(s_r[h * 32 + lane], zi, part_a);
        }
    }
#pragma unroll
    for (int h = 0; h < TR / 32; ++h) {
        const int row = r0 + h * 32 + lane;
        if (row < r1) {
            d.z[row] = zv[h];
            if (init) d.p[row] = zv[h];
        }
    }
    __syncwarp();
}

template <int TR, int MINB, int FMT>
__global__ void __launch_bounds__(kNT, MINB) k_pcg_batched(BatchDev d) {
    __shared__ __align__(16) float s_rh[kWarps][TR];
    __shared__ __align__(16) double s_r[kWarps][TR];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;

    auto per_tile = [&](auto &&fn) {
        for (int t = gw; t < d.ntiles; t += nw) {
            const TileInfo ti = load_tile(d, t);
            double a = 0.0, b2 = 0.0;
            fn(t, ti, a, b2);
            a = warp_sum(a);
            b2 = warp_sum(b2);
            if (lane == 0) {
                d.part[2 * t] = a;
                d.part[2 * t + 1] = b2;
            }
        }
    };
    // the same per-tile work over the list of running tiles (built by build_list); the next
    // listed tile's description is loaded while the current one is processed. partials: how
    // many per-tile sums the phase keeps (0, 1: a, 2: a and b2); each costs a warp tree of
    // five FP64 adds per tile, so a phase sums only what it uses.
    auto per_listed = [&](int cnt_slot, int partials, auto &&fn) {
        const int cnt = __ldcg(d.nlist + cnt_slot);
        const int32_t *lst = d.alist + (size_t)cnt_slot * d.ntiles;
        int t = gw < cnt ? __ldcg(lst + gw) : 0;
        TileInfo ti = load_tile(d, gw < cnt ? t : 0);
        for (int i = gw; i < cnt; i += nw) {
            const int tn = i + nw < cnt ? __ldcg(lst + i + nw) : t;
            const TileInfo tin = load_tile(d, tn);
            double a = 0.0, b2 = 0.0;
            fn(t, ti, a, b2);
            if (partials > 0) {
                a = warp_sum(a);
                if (partials > 1) b2 = warp_sum(b2);
                if (lane == 0) {
                    d.part[2 * t] = a;
                    if (partials > 1) d.part[2 * t + 1] = b2;
                }
            }
            t = tn;
            ti = tin;
        }
    };
    // List of the tiles whose system is running, appended to list `sl`, whose length must be
    // zero. Each CTA scans a contiguous range of tiles and reserves room for all it keeps with
    // one atomic per 256 tiles (the ranges land in any order). A grid barrier must follow before
    // the list is read. The list not in use has its length cleared in phase B, after the last
    // read of its old contents.
    __shared__ int s_wcnt[kWarps];
    __shared__ int s_lbase;
    auto build_list = [&](int sl) {
        const int per = (d.ntiles + gridDim.x - 1) / gridDim.x;
        const int c0 = blockIdx.x * per, c1 = min(d.ntiles, c0 + per);
        for (int t0 = c0; t0 < c1; t0 += kNT) {
            const int t = t0 + threadIdx.x;
            const bool keep = t < c1 && __ldcg(d.state + d.tile_sys[t]) == kRunning;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_wcnt[warp] = __popc(m);
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int w = 0; w < kWarps; ++w) {
                    const int c = s_wcnt[w];
                    s_wcnt[w] = tot;
                    tot += c;
                }
                s_lbase = tot > 0 ? atomicAdd(d.nlist + sl, tot) : 0;
            }
            __syncthreads();
            if (keep) d.alist[(size_t)sl * d.ntiles + s_lbase + s_wcnt[warp] + __popc(m & ((1u << lane) - 1u))] = t;
            __syncthreads();
        }
    };
    // Fixed-order sums of system s's tile partials by the whole CTA (every thread of the CTA
    // must call it; the results are valid in every thread). One CTA per system keeps the
    // largest systems' sums short.
    __shared__ double s_sum[kWarps];
    auto sys_sum2 = [&](int s, double &a, double &b2) {
        double va = 0.0, vb = 0.0;
        for (int t = d.sys_tile[s] + threadIdx.x; t < d.sys_tile[s + 1]; t += kNT) {
            va += __ldcg(d.part + 2 * t);
            vb += __ldcg(d.part + 2 * t + 1);
        }
        a = block_sum<kNT>(va, s_sum);
        b2 = block_sum<kNT>(vb, s_sum);
    };
    auto sys_sum = [&](int s) {
        double va = 0.0;
        for (int t = d.sys_tile[s] + threadIdx.x; t < d.sys_tile[s + 1]; t += kNT) va += __ldcg(d.part + 2 * t);
        return block_sum<kNT>(va, s_sum);
    };

    // which list length is current: it alternates at every list build; the loop ends with an
    // empty list in the current slot, so a restart builds into it again
    int slot = 0;
    // ---- start: r = b - A x, relres, then z = M^-1 r, p = z, rho ----------------------
    for (int restart = 0; restart < 3; ++restart) {
        per_tile([&](int, const TileInfo &ti, double &a, double &b2) {
            if (restart > 0 && __ldcg(d.state + ti.sys) != kRunning) return;
            tile_spmv<TR>(d, ti, d.x, 1, a, b2);
        });
        if (!grid_barrier(d)) return;
        for (int s = blockIdx.x; s < d.nsys; s += gridDim.x) {
            if (restart > 0 && __ldcg(d.state + s) != kRunning) continue;
            double rr, bb;
            sys_sum2(s, rr, bb);
            if (threadIdx.x == 0) {
                if (restart == 0) {
                    d.bnorm[s] = sqrt(bb);
                    d.iter[s] = 0;
                    d.restarts[s] = 0;
                }
                const double bn = d.bnorm[s];
                const double rel = bn > 0.0 ? sqrt(rr) / bn : 0.0;
                d.relres[s] = rel;
                d.true_relres[s] = rel;
                d.xpend[s] = 0;
                if (bn == 0.0) d.state[s] = kConverged;
                else if (!(rel < 1.0e308)) d.state[s] = kBreakdown;
                else if (rel <= d.tol) d.state[s] = kConverged;
                else if (d.iter[s] >= d.maxit) d.state[s] = kMaxit;
                else d.state[s] = kRunning;
            }
        }
        if (!grid_barrier(d)) return;
        per_tile([&](int, const TileInfo &ti, double &a, double &b2) {
            if (__ldcg(d.state + ti.sys) != kRunning) return;
            tile_apply<TR, FMT>(d, ti, 0.0, 0, 1, s_rh[warp], s_r[warp], a, b2);
        });
        if (!grid_barrier(d)) return;
        for (int s = blockIdx.x; s < d.nsys; s += gridDim.x) {
            if (__ldcg(d.state + s) != kRunning) continue;
            const double rz = sys_sum(s);
            if (threadIdx.x == 0) {
                d.rho[s] = rz;
                if (!finite_pos(rz)) d.state[s] = kBreakdown;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) *d.active = 1;
        if (!grid_barrier(d)) return;
        build_list(slot);
        if (!grid_barrier(d)) return;

        // ---- iterations --------------------------------------------------------------
        while (*((volatile int32_t *)d.active) != 0) {
            // A: q = A p, p.q (the previous iteration's list decision has been read)
            if (blockIdx.x == 0 && threadIdx.x == 0) *d.changed = 0;
            per_listed(slot, 1, [&](int, const TileInfo &ti, double &a, double &b2) {
                tile_spmv<TR>(d, ti, d.p, 0, a, b2);
            });
            if (!grid_barrier(d)) return;
            // B: alpha per system; the previous iteration's x updates are done
            if (blockIdx.x == 0 && threadIdx.x == 0) d.nlist[slot ^ 1] = 0;
            for (int s = blockIdx.x; s < d.nsys; s += gridDim.x) {
                if (threadIdx.x == 0) d.xpend[s] = 0;
                if (__ldcg(d.state + s) != kRunning) continue;
                const double sigma = sys_sum(s);
                if (threadIdx.x == 0) {
                    if (!finite_pos(sigma)) {
                        d.state[s] = kBreakdownSigma;
                        atomicOr(d.changed, 1);
                    } else {
                        d.alpha[s] = d.rho[s] / sigma;
                    }
                }
            }
            if (!grid_barrier(d)) return;
            // C: r -= alpha q, z = M^-1 r, r.r and r.z
            // (no per-tile state test: a system whose sigma broke down in B keeps a stale alpha
            // here, and its r, z and partial sums are never read again, so the tile's loads
            // need not wait for the state)
            per_listed(slot, 2, [&](int, const TileInfo &ti, double &a, double &b2) {
                tile_apply<TR, FMT>(d, ti, __ldcg(d.alpha + ti.sys), 1, 0, s_rh[warp], s_r[warp], a, b2);
            });
            if (!grid_barrier(d)) return;
            // D: convergence and beta per system; count the systems still running
            int my_active = 0;
            for (int s = blockIdx.x; s < d.nsys; s += gridDim.x) {
                if (__ldcg(d.state + s) != kRunning) continue;
                double rz, rr;
                sys_sum2(s, rz, rr);
                if (threadIdx.x == 0) {
                    const int it = d.iter[s] + 1;
                    d.iter[s] = it;
                    d.xpend[s] = 1;
                    const double rel = sqrt(rr) / d.bnorm[s];
                    d.relres[s] = rel;
                    if (!(rel < 1.0e308)) d.state[s] = kBreakdown;
                    else if (rel <= d.tol) d.state[s] = kConverged;
                    else if (it >= d.maxit) d.state[s] = kMaxit;
                    else if (!finite_pos(rz)) d.state[s] = kBreakdown;
                    else {
                        d.beta[s] = rz / d.rho[s];
                        d.rho[s] = rz;
                        my_active = 1;
                    }
                    if (!my_active) atomicOr(d.changed, 1);
                }
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) *d.active = 0;
            if (!grid_barrier(d)) return;
            if (threadIdx.x == 0 && my_active) atomicOr(d.active, 1);
            // the list changes only when a system stopped (B or D of this iteration)
            const bool rebuild = __ldcg(d.changed) != 0;
            // E: x += alpha p, p = z + beta p (the list still holds the systems D just stopped);
            // all loads of the tile's rows before its stores
            // (the rows are loaded together with the system's flags and scalars, not after them)
            per_listed(slot, 0, [&](int, const TileInfo &ti, double &, double &) {
                double pv[TR / 32], xv[TR / 32], zv[TR / 32];
#pragma unroll
                for (int h = 0; h < TR / 32; ++h) {
                    const int row = ti.r0 + h * 32 + lane;
                    if (row < ti.r1) {
                        pv[h] = d.p[row];
                        xv[h] = d.x[row];
                        zv[h] = d.z[row];
                    }
                }
                const int s = ti.sys;
                const int xp = __ldcg(d.xpend + s), run = __ldcg(d.state + s) == kRunning;
                const double al = __ldcg(d.alpha + s), be = __ldcg(d.beta + s);
#pragma unroll
                for (int h = 0; h < TR / 32; ++h) {
                    const int row = ti.r0 + h * 32 + lane;
                    if (row < ti.r1) {
                        if (xp) d.x[row] = fma(al, pv[h], xv[h]);
                        if (run) d.p[row] = fma(be, pv[h], zv[h]);
                    }
                }
            });
            if (rebuild) {
                slot ^= 1;
                build_list(slot);
            }
            if (!grid_barrier(d)) return;
        }
        for (int s = blockIdx.x; s < d.nsys; s += gridDim.x)
            if (threadIdx.x == 0) d.xpend[s] = 0;
        // ---- true residual of the converged systems; restart those that miss tol -----
        per_tile([&](int, const TileInfo &ti, double &a, double &b2) {
            if (__ldcg(d.state + ti.sys) != kConverged) return;
            tile_spmv<TR>(d, ti, d.x, 1, a, b2);
        });
        if (!grid_barrier(d)) return;
        int again = 0;
        for (int s = blockIdx.x; s < d.nsys; s += gridDim.x) {
            if (__ldcg(d.state + s) != kConverged) continue;
            const double rr = sys_sum(s);
            if (threadIdx.x == 0) {
                const double rel = d.bnorm[s] > 0.0 ? sqrt(rr) / d.bnorm[s] : 0.0;
                d.true_relres[s] = rel;
                if (rel > d.tol && d.iter[s] < d.maxit && restart < 2) {
                    d.state[s] = kRunning;
                    d.restarts[s] += 1;
                    again = 1;
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) *d.active = 0;
        if (!grid_barrier(d)) return;
        if (threadIdx.x == 0 && again) atomicOr(d.active, 1);
        if (!grid_barrier(d)) return;
        if (*((volatile int32_t *)d.active) == 0) return;
    }
}

}  // namespace mpbjac

using namespace mpbjac;

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
struct bjac_batch {
    int nsys = 0, n_tot = 0, nnz_tot = 0, nb_tot = 0, ntiles = 0, tile_rows = 32;
    int slot_eb = 8;                            // bytes per entry of the pool slots
    cudaStream_t stream = nullptr;
    std::vector<int32_t> sys_row, sys_tile, sys_blk;
    int32_t *rowptr = nullptr, *colidx = nullptr;
    double *val = nullptr;
    int32_t *block_ptr = nullptr;
    int64_t *goff = nullptr;
    uint8_t *fmt = nullptr;
    float *scale = nullptr;
    int64_t *qoff = nullptr;
    uint8_t *pool = nullptr;
    double *feat = nullptr, *kap = nullptr;
    int *status = nullptr;
    int32_t *tile_row = nullptr, *tile_sys = nullptr, *tile_blk = nullptr, *d_sys_tile = nullptr;
    double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *part = nullptr;
    double *sd = nullptr;          // per-system doubles: bnorm rho alpha beta relres true_relres
    int32_t *si = nullptr;         // per-system ints: iter state xpend restarts
    unsigned int *ctl = nullptr;   // barrier count, generation, err, active, list lengths [2]
    int32_t *soff = nullptr, *scol = nullptr, *alist = nullptr;   // sliced-ELLPACK tiles, tile lists
    int4 *tinfo = nullptr;          // per-tile descriptions (two int4 each)
    double *sval = nullptr;
    std::vector<int32_t> h_bp;      // host copy of the concatenated block offsets
    int grid = 0;
    float tune_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // timings of the kernel variants
    int variant = 0;
    bool fp32_only = false;                  // every block binary32: the kernels for that format
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double tol_cached = -1.0;
    int maxit_cached = -1;
    int force_timeout = 0;                   // test hook: barriers wait for one CTA too many
    int force_cached = 0;
    int32_t blocks_per_fmt[4] = {0, 0, 0, 0};
    float setup_ms = 0.0f;
};

static void free_batch(bjac_batch *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    void *ptrs[] = {h->rowptr, h->colidx, h->val, h->block_ptr, h->goff, h->fmt, h->scale, h->qoff, h->pool, h->feat,
                    h->kap, h->status, h->tile_row, h->tile_sys, h->tile_blk, h->d_sys_tile, h->b, h->x, h->r, h->z,
                    h->p, h->q, h->part, h->sd, h->si, h->ctl, h->soff, h->scol, h->sval, h->alist, h->tinfo};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete h;
}

__global__ void k_concat_csr(int rows, int row0, int nz0, const int32_t *rp, const int32_t *ci, const double *v,
                             int32_t *rp_out, int32_t *ci_out, double *v_out) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int i = tid; i < rows; i += stride) rp_out[row0 + i] = nz0 + rp[i];
    const int nnz = rp[rows];
    for (int k = tid; k < nnz; k += stride) {
        ci_out[nz0 + k] = row0 + ci[k];
        v_out[nz0 + k] = v[k];
    }
}

static BatchDev batch_dev(bjac_batch *h, double tol, int maxit) {
    BatchDev d{};
    d.n_tot = h->n_tot;
    d.slot_eb = h->slot_eb;
    d.nsys = h->nsys;
    d.ntiles = h->ntiles;
    d.rowptr = h->rowptr;
    d.colidx = h->colidx;
    d.val = h->val;
    d.block_ptr = h->block_ptr;
    d.fmt = h->fmt;
    d.scale = h->scale;
    d.qoff = h->qoff;
    d.pool = h->pool;
    d.tile_row = h->tile_row;
    d.tile_sys = h->tile_sys;
    d.tile_blk = h->tile_blk;
    d.sys_tile = h->d_sys_tile;
    d.b = h->b;
    d.x = h->x;
    d.r = h->r;
    d.z = h->z;
    d.p = h->p;
    d.q = h->q;
    d.part = h->part;
    const int S = h->nsys;
    d.bnorm = h->sd;
    d.rho = h->sd + S;
    d.alpha = h->sd + 2 * S;
    d.beta = h->sd + 3 * S;
    d.relres = h->sd + 4 * S;
    d.true_relres = h->sd + 5 * S;
    d.iter = h->si;
    d.state = h->si + S;
    d.xpend = h->si + 2 * S;
    d.restarts = h->si + 3 * S;
    d.tol = tol;
    d.maxit = maxit;
    d.bar_count = h->ctl;
    d.bar_gen = h->ctl + 1;
    d.err = reinterpret_cast<int32_t *>(h->ctl + 2);
    d.active = reinterpret_cast<int32_t *>(h->ctl + 3);
    d.bar_extra = h->force_timeout ? 1 : 0;
    d.nlist = reinterpret_cast<int32_t *>(h->ctl + 4);
    d.changed = reinterpret_cast<int32_t *>(h->ctl + 6);
    d.soff = h->soff;
    d.tinfo = h->tinfo;
    d.scol = h->scol;
    d.sval = h->sval;
    d.alist = h->alist;
    return d;
}

// kernel variants the setup times: tile height x CTAs per SM the registers are sized for; a
// batch whose blocks are all binary32 (the usual batched format) also gets kernels compiled for
// that format alone, which need fewer registers
constexpr int kBatchVariants = 8;
constexpr int kVarTR[kBatchVariants] = {32, 32, 32, 64, 64, 64, 128, 128};
[[maybe_unused]] constexpr int kVarMinB[kBatchVariants] = {2, 4, 6, 2, 4, 6, 4, 6};   // as instantiated below

template <int TR, int MINB, int FMT>
static int launch_batched_t(const BatchDev &d, cudaStream_t st, int grid) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kNT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MPB_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_batched<TR, MINB, FMT>, d));
    return MPBJAC_OK;
}

template <int FMT>
static int launch_batched_f(int variant, const BatchDev &d, cudaStream_t st, int grid) {
    switch (variant) {
        case 0: return launch_batched_t<32, 2, FMT>(d, st, grid);
        case 1: return launch_batched_t<32, 4, FMT>(d, st, grid);
        case 2: return launch_batched_t<32, 6, FMT>(d, st, grid);
        case 3: return launch_batched_t<64, 2, FMT>(d, st, grid);
        case 4: return launch_batched_t<64, 4, FMT>(d, st, grid);
        case 5: return launch_batched_t<64, 6, FMT>(d, st, grid);
        case 6: return launch_batched_t<128, 4, FMT>(d, st, grid);
        default: return launch_batched_t<128, 6, FMT>(d, st, grid);
    }
}

static int launch_batched(int variant, bool fp32_only, const BatchDev &d, cudaStream_t st, int grid) {
    return fp32_only ? launch_batched_f<BJAC_FP32>(variant, d, st, grid) : launch_batched_f<-1>(variant, d, st, grid);
}

template <int TR, int MINB, int FMT>
static int per_sm_of() {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_batched<TR, MINB, FMT>, kNT, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    return per;
}

template <int FMT>
static int per_sm_f(int variant) {
    switch (variant) {
        case 0: return per_sm_of<32, 2, FMT>();
        case 1: return per_sm_of<32, 4, FMT>();
        case 2: return per_sm_of<32, 6, FMT>();
        case 3: return per_sm_of<64, 2, FMT>();
        case 4: return per_sm_of<64, 4, FMT>();
        case 5: return per_sm_of<64, 6, FMT>();
        case 6: return per_sm_of<128, 4, FMT>();
        default: return per_sm_of<128, 6, FMT>();
    }
}

// CTAs of a variant that are co-resident on the GPU (the cooperative grid)
static int max_coresident(int variant, bool fp32_only) {
    return sm_count() * (fp32_only ? per_sm_f<BJAC_FP32>(variant) : per_sm_f<-1>(variant));
}

// variant chosen per batch shape (systems, rows, nonzeros, blocks, all binary32)
struct BatchTuneKey {
    int nsys, n, nnz, nb;
    bool fp32_only;
    bool operator==(const BatchTuneKey &o) const {
        return nsys == o.nsys && n == o.n && nnz == o.nnz && nb == o.nb && fp32_only == o.fp32_only;
    }
};
struct BatchTune {
    BatchTuneKey key;
    int variant;
    float ms[kBatchVariants];
};
static std::vector<BatchTune> g_batch_tune;

// one warp per 32-row slice of a tile: its rows' entries column-major, padded with (0, -1)
__global__ void k_batch_ell(int nslices, int spt, const int32_t *__restrict__ tile_row,
                            const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                            const double *__restrict__ val, const int32_t *__restrict__ soff,
                            int32_t *__restrict__ scol, double *__restrict__ sval) {
    const int lane = threadIdx.x & 31;
    const int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nslices) return;
    const int t = sl / spt, hh = sl - t * spt;
    const int r0 = tile_row[t] + 32 * hh, r1 = tile_row[t + 1];
    const int o0 = soff[sl], len = (soff[sl + 1] - o0) >> 5;
    const int row = r0 + lane;
    const int lo = row < r1 ? rowptr[row] : 0;
    const int rl = row < r1 ? rowptr[row + 1] - lo : 0;
    for (int j = 0; j < len; ++j) {
        const size_t k = (size_t)o0 + 32 * (size_t)j + lane;
        const bool in = j < rl;
        sval[k] = in ? val[lo + j] : 0.0;
        scol[k] = in ? colidx[lo + j] : -1;
    }
}

// stored length of every 32-row slice of every tile (its longest row): one warp per slice
__global__ void k_batch_slice_len(int nslices, int spt, const int32_t *__restrict__ tile_row,
                                  const int32_t *__restrict__ rowptr, int32_t *__restrict__ slen) {
    const int lane = threadIdx.x & 31;
    const int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nslices) return;
    const int t = sl / spt, hh = sl - t * spt;
    const int r0 = tile_row[t] + 32 * hh, r1 = min(tile_row[t + 1], r0 + 32);
    const int row = r0 + lane;
    int len = row < r1 ? rowptr[row + 1] - rowptr[row] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) slen[sl] = len;
}

static int build_tiles(bjac_batch *h, int tr, const std::vector<int32_t> &bp) {
    // tiles of at most tr rows, cut at system boundaries and at block boundaries
    std::vector<int32_t> trow, tsys, tblk;
    h->sys_tile.assign(h->nsys + 1, 0);
    int bk = 0;
    for (int s = 0; s < h->nsys; ++s) {
        h->sys_tile[s] = (int)tsys.size();
        int row = h->sys_row[s];
        const int end = h->sys_row[s + 1];
        while (row < end) {
            while (bp[bk + 1] <= row) ++bk;
            int stop = std::min(row + tr, end);
            // do not split a block: end at the last block boundary inside [row, row + tr]
            int k = bk;
            int last = row;
            while (k < h->nb_tot && bp[k + 1] <= stop) last = bp[++k];
            if (last == row) last = bp[bk + 1];     // a block longer than tr (never with bs <= 32)
            trow.push_back(row);
            tsys.push_back(s);
            tblk.push_back(bk);
            row = last;
        }
    }
    h->sys_tile[h->nsys] = (int)tsys.size();
    trow.push_back(h->n_tot);
    h->ntiles = (int)tsys.size();
    cudaFree(h->tile_row);
    cudaFree(h->tile_sys);
    cudaFree(h->tile_blk);
    MPB_CUDA(cudaMalloc(&h->tile_row, sizeof(int32_t) * trow.size()));
    MPB_CUDA(cudaMalloc(&h->tile_sys, sizeof(int32_t) * tsys.size()));
    MPB_CUDA(cudaMalloc(&h->tile_blk, sizeof(int32_t) * tblk.size()));
    MPB_CUDA(cudaMemcpy(h->tile_row, trow.data(), sizeof(int32_t) * trow.size(), cudaMemcpyHostToDevice));
    MPB_CUDA(cudaMemcpy(h->tile_sys, tsys.data(), sizeof(int32_t) * tsys.size(), cudaMemcpyHostToDevice));
    MPB_CUDA(cudaMemcpy(h->tile_blk, tblk.data(), sizeof(int32_t) * tblk.size(), cudaMemcpyHostToDevice));
    MPB_CUDA(cudaMemcpy(h->d_sys_tile, h->sys_tile.data(), sizeof(int32_t) * (h->nsys + 1), cudaMemcpyHostToDevice));
    cudaFree(h->part);
    MPB_CUDA(cudaMalloc(&h->part, sizeof(double) * 2 * h->ntiles));
    // sliced-ELLPACK copy of every tile (32-row slices padded to their longest row)
    const int spt = tr / 32;
    const size_t nsl = (size_t)h->ntiles * spt;
    std::vector<int32_t> so(nsl + 1), slen(nsl, 0);
    {
        // the slices' stored lengths on the device (one warp per slice), read back once
        int32_t *dlen = nullptr;
        MPB_CUDA(cudaMalloc(&dlen, sizeof(int32_t) * std::max<size_t>(1, nsl)));
        const int grid = (int)((nsl * 32 + 255) / 256);
        k_batch_slice_len<<<grid, 256, 0, h->stream>>>((int)nsl, spt, h->tile_row, h->rowptr, dlen);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(slen.data(), dlen, sizeof(int32_t) * nsl, cudaMemcpyDeviceToHost,
                                                  h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(dlen);
        if (e != cudaSuccess) return cuda_fail(e, "slice lengths of the batch");
    }
    long long acc = 0;
    for (size_t k = 0; k < nsl; ++k) {
        so[k] = (int32_t)acc;
        if (slen[k] > 0xFFFF) return fail(MPBJAC_ERR_UNSUPPORTED, "the batched solver takes rows of at most 65535 entries");
        acc += 32ll * slen[k];
        if (acc > (long long)INT32_MAX - 64) return fail(MPBJAC_ERR_INVALID_ARG, "batch too large for int32");
    }
    so[nsl] = (int32_t)acc;
    // tile descriptions: rows, system, first block, common block size, slice offsets
    std::vector<int32_t> ti((size_t)h->ntiles * 8);
    for (int t = 0; t < h->ntiles; ++t) {
        int32_t *e = &ti[(size_t)t * 8];
        e[0] = trow[t];
        e[1] = trow[t + 1];
        e[2] = tsys[t];
        e[3] = tblk[t];
        int ubs = bp[tblk[t] + 1] - bp[tblk[t]];
        for (int k = tblk[t]; k < h->nb_tot && bp[k] < trow[t + 1]; ++k)
            if (bp[k + 1] - bp[k] != ubs) ubs = 0;
        e[4] = ubs;
        e[5] = so[(size_t)t * spt];
        auto ln = [&](int k) { return k < spt ? slen[(size_t)t * spt + k] : 0; };
        e[6] = (int32_t)((uint32_t)ln(0) | ((uint32_t)ln(1) << 16));
        e[7] = (int32_t)((uint32_t)ln(2) | ((uint32_t)ln(3) << 16));
    }
    cudaFree(h->tinfo);
    h->tinfo = nullptr;
    MPB_CUDA(cudaMalloc(&h->tinfo, sizeof(int32_t) * ti.size()));
    MPB_CUDA(cudaMemcpy(h->tinfo, ti.data(), sizeof(int32_t) * ti.size(), cudaMemcpyHostToDevice));
    cudaFree(h->soff);
    cudaFree(h->scol);
    cudaFree(h->sval);
    cudaFree(h->alist);
    h->soff = nullptr;
    h->scol = nullptr;
    h->sval = nullptr;
    h->alist = nullptr;
    MPB_CUDA(cudaMalloc(&h->soff, sizeof(int32_t) * (nsl + 1)));
    MPB_CUDA(cudaMalloc(&h->scol, sizeof(int32_t) * std::max(1ll, acc)));
    MPB_CUDA(cudaMalloc(&h->sval, sizeof(double) * std::max(1ll, acc)));
    MPB_CUDA(cudaMalloc(&h->alist, sizeof(int32_t) * 2 * (size_t)h->ntiles));
    MPB_CUDA(cudaMemcpy(h->soff, so.data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice));
    const int grid = (int)((nsl * 32 + 255) / 256);
    k_batch_ell<<<grid, 256, 0, h->stream>>>((int)nsl, spt, h->tile_row, h->rowptr, h->colidx, h->val, h->soff,
                                             h->scol, h->sval);
    MPB_CUDA(cudaGetLastError());
    MPB_CUDA(cudaStreamSynchronize(h->stream));
    h->tile_rows = tr;
    return MPBJAC_OK;
}

static int run_batched(bjac_batch *h, double tol, int maxit, cudaStream_t st, bool use_graph) {
    BatchDev d = batch_dev(h, tol, maxit);
    MPB_CUDA(cudaMemsetAsync(h->ctl, 0, 8 * sizeof(unsigned int), st));
    if (!use_graph) return launch_batched(h->variant, h->fp32_only, d, st, h->grid);
    if (!h->exec || h->tol_cached != tol || h->maxit_cached != maxit || h->force_cached != h->force_timeout) {
        if (h->exec) cudaGraphExecDestroy(h->exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        h->exec = nullptr;
        h->graph = nullptr;
        cudaStream_t cs;
        MPB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        MPB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int rc = launch_batched(h->variant, h->fp32_only, d, cs, h->grid);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "capture of the batched kernel");
        e = cudaGraphInstantiate(&h->exec, g, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cudaGraphInstantiate (batched)"); }
        h->graph = g;
        h->tol_cached = tol;
        h->maxit_cached = maxit;
        h->force_cached = h->force_timeout;
    }
    MPB_CUDA(cudaGraphLaunch(h->exec, st));
    return MPBJAC_OK;
}

extern "C" int bjac_batch_setup(int32_t nsys, const bjac_csr *A, const int32_t *const *block_ptr, const int32_t *nb,
                                const bjac_policy *policy, bjac_batch **out) {
    if (!out) return fail(MPBJAC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nsys < 1 || !A || !block_ptr || !nb || !policy) return fail(MPBJAC_ERR_INVALID_ARG, "NULL argument or nsys < 1");
    const bjac_policy &P = *policy;
    if (P.select != BJAC_SELECT_UNIFORM && P.select != BJAC_SELECT_FIXED && P.select != BJAC_SELECT_RULE &&
        P.select != BJAC_SELECT_GIVEN)
        return fail(MPBJAC_ERR_UNSUPPORTED, "the batched solver takes uniform, fixed, rule or given selection");
    if (P.select == BJAC_SELECT_GIVEN && !P.block_fmt)
        return fail(MPBJAC_ERR_INVALID_ARG, "SELECT_GIVEN needs block_fmt (every block of every system)");
    if (P.temporal != BJAC_TEMPORAL_NONE) return fail(MPBJAC_ERR_UNSUPPORTED, "no aMP switching in the batched solver");
    long long n_tot = 0, nnz_tot = 0, nb_tot = 0;
    for (int s = 0; s < nsys; ++s) {
        if (A[s].n <= 0 || A[s].nnz < 0 || !A[s].rowptr) return fail(MPBJAC_ERR_INVALID_ARG, "bad CSR in the batch");
        if (!block_ptr[s] || nb[s] < 1 || block_ptr[s][0] != 0 || block_ptr[s][nb[s]] != A[s].n)
            return fail(MPBJAC_ERR_INVALID_ARG, "bad block_ptr in the batch");
        for (int k = 0; k < nb[s]; ++k) {
            const int bs = block_ptr[s][k + 1] - block_ptr[s][k];
            if (bs < 1 || bs > 32) return fail(MPBJAC_ERR_INVALID_ARG, "batched blocks need 1..32 rows");
        }
        n_tot += A[s].n;
        nnz_tot += A[s].nnz;
        nb_tot += nb[s];
    }
    if (n_tot >= (1ll << 31) || nnz_tot >= (1ll << 31)) return fail(MPBJAC_ERR_INVALID_ARG, "batch too large for int32");
    if (P.select == BJAC_SELECT_GIVEN)
        for (long long k = 0; k < nb_tot; ++k)
            if (P.block_fmt[k] > BJAC_FP16S) return fail(MPBJAC_ERR_INVALID_ARG, "block_fmt entries must be 0..3");
    bjac_batch *h = new bjac_batch();
    auto bail = [&](int rc) { free_batch(h); return rc; };
    h->nsys = nsys;
    h->n_tot = (int)n_tot;
    h->nnz_tot = (int)nnz_tot;
    h->nb_tot = (int)nb_tot;
    h->stream = (cudaStream_t)P.stream;
    cudaStream_t st = h->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    h->sys_row.assign(nsys + 1, 0);
    h->sys_blk.assign(nsys + 1, 0);
    std::vector<int32_t> bp(nb_tot + 1, 0);
    std::vector<int64_t> goff(nb_tot + 1, 0);
    {
        int row = 0, blk = 0;
        for (int s = 0; s < nsys; ++s) {
            h->sys_row[s] = row;
            h->sys_blk[s] = blk;
            for (int k = 0; k < nb[s]; ++k) bp[blk + k] = row + block_ptr[s][k];
            row += A[s].n;
            blk += nb[s];
        }
        h->sys_row[nsys] = row;
        h->sys_blk[nsys] = blk;
        bp[nb_tot] = row;
        h->h_bp = bp;
        for (long long k = 0; k < nb_tot; ++k) {
            const int64_t bs = bp[k + 1] - bp[k];
            goff[k + 1] = goff[k] + bs * bs;
        }
    }
#define BTRY(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call)); } while (0)
    BTRY(cudaMalloc(&h->rowptr, sizeof(int32_t) * (n_tot + 1)));
    BTRY(cudaMalloc(&h->colidx, sizeof(int32_t) * std::max(1ll, nnz_tot)));
    BTRY(cudaMalloc(&h->val, sizeof(double) * std::max(1ll, nnz_tot)));
    {
        int row = 0, nz = 0;
        for (int s = 0; s < nsys; ++s) {
            k_concat_csr<<<std::max(1, std::min(sm_count() * 4, (A[s].nnz + 255) / 256)), 256, 0, st>>>(
                A[s].n, row, nz, A[s].rowptr, A[s].colidx, A[s].val, h->rowptr, h->colidx, h->val);
            row += A[s].n;
            nz += A[s].nnz;
        }
        const int32_t last = nz;
        BTRY(cudaMemcpyAsync(h->rowptr + n_tot, &last, sizeof(int32_t), cudaMemcpyHostToDevice, st));
        BTRY(cudaStreamSynchronize(st));
    }
    BTRY(cudaMalloc(&h->block_ptr, sizeof(int32_t) * (nb_tot + 1)));
    BTRY(cudaMalloc(&h->goff, sizeof(int64_t) * (nb_tot + 1)));
    BTRY(cudaMalloc(&h->fmt, nb_tot));
    BTRY(cudaMalloc(&h->scale, sizeof(float) * nb_tot));
    BTRY(cudaMalloc(&h->qoff, sizeof(int64_t) * (nb_tot + 1)));
    BTRY(cudaMalloc(&h->feat, sizeof(double) * 12 * nb_tot));
    BTRY(cudaMalloc(&h->kap, sizeof(double) * 2 * nb_tot));
    BTRY(cudaMalloc(&h->status, 2 * sizeof(int)));
    BTRY(cudaMemcpy(h->block_ptr, bp.data(), sizeof(int32_t) * (nb_tot + 1), cudaMemcpyHostToDevice));
    BTRY(cudaMemcpy(h->goff, goff.data(), sizeof(int64_t) * (nb_tot + 1), cudaMemcpyHostToDevice));
    BTRY(cudaMemset(h->status, 0, 2 * sizeof(int)));
    // pool: fixed format -> compact offsets now; rule -> the binary64 layout (room for any format)
    const int ffmt = P.select == BJAC_SELECT_UNIFORM ? BJAC_FP64 : P.fixed_fmt;
    std::vector<int64_t> qoff(nb_tot + 1, 0);
    for (long long k = 0; k < nb_tot; ++k) {
        const int64_t bs = bp[k + 1] - bp[k];
        const int by = (P.select == BJAC_SELECT_RULE || P.select == BJAC_SELECT_GIVEN)
                           ? 8 : (ffmt == BJAC_FP64 ? 8 : ffmt == BJAC_FP32 ? 4 : 2);
        h->slot_eb = by;
        qoff[k + 1] = qoff[k] + ((bs * bs * by + 15) & ~int64_t(15));
    }
    BTRY(cudaMalloc(&h->pool, std::max<int64_t>(16, qoff[nb_tot])));
    BTRY(cudaMemcpy(h->qoff, qoff.data(), sizeof(int64_t) * (nb_tot + 1), cudaMemcpyHostToDevice));
    SetupArgs a{};
    a.n = h->n_tot;
    a.rowptr = h->rowptr;
    a.colidx = h->colidx;
    a.val = h->val;
    a.block_ptr = h->block_ptr;
    a.nb = h->nb_tot;
    a.goff = h->goff;
    a.G = nullptr;
    a.select = P.select;
    a.fixed_fmt = ffmt;
    a.theta = P.theta > 0 ? P.theta : 0.1;
    a.fmt = h->fmt;
    a.scale = h->scale;
    a.qoff = h->qoff;
    a.pool = h->pool;       // the rule / given paths write each block in its format at its slot
    if (P.select == BJAC_SELECT_GIVEN) {
        BTRY(cudaMemcpy(h->fmt, P.block_fmt, nb_tot, cudaMemcpyHostToDevice));
        a.given = h->fmt;
    }
    a.feat = h->feat;
    a.kap = h->kap;
    a.status = h->status;
    int rc = launch_setup_blocks(a, 32, nullptr, st);
    if (rc) return bail(rc);
    int hstat[2] = {0, 0};
    BTRY(cudaMemcpyAsync(hstat, h->status, sizeof(hstat), cudaMemcpyDeviceToHost, st));
    std::vector<uint8_t> hf(nb_tot);
    BTRY(cudaMemcpyAsync(hf.data(), h->fmt, nb_tot, cudaMemcpyDeviceToHost, st));
    BTRY(cudaStreamSynchronize(st));
    if (hstat[0] != 0) return bail(fail(MPBJAC_ERR_NOT_SPD, "a diagonal block of the batch is not positive definite"));
    for (uint8_t f : hf) h->blocks_per_fmt[f & 3] += 1;
    h->fp32_only = h->blocks_per_fmt[BJAC_FP32] == nb_tot;
    // vectors and per-system state
    BTRY(cudaMalloc(&h->b, sizeof(double) * n_tot));
    BTRY(cudaMalloc(&h->x, sizeof(double) * n_tot));
    BTRY(cudaMalloc(&h->r, sizeof(double) * n_tot));
    BTRY(cudaMalloc(&h->z, sizeof(double) * n_tot));
    BTRY(cudaMalloc(&h->p, sizeof(double) * n_tot));
    BTRY(cudaMalloc(&h->q, sizeof(double) * n_tot));
    BTRY(cudaMalloc(&h->sd, sizeof(double) * 6 * nsys));
    BTRY(cudaMalloc(&h->si, sizeof(int32_t) * 4 * nsys));
    BTRY(cudaMalloc(&h->ctl, sizeof(unsigned int) * 8));
    BTRY(cudaMalloc(&h->d_sys_tile, sizeof(int32_t) * (nsys + 1)));
    // autotuner: tile height (32 or 64 rows per warp task) and CTAs per SM (2, 4, 6: the
    // register budget of the kernel) timed on 20 iterations of this batch; the choice is kept
    // per batch shape for the life of the process
    const BatchTuneKey key{nsys, (int)n_tot, (int)nnz_tot, (int)nb_tot, h->fp32_only};
    const BatchTune *cached = nullptr;
    for (const auto &e : g_batch_tune)
        if (e.key == key) cached = &e;
    if (cached) {
        for (int v = 0; v < kBatchVariants; ++v) h->tune_ms[v] = cached->ms[v];
        rc = build_tiles(h, kVarTR[cached->variant], bp);
        if (rc) return bail(rc);
        h->variant = cached->variant;
        h->grid = max_coresident(cached->variant, h->fp32_only);
    } else {
        BTRY(cudaMemsetAsync(h->b, 0, sizeof(double) * n_tot, st));
        std::vector<double> ones(n_tot, 1.0);
        BTRY(cudaMemcpy(h->b, ones.data(), sizeof(double) * n_tot, cudaMemcpyHostToDevice));
        float best = 1e30f;
        int best_v = 0;
        for (int v = 0; v < kBatchVariants; ++v) {
            const int tr = kVarTR[v];
            if (v == 0 || kVarTR[v - 1] != tr) {
                rc = build_tiles(h, tr, bp);
                if (rc) return bail(rc);
            }
            h->variant = v;
            h->grid = max_coresident(v, h->fp32_only);
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                BTRY(cudaMemsetAsync(h->x, 0, sizeof(double) * n_tot, st));
                BTRY(cudaEventRecord(e1, st));
                cudaEvent_t e2;
                cudaEventCreate(&e2);
                rc = run_batched(h, 0.0, 20, st, false);
                if (rc) return bail(rc);
                BTRY(cudaEventRecord(e2, st));
                BTRY(cudaEventSynchronize(e2));
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e1, e2);
                cudaEventDestroy(e2);
                if (rep > 0) t = std::min(t, ms);
            }
            h->tune_ms[v] = t;
            if (t < best) { best = t; best_v = v; }
        }
        if (kVarTR[best_v] != kVarTR[kBatchVariants - 1]) {
            rc = build_tiles(h, kVarTR[best_v], bp);
            if (rc) return bail(rc);
        }
        h->variant = best_v;
        h->grid = max_coresident(best_v, h->fp32_only);
        BatchTune e{key, best_v, {}};
        for (int v = 0; v < kBatchVariants; ++v) e.ms[v] = h->tune_ms[v];
        g_batch_tune.push_back(e);
    }
#undef BTRY
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&h->setup_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = h;
    return MPBJAC_OK;
}

extern "C" int pcg_solve_batched(bjac_batch *h, const double *const *b, double *const *x, double tol, int32_t maxit,
                                 pcg_stats *stats) {
    if (!h || !b || !x) return fail(MPBJAC_ERR_INVALID_ARG, "NULL argument");
    if (maxit < 0 || !(tol >= 0.0)) return fail(MPBJAC_ERR_INVALID_ARG, "need maxit >= 0 and tol >= 0");
    cudaStream_t st = h->stream;
    cudaEvent_t e0, e1;
    MPB_CUDA(cudaEventCreate(&e0));
    MPB_CUDA(cudaEventCreate(&e1));
    MPB_CUDA(cudaEventRecord(e0, st));
    for (int s = 0; s < h->nsys; ++s) {
        const size_t rows = (size_t)(h->sys_row[s + 1] - h->sys_row[s]);
        MPB_CUDA(cudaMemcpyAsync(h->b + h->sys_row[s], b[s], rows * 8, cudaMemcpyDeviceToDevice, st));
        MPB_CUDA(cudaMemcpyAsync(h->x + h->sys_row[s], x[s], rows * 8, cudaMemcpyDeviceToDevice, st));
    }
    int rc = run_batched(h, tol, maxit, st, true);
    if (rc) return rc;
    for (int s = 0; s < h->nsys; ++s) {
        const size_t rows = (size_t)(h->sys_row[s + 1] - h->sys_row[s]);
        MPB_CUDA(cudaMemcpyAsync(x[s], h->x + h->sys_row[s], rows * 8, cudaMemcpyDeviceToDevice, st));
    }
    MPB_CUDA(cudaEventRecord(e1, st));
    MPB_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int S = h->nsys;
    std::vector<double> sd(6 * (size_t)S);
    std::vector<int32_t> si(4 * (size_t)S);
    unsigned int ctl[4];
    MPB_CUDA(cudaMemcpy(sd.data(), h->sd, sizeof(double) * 6 * S, cudaMemcpyDeviceToHost));
    MPB_CUDA(cudaMemcpy(si.data(), h->si, sizeof(int32_t) * 4 * S, cudaMemcpyDeviceToHost));
    MPB_CUDA(cudaMemcpy(ctl, h->ctl, sizeof(ctl), cudaMemcpyDeviceToHost));
    if ((int)ctl[2] != 0) return fail(MPBJAC_ERR_TIMEOUT, "a grid barrier of the batched kernel timed out");
    int worst = MPBJAC_OK;
    for (int s = 0; s < S; ++s) {
        const int state = si[S + s];
        int status;
        if (state == kBreakdown || state == kBreakdownSigma) status = MPBJAC_ERR_BREAKDOWN;
        else if (state == kConverged && sd[5 * S + s] <= tol) status = MPBJAC_OK;
        else status = MPBJAC_NOT_CONVERGED;
        if (status < 0) worst = status;
        else if (worst == MPBJAC_OK && status > 0) worst = status;
        if (stats) {
            pcg_stats &o = stats[s];
            memset(&o, 0, sizeof(o));
            o.iters = si[s];
            o.converged = status == MPBJAC_OK;
            o.status = status;
            o.restarts = si[3 * S + s];
            o.relres = sd[4 * S + s];
            o.true_relres = sd[5 * S + s];
            o.graph_launches = 1;
            o.kernel_launches = 1;      // the persistent kernel (shared by all systems)
            for (int i = 0; i < 4; ++i) o.blocks_per_fmt[i] = h->blocks_per_fmt[i];
            o.setup_ms = h->setup_ms;
            o.solve_ms = ms;
        }
    }
    return worst;
}

extern "C" void bjac_batch_destroy(bjac_batch *h) { free_batch(h); }

extern "C" int bjac_batch_force_timeout(bjac_batch *h, int32_t on) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "batch is NULL");
    if (on != 0 && on != 1) return fail(MPBJAC_ERR_INVALID_ARG, "on must be 0 or 1");
    h->force_timeout = on;
    return MPBJAC_OK;
}

extern "C" int bjac_batch_info(const bjac_batch *h, int32_t *ntiles, int32_t *tile_rows, int32_t *grid,
                               float *tune_ms) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "batch is NULL");
    if (ntiles) *ntiles = h->ntiles;
    if (tile_rows) *tile_rows = h->tile_rows;
    if (grid) *grid = h->grid;
    if (tune_ms)
        for (int v = 0; v < kBatchVariants; ++v) tune_ms[v] = h->tune_ms[v];
    return MPBJAC_OK;
}

extern "C" int bjac_batch_set_variant(bjac_batch *h, int32_t variant) {
    if (!h) return fail(MPBJAC_ERR_INVALID_ARG, "batch is NULL");
    if (variant < 0 || variant >= kBatchVariants) return fail(MPBJAC_ERR_INVALID_ARG, "variant must be 0..7");
    MPB_CUDA(cudaStreamSynchronize(h->stream));
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    if (kVarTR[variant] != kVarTR[h->variant]) {
        const int rc = build_tiles(h, kVarTR[variant], h->h_bp);
        if (rc) return rc;
    }
    h->variant = variant;
    h->grid = max_coresident(variant, h->fp32_only);
    return MPBJAC_OK;
}
