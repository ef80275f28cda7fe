// FP32 pair-distance tiles of the SIMT kernels (the refinement's run tiles and
// the recall estimator's query x sample tiles): a block of RF_THREADS threads
// computes a T x T tile of squared Euclidean distances in the canonical order
// (one accumulator per pair, coordinates in ascending order, the difference
// and its square as two FMAs), so every pair has the bits of pair_d2_seq.
#pragma once

#include "common.cuh"

namespace gkm {

constexpr int RF_THREADS = 256;
constexpr int RF_WARPS = RF_THREADS / 32;
constexpr int RF_DK = 32;  // coordinates staged per step

template <int T>
struct RefineTile {
    static constexpr int XR = 2 * T + 4;  // stride of a staged coordinate of the row samples (each value twice)
    static constexpr int XC = T + 4;      // stride of a staged coordinate of the column samples
    static constexpr int DS = T + 1;      // padded stride of the distance tile
    static constexpr int Q = T / 16;      // consecutive rows, and columns, per thread
    // staging buffers: two for the 64-wide tile (one stage consumed while the next is stored), one for the
    // 128-wide tile (two would halve its blocks per SM); the distance tile reuses them (written after the
    // last stage)
    static constexpr int NBUF = T == 64 ? 2 : 1;
    static constexpr size_t buf_floats = (size_t)RF_DK * (XR + XC);
    static constexpr size_t stage_floats = NBUF * buf_floats;
    static constexpr size_t tile_floats = (size_t)T * DS;
    static constexpr size_t fixed_bytes =
        sizeof(float) * (stage_floats > tile_floats ? stage_floats : tile_floats) + sizeof(int) * 2 * T;
    // per warp: row keys (kappa), merged-row keys (kappa), candidate keys (T), dup bits
    __host__ __device__ static size_t warp_bytes(int kappa)
    {
        return sizeof(uint64_t) * (size_t)(2 * kappa + T) + 4 * sizeof(unsigned);
    }
    static_assert(fixed_bytes % 8 == 0, "the per-warp key buffers need 8-byte alignment");
    __host__ __device__ static size_t smem_bytes(int kappa) { return fixed_bytes + RF_WARPS * warp_bytes(kappa); }
};

// 16 bytes of sample elements (4 FP32 or 8 BF16) widened to floats.
template <typename XT>
__device__ __forceinline__ void widen16(const uint4 &q, float (&v)[16 / sizeof(XT)])
{
    if constexpr (sizeof(XT) == 4) {
        v[0] = __uint_as_float(q.x), v[1] = __uint_as_float(q.y), v[2] = __uint_as_float(q.z),
        v[3] = __uint_as_float(q.w);
    } else {
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
}

// Rows whose stage segments can be read as aligned 16-byte vectors: d and the row stride multiples of the
// vector, the base 16-byte aligned (then every segment t0 .. t0 + RF_DK of a row is).
template <typename XT>
__host__ __device__ inline bool tile_vec16(const XT *X, int d, int64_t ld)
{
    constexpr int E = 16 / (int)sizeof(XT);
    return d % E == 0 && ld % E == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
}

// Pair distances of one T x T tile into dt[row * DS + col]: rows are the samples rid[0 .. nr),
// columns the samples cid[] (SAME: the rows again).  stage points at the block's staging area
// (RefineTile<T>::stage_floats floats), dt at the distance tile, which may alias it.  Called by all threads
// of the block; the caller synchronises before reading dt.  VEC: the rows meet tile_vec16, and each stage is
// fetched as 16-byte vectors (one load per 4 or 8 elements) instead of element by element.
template <int T, bool SAME, bool VEC, typename XT>
__device__ __forceinline__ void tile_distances(const XT *__restrict__ X, int d, int64_t ld, const int *rid,
                                               const int *cid, int nr, float *stage, float *dt)
{
    using TL = RefineTile<T>;
    constexpr int XR = TL::XR, XC = TL::XC, DS = TL::DS, Q = TL::Q;
    const int tid = threadIdx.x;
    // this thread: rows Q by .. Q by + Q - 1, columns Q bx .. Q bx + Q - 1 of the tile.  Two tiles: block
    // (by, bx) = (tid / 16, tid % 16), and warps whose rows all lie beyond the run skip the arithmetic.  A run's
    // own tile (SAME) is symmetric, d(i, j) = d(j, i) bit for bit (the difference only changes sign): only the
    // nb (nb + 1) / 2 blocks with by <= bx < nb = ceil(nr / Q) hold pairs of the run, and they go to threads
    // 0, 1, ... row by row (a run of 50 fills 91 threads, three warps; the other warps skip the arithmetic);
    // each block is also written mirrored.
    int by = tid >> 4, bx = tid & 15;
    bool rows_live;
    if constexpr (SAME) {
        // the arithmetic goes to the block's warps rot, rot + 1, ... (rot = blockIdx.x % 4): each warp of an SM
        // issues on scheduler (its index % 4), so blocks that share an SM spread their few busy warps over all
        // four schedulers instead of all starting at scheduler 0
        const int rot = (int)(blockIdx.x & 3) * 32;
        const int nb = (nr + Q - 1) / Q;
        int t = (tid - rot) & (RF_THREADS - 1), r = 0;
        while (r < nb && t >= nb - r) {
            t -= nb - r;
            r++;
        }
        by = r;
        bx = r + t;
        rows_live = r < nb;
    } else {
        rows_live = Q * by < nr;
    }
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 acc[Q][Q / 2];
#pragma unroll
    for (int a = 0; a < Q; a++)
#pragma unroll
        for (int b = 0; b < Q / 2; b++)
            acc[a][b] = make_float2(0.f, 0.f);
    // coordinates t0 .. t0+31 of the row and column samples, zero padded, are loaded into
    // registers one stage ahead (their loads in flight during the previous stage's arithmetic)
    constexpr int PER = T * RF_DK / RF_THREADS;
    constexpr int E = 16 / (int)sizeof(XT), CPR = RF_DK / E;  // vector path: elements per vector, vectors per row
    constexpr int PERV = T * CPR / RF_THREADS;
    static_assert(PERV >= 1 && (T * CPR) % RF_THREADS == 0, "whole vectors per thread");
    float pr_v[VEC ? 1 : PER], pc_v[(SAME || VEC) ? 1 : PER];
    uint4 qr[VEC ? PERV : 1], qc[(SAME || !VEC) ? 1 : PERV];
    auto fetch = [&](int t0) {
        if constexpr (VEC) {
#pragma unroll
            for (int p = 0; p < PERV; p++) {
                const int e = tid + p * RF_THREADS, row = e / CPR, t = t0 + (e % CPR) * E;
                const int a = rid[row];
                qr[p] = (a >= 0 && t < d) ? __ldg(reinterpret_cast<const uint4 *>(X + (int64_t)a * ld + t))
                                          : make_uint4(0u, 0u, 0u, 0u);
                if constexpr (!SAME) {
                    const int b = cid[row];
                    qc[p] = (b >= 0 && t < d) ? __ldg(reinterpret_cast<const uint4 *>(X + (int64_t)b * ld + t))
                                              : make_uint4(0u, 0u, 0u, 0u);
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < PER; p++) {
                const int e = tid + p * RF_THREADS, row = e / RF_DK, t = t0 + e % RF_DK;
                const int a = rid[row];
                pr_v[p] = (a >= 0 && t < d) ? ldx(X + (int64_t)a * ld + t) : 0.f;
                if constexpr (!SAME) {
                    const int b = cid[row];
                    pc_v[p] = (b >= 0 && t < d) ? ldx(X + (int64_t)b * ld + t) : 0.f;
                }
            }
        }
    };
    // stage s of the coordinates goes to buffer s % NBUF (rows [RF_DK][XR], then columns [RF_DK][XC]); with
    // two buffers the next stage is stored while the current one is consumed, one barrier per stage
    auto store = [&](float *buf) {
        float *br = buf, *bc = buf + RF_DK * XR;
        if constexpr (VEC) {
#pragma unroll
            for (int p = 0; p < PERV; p++) {
                const int e = tid + p * RF_THREADS, row = e / CPR, tt0 = (e % CPR) * E;
                float v[E], w[E];
                widen16<XT>(qr[p], v);
                if constexpr (!SAME)
                    widen16<XT>(qc[p], w);
#pragma unroll
                for (int j = 0; j < E; j++) {
                    *reinterpret_cast<float2 *>(br + (tt0 + j) * XR + 2 * row) = make_float2(v[j], v[j]);
                    bc[(tt0 + j) * XC + row] = SAME ? v[j] : w[j];
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < PER; p++) {
                const int e = tid + p * RF_THREADS, row = e / RF_DK, tt = e % RF_DK;
                *reinterpret_cast<float2 *>(br + tt * XR + 2 * row) = make_float2(pr_v[p], pr_v[p]);
                if constexpr (SAME)
                    bc[tt * XC + row] = pr_v[p];
                else
                    bc[tt * XC + row] = pc_v[p];
            }
        }
    };
    constexpr int NBUF = TL::NBUF;
    fetch(0);
    store(stage);
    __syncthreads();
    for (int t0 = 0, sidx = 0; t0 < d; t0 += RF_DK, sidx = (sidx + 1) % NBUF) {
        const float *cur = stage + sidx * TL::buf_floats;
        const bool more = t0 + RF_DK < d;
        if (more)
            fetch(t0 + RF_DK);
        const int tmax = min(RF_DK, d - t0);
        if (rows_live) {
            // one staged coordinate: the thread's Q rows (each value twice) and Q columns, then the Q x Q pairs
            auto step = [&](int tt) {
                float2 vr[Q], vc[Q / 2];
                const float4 *pr = reinterpret_cast<const float4 *>(cur + tt * XR + 2 * Q * by);
                const float4 *pc = reinterpret_cast<const float4 *>(cur + RF_DK * XR + tt * XC + Q * bx);
#pragma unroll
                for (int q = 0; q < Q / 2; q++) {
                    const float4 r4 = pr[q];
                    vr[2 * q] = make_float2(r4.x, r4.y);
                    vr[2 * q + 1] = make_float2(r4.z, r4.w);
                }
#pragma unroll
                for (int q = 0; q < Q / 4; q++) {
                    const float4 c4 = pc[q];
                    vc[2 * q] = make_float2(c4.x, c4.y);
                    vc[2 * q + 1] = make_float2(c4.z, c4.w);
                }
#pragma unroll
                for (int a = 0; a < Q; a++)
#pragma unroll
                    for (int b = 0; b < Q / 2; b++) {
                        const float2 e = __ffma2_rn(vc[b], m1, vr[a]);
                        acc[a][b] = __ffma2_rn(e, e, acc[a][b]);
                    }
            };
            if (T == 64 && tmax == RF_DK) {  // a full stage of the 64-wide tile, unrolled (the next coordinates'
                                              // loads overlap this one's FMAs; the 128-wide tile has no registers
                                              // to spare)
#pragma unroll 4
                for (int tt = 0; tt < RF_DK; tt++)
                    step(tt);
            } else {
                for (int tt = 0; tt < tmax; tt++)
                    step(tt);
            }
        }
        if constexpr (NBUF == 2) {
            if (more)
                store(stage + (sidx ^ 1) * TL::buf_floats);  // read last in the previous stage, before its barrier
            __syncthreads();
        } else {
            __syncthreads();  // every thread is done with the buffer
            if (more) {
                store(stage);
                __syncthreads();
            }
        }
    }
    if (rows_live) {
#pragma unroll
        for (int a = 0; a < Q; a++)
#pragma unroll
            for (int b = 0; b < Q / 2; b++) {
                dt[(Q * by + a) * DS + Q * bx + 2 * b] = acc[a][b].x;
                dt[(Q * by + a) * DS + Q * bx + 2 * b + 1] = acc[a][b].y;
                if (SAME && by != bx) {
                    dt[(Q * bx + 2 * b) * DS + Q * by + a] = acc[a][b].x;
                    dt[(Q * bx + 2 * b + 1) * DS + Q * by + a] = acc[a][b].y;
                }
            }
    }
}

// A run's own 64 x 64 tile (rows = columns = rid[0 .. nr)) computed by a group of NC threads of the block, with
// index ct in [0, NC), that synchronise on named barrier bar (the rest of the block does other work meanwhile):
// the arithmetic, the stages and the pair order of tile_distances<64, true, VEC>, so every distance has the same
// bits.  Nothing is written to a distance tile: a thread that holds a block of pairs (returns true) gets the
// block's position (by, bx) and its Q x Q distances in acc, for the caller to store when the tile is free.
template <int NC, bool VEC, typename XT>
__device__ __forceinline__ bool tile_distances_group(const XT *__restrict__ X, int d, int64_t ld, const int *rid,
                                                     int nr, float *stage, int ct, int bar,
                                                     float2 (&acc)[RefineTile<64>::Q][RefineTile<64>::Q / 2],
                                                     int &by_out, int &bx_out)
{
    constexpr int T = 64;
    using TL = RefineTile<T>;
    constexpr int XR = TL::XR, XC = TL::XC, Q = TL::Q;
    static_assert(NC % 32 == 0 && NC >= 136, "the group covers the 136 pair blocks of a 64-row triangle");
    const int nb = (nr + Q - 1) / Q;
    int t = ct, r = 0;
    while (r < nb && t >= nb - r) {
        t -= nb - r;
        r++;
    }
    const int by = r, bx = r + t;
    const bool rows_live = r < nb;
    by_out = by, bx_out = bx;
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int a = 0; a < Q; a++)
#pragma unroll
        for (int b = 0; b < Q / 2; b++)
            acc[a][b] = make_float2(0.f, 0.f);
    // stage loads: 16-byte vectors (VEC) or elements, shared out over the NC threads
    constexpr int E = 16 / (int)sizeof(XT), CPR = RF_DK / E;
    constexpr int NV = T * CPR, NS = T * RF_DK;
    constexpr int PV = (NV + NC - 1) / NC, PS = (NS + NC - 1) / NC;
    uint4 qr[VEC ? PV : 1];
    float pr[VEC ? 1 : PS];
    auto fetch = [&](int t0) {
        if constexpr (VEC) {
#pragma unroll
            for (int p = 0; p < PV; p++) {
                const int e = ct + p * NC, row = e / CPR, tt = t0 + (e % CPR) * E;
                const int a = e < NV ? rid[row] : -1;
                qr[p] = (a >= 0 && tt < d) ? __ldg(reinterpret_cast<const uint4 *>(X + (int64_t)a * ld + tt))
                                           : make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
#pragma unroll
            for (int p = 0; p < PS; p++) {
                const int e = ct + p * NC, row = e / RF_DK, tt = t0 + e % RF_DK;
                const int a = e < NS ? rid[row] : -1;
                pr[p] = (a >= 0 && tt < d) ? ldx(X + (int64_t)a * ld + tt) : 0.f;
            }
        }
    };
    auto store = [&](float *buf) {
        float *br = buf, *bc = buf + RF_DK * XR;
        if constexpr (VEC) {
#pragma unroll
            for (int p = 0; p < PV; p++) {
                const int e = ct + p * NC;
                if (e < NV) {
                    const int row = e / CPR, tt0 = (e % CPR) * E;
                    float v[E];
                    widen16<XT>(qr[p], v);
#pragma unroll
                    for (int j = 0; j < E; j++) {
                        *reinterpret_cast<float2 *>(br + (tt0 + j) * XR + 2 * row) = make_float2(v[j], v[j]);
                        bc[(tt0 + j) * XC + row] = v[j];
                    }
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < PS; p++) {
                const int e = ct + p * NC;
                if (e < NS) {
                    const int row = e / RF_DK, tt = e % RF_DK;
                    *reinterpret_cast<float2 *>(br + tt * XR + 2 * row) = make_float2(pr[p], pr[p]);
                    bc[tt * XC + row] = pr[p];
                }
            }
        }
    };
    fetch(0);
    store(stage);
    bar_sync(bar, NC);
    for (int t0 = 0, sidx = 0; t0 < d; t0 += RF_DK, sidx ^= 1) {
        const float *cur = stage + sidx * TL::buf_floats;
        const bool more = t0 + RF_DK < d;
        if (more)
            fetch(t0 + RF_DK);
        const int tmax = min(RF_DK, d - t0);
        if (rows_live) {
            auto step = [&](int tt) {
                float2 vr[Q], vc[Q / 2];
                const float4 *prr = reinterpret_cast<const float4 *>(cur + tt * XR + 2 * Q * by);
                const float4 *pc = reinterpret_cast<const float4 *>(cur + RF_DK * XR + tt * XC + Q * bx);
#pragma unroll
                for (int q = 0; q < Q / 2; q++) {
                    const float4 r4 = prr[q];
                    vr[2 * q] = make_float2(r4.x, r4.y);
                    vr[2 * q + 1] = make_float2(r4.z, r4.w);
                }
#pragma unroll
                for (int q = 0; q < Q / 4; q++) {
                    const float4 c4 = pc[q];
                    vc[2 * q] = make_float2(c4.x, c4.y);
                    vc[2 * q + 1] = make_float2(c4.z, c4.w);
                }
#pragma unroll
                for (int a = 0; a < Q; a++)
#pragma unroll
                    for (int b = 0; b < Q / 2; b++) {
                        const float2 e = __ffma2_rn(vc[b], m1, vr[a]);
                        acc[a][b] = __ffma2_rn(e, e, acc[a][b]);
                    }
            };
            if (tmax == RF_DK) {
#pragma unroll 4
                for (int tt = 0; tt < RF_DK; tt++)
                    step(tt);
            } else {
                for (int tt = 0; tt < tmax; tt++)
                    step(tt);
            }
        }
        if (more)
            store(stage + (sidx ^ 1) * TL::buf_floats);  // read last in the previous stage, before its barrier
        bar_sync(bar, NC);
    }
    return rows_live;
}

}  // namespace gkm
