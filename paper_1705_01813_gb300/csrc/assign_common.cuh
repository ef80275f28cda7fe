// Helpers shared by the assignment kernels (SIMT and tensor-core): the
// per-lane partial squared distance in the fixed order of the FP32 path and
// the warp reductions that complete it.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gkm {

// Warp sums of G per-lane partial values (G = 2, 4, ..., 32 candidates) at
// once.  The first log2 G exchange steps pair lanes across bit 4, 3, ... and
// halve the values each lane holds; the remaining lane bits are summed with a
// plain xor butterfly.  Every candidate's total is thus formed with the tree
// of warp_total (bit 4 first, then 3, 2, 1, 0), so all three give the same
// bits.  Afterwards lane l holds the total of candidate l / (32 / G).
template <int G>
__device__ __forceinline__ float transpose_reduce(float (&v)[G])
{
    static_assert(G >= 2 && G <= 32 && (G & (G - 1)) == 0, "G must be a power of two in [2, 32]");
    const int lane = lane_id();
#pragma unroll
    for (int h = G / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < h; j++) {
            float send = upper ? v[j] : v[j + h];
            float keep = upper ? v[j + h] : v[j];
            v[j] = keep + __shfl_xor_sync(FULL_MASK, send, o);
        }
    }
    float t = v[0];
#pragma unroll
    for (int o = 16 / G; o >= 1; o >>= 1)
        t += __shfl_xor_sync(FULL_MASK, t, o);
    return t;
}

__device__ __forceinline__ float transpose_reduce32(float (&v)[32]) { return transpose_reduce<32>(v); }

// Partial (per lane) squared distance of x (registers) to a row of 16-byte
// vectors, in the accumulation order of the assignment kernels: two
// accumulators, (a0, a1) += (e0^2, e1^2), then += (e2^2, e3^2) per vector,
// each a round-to-nearest FMA, and a0 + a1 at the end.  The packed FP32x2 FMA
// of sm_100+ performs each pair at once with the same roundings; e = x - c is
// formed as fma(c, -1, x), which is x - c rounded once.
template <int NV, typename RowLoad>
__device__ __forceinline__ float lane_partial(const float4 (&xv)[NV], int d4, RowLoad load)
{
    const int lane = lane_id();
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int v = 0; v < NV; v++) {
        const int col = lane + 32 * v;
        if (col < d4) {
            const float4 cv = load(col);
            const float2 e01 = __ffma2_rn(make_float2(cv.x, cv.y), m1, make_float2(xv[v].x, xv[v].y));
            const float2 e23 = __ffma2_rn(make_float2(cv.z, cv.w), m1, make_float2(xv[v].z, xv[v].w));
            a = __ffma2_rn(e01, e01, a);
            a = __ffma2_rn(e23, e23, a);
        }
    }
    return a.x + a.y;
}

// Partial squared distance of x to a row of an int8 shadow (4 values per 32-bit word, each stored as q + 128,
// the row's values being q s with |q| <= 127): word col holds the values of vector col.  Each byte is widened
// exactly (the float 2^23 + u, minus 2^23 + 128) and e = x - q s is one fma (the product q s is exact inside it),
// so the partial is the FP32 sum of (x - c~)^2 for the shadow values c~ = q s.
template <int NV, typename RowLoad>
__device__ __forceinline__ float lane_partial_q8(const float4 (&xv)[NV], int d4, float neg_s, RowLoad load)
{
    const int lane = lane_id();
    const float2 ns2 = make_float2(neg_s, neg_s);
    const float2 off2 = make_float2(-8388736.f, -8388736.f);  // -(2^23 + 128)
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int v = 0; v < NV; v++) {
        const int col = lane + 32 * v;
        if (col < d4) {
            const uint32_t w = load(col);
            const float2 u01 = make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540)),
                                           __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7541)));
            const float2 u23 = make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7542)),
                                           __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7543)));
            const float2 q01 = __fadd2_rn(u01, off2), q23 = __fadd2_rn(u23, off2);
            const float2 e01 = __ffma2_rn(q01, ns2, make_float2(xv[v].x, xv[v].y));
            const float2 e23 = __ffma2_rn(q23, ns2, make_float2(xv[v].z, xv[v].w));
            a = __ffma2_rn(e01, e01, a);
            a = __ffma2_rn(e23, e23, a);
        }
    }
    return a.x + a.y;
}

// The same partial for a row of the lane-major int8 shadow (d a multiple of 128): the NV words lane l needs,
// those of vectors l, l + 32, ..., are contiguous, so they arrive in one load (NV = 4: 16 bytes); the values,
// their order and the result are those of lane_partial_q8 on the row-major shadow.
template <int NV>
__device__ __forceinline__ float lane_partial_q8w(const float4 (&xv)[NV], float neg_s, const uint32_t (&w)[NV])
{
    const float2 ns2 = make_float2(neg_s, neg_s);
    const float2 off2 = make_float2(-8388736.f, -8388736.f);  // -(2^23 + 128)
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int v = 0; v < NV; v++) {
        const float2 u01 = make_float2(__uint_as_float(__byte_perm(w[v], 0x4B000000u, 0x7540)),
                                       __uint_as_float(__byte_perm(w[v], 0x4B000000u, 0x7541)));
        const float2 u23 = make_float2(__uint_as_float(__byte_perm(w[v], 0x4B000000u, 0x7542)),
                                       __uint_as_float(__byte_perm(w[v], 0x4B000000u, 0x7543)));
        const float2 q01 = __fadd2_rn(u01, off2), q23 = __fadd2_rn(u23, off2);
        const float2 e01 = __ffma2_rn(q01, ns2, make_float2(xv[v].x, xv[v].y));
        const float2 e23 = __ffma2_rn(q23, ns2, make_float2(xv[v].z, xv[v].w));
        a = __ffma2_rn(e01, e01, a);
        a = __ffma2_rn(e23, e23, a);
    }
    return a.x + a.y;
}

// The NV words of this lane from a lane-major int8 shadow row (row points at the row's first word).
template <int NV>
__device__ __forceinline__ void load_q8w(const uint32_t *__restrict__ row, uint32_t (&w)[NV])
{
    const int lane = lane_id();
    if constexpr (NV % 4 == 0) {
#pragma unroll
        for (int h = 0; h < NV / 4; h++) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(row) + lane * (NV / 4) + h);
            w[4 * h] = q.x, w[4 * h + 1] = q.y, w[4 * h + 2] = q.z, w[4 * h + 3] = q.w;
        }
    } else if constexpr (NV == 2) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row) + lane);
        w[0] = q.x, w[1] = q.y;
    } else {
        w[0] = __ldg(row + lane);
    }
}

// Complete one candidate's distance from the lane partials: the xor butterfly
// pairs lanes by bit 4, then 3, 2, 1, 0, which is the grouping of
// transpose_reduce32, so the total has the same bits as there.
__device__ __forceinline__ float warp_total(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

}  // namespace gkm
