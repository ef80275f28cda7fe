// Helpers shared by the assignment kernels (SIMT and tensor-core): the
// per-lane partial squared distance in the fixed order of the FP32 path and
// the warp reductions that complete it.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gkm {

// Sum of 32 per-lane partial values for 32 candidates at once: after the five
// exchange steps lane l holds the total over the warp of v[l] (31 shuffles in
// all, instead of 5 per candidate).
__device__ __forceinline__ float transpose_reduce32(float (&v)[32])
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < o; j++) {
            float send = upper ? v[j] : v[j + o];
            float keep = upper ? v[j + o] : v[j];
            v[j] = keep + __shfl_xor_sync(FULL_MASK, send, o);
        }
    }
    return v[0];
}

__device__ __forceinline__ float4 bf16x4_to_float4(uint2 v)
{
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&v.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&v.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

// Partial (per lane) squared distance of x (registers) to a row of 16-byte
// vectors, in the accumulation order of k_assign_rows.
template <int NV, typename RowLoad>
__device__ __forceinline__ float lane_partial(const float4 (&xv)[NV], int d4, RowLoad load)
{
    const int lane = lane_id();
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        const int col = lane + 32 * v;
        if (col < d4) {
            const float4 cv = load(col);
            const float e0 = xv[v].x - cv.x, e1 = xv[v].y - cv.y, e2 = xv[v].z - cv.z, e3 = xv[v].w - cv.w;
            a0 = fmaf(e0, e0, a0);
            a1 = fmaf(e1, e1, a1);
            a0 = fmaf(e2, e2, a0);
            a1 = fmaf(e3, e3, a1);
        }
    }
    return a0 + a1;
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
