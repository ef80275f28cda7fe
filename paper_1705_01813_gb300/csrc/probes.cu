// Measurement probes: the ceilings the assignment's roofline is read against
// where HBM is not the bound.
//
// k_probe_gather reads whole table rows chosen by an index list the way the
// assignment reads candidate centroid rows: one warp per row, 16 bytes per
// lane per load, eight rows of a warp in flight together; a 5 MB table stays
// in L2 (the SIFT-shaped centroid table), a 2 GB one does not (the
// deep-feature one).  k_probe_fma runs independent packed FP32x2 FMA chains
// (the instruction of the distance loops).  Both write one value per warp so
// that the work cannot be dropped.
#include "common.cuh"

namespace gkm {

constexpr int PG_WARPS = 8;
constexpr int PG_ROWS = 8;  // rows in flight per warp

template <int NV>
__global__ void __launch_bounds__(PG_WARPS * 32) k_probe_gather(const float4 *__restrict__ table, int64_t rows,
                                                                int row4, const int32_t *__restrict__ idx,
                                                                int64_t count, float *__restrict__ sink)
{
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int64_t warp = (int64_t)blockIdx.x * PG_WARPS + w, nwarps = (int64_t)gridDim.x * PG_WARPS;
    float acc = 0.f;
    for (int64_t j0 = warp * PG_ROWS; j0 < count; j0 += nwarps * PG_ROWS) {
        float4 v[PG_ROWS][NV];
#pragma unroll
        for (int r = 0; r < PG_ROWS; r++) {
            const int64_t j = j0 + r;
            int row = j < count ? __ldg(idx + j) : -1;
            row = row < rows ? row : -1;  // indices outside the table read nothing
#pragma unroll
            for (int q = 0; q < NV; q++) {
                const int col = lane + 32 * q;
                v[r][q] = (row >= 0 && col < row4) ? __ldg(table + (int64_t)row * row4 + col)
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int r = 0; r < PG_ROWS; r++)
#pragma unroll
            for (int q = 0; q < NV; q++)
                acc += (v[r][q].x + v[r][q].y) + (v[r][q].z + v[r][q].w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(FULL_MASK, acc, o);
    if (lane == 0)
        sink[warp] = acc;
}

__global__ void __launch_bounds__(256) k_probe_fma(float *__restrict__ sink, int64_t iters)
{
    float2 a[8];
    const float s = 1e-7f * (float)(threadIdx.x + 1);
#pragma unroll
    for (int j = 0; j < 8; j++)
        a[j] = make_float2(s * (j + 1), -s * (j + 1));
    const float2 m = make_float2(0.9999999f, 0.9999999f), c = make_float2(1e-9f, -1e-9f);
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < 8; j++)
            a[j] = __ffma2_rn(a[j], m, c);
    }
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++)
        t += a[j].x + a[j].y;
    if ((threadIdx.x & 31) == 0)
        sink[((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5] = t;
}

// both probes: 152 x 8 blocks of 8 warps, one sink value per warp (PROBE_SINK floats)
static_assert(PROBE_SINK == 152 * 8 * PG_WARPS, "sink size");

cudaError_t launch_probe_gather(const float *table, int64_t rows, int row_floats, const int32_t *idx, int64_t count,
                                float *sink, cudaStream_t s)
{
    const int row4 = row_floats / 4;
    const float4 *t4 = reinterpret_cast<const float4 *>(table);
    const int grid = 152 * 8;
    if (row4 <= 32)
        k_probe_gather<1><<<grid, PG_WARPS * 32, 0, s>>>(t4, rows, row4, idx, count, sink);
    else if (row4 <= 64)
        k_probe_gather<2><<<grid, PG_WARPS * 32, 0, s>>>(t4, rows, row4, idx, count, sink);
    else
        k_probe_gather<4><<<grid, PG_WARPS * 32, 0, s>>>(t4, rows, row4, idx, count, sink);
    return cudaGetLastError();
}

cudaError_t launch_probe_fma(float *sink, int64_t iters, cudaStream_t s)
{
    k_probe_fma<<<152 * 8, 256, 0, s>>>(sink, iters);
    return cudaGetLastError();
}

}  // namespace gkm
