// Measurement probes of the benchmark (not part of libgkm): the ceilings the
// assignment's roofline is read against where HBM is not the bound.
//
// k_probe_gather reads whole table rows chosen by an index list the way the
// assignment reads candidate centroid rows: one warp per row, 16 bytes per
// lane per load, eight rows of a warp in flight together; a 5 MB table stays
// in L2 (the SIFT-shaped centroid table), a 2 GB one does not (the
// deep-feature one).  k_probe_fma runs independent packed FP32x2 FMA chains
// (the instruction of the distance loops).  Both write one value per warp so
// that the work cannot be dropped.
//
// Built into libgkm_probes.so by benchlib/probes.py; the entry points below
// return 0 on success, 1 on a bad argument, 2 on a CUDA launch error.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PG_WARPS = 8;
constexpr int PG_ROWS = 8;        // rows in flight per warp
constexpr int GRID = 152 * 8;     // both probes: 152 x 8 blocks
constexpr int SINK = GRID * PG_WARPS;  // one sink value per warp

template <int NV>
__global__ void __launch_bounds__(PG_WARPS * 32) k_probe_gather(const float4 *__restrict__ table, int64_t rows,
                                                                int row4, const int32_t *__restrict__ idx,
                                                                int64_t count, float *__restrict__ sink)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * PG_WARPS + w, nwarps = (int64_t)gridDim.x * PG_WARPS;
    float acc = 0.f;
    for (int64_t j0 = warp * PG_ROWS; j0 < count; j0 += nwarps * PG_ROWS) {
        float4 v[PG_ROWS][NV];
#pragma unroll
        for (int r = 0; r < PG_ROWS; r++) {
            const int64_t j = j0 + r;
            int row = j < count ? __ldg(idx + j) : -1;
            row = (row >= 0 && row < rows) ? row : -1;  // indices outside the table read nothing
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
        acc += __shfl_xor_sync(FULL, acc, o);
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

}  // namespace

extern "C" {

__attribute__((visibility("default"))) int gkb_probe_sink_floats(void) { return SINK; }

// For j < count, one warp reads row idx[j] of table (rows x row_floats FP32,
// row-major, 16-byte aligned; row_floats a multiple of 4 up to 512) in
// 16-byte loads.  Bytes read: count x row_floats x 4.  sink: SINK floats.
__attribute__((visibility("default"))) int gkb_probe_gather(const float *table, int64_t rows, int32_t row_floats,
                                                            const int32_t *idx, int64_t count, float *sink,
                                                            void *stream)
{
    if (!table || !idx || !sink || rows < 1 || rows > INT32_MAX || count < 0)
        return 1;
    if (row_floats < 4 || row_floats > 512 || row_floats % 4 != 0 || (reinterpret_cast<uintptr_t>(table) & 15))
        return 1;
    const int row4 = row_floats / 4;
    const float4 *t4 = reinterpret_cast<const float4 *>(table);
    cudaStream_t s = (cudaStream_t)stream;
    if (row4 <= 32)
        k_probe_gather<1><<<GRID, PG_WARPS * 32, 0, s>>>(t4, rows, row4, idx, count, sink);
    else if (row4 <= 64)
        k_probe_gather<2><<<GRID, PG_WARPS * 32, 0, s>>>(t4, rows, row4, idx, count, sink);
    else
        k_probe_gather<4><<<GRID, PG_WARPS * 32, 0, s>>>(t4, rows, row4, idx, count, sink);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// Every thread runs eight independent chains of `iters` packed FP32x2 FMAs:
// 32 x iters FLOP per thread, GRID x 256 threads.
__attribute__((visibility("default"))) int gkb_probe_fma(float *sink, int64_t iters, void *stream)
{
    if (!sink || iters < 0)
        return 1;
    k_probe_fma<<<GRID, 256, 0, (cudaStream_t)stream>>>(sink, iters);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
