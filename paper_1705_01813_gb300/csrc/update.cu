// Centroid update as a segmented mean over the CSR grouping (Sec. 1: each
// centroid becomes the average of its members), with the composite vectors
// D_r of Eq. 2 and the distortion after the update from the Eq. 2 identity
//     n E = sum_i ||x_i||^2 - sum_r D_r'D_r / n_r.
//
// One warp per cluster.  The warp is split into G groups of L lanes
// (L = lanes needed to cover a row with VEC-wide loads, at most 32); group g
// sums members g, g + G, ... and lane s of a group owns row columns
// s, s + L, ... (in VEC-wide vectors).  Sums are compensated (Kahan) FP32,
// widened to FP64 before groups are combined, so the composite vectors keep
// about FP64 accuracy without FP64 arithmetic per element.
#include "common.cuh"

namespace gkm {

constexpr int UP_WARPS = 8;
constexpr int UP_CPL = 8;  // vectors per lane per column block

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <int VEC>
struct VecT;
template <>
struct VecT<4> {
    using T = float4;
};
template <>
struct VecT<1> {
    using T = float;
};

__device__ __forceinline__ float comp(const float4 &v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }
__device__ __forceinline__ float comp(const float &v, int) { return v; }

template <int VEC>
__global__ void __launch_bounds__(UP_WARPS * 32) k_update(const float *__restrict__ X, int d, int64_t ld,
                                                          const int32_t *__restrict__ off,
                                                          const int32_t *__restrict__ mem, int k,
                                                          float *__restrict__ C, int32_t *__restrict__ counts,
                                                          double *__restrict__ contrib)
{
    using V = typename VecT<VEC>::T;
    const int lane = lane_id();
    const int nv = d / VEC;  // vectors per row
    int L = 1;
    while (L < 32 && L < nv)
        L <<= 1;
    const int G = 32 / L;
    const int g = lane / L, sub = lane % L;
    const int64_t ldv = ld / VEC;
    const V *Xv = reinterpret_cast<const V *>(X);

    for (int r = blockIdx.x * UP_WARPS + (threadIdx.x >> 5); r < k; r += gridDim.x * UP_WARPS) {
        const int beg = off[r], m = off[r + 1] - beg;
        if (counts)
            counts[r] = m;
        if (m == 0) {
            if (lane == 0)
                contrib[r] = 0.0;
            continue;
        }
        double sq_lane = 0.0, dd_lane = 0.0;
        for (int cb = 0; cb < nv; cb += L * UP_CPL) {
            float s[UP_CPL][VEC], c[UP_CPL][VEC];
            float qs = 0.f, qc = 0.f;
#pragma unroll
            for (int u = 0; u < UP_CPL; u++)
#pragma unroll
                for (int q = 0; q < VEC; q++)
                    s[u][q] = c[u][q] = 0.f;
            for (int p = g; p < m; p += G) {
                const V *row = Xv + (int64_t)mem[beg + p] * ldv;
                V v[UP_CPL];
#pragma unroll
                for (int u = 0; u < UP_CPL; u++) {
                    int col = cb + sub + u * L;
                    if (col < nv)
                        v[u] = row[col];
                }
#pragma unroll
                for (int u = 0; u < UP_CPL; u++) {
                    int col = cb + sub + u * L;
                    if (col < nv) {
#pragma unroll
                        for (int q = 0; q < VEC; q++) {
                            float x = comp(v[u], q);
                            kahan_add(s[u][q], c[u][q], x);
                            // x^2 = p + e exactly (e from one fma); p is summed, e folded
                            // into the compensation term (true sum ~ qs - qc)
                            float p2 = x * x;
                            float e2 = fmaf(x, x, -p2);
                            kahan_add(qs, qc, p2);
                            qc -= e2;
                        }
                    }
                }
            }
            sq_lane += (double)qs - (double)qc;
            // widen, combine the G groups, write the means of this column block
#pragma unroll
            for (int u = 0; u < UP_CPL; u++) {
                int col = cb + sub + u * L;
#pragma unroll
                for (int q = 0; q < VEC; q++) {
                    double S = (double)s[u][q] - (double)c[u][q];
                    for (int o = L; o < 32; o <<= 1)
                        S += __shfl_xor_sync(FULL_MASK, S, o);
                    if (col < nv && g == 0) {
                        C[(int64_t)r * d + (int64_t)col * VEC + q] = (float)(S / (double)m);
                        dd_lane += S * S;
                    }
                }
            }
        }
        for (int o = 1; o < 32; o <<= 1) {
            sq_lane += __shfl_xor_sync(FULL_MASK, sq_lane, o);
            dd_lane += __shfl_xor_sync(FULL_MASK, dd_lane, o);
        }
        if (lane == 0)
            contrib[r] = sq_lane - dd_lane / (double)m;
    }
}

// Deterministic FP64 sum of `count` values (one block, fixed order).
__global__ void __launch_bounds__(1024) k_sum_f64(const double *__restrict__ v, int64_t count,
                                                  double *__restrict__ out)
{
    __shared__ double s[1024];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += 1024)
        a += v[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *out = s[0];
}

size_t update_scratch_bytes(int64_t, int32_t k) { return ((size_t)k * sizeof(double) + 255) & ~size_t(255); }

cudaError_t launch_update(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2,
                          void *scratch, cudaStream_t s)
{
    (void)n;
    double *contrib = static_cast<double *>(scratch);
    int64_t blocks = ((int64_t)k + UP_WARPS - 1) / UP_WARPS;
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    bool vec4 = (d % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    if (vec4)
        k_update<4><<<(unsigned)blocks, UP_WARPS * 32, 0, s>>>(X, (int)d, ld, offsets, members, k, C, counts,
                                                                contrib);
    else
        k_update<1><<<(unsigned)blocks, UP_WARPS * 32, 0, s>>>(X, (int)d, ld, offsets, members, k, C, counts,
                                                                contrib);
    if (sum_d2)
        k_sum_f64<<<1, 1024, 0, s>>>(contrib, k, sum_d2);
    return cudaGetLastError();
}

}  // namespace gkm
