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

// Accumulate one loaded row slice into the compensated sums.
template <int VEC, int CPL>
__device__ __forceinline__ void accumulate(const typename VecT<VEC>::T (&v)[CPL], float (&s)[CPL][VEC],
                                           float (&c)[CPL][VEC], float &qs, float &qc, int cb, int sub, int L, int nv)
{
#pragma unroll
    for (int u = 0; u < CPL; u++) {
        if (cb + sub + u * L < nv) {
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

// CPL: row vectors per lane per column block (chosen from d by the launcher).
template <int VEC, int CPL>
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
        if (counts && lane == 0)
            counts[r] = m;
        if (m == 0) {
            if (lane == 0)
                contrib[r] = 0.0;
            continue;
        }
        double sq_lane = 0.0, dd_lane = 0.0;
        for (int cb = 0; cb < nv; cb += L * CPL) {
            float s[CPL][VEC], c[CPL][VEC];
            float qs = 0.f, qc = 0.f;
#pragma unroll
            for (int u = 0; u < CPL; u++)
#pragma unroll
                for (int q = 0; q < VEC; q++)
                    s[u][q] = c[u][q] = 0.f;
            // members in batches of 32 ids (one coalesced load), handed to the
            // lane groups by shuffles; two members per group in flight
            for (int b0 = 0; b0 < m; b0 += 32) {
                const int nb = min(32, m - b0);
                const int my_id = lane < nb ? mem[beg + b0 + lane] : 0;
                for (int j = 0; j < nb; j += 2 * G) {
                    const int p0 = j + g, p1 = j + G + g;
                    const int id0 = __shfl_sync(FULL_MASK, my_id, p0 & 31);
                    const int id1 = __shfl_sync(FULL_MASK, my_id, p1 & 31);
                    V v0[CPL], v1[CPL];
                    const V *row0 = Xv + (int64_t)id0 * ldv;
                    const V *row1 = Xv + (int64_t)id1 * ldv;
#pragma unroll
                    for (int u = 0; u < CPL; u++) {
                        int col = cb + sub + u * L;
                        if (col < nv && p0 < nb)
                            v0[u] = __ldcs(row0 + col);
                        if (col < nv && p1 < nb)
                            v1[u] = __ldcs(row1 + col);
                    }
                    if (p0 < nb)
                        accumulate<VEC, CPL>(v0, s, c, qs, qc, cb, sub, L, nv);
                    if (p1 < nb)
                        accumulate<VEC, CPL>(v1, s, c, qs, qc, cb, sub, L, nv);
                }
            }
            sq_lane += (double)qs - (double)qc;
            // widen, combine the G groups, write the means of this column block
#pragma unroll
            for (int u = 0; u < CPL; u++) {
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
    if (blocks > 152 * 64)
        blocks = 152 * 64;
    bool vec4 = (d % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const int nv = vec4 ? (int)(d / 4) : (int)d;
    const int L = nv >= 32 ? 32 : (nv >= 16 ? 16 : nv >= 8 ? 8 : nv >= 4 ? 4 : nv >= 2 ? 2 : 1);
    const int need = (nv + L - 1) / L;  // vectors per lane to cover a row in one column block
    const unsigned grid = (unsigned)blocks;
    const int dd = (int)d;
#define GK_UPD(VEC, CPL) \
    k_update<VEC, CPL><<<grid, UP_WARPS * 32, 0, s>>>(X, dd, ld, offsets, members, k, C, counts, contrib)
    if (vec4) {
        if (need <= 1)
            GK_UPD(4, 1);
        else if (need <= 2)
            GK_UPD(4, 2);
        else if (need <= 4)
            GK_UPD(4, 4);
        else
            GK_UPD(4, 8);
    } else {
        if (need <= 1)
            GK_UPD(1, 1);
        else if (need <= 2)
            GK_UPD(1, 2);
        else if (need <= 4)
            GK_UPD(1, 4);
        else
            GK_UPD(1, 8);
    }
#undef GK_UPD
    if (sum_d2)
        k_sum_f64<<<1, 1024, 0, s>>>(contrib, k, sum_d2);
    return cudaGetLastError();
}

}  // namespace gkm
