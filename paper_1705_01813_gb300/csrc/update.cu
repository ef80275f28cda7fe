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

constexpr int UP_WARPS = 4;

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

// One block of UP_WARPS warps per cluster.  Each warp is split into G groups
// of L lanes; the W * G groups of the block take members g, g + W G, ... of
// the cluster (UNR of them in flight per group), and lane s of a group owns
// row vectors s, s + L, ... (CPL of them per column block).  Group sums are
// widened to FP64, combined across the groups of a warp by shuffles and across
// the warps through shared memory in a fixed order (reproducible bits).
template <int VEC, int CPL>
__global__ void __launch_bounds__(UP_WARPS * 32) k_update(const float *__restrict__ X, int d, int64_t ld,
                                                          const int32_t *__restrict__ off,
                                                          const int32_t *__restrict__ mem, int k,
                                                          float *__restrict__ C, int32_t *__restrict__ counts,
                                                          double *__restrict__ contrib)
{
    using V = typename VecT<VEC>::T;
    constexpr int UNR = CPL >= 8 ? 1 : (CPL >= 4 ? 2 : 4);  // member rows in flight per group
    __shared__ double s_part[UP_WARPS][32 * CPL * VEC];
    __shared__ double s_sq[UP_WARPS];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int nv = d / VEC;  // vectors per row
    int L = 1;
    while (L < 32 && L < nv)
        L <<= 1;
    const int G = 32 / L;
    const int g = lane / L, sub = lane % L;
    const int gstride = UP_WARPS * G, gidx = w * G + g;
    const int64_t ldv = ld / VEC;
    const V *Xv = reinterpret_cast<const V *>(X);

    const int r = blockIdx.x;
    if (r >= k)
        return;
    const int beg = off[r], m = off[r + 1] - beg;
    if (counts && threadIdx.x == 0)
        counts[r] = m;
    if (m == 0) {
        if (threadIdx.x == 0)
            contrib[r] = 0.0;
        return;
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
        for (int p0 = gidx; p0 < m; p0 += UNR * gstride) {
            V v[UNR][CPL];
#pragma unroll
            for (int z = 0; z < UNR; z++) {
                const int p = p0 + z * gstride;
                if (p < m) {
                    const V *row = Xv + (int64_t)__ldg(mem + beg + p) * ldv;
#pragma unroll
                    for (int u = 0; u < CPL; u++) {
                        const int col = cb + sub + u * L;
                        if (col < nv)
                            v[z][u] = __ldcs(row + col);
                    }
                }
            }
#pragma unroll
            for (int z = 0; z < UNR; z++)
                if (p0 + z * gstride < m)
                    accumulate<VEC, CPL>(v[z], s, c, qs, qc, cb, sub, L, nv);
        }
        sq_lane += (double)qs - (double)qc;
        // widen, combine the G groups of the warp, then the warps of the block
#pragma unroll
        for (int u = 0; u < CPL; u++) {
#pragma unroll
            for (int q = 0; q < VEC; q++) {
                double S = (double)s[u][q] - (double)c[u][q];
                for (int o = L; o < 32; o <<= 1)
                    S += __shfl_xor_sync(FULL_MASK, S, o);
                if (g == 0)
                    s_part[w][(u * L + sub) * VEC + q] = S;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < L * CPL * VEC; e += UP_WARPS * 32) {
            // entry e = (u * L + sb) * VEC + q holds column vector cb + sb + u * L, component q
            const int u = (e / VEC) / L, sb = (e / VEC) % L;
            const int colv = cb + sb + u * L;
            if (colv < nv) {
                double S = 0.0;
                for (int ww = 0; ww < UP_WARPS; ww++)
                    S += s_part[ww][e];
                C[(int64_t)r * d + (int64_t)colv * VEC + (e % VEC)] = (float)(S / (double)m);
                dd_lane += S * S;
            }
        }
        __syncthreads();
    }
    // sum of ||x||^2 over all lanes, sum of D_t^2 over the threads that wrote means
    for (int o = 1; o < 32; o <<= 1) {
        sq_lane += __shfl_xor_sync(FULL_MASK, sq_lane, o);
        dd_lane += __shfl_xor_sync(FULL_MASK, dd_lane, o);
    }
    if (lane == 0) {
        s_sq[w] = sq_lane;
        s_part[w][0] = dd_lane;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sq = 0.0, dd = 0.0;
        for (int ww = 0; ww < UP_WARPS; ww++) {
            sq += s_sq[ww];
            dd += s_part[ww][0];
        }
        contrib[r] = sq - dd / (double)m;
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
    const int64_t blocks = k;
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
