// Centroid update as a segmented mean over the CSR grouping (Sec. 1: each
// centroid becomes the average of its members), with the composite vectors
// D_r of Eq. 2 and the distortion after the update from the Eq. 2 identity
//     n E = sum_i ||x_i||^2 - sum_r D_r'D_r / n_r.
//
// One block per cluster; each warp is split into G groups of L lanes
// (L = lanes needed to cover a row with VEC-wide loads, at most 32); a group
// sums every (warps x G)-th member and lane s of a group owns row columns
// s, s + L, ... (in VEC-wide vectors).  Sums are compensated (Kahan) FP32 and
// combined as exact double-float pairs, so the composite vectors keep the
// accuracy of the compensated sums with FP32 arithmetic only; FP64 appears
// once per cluster, in the distortion term.
#include "common.cuh"

#include <cuda_bf16.h>

#include <type_traits>

namespace gkm {

constexpr int UP_WARPS = 4;
constexpr int UP_MCHUNK = 1024;  // member ids staged in shared memory at a time
constexpr int UP_RV = 8;         // 16-byte vectors per lane and pipeline stage (PIPE kernels): 8 / CPL rows

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Double-float values (hi + lo, two FP32 numbers) and the error-free
// transformations that add them (Knuth's two-sum, Dekker's fast two-sum):
// cross-group and cross-warp combination, squares and the mean are done in
// FP32 arithmetic with about 44 bits of precision, which keeps the Kahan sums
// exact and spares the GPU's slow FP64 units.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF fast_two_sum(float a, float b)  // |a| >= |b| or a == 0
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return fast_two_sum(s, e + a.lo + b.lo);
}

__device__ __forceinline__ DF df_shfl_xor(DF a, int o)
{
    return {__shfl_xor_sync(FULL_MASK, a.hi, o), __shfl_xor_sync(FULL_MASK, a.lo, o)};
}

// a^2 (the lo^2 term is below the pair's precision)
__device__ __forceinline__ DF df_sqr(DF a)
{
    const float p = a.hi * a.hi;
    const float e = fmaf(a.hi, a.hi, -p);
    return fast_two_sum(p, fmaf(2.f * a.hi, a.lo, e));
}

// a / m rounded to FP32: q = a.hi / m (IEEE), whose remainder a.hi - q m is
// exact in one fma, corrected by (remainder + a.lo) / m.
__device__ __forceinline__ float df_div(DF a, float mf, float inv_m)
{
    const float q = a.hi / mf;
    const float r = fmaf(-q, mf, a.hi) + a.lo;
    return q + r * inv_m;
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

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

// The Kahan step of kahan_add on two sums at once, in packed FP32x2 instructions with the same roundings (a - b
// as fma(b, -1, a), a + b as fma(a, 1, b): each rounded once, as the scalar operations are).
__device__ __forceinline__ void kahan_add2(float &s0, float &s1, float &c0, float &c1, float2 x)
{
    const float2 m1 = make_float2(-1.f, -1.f), p1 = make_float2(1.f, 1.f);
    const float2 S = make_float2(s0, s1), Cc = make_float2(c0, c1);
    const float2 y = __ffma2_rn(Cc, m1, x);                     // x - c
    const float2 t = __ffma2_rn(S, p1, y);                      // s + y
    const float2 cn = __ffma2_rn(y, m1, __ffma2_rn(S, m1, t));  // (t - s) - y
    s0 = t.x, s1 = t.y, c0 = cn.x, c1 = cn.y;
}

// Accumulate one loaded row slice into the compensated sums: per coordinate the Kahan sum of x, and the sum of
// squares as two compensated chains (qs.x takes the even coordinates of a vector, qs.y the odd ones), each
// square x^2 = p + e split exactly (e from one fma), p summed and e folded into the compensation term (the true
// sum being about qs - qc).  16-byte vectors run in packed FP32x2 instructions.  EXACT_SQ: every x * x is exact
// in FP32 (BF16 samples: 8 significant bits), so the fma that splits off the square's rounding error would give 0
// and is skipped (same bits).
template <int VEC, int CPL, bool EXACT_SQ = false>
__device__ __forceinline__ void accumulate(const typename VecT<VEC>::T (&v)[CPL], float (&s)[CPL][VEC],
                                           float (&c)[CPL][VEC], float2 &qs, float2 &qc, int cb, int sub, int L,
                                           int nv)
{
#pragma unroll
    for (int u = 0; u < CPL; u++) {
        if (cb + sub + u * L < nv) {
            if constexpr (VEC == 4) {
                const float2 m1 = make_float2(-1.f, -1.f), z2 = make_float2(0.f, 0.f);
                const float2 xa = make_float2(comp(v[u], 0), comp(v[u], 1));
                const float2 xb = make_float2(comp(v[u], 2), comp(v[u], 3));
                kahan_add2(s[u][0], s[u][1], c[u][0], c[u][1], xa);
                kahan_add2(s[u][2], s[u][3], c[u][2], c[u][3], xb);
                const float2 pa = __ffma2_rn(xa, xa, z2), pb = __ffma2_rn(xb, xb, z2);
                kahan_add2(qs.x, qs.y, qc.x, qc.y, pa);
                if constexpr (!EXACT_SQ)
                    qc = __ffma2_rn(__ffma2_rn(xa, xa, make_float2(-pa.x, -pa.y)), m1, qc);
                kahan_add2(qs.x, qs.y, qc.x, qc.y, pb);
                if constexpr (!EXACT_SQ)
                    qc = __ffma2_rn(__ffma2_rn(xb, xb, make_float2(-pb.x, -pb.y)), m1, qc);
            } else {
#pragma unroll
                for (int q = 0; q < VEC; q++) {
                    const float x = comp(v[u], q);
                    kahan_add(s[u][q], c[u][q], x);
                    const float p2 = x * x;
                    kahan_add(qs.x, qc.x, p2);
                    if constexpr (!EXACT_SQ)
                        qc.x -= fmaf(x, x, -p2);
                }
            }
        }
    }
}

// The sum of squares of a lane's compensated chains, as a double-float value.
__device__ __forceinline__ DF chains_sum(float2 qs, float2 qc)
{
    return df_add(fast_two_sum(qs.x, -qc.x), fast_two_sum(qs.y, -qc.y));
}

// One block of UP_WARPS warps per cluster.  Each warp is split into G groups
// of L lanes; the W * G groups of the block take members g, g + W G, ... of
// the cluster (UNR of them in flight per group), and lane s of a group owns
// row vectors s, s + L, ... (CPL of them per column block).  Group sums are
// combined (double-float) across the groups of a warp by shuffles and across
// the warps through shared memory in a fixed order (reproducible bits).
// PIPE (16-byte vectors): the member rows are streamed into a two-stage
// shared-memory ring with cp.async, UP_RV / CPL rows per group and stage, so the
// next stage's loads are in flight while the current one is summed; the
// summation order is the same.  The ring shares its memory with the partial
// sums of the epilogue, which run after it.
// One VEC-wide vector of a sample row as floats (BF16 samples are widened).
template <int VEC, typename XT>
__device__ __forceinline__ typename VecT<VEC>::T load_vec(const XT *p)
{
    if constexpr (VEC == 4)
        return ldx4<XT, true>(p);
    else
        return ldx(p);
}

template <int VEC, int CPL, bool PIPE, typename XT>
__global__ void __launch_bounds__(UP_WARPS * 32) k_update(const XT *__restrict__ X, int d, int64_t ld,
                                                          const int32_t *__restrict__ off,
                                                          const int32_t *__restrict__ mem, int k, int small_max,
                                                          float *__restrict__ C, int32_t *__restrict__ counts,
                                                          double *__restrict__ contrib, DevStatus *st)
{
    using V = typename VecT<VEC>::T;
    static_assert(!PIPE || std::is_same_v<XT, float>, "the cp.async ring moves FP32 rows");
    constexpr int UNR = CPL >= 8 ? 1 : (CPL >= 4 ? 2 : (CPL >= 2 ? 4 : 4));  // member rows in flight per group
    constexpr int R = PIPE ? UP_RV / CPL : 1;  // rows per group and stage
    constexpr size_t PART_BYTES = sizeof(float2) * UP_WARPS * 32 * CPL * VEC;
    constexpr size_t RING_BYTES = PIPE ? sizeof(float4) * UP_WARPS * 2 * R * 32 * CPL : 0;
    __shared__ __align__(16) unsigned char s_buf[PART_BYTES > RING_BYTES ? PART_BYTES : RING_BYTES];
    auto s_part = reinterpret_cast<float2 (*)[32 * CPL * VEC]>(s_buf);
    __shared__ float2 s_sq[UP_WARPS], s_dd[UP_WARPS];
    __shared__ int s_mem[UP_MCHUNK];
    static_assert(!PIPE || (VEC == 4 && UP_RV % CPL == 0), "the pipelined variant moves 16-byte vectors");
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

    // clusters r = blockIdx.x, + gridDim.x, ...; those of at most small_max members are k_update_small's
    for (int r = blockIdx.x; r < k; r += gridDim.x) {
    const int beg = off[r], m = off[r + 1] - beg;
    if (m <= small_max)
        continue;
    if (counts && threadIdx.x == 0)
        counts[r] = m;
    if (m == 0) {
        if (threadIdx.x == 0)
            contrib[r] = 0.0;
        continue;
    }
    const float mf = (float)m, inv_m = 1.0f / mf;
    DF sq_lane = {0.f, 0.f}, dd_lane = {0.f, 0.f};
    for (int cb = 0; cb < nv; cb += L * CPL) {
        float s[CPL][VEC], c[CPL][VEC];
        float2 qs = make_float2(0.f, 0.f), qc = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < CPL; u++)
#pragma unroll
            for (int q = 0; q < VEC; q++)
                s[u][q] = c[u][q] = 0.f;
        // the member ids of a chunk are staged in shared memory first, so each row
        // load waits for one memory round trip instead of two
        for (int mb = 0; mb < m; mb += UP_MCHUNK) {
            const int mc = min(UP_MCHUNK, m - mb);
            __syncthreads();  // the previous chunk's ids are no longer read
            for (int q = threadIdx.x; q < mc; q += UP_WARPS * 32)
                s_mem[q] = __ldg(mem + beg + mb + q);
            __syncthreads();
            if constexpr (PIPE) {
                float4 *ring = reinterpret_cast<float4 *>(s_buf) + w * (2 * R * 32 * CPL);  // [stage][row][u][lane]
                const int wlead = w * G;                       // the warp's first group has the most rows
                const int njw = mc > wlead ? (mc - wlead + gstride - 1) / gstride : 0;
                const int nst = (njw + R - 1) / R;
                auto issue = [&](int t) {
                    float4 *buf = ring + (t & 1) * (R * 32 * CPL);
#pragma unroll
                    for (int z = 0; z < R; z++) {
                        const int p = gidx + gstride * (t * R + z);
                        if (p < mc) {
                            const V *row = Xv + (int64_t)s_mem[p] * ldv;
#pragma unroll
                            for (int u = 0; u < CPL; u++) {
                                const int col = cb + sub + u * L;
                                if (col < nv)
                                    cp_async16(buf + (z * CPL + u) * 32 + lane, row + col);
                            }
                        }
                    }
                    cp_async_commit();
                };
                if (nst > 0)
                    issue(0);
                for (int t = 0; t < nst; t++) {
                    if (t + 1 < nst)
                        issue(t + 1);
                    else
                        cp_async_commit();  // empty group: the wait below always leaves one
                    cp_async_wait<1>();
                    __syncwarp();
                    const float4 *buf = ring + (t & 1) * (R * 32 * CPL);
#pragma unroll
                    for (int z = 0; z < R; z++) {
                        if (gidx + gstride * (t * R + z) < mc) {
                            V vz[CPL];
#pragma unroll
                            for (int u = 0; u < CPL; u++)
                                vz[u] = buf[(z * CPL + u) * 32 + lane];
                            accumulate<VEC, CPL, std::is_same_v<XT, __nv_bfloat16>>(vz, s, c, qs, qc, cb, sub, L, nv);
                        }
                    }
                    __syncwarp();  // stage t & 1 is refilled by issue(t + 2)
                }
            } else {
                for (int p0 = gidx; p0 < mc; p0 += UNR * gstride) {
                    V v[UNR][CPL];
#pragma unroll
                    for (int z = 0; z < UNR; z++) {
                        const int p = p0 + z * gstride;
                        if (p < mc) {
                            const XT *rowx = X + (int64_t)s_mem[p] * ld;
#pragma unroll
                            for (int u = 0; u < CPL; u++) {
                                const int col = cb + sub + u * L;
                                if (col < nv)
                                    v[z][u] = load_vec<VEC>(rowx + (int64_t)col * VEC);
                            }
                        }
                    }
#pragma unroll
                    for (int z = 0; z < UNR; z++)
                        if (p0 + z * gstride < mc)
                            accumulate<VEC, CPL, std::is_same_v<XT, __nv_bfloat16>>(v[z], s, c, qs, qc, cb, sub, L, nv);
                }
            }
        }
        if constexpr (PIPE)
            __syncthreads();  // every warp is done with the ring before the partial sums overwrite it
        sq_lane = df_add(sq_lane, chains_sum(qs, qc));
        // combine the G groups of the warp, then the warps of the block, in a fixed order
#pragma unroll
        for (int u = 0; u < CPL; u++) {
#pragma unroll
            for (int q = 0; q < VEC; q++) {
                DF S = fast_two_sum(s[u][q], -c[u][q]);  // the Kahan sum s - c, exactly
                for (int o = L; o < 32; o <<= 1)
                    S = df_add(S, df_shfl_xor(S, o));
                if (g == 0)
                    s_part[w][(u * L + sub) * VEC + q] = make_float2(S.hi, S.lo);
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < L * CPL * VEC; e += UP_WARPS * 32) {
            // entry e = (u * L + sb) * VEC + q holds column vector cb + sb + u * L, component q
            const int u = (e / VEC) / L, sb = (e / VEC) % L;
            const int colv = cb + sb + u * L;
            if (colv < nv) {
                DF S = {s_part[0][e].x, s_part[0][e].y};
                for (int ww = 1; ww < UP_WARPS; ww++)
                    S = df_add(S, DF{s_part[ww][e].x, s_part[ww][e].y});
                C[(int64_t)r * d + (int64_t)colv * VEC + (e % VEC)] = df_div(S, mf, inv_m);
                dd_lane = df_add(dd_lane, df_sqr(S));
            }
        }
        __syncthreads();
    }
    // sum of ||x||^2 over all lanes, sum of D_t^2 over the threads that wrote means
    for (int o = 1; o < 32; o <<= 1) {
        sq_lane = df_add(sq_lane, df_shfl_xor(sq_lane, o));
        dd_lane = df_add(dd_lane, df_shfl_xor(dd_lane, o));
    }
    if (lane == 0) {
        s_sq[w] = make_float2(sq_lane.hi, sq_lane.lo);
        s_dd[w] = make_float2(dd_lane.hi, dd_lane.lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DF sq = {s_sq[0].x, s_sq[0].y}, dd = {s_dd[0].x, s_dd[0].y};
        for (int ww = 1; ww < UP_WARPS; ww++) {
            sq = df_add(sq, DF{s_sq[ww].x, s_sq[ww].y});
            dd = df_add(dd, DF{s_dd[ww].x, s_dd[ww].y});
        }
        const double cr = df_to_double(sq) - df_to_double(dd) / (double)m;
        contrib[r] = cr;
        if (!isfinite(cr))  // a non-finite sample in the cluster (Inf or NaN spreads into its sums)
            flag_error(st, GK_ERR_NUMERIC, (unsigned)r);
    }
    __syncthreads();  // s_sq / s_dd are read above before the next cluster writes them
    }
}

// Clusters of at most maxm members, one warp each (the deep-feature workload's clusters hold about ten):
// lane l owns row vectors l, l + 32, ... (NVL of them); the members' rows stream through the warp RIF at a
// time, and every coordinate is summed over the members in member order with compensated FP32 arithmetic,
// then combined and divided as in k_update.  No shared memory and no block barrier, so a cluster costs a
// few dependent loads instead of a block's set-up.
constexpr int US_WARPS = 8;
// Largest cluster of the warp kernel: 32 members for rows of at most 128 values (larger clusters of such rows are
// faster in k_update's block: 1M x 128 FP32, clusters of about 100: 0.173 against 0.223 ms per call), 128 members
// for wider rows (10M x 512 BF16, clusters of about 10 and 50: 3.8 against 5.1 ms).  The rule depends on the row
// width only, so BF16 samples and their FP32 widening take the same kernel for every cluster.
constexpr int US_MAXM_NARROW = 32;
constexpr int US_MAXM_WIDE = 128;

// A row vector of 4 elements as loaded (16 bytes of FP32, 8 bytes of BF16), widened when it is summed.
template <typename XT>
struct RawVec;
template <>
struct RawVec<float> {
    using T = float4;
    __device__ static T load(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
    __device__ static float4 widen(T v) { return v; }
    __device__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct RawVec<__nv_bfloat16> {
    using T = uint2;
    __device__ static T load(const __nv_bfloat16 *p) { return __ldcs(reinterpret_cast<const uint2 *>(p)); }
    __device__ static float4 widen(T v) { return bf16x4_to_float4(v); }
    __device__ static T zero() { return make_uint2(0u, 0u); }
};

template <int NVL, typename XT>
__global__ void __launch_bounds__(US_WARPS * 32, 3) k_update_small(const XT *__restrict__ X, int d, int64_t ld,
                                                                const int32_t *__restrict__ off,
                                                                const int32_t *__restrict__ mem, int k, int maxm,
                                                                float *__restrict__ C, int32_t *__restrict__ counts,
                                                                double *__restrict__ contrib, DevStatus *st)
{
    constexpr int RIF = NVL == 1 ? 8 : NVL == 2 ? 4 : 2;  // member rows in flight (registers allowing)
    using RV = RawVec<XT>;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int nv = d / 4;
    for (int r = blockIdx.x * US_WARPS + w; r < k; r += gridDim.x * US_WARPS) {
        const int beg = off[r], m = off[r + 1] - beg;
        if (m > maxm)
            continue;  // a cluster of k_update
        if (counts && lane == 0)
            counts[r] = m;
        if (m == 0) {
            if (lane == 0)
                contrib[r] = 0.0;
            continue;
        }
        // member ids 32 at a time (lane l holds id p + l of the current 32), the next 32 loaded one chunk ahead
        int myid = lane < m ? __ldg(mem + beg + lane) : 0;
        int nxtid = 32 + lane < m ? __ldg(mem + beg + 32 + lane) : 0;
        float s[NVL][4], c[NVL][4];
#pragma unroll
        for (int u = 0; u < NVL; u++)
#pragma unroll
            for (int q = 0; q < 4; q++)
                s[u][q] = c[u][q] = 0.f;
        float2 qs = make_float2(0.f, 0.f), qc = make_float2(0.f, 0.f);
        for (int p0 = 0; p0 < m; p0 += RIF) {
            if (p0 > 0 && (p0 & 31) == 0) {  // RIF divides 32
                myid = nxtid;
                nxtid = p0 + 32 + lane < m ? __ldg(mem + beg + p0 + 32 + lane) : 0;
            }
            typename RV::T raw[RIF][NVL];
#pragma unroll
            for (int z = 0; z < RIF; z++) {
                const int a = __shfl_sync(FULL_MASK, myid, (p0 + z) & 31);
                const XT *row = X + (int64_t)a * ld;
#pragma unroll
                for (int u = 0; u < NVL; u++) {
                    const int col = lane + 32 * u;
                    raw[z][u] = (p0 + z < m && col < nv) ? RV::load(row + 4 * col) : RV::zero();
                }
            }
#pragma unroll
            for (int z = 0; z < RIF; z++) {
                if (p0 + z < m) {
                    float4 v[NVL];
#pragma unroll
                    for (int u = 0; u < NVL; u++)
                        v[u] = RV::widen(raw[z][u]);
                    accumulate<4, NVL, std::is_same_v<XT, __nv_bfloat16>>(v, s, c, qs, qc, 0, lane, 32, nv);
                }
            }
        }
        const float mf = (float)m, inv_m = 1.0f / mf;
        DF sq = chains_sum(qs, qc), dd = {0.f, 0.f};
#pragma unroll
        for (int u = 0; u < NVL; u++) {
            const int col = lane + 32 * u;
            if (col < nv) {
                float out[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const DF S = fast_two_sum(s[u][q], -c[u][q]);  // the Kahan sum s - c, exactly
                    out[q] = df_div(S, mf, inv_m);
                    dd = df_add(dd, df_sqr(S));
                }
                *reinterpret_cast<float4 *>(C + (int64_t)r * d + 4 * col) = make_float4(out[0], out[1], out[2], out[3]);
            }
        }
        for (int o = 1; o < 32; o <<= 1) {
            sq = df_add(sq, df_shfl_xor(sq, o));
            dd = df_add(dd, df_shfl_xor(dd, o));
        }
        if (lane == 0) {
            const double cr = df_to_double(sq) - df_to_double(dd) / (double)m;
            contrib[r] = cr;
            if (!isfinite(cr))
                flag_error(st, GK_ERR_NUMERIC, (unsigned)r);
        }
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

const double *update_contrib(const void *scratch) { return static_cast<const double *>(scratch); }

template <typename XT>
static cudaError_t update_t(const XT *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                            const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2,
                            void *scratch, DevStatus *st, cudaStream_t s)
{
    double *contrib = static_cast<double *>(scratch);
    const bool vec4 = x_vec4(X, d, ld);
    const int nv = vec4 ? (int)(d / 4) : (int)d;
    const int L = nv >= 32 ? 32 : (nv >= 16 ? 16 : nv >= 8 ? 8 : nv >= 4 ? 4 : nv >= 2 ? 2 : 1);
    const int need = (nv + L - 1) / L;  // vectors per lane to cover a row in one column block
    const int dd = (int)d;
    constexpr bool PIPE = std::is_same_v<XT, float>;  // FP32 rows stream through the cp.async ring
    // clusters of at most small_max members go to the warp-per-cluster kernel where rows are 16-byte vectors of
    // at most 4 per lane and the centroid rows 16-byte aligned; the block kernel takes the others (which kernel
    // sums a cluster depends on its size and the row width only)
    const bool small = vec4 && nv <= 32 * 4 && d % 4 == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
    const int small_max = small ? (nv > 32 ? US_MAXM_WIDE : US_MAXM_NARROW) : -1;
    cudaError_t e;
    if (small) {
        int g = 0;
#define GK_UPS(NVL)                                                                                                \
    do {                                                                                                         \
        if ((e = resident_grid(reinterpret_cast<const void *>(k_update_small<NVL, XT>), US_WARPS * 32, 0, &g)) !=   \
            cudaSuccess)                                                                                         \
            return e;                                                                                            \
        k_update_small<NVL, XT><<<(unsigned)g, US_WARPS * 32, 0, s>>>(X, dd, ld, offsets, members, k, small_max, \
                                                                      C, counts, contrib, st);                   \
    } while (0)
        if (nv <= 32)
            GK_UPS(1);
        else if (nv <= 64)
            GK_UPS(2);
        else
            GK_UPS(4);
#undef GK_UPS
    }
    // the block kernel walks the clusters grid-stride on a one-wave grid (at most k blocks)
    int bg = 0;
    if ((e = resident_grid(reinterpret_cast<const void *>(vec4 ? (need <= 1 ? (const void *)k_update<4, 1, PIPE, XT>
                                                                             : need <= 2 ? (const void *)k_update<4, 2, PIPE, XT>
                                                                             : need <= 4 ? (const void *)k_update<4, 4, PIPE, XT>
                                                                                         : (const void *)k_update<4, 8, PIPE, XT>)
                                                                 : (need <= 1 ? (const void *)k_update<1, 1, false, XT>
                                                                             : need <= 2 ? (const void *)k_update<1, 2, false, XT>
                                                                             : need <= 4 ? (const void *)k_update<1, 4, false, XT>
                                                                                         : (const void *)k_update<1, 8, false, XT>)),
                           UP_WARPS * 32, 0, &bg)) != cudaSuccess)
        return e;
    // one block per cluster while the clusters are mostly the block kernel's (the hardware then hands clusters
    // of uneven sizes to SMs as blocks finish); where most clusters are small, a one-wave grid walks the few
    // large ones instead of launching a block per cluster that would return at once.  Which block sums a
    // cluster changes none of its bits.
    const bool mostly_small = small && n <= (int64_t)k * small_max;
    const unsigned grid = (unsigned)(mostly_small ? (k < bg ? k : bg) : k);
#define GK_UPD(VEC, CPL, P) \
    k_update<VEC, CPL, P, XT><<<grid, UP_WARPS * 32, 0, s>>>(X, dd, ld, offsets, members, k, small_max, C, counts, \
                                                             contrib, st)
    if (vec4) {
        if (need <= 1)
            GK_UPD(4, 1, PIPE);
        else if (need <= 2)
            GK_UPD(4, 2, PIPE);
        else if (need <= 4)
            GK_UPD(4, 4, PIPE);
        else
            GK_UPD(4, 8, PIPE);
    } else {
        if (need <= 1)
            GK_UPD(1, 1, false);
        else if (need <= 2)
            GK_UPD(1, 2, false);
        else if (need <= 4)
            GK_UPD(1, 4, false);
        else
            GK_UPD(1, 8, false);
    }
#undef GK_UPD
    if (sum_d2)
        k_sum_f64<<<1, 1024, 0, s>>>(contrib, k, sum_d2);
    return cudaGetLastError();
}

cudaError_t launch_update(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2,
                          void *scratch, DevStatus *st, cudaStream_t s)
{
    if (bf16)
        return update_t(static_cast<const __nv_bfloat16 *>(X), n, d, ld, offsets, members, k, C, counts, sum_d2,
                        scratch, st, s);
    return update_t(static_cast<const float *>(X), n, d, ld, offsets, members, k, C, counts, sum_d2, scratch, st, s);
}

}  // namespace gkm
