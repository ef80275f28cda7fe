// Graph-guided assignment (Alg. 2 candidate loop with the closest-centroid
// rule of Sec. 4.2, "GK-means^-"):
//   Q_i = { L[i] } u { L[G[i][j]] : j < kappa }          (candidate clusters)
//   L'[i] = argmin over r in Q_i of (||x_i - C_r||^2, r)  (ties -> smaller label)
//
// One warp per sample.  The warp stages x_i in shared memory, gathers the
// kappa + 1 candidate labels 32 at a time and removes repeats with
// __match_any_sync plus a scan of the labels already kept, then each lane
// takes candidates lane, lane + 32, ... and computes their distances with
// 16-byte centroid loads; a shuffle reduction picks the (distance, label)
// minimum.  Per-block FP64 partial sums of the winning distances and the
// count of changed labels are reduced in a fixed order afterwards, so every
// run gives the same bits.
#include "assign_common.cuh"
#include "common.cuh"

#include <cuda_bf16.h>

#include <type_traits>

namespace gkm {

bool assign_tc_supported(int64_t d, int64_t ld, const float *X, const float *C, int32_t kappa);
cudaError_t launch_assign_tc(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                             const float *C, const __nv_bfloat16 *Cb, const float *delta, const float *cnorm,
                             int32_t k, const int32_t *labels_in, const int32_t *members, int32_t *sel_lab,
                             int32_t *sel_n, int32_t *tile_flag, DevStatus *st, cudaStream_t s);

constexpr int AS_WARPS = 8;
constexpr int AS_BLOCKS = 152 * 8;  // fixed grid: the FP64 partial sums have a fixed order
// The row kernels for d <= 256 fit six blocks per SM (at most 40 registers a thread: more warps in flight
// for the latency-bound centroid gathers).  Every row kernel runs on a grid of the blocks resident at once
// (resident_grid), one wave; the distortion sums do not depend on it: k_assign_reduce forms them on its
// own fixed grid.
constexpr int AS_ROWS_PER_SM = 6;
constexpr int AS_QCAP = MAX_KAPPA + 1;
constexpr int AS_TILE = 128;  // samples per tile of the tensor-core assignment

template <int VEC>
__device__ __forceinline__ float cand_d2(const float *__restrict__ xs, const float *__restrict__ c, int d);

template <>
__device__ __forceinline__ float cand_d2<4>(const float *__restrict__ xs, const float *__restrict__ c, int d)
{
    const float4 *x4 = reinterpret_cast<const float4 *>(xs);
    const float4 *c4 = reinterpret_cast<const float4 *>(c);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const int nv = d >> 2;
#pragma unroll 4
    for (int t = 0; t < nv; t++) {
        float4 xv = x4[t];
        float4 cv = __ldg(c4 + t);
        float e0 = xv.x - cv.x, e1 = xv.y - cv.y, e2 = xv.z - cv.z, e3 = xv.w - cv.w;
        a0 = fmaf(e0, e0, a0);
        a1 = fmaf(e1, e1, a1);
        a2 = fmaf(e2, e2, a2);
        a3 = fmaf(e3, e3, a3);
    }
    return (a0 + a1) + (a2 + a3);
}

template <>
__device__ __forceinline__ float cand_d2<1>(const float *__restrict__ xs, const float *__restrict__ c, int d)
{
    float a0 = 0.f, a1 = 0.f;
    int t = 0;
    for (; t + 1 < d; t += 2) {
        float e0 = xs[t] - __ldg(c + t), e1 = xs[t + 1] - __ldg(c + t + 1);
        a0 = fmaf(e0, e0, a0);
        a1 = fmaf(e1, e1, a1);
    }
    if (t < d) {
        float e0 = xs[t] - __ldg(c + t);
        a0 = fmaf(e0, e0, a0);
    }
    return a0 + a1;
}

template <int VEC, typename XT>
__global__ void __launch_bounds__(AS_WARPS * 32) k_assign(const XT *__restrict__ X, int64_t n, int d, int64_t ld,
                                                          const int32_t *__restrict__ G, int kappa,
                                                          const float *__restrict__ C, int k,
                                                          const int32_t *__restrict__ Lin,
                                                          int32_t *__restrict__ Lout, float *__restrict__ best_out,
                                                          DevStatus *st)
{
    extern __shared__ __align__(16) float smem[];
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int dpad = (d + 3) & ~3;
    float *xs = smem + w * dpad;
    int *qlist = reinterpret_cast<int *>(smem + AS_WARPS * dpad) + w * AS_QCAP;

    const int ncand = kappa + 1;
    for (int64_t i = (int64_t)blockIdx.x * AS_WARPS + w; i < n; i += (int64_t)gridDim.x * AS_WARPS) {
        // stage x_i
        const XT *xi = X + i * ld;
        if (VEC == 4) {
            for (int t = lane; t < (d >> 2); t += 32)
                reinterpret_cast<float4 *>(xs)[t] = ldx4<XT>(xi + 4 * t);
        } else {
            for (int t = lane; t < d; t += 32)
                xs[t] = ldx(xi + t);
        }
        // candidate labels: slot 0 is the own label, slot 1 + j the label of neighbour j
        const int own = Lin[i];
        int u = 0;
        for (int c0 = 0; c0 < ncand; c0 += 32) {
            int c = c0 + lane;
            int lab = -1;
            if (c == 0) {
                lab = own;
            } else if (c < ncand) {
                int nb = G[i * kappa + (c - 1)];
                if ((unsigned)nb < (unsigned)n)
                    lab = Lin[nb];
                else
                    flag_error(st, GK_ERR_INVALID, (unsigned)i);
            }
            if (c < ncand && (unsigned)lab >= (unsigned)k) {
                flag_error(st, GK_ERR_INVALID, (unsigned)i);
                lab = -1;
            }
            unsigned peers = __match_any_sync(FULL_MASK, lab);
            bool keep = lab >= 0 && (peers & lanemask_lt()) == 0u;
            if (keep)
                for (int q = 0; q < u; q++)
                    if (qlist[q] == lab) {
                        keep = false;
                        break;
                    }
            unsigned keeps = __ballot_sync(FULL_MASK, keep);
            __syncwarp();
            if (keep)
                qlist[u + __popc(keeps & lanemask_lt())] = lab;
            u += __popc(keeps);
            __syncwarp();
        }
        // distances to the kept centroids, lane-parallel over candidates
        float bd = __int_as_float(0x7f800000);
        int br = 0x7fffffff;
        for (int q = lane; q < u; q += 32) {
            int r = qlist[q];
            float dv = cand_d2<VEC>(xs, C + (int64_t)r * d, d);
            if (key_less(dv, r, bd, br)) {
                bd = dv;
                br = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float od = __shfl_xor_sync(FULL_MASK, bd, o);
            int orr = __shfl_xor_sync(FULL_MASK, br, o);
            if (key_less(od, orr, bd, br)) {
                bd = od;
                br = orr;
            }
        }
        if (lane == 0) {
            if (br == 0x7fffffff)  // no valid candidate (own label out of range): keep the input label
                br = own, bd = 0.f;
            Lout[i] = br;
            if (best_out)
                best_out[i] = bd;
        }
        __syncwarp();
    }
}

// Coalesced variant for 16-byte rows (d % 4 == 0, d <= 32 * 4 * NV): the warp
// keeps x_i in registers (lane l owns vectors l, l + 32, ...).  Repeated
// candidate labels are dropped with __match_any_sync inside each batch of 32
// and, across batches, with a per-warp open-addressing set in shared memory
// (one atomicCAS per new label).  Distances are taken AS_G candidates at a
// time (AS_G / 2 for rows over 512 floats): each lane loads one 16-byte vector
// of every centroid of the group, and transpose_reduce completes the group's
// sums together.  The candidate list is padded to a multiple of the group with
// its first entry, whose second evaluation
// cannot change the (distance, label) minimum.
constexpr int AS_G = 8;
constexpr int AS_HASH = 256;                                  // slots of the per-warp label set
constexpr int AS_QROW = (AS_QCAP + AS_G + 3) / 4 * 4;         // candidate list row, padding included
static_assert(AS_HASH > AS_QCAP, "the label set must never fill up");

template <int NV, typename XT, int GS>
__global__ void __launch_bounds__(AS_WARPS * 32, NV <= 2 ? AS_ROWS_PER_SM : 4) k_assign_rows(const XT *__restrict__ X, int64_t n, int d,
                                                               int64_t ld, const int32_t *__restrict__ G, int kappa,
                                                               const float *__restrict__ C, int k,
                                                               const int32_t *__restrict__ Lin,
                                                               int32_t *__restrict__ Lout,
                                                               float *__restrict__ best_out, DevStatus *st)
{
    __shared__ __align__(16) int s_q[AS_WARPS][AS_QROW];
    __shared__ __align__(16) int s_h[AS_WARPS][AS_HASH];
    const int w = threadIdx.x >> 5, lane = lane_id();
    int *qlist = s_q[w];
    int *tab = s_h[w];
    static_assert(GS == 4 || GS == 8, "candidates per group: 4 or 8");
    const int d4 = d >> 2;
    const float4 *C4 = reinterpret_cast<const float4 *>(C);
    const int ncand = kappa + 1;

    for (int64_t i = (int64_t)blockIdx.x * AS_WARPS + w; i < n; i += (int64_t)gridDim.x * AS_WARPS) {
        const XT *xrow = X + i * ld;
        float4 xv[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            int col = lane + 32 * v;
            xv[v] = col < d4 ? ldx4<XT, true>(xrow + 4 * col) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = lane * 4; q < AS_HASH; q += 128)
            *reinterpret_cast<int4 *>(tab + q) = make_int4(-1, -1, -1, -1);
        __syncwarp();
        // candidate labels: slot 0 is the own label, slot 1 + j the label of neighbour j
        const int own = Lin[i];
        int u = 0;
        for (int c0 = 0; c0 < ncand; c0 += 32) {
            int c = c0 + lane;
            int lab = -1;
            if (c == 0) {
                lab = own;
            } else if (c < ncand) {
                int nb = __ldcs(G + i * kappa + (c - 1));
                if ((unsigned)nb < (unsigned)n)
                    lab = Lin[nb];
                else
                    flag_error(st, GK_ERR_INVALID, (unsigned)i);
            }
            if (c < ncand && (unsigned)lab >= (unsigned)k) {
                flag_error(st, GK_ERR_INVALID, (unsigned)i);
                lab = -1;
            }
            const unsigned peers = __match_any_sync(FULL_MASK, lab);
            bool fresh = false;
            if (lab >= 0 && (peers & lanemask_lt()) == 0u) {
                unsigned h = ((unsigned)lab * 0x9E3779B1u) >> 24;  // 8-bit multiplicative hash
                for (int probe = 0; probe < AS_HASH; probe++) {    // the set is never full: ends early
                    const int old = atomicCAS(tab + h, -1, lab);
                    if (old == -1) {
                        fresh = true;
                        break;
                    }
                    if (old == lab)
                        break;
                    h = (h + 1) & (AS_HASH - 1);
                }
            }
            const unsigned fr = __ballot_sync(FULL_MASK, fresh);
            if (fresh)
                qlist[u + __popc(fr & lanemask_lt())] = lab;
            u += __popc(fr);
        }
        __syncwarp();
        if (u > 0 && lane < GS)
            qlist[u + lane] = qlist[0];
        __syncwarp();

        float bd = __int_as_float(0x7f800000);
        int br = 0x7fffffff;
        for (int g0 = 0; g0 < u; g0 += GS) {
            int lab[GS];
#pragma unroll
            for (int c = 0; c < GS; c += 4) {
                const int4 q4 = *reinterpret_cast<const int4 *>(qlist + g0 + c);
                lab[c] = q4.x;
                lab[c + 1] = q4.y;
                lab[c + 2] = q4.z;
                lab[c + 3] = q4.w;
            }
            float part[GS];
#pragma unroll
            for (int c = 0; c < GS; c++) {
                const float4 *row = C4 + (int64_t)lab[c] * d4;
                part[c] = lane_partial<NV>(xv, d4, [&](int col) { return __ldg(row + col); });
            }
            const float tot = transpose_reduce<GS>(part);
            const int r = qlist[g0 + lane / (32 / GS)];
            if (key_less(tot, r, bd, br)) {
                bd = tot;
                br = r;
            }
        }
        // lanes that share bits 4 .. log2(32 / GS) hold the same candidates
#pragma unroll
        for (int o = 16; o >= 32 / GS; o >>= 1) {
            float od = __shfl_xor_sync(FULL_MASK, bd, o);
            int orr = __shfl_xor_sync(FULL_MASK, br, o);
            if (key_less(od, orr, bd, br)) {
                bd = od;
                br = orr;
            }
        }
        if (lane == 0) {
            if (br == 0x7fffffff)  // no valid candidate (own label out of range): keep the input label
                br = own, bd = 0.f;
            Lout[i] = br;
            if (best_out)
                best_out[i] = bd;
        }
        __syncwarp();
    }
}

// k_assign_rows with the candidate distances screened against a shadow copy of
// the centroids: BF16 rows (FMT 0, half the bytes per candidate row) or int8
// rows with a per-row scale (FMT 1, a quarter).  Pass 1 takes every
// candidate's distance D~ to the shadow row as k_assign_rows does (same lane
// layout, same candidate groups, shadow values widened exactly); with delta_r >=
// ||C_r - Cb_r||, |D - D~| <= delta_r (2 sqrt(D~) + delta_r) for the exact
// distances D, D~, and adding the FP32 rounding of both sums gives a bound E_r.
// Pass 2 recomputes, one at a time and against C, every candidate whose lower
// value D~ - E_r does not exceed the smallest upper value D~ + E_r (usually the
// winner alone), with the lane partials and summation tree of k_assign_rows,
// so the winner and its distance are that kernel's bit for bit.  The samples
// (FP32 or BF16, widened exactly) enter both passes unrounded: the bound covers
// the centroids' rounding alone.
// Shadow formats of the screening: FMT 0 BF16 rows (4 values per 8 bytes), FMT 1 int8 rows with a per-row
// scale s_r (4 values per 4 bytes; see lane_partial_q8), half the bytes again; FMT 2 the same int8 rows stored
// lane-major (d a multiple of 128), so that a lane's share of a row is one vector load.
template <int NV, typename XT, int GS, int FMT>
__global__ void __launch_bounds__(AS_WARPS * 32, NV <= 2 ? AS_ROWS_PER_SM : (NV == 4 ? 4 : 3)) k_assign_rows_scr(
    const XT *__restrict__ X, int64_t n, int d, int64_t ld, const int32_t *__restrict__ G, int kappa,
    const float *__restrict__ C, const void *__restrict__ Cs, const float *__restrict__ delta,
    const float *__restrict__ scale, int k, const int32_t *__restrict__ Lin, int32_t *__restrict__ Lout,
    float *__restrict__ best_out, DevStatus *st)
{
    __shared__ __align__(16) int s_q[AS_WARPS][AS_QROW];
    __shared__ __align__(16) int s_h[AS_WARPS][AS_HASH];
    __shared__ float s_lo[AS_WARPS][AS_QROW];
    const int w = threadIdx.x >> 5, lane = lane_id();
    int *qlist = s_q[w];
    int *tab = s_h[w];
    float *lov = s_lo[w];
    static_assert(GS == 4 || GS == 8, "candidates per group: 4 or 8");
    const int d4 = d >> 2;
    const float4 *C4 = reinterpret_cast<const float4 *>(C);
    const uint2 *Cb4 = static_cast<const uint2 *>(Cs);       // FMT 0: 4 BF16 per 8 bytes
    const uint32_t *Cq4 = static_cast<const uint32_t *>(Cs);  // FMT 1: 4 int8 per 4 bytes
    const float gam = (float)(d + 8) * 5.9604645e-8f;         // FP32 rounding of a d-term sum, relative
    const int ncand = kappa + 1;

    for (int64_t i = (int64_t)blockIdx.x * AS_WARPS + w; i < n; i += (int64_t)gridDim.x * AS_WARPS) {
        const XT *xrow = X + i * ld;
        float4 xv[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            int col = lane + 32 * v;
            xv[v] = col < d4 ? ldx4<XT, true>(xrow + 4 * col) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = lane * 4; q < AS_HASH; q += 128)
            *reinterpret_cast<int4 *>(tab + q) = make_int4(-1, -1, -1, -1);
        __syncwarp();
        const int own = Lin[i];
        int u = 0;
        for (int c0 = 0; c0 < ncand; c0 += 32) {
            int c = c0 + lane;
            int lab = -1;
            if (c == 0) {
                lab = own;
            } else if (c < ncand) {
                int nb = __ldcs(G + i * kappa + (c - 1));
                if ((unsigned)nb < (unsigned)n)
                    lab = Lin[nb];
                else
                    flag_error(st, GK_ERR_INVALID, (unsigned)i);
            }
            if (c < ncand && (unsigned)lab >= (unsigned)k) {
                flag_error(st, GK_ERR_INVALID, (unsigned)i);
                lab = -1;
            }
            const unsigned peers = __match_any_sync(FULL_MASK, lab);
            bool fresh = false;
            if (lab >= 0 && (peers & lanemask_lt()) == 0u) {
                unsigned h = ((unsigned)lab * 0x9E3779B1u) >> 24;
                for (int probe = 0; probe < AS_HASH; probe++) {
                    const int old = atomicCAS(tab + h, -1, lab);
                    if (old == -1) {
                        fresh = true;
                        break;
                    }
                    if (old == lab)
                        break;
                    h = (h + 1) & (AS_HASH - 1);
                }
            }
            const unsigned fr = __ballot_sync(FULL_MASK, fresh);
            if (fresh)
                qlist[u + __popc(fr & lanemask_lt())] = lab;
            u += __popc(fr);
        }
        __syncwarp();
        if (u > 0 && lane < GS)
            qlist[u + lane] = qlist[0];
        __syncwarp();

        // pass 1: BF16 distances with their bounds
        float best_up = __int_as_float(0x7f800000);
        for (int g0 = 0; g0 < u; g0 += GS) {
            int lab[GS];
#pragma unroll
            for (int c = 0; c < GS; c += 4) {
                const int4 q4 = *reinterpret_cast<const int4 *>(qlist + g0 + c);
                lab[c] = q4.x;
                lab[c + 1] = q4.y;
                lab[c + 2] = q4.z;
                lab[c + 3] = q4.w;
            }
            float part[GS];
#pragma unroll
            for (int c = 0; c < GS; c++) {
                if constexpr (FMT == 0) {
                    const uint2 *row = Cb4 + (int64_t)lab[c] * d4;
                    part[c] = lane_partial<NV>(xv, d4, [&](int col) { return bf16x4_to_float4(__ldg(row + col)); });
                } else if constexpr (FMT == 1) {
                    const uint32_t *row = Cq4 + (int64_t)lab[c] * d4;
                    part[c] = lane_partial_q8<NV>(xv, d4, -__ldg(scale + lab[c]),
                                                  [&](int col) { return __ldg(row + col); });
                } else {  // FMT 2: lane-major int8 rows, d = 128 NV
                    uint32_t wq[NV];
                    load_q8w<NV>(Cq4 + (int64_t)lab[c] * d4, wq);
                    part[c] = lane_partial_q8w<NV>(xv, -__ldg(scale + lab[c]), wq);
                }
            }
            const float dt = transpose_reduce<GS>(part);
            const int cl = lane / (32 / GS);
            const float dl = __ldg(delta + qlist[g0 + cl]);
            const float sq = sqrtf(fmaxf(dt, 0.f));
            const float e = 1.01f * (dl * (2.f * sq + dl) + gam * (2.f * dt + dl * (2.f * sq + dl)));
            if (lane % (32 / GS) == 0)
                lov[g0 + cl] = dt - e;
            best_up = fminf(best_up, dt + e);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            best_up = fminf(best_up, __shfl_xor_sync(FULL_MASK, best_up, o));
        __syncwarp();
        // pass 2: exact FP32 distances of the candidates that may be the minimum
        float bd = __int_as_float(0x7f800000);
        int br = 0x7fffffff;
        for (int g0 = 0; g0 < u; g0 += 32) {
            const int cnt = min(32, u - g0);
            unsigned sel = __ballot_sync(FULL_MASK, lane < cnt && lov[g0 + lane] <= best_up);
            while (sel) {
                const int c = __ffs(sel) - 1;
                sel &= sel - 1;
                const int r = qlist[g0 + c];
                const float4 *row = C4 + (int64_t)r * d4;
                const float tot = warp_total(lane_partial<NV>(xv, d4, [&](int col) { return __ldg(row + col); }));
                if (key_less(tot, r, bd, br)) {
                    bd = tot;
                    br = r;
                }
            }
        }
        if (lane == 0) {
            if (br == 0x7fffffff)  // no valid candidate (own label out of range): keep the input label
                br = own, bd = 0.f;
            Lout[i] = br;
            if (best_out)
                best_out[i] = bd;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// BF16 shadow of the centroids: Cb = bf16(C) and delta_r >= ||C_r - Cb_r||.
// ---------------------------------------------------------------------------
__global__ void k_shadow_bf16(const float *__restrict__ C, int k, int d, __nv_bfloat16 *__restrict__ Cb,
                              float *__restrict__ delta, float *__restrict__ cnorm)
{
    const int lane = lane_id();
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < k; r += gridDim.x * (blockDim.x >> 5)) {
        double e = 0.0, c2 = 0.0;
        for (int t = lane; t < d; t += 32) {
            const float c = C[(int64_t)r * d + t];
            const __nv_bfloat16 b = __float2bfloat16_rn(c);
            Cb[(int64_t)r * d + t] = b;
            const double diff = (double)c - (double)__bfloat162float(b);
            e += diff * diff;
            c2 += (double)c * (double)c;
        }
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(FULL_MASK, e, o);
            c2 += __shfl_xor_sync(FULL_MASK, c2, o);
        }
        if (lane == 0) {
            delta[r] = (float)(sqrt(e) * (1.0 + 1e-6)) + 1e-30f;  // rounded up
            cnorm[r] = (float)c2;                                 // ||C_r||^2 (a bound input only)
        }
    }
}

// Int8 shadow of the centroids: per row r the scale s_r = max_t |C_rt| / 127 (1 for a zero row), codes
// q_rt = rint(C_rt / s_r) (the quotient taken as a product with 1 / s_r) clamped to [-127, 127] and stored as
// q + 128, four per 32-bit word in the order of the row's values, and delta_r >= ||C_r - q_r s_r||, in FP32
// only.  Each error v - q s is formed as (v - p) - e with p = fl(q s) and e = fma(q, s, -p) (q s = p + e
// exactly); v - p is exact where p/2 <= v <= 2p (Sterbenz; |q| >= 1 puts v within half a step of q s), so the
// computed error is within 2u |v - q s| + 1.01 u^2 max|C_r| of the true one (u = 2^-24).  The errors are squared
// in units of w = max(s, FLT_MIN) (so that no square of a row of tiny values falls below the normal range) and
// summed in FP32 (d fma steps and the warp's 5 additions: relative error below gamma_(d+5), one more u for the
// division by w); delta_r inflates the square root by (d + 24) 1.2e-7 and 1e-5 (the 1 / (1 - 2u) above and this
// evaluation's own roundings) and adds sqrt(d) 4e-15 max|C_r| (the absolute term, which also covers squares
// below the normal range): a rigorous upper bound, no FP64.
__global__ void k_shadow_i8(const float *__restrict__ C, int k, int d, bool lane_major, uint32_t *__restrict__ Cq,
                            float *__restrict__ delta, float *__restrict__ scale)
{
    const int lane = lane_id();
    const int d4 = d >> 2;
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < k; r += gridDim.x * (blockDim.x >> 5)) {
        const float4 *row = reinterpret_cast<const float4 *>(C + (int64_t)r * d);
        float mx = 0.f;
        for (int col = lane; col < d4; col += 32) {
            const float4 v = row[col];
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        for (int o = 16; o > 0; o >>= 1)
            mx = fmaxf(mx, __shfl_xor_sync(FULL_MASK, mx, o));
        const float sc = mx > 0.f ? mx / 127.f : 1.f;
        const float inv = 1.f / sc;
        const float wu = fmaxf(sc, 1.17549435e-38f), winv = 1.f / wu;  // error unit (FLT_MIN at least)
        float e = 0.f;
        for (int col = lane; col < d4; col += 32) {
            const float4 v = row[col];
            const float vals[4] = {v.x, v.y, v.z, v.w};
            uint32_t word = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float qf = fminf(127.f, fmaxf(-127.f, rintf(vals[q] * inv)));
                word |= (uint32_t)((int)qf + 128) << (8 * q);
                const float p = qf * sc;
                const float pe = fmaf(qf, sc, -p);  // q s = p + pe exactly
                const float z = ((vals[q] - p) - pe) * winv;
                e = fmaf(z, z, e);
            }
            // row-major: word col; lane-major (d4 = 32 nv): the word of vector col = l + 32 v goes to l nv + v
            const int nv = d4 >> 5;
            Cq[(int64_t)r * d4 + (lane_major ? (col & 31) * nv + (col >> 5) : col)] = word;
        }
        for (int o = 16; o > 0; o >>= 1)
            e += __shfl_xor_sync(FULL_MASK, e, o);
        if (lane == 0) {
            delta[r] = sqrtf(e * (1.f + (float)(d + 24) * 1.2e-7f)) * 1.00001f * wu + sqrtf((float)d) * 4e-15f * mx +
                       1e-30f;
            scale[r] = sc;
        }
    }
}

// k_assign_rows with the candidate distances first taken against the BF16
// shadow Cb (half the bytes per candidate row).  With delta_r >= ||C_r - Cb_r||,
// |D - D~| <= delta_r (2 sqrt(D~) + delta_r) for the exact distances D, D~ to
// C_r and Cb_r; adding the FP32 rounding of both sums gives a bound E_r, and
// every candidate whose lower value D~ - E_r does not exceed the smallest upper
// value D~ + E_r is recomputed against C with the FP32 kernel's order (same
// lane partials, same reduction tree), so the winner and its distance are the
// FP32 kernel's bit for bit.
template <int NV, bool TILES>
__global__ void __launch_bounds__(AS_WARPS * 32) k_assign_rows_bf(const float *__restrict__ X, int64_t n, int d,
                                                                  int64_t ld, const int32_t *__restrict__ G,
                                                                  int kappa, const float *__restrict__ C,
                                                                  const __nv_bfloat16 *__restrict__ Cb,
                                                                  const float *__restrict__ delta, int k,
                                                                  const int32_t *__restrict__ Lin,
                                                                  int32_t *__restrict__ Lout,
                                                                  float *__restrict__ best_out,
                                                                  const int32_t *__restrict__ tmem_members, const int32_t *__restrict__ tile_flag,
                                                               const int32_t *__restrict__ sel_lab,
                                                               const int32_t *__restrict__ sel_n, DevStatus *st)
{
    __shared__ int s_q[AS_WARPS][AS_QCAP];
    __shared__ float s_lo[AS_WARPS][AS_QCAP + 31];
    const int w = threadIdx.x >> 5, lane = lane_id();
    int *qlist = s_q[w];
    const int d4 = d >> 2;
    const float4 *C4 = reinterpret_cast<const float4 *>(C);
    const uint2 *Cb4 = reinterpret_cast<const uint2 *>(Cb);  // 4 BF16 per 8 bytes
    const float gam = (float)(d + 8) * 5.9604645e-8f;         // FP32 rounding of a d-term sum, relative

    const int ncand = kappa + 1;
    for (int64_t p = (int64_t)blockIdx.x * AS_WARPS + w; p < n; p += (int64_t)gridDim.x * AS_WARPS) {
        int64_t i = p;
        int nl = -1;  // >= 0: the tensor-core screening left nl candidates for the exact pass
        if (TILES) {
            i = tmem_members[p];
            if (!tile_flag[p / AS_TILE])
                nl = sel_n[i];
        }
        const float4 *x4 = reinterpret_cast<const float4 *>(X + i * ld);
        float4 xv[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            int col = lane + 32 * v;
            xv[v] = col < d4 ? __ldcs(x4 + col) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int own = Lin[i];
        float bd = __int_as_float(0x7f800000);
        int br = 0x7fffffff;
        if (nl >= 0) {
            // exact FP32 distances of the screened labels (same lane partials and reduction grouping)
            const int mine = lane < nl ? __ldg(sel_lab + i * 8 + lane) : 0;
#pragma unroll 4
            for (int z = 0; z < nl; z++) {
                const int r = __shfl_sync(FULL_MASK, mine, z);
                const float4 *row = C4 + (int64_t)r * d4;
                const float tot = warp_total(lane_partial<NV>(xv, d4, [&](int col) { return __ldg(row + col); }));
                if (key_less(tot, r, bd, br)) {
                    bd = tot;
                    br = r;
                }
            }
        } else {
            int u = 0;
            for (int c0 = 0; c0 < ncand; c0 += 32) {
                int c = c0 + lane;
                int lab = -1;
                if (c == 0) {
                    lab = own;
                } else if (c < ncand) {
                    int nb = __ldcs(G + i * kappa + (c - 1));
                    if ((unsigned)nb < (unsigned)n)
                        lab = Lin[nb];
                    else
                        flag_error(st, GK_ERR_INVALID, (unsigned)i);
                }
                if (c < ncand && (unsigned)lab >= (unsigned)k) {
                    flag_error(st, GK_ERR_INVALID, (unsigned)i);
                    lab = -1;
                }
                unsigned peers = __match_any_sync(FULL_MASK, lab);
                bool keep = lab >= 0 && (peers & lanemask_lt()) == 0u;
                if (keep)
                    for (int q = 0; q < u; q++)
                        if (qlist[q] == lab) {
                            keep = false;
                            break;
                        }
                unsigned keeps = __ballot_sync(FULL_MASK, keep);
                __syncwarp();
                if (keep)
                    qlist[u + __popc(keeps & lanemask_lt())] = lab;
                u += __popc(keeps);
                __syncwarp();
            }
            // pass 1: BF16 distances of every candidate (lane l holds candidate g0 + l of each group)
            float *lov = s_lo[w];
            float best_up = __int_as_float(0x7f800000);
    #pragma unroll 1
            for (int g0 = 0; g0 < u; g0 += 32) {
                const int cnt = min(32, u - g0);
                float part[32];
    #pragma unroll
                for (int c = 0; c < 32; c++) {
                    float acc = 0.f;
                    if (c < cnt) {
                        const uint2 *row = Cb4 + (int64_t)qlist[g0 + c] * d4;
                        acc = lane_partial<NV>(xv, d4, [&](int col) { return bf16x4_to_float4(__ldg(row + col)); });
                    }
                    part[c] = acc;
                }
                const float dt = transpose_reduce32(part);
                if (lane < cnt) {
                    const float dl = delta[qlist[g0 + lane]];
                    const float sq = sqrtf(fmaxf(dt, 0.f));
                    const float e = 1.01f * (dl * (2.f * sq + dl) + gam * (2.f * dt + dl * (2.f * sq + dl)));
                    lov[g0 + lane] = dt - e;
                    best_up = fminf(best_up, dt + e);
                }
            }
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                best_up = fminf(best_up, __shfl_xor_sync(FULL_MASK, best_up, o));
            __syncwarp();
            // pass 2: FP32 distances of the candidates that may be the minimum, one at a
            // time; the xor butterfly groups the lane partials as transpose_reduce32 does,
            // so each total has the bits of the FP32 kernel
    #pragma unroll 1
            for (int g0 = 0; g0 < u; g0 += 32) {
                const int cnt = min(32, u - g0);
                unsigned sel = __ballot_sync(FULL_MASK, lane < cnt && lov[g0 + lane] <= best_up);
                while (sel) {
                    const int c = __ffs(sel) - 1;
                    sel &= sel - 1;
                    const int r = qlist[g0 + c];
                    const float4 *row = C4 + (int64_t)r * d4;
                    float tot = lane_partial<NV>(xv, d4, [&](int col) { return __ldg(row + col); });
    #pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
                        tot += __shfl_xor_sync(FULL_MASK, tot, o);
                    if (key_less(tot, r, bd, br)) {
                        bd = tot;
                        br = r;
                    }
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float od = __shfl_xor_sync(FULL_MASK, bd, o);
            int orr = __shfl_xor_sync(FULL_MASK, br, o);
            if (key_less(od, orr, bd, br)) {
                bd = od;
                br = orr;
            }
        }
        if (lane == 0) {
            if (br == 0x7fffffff)  // no valid candidate (own label out of range): keep the input label
                br = own, bd = 0.f;
            Lout[i] = br;
            if (best_out)
                best_out[i] = bd;
        }
        __syncwarp();
    }
}

// Per-block FP64 sums of best[] and counts of changed labels over fixed index
// ranges (the same for every kernel that produced best[]), so the total has
// the same bits whichever assignment kernel ran.
__global__ void __launch_bounds__(256) k_assign_reduce(const float *__restrict__ best,
                                                       const int32_t *__restrict__ Lin,
                                                       const int32_t *__restrict__ Lout, int64_t n,
                                                       double *__restrict__ blk_sum,
                                                       unsigned long long *__restrict__ blk_changed)
{
    __shared__ double s[256];
    __shared__ unsigned long long c[256];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    double a = 0.0;
    unsigned long long ch = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) {
        a += (double)best[i];
        ch += Lin[i] != Lout[i] ? 1ull : 0ull;
    }
    s[threadIdx.x] = a;
    c[threadIdx.x] = ch;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s[threadIdx.x] += s[threadIdx.x + o];
            c[threadIdx.x] += c[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        blk_sum[blockIdx.x] = s[0];
        blk_changed[blockIdx.x] = c[0];
    }
}

__global__ void __launch_bounds__(1024) k_assign_finish(const double *__restrict__ blk_sum,
                                                        const unsigned long long *__restrict__ blk_changed, int nb,
                                                        double *__restrict__ sum_d2, int64_t *__restrict__ n_changed)
{
    __shared__ double s[1024];
    __shared__ unsigned long long c[1024];
    double a = 0.0;
    unsigned long long b = 0;
    for (int i = threadIdx.x; i < nb; i += 1024) {
        a += blk_sum[i];
        b += blk_changed[i];
    }
    s[threadIdx.x] = a;
    c[threadIdx.x] = b;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s[threadIdx.x] += s[threadIdx.x + w];
            c[threadIdx.x] += c[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (sum_d2)
            *sum_d2 = s[0];
        if (n_changed)
            *n_changed = (int64_t)c[0];
    }
}

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

size_t assign_scratch_bytes(int64_t n, int32_t k, int64_t d)
{
    const size_t part = al256((size_t)AS_BLOCKS * (sizeof(double) + sizeof(unsigned long long)));
    const size_t shadow = al256((size_t)k * (size_t)d * 2) + 2 * al256((size_t)k * 4);
    const size_t best = al256((size_t)n * 4);
    const size_t tiles = al256((size_t)((n + AS_TILE - 1) / AS_TILE) * 4);
    const size_t sel = al256((size_t)n * 8 * 4) + al256((size_t)n * 4);
    return part + shadow + best + tiles + sel;
}

template <typename XT>
static cudaError_t assign_t(const XT *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                            const float *C, int32_t k, const int32_t *labels_in, int32_t *labels_out, float *best_d2,
                            double *sum_d2, int64_t *n_changed, void *scratch, DevStatus *st, cudaStream_t s,
                            int precision, const int32_t *members)
{
    char *sp = static_cast<char *>(scratch);
    double *blk_sum = reinterpret_cast<double *>(sp);
    unsigned long long *blk_chg = reinterpret_cast<unsigned long long *>(blk_sum + AS_BLOCKS);
    sp += al256((size_t)AS_BLOCKS * (sizeof(double) + sizeof(unsigned long long)));
    __nv_bfloat16 *Cb = reinterpret_cast<__nv_bfloat16 *>(sp);
    sp += al256((size_t)k * (size_t)d * 2);
    float *delta = reinterpret_cast<float *>(sp);
    sp += al256((size_t)k * 4);
    float *cnorm = reinterpret_cast<float *>(sp);
    sp += al256((size_t)k * 4);
    float *best = best_d2 ? best_d2 : reinterpret_cast<float *>(sp);
    sp += al256((size_t)n * 4);
    int32_t *tile_flag = reinterpret_cast<int32_t *>(sp);
    sp += al256((size_t)((n + AS_TILE - 1) / AS_TILE) * 4);
    int32_t *sel_lab = reinterpret_cast<int32_t *>(sp);
    sp += al256((size_t)n * 8 * 4);
    int32_t *sel_n = reinterpret_cast<int32_t *>(sp);

    const bool vec4 = x_vec4(X, d, ld) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
    const int d4 = (int)(d / 4);
    // candidates per group of the row kernels (a tile shape: every width gives the same bits, transpose_reduce
    // forms each total with warp_total's tree): 8 by default, 4 for rows of more than 512 values, where 8 would
    // not keep the loads in registers; a caller (the autotuner) may ask for 4 or 8
    const int gw = (precision >> 8) & 0xff;
    precision &= 0xff;
    cudaError_t e;
    int grid = 0;
    bool done = false;
    if ((precision == 2 || precision == 4) && vec4 && d4 <= 32 * 8) {
        // the shadow: BF16 (2) or int8 with a per-row scale (4); the int8 codes take the BF16 shadow's space
        const int sgrid = (k + 7) / 8 < 152 * 16 ? (k + 7) / 8 : 152 * 16;
        // int8 rows lane-major where every lane owns whole vectors (d a multiple of 128): one load per lane and row
        const bool lane_major = precision == 4 && d % 128 == 0;
        if (precision == 2)
            k_shadow_bf16<<<sgrid, 256, 0, s>>>(C, k, (int)d, Cb, delta, cnorm);
        else
            k_shadow_i8<<<sgrid, 256, 0, s>>>(C, k, (int)d, lane_major, reinterpret_cast<uint32_t *>(Cb), delta,
                                              cnorm);
#define GK_ASB8F(NV, GS, F)                                                                                      \
    do {                                                                                                         \
        if ((e = resident_grid(reinterpret_cast<const void *>(k_assign_rows_scr<NV, XT, GS, F>), AS_WARPS * 32,  \
                               0, &grid)) != cudaSuccess)                                                        \
            return e;                                                                                            \
        k_assign_rows_scr<NV, XT, GS, F><<<grid, AS_WARPS * 32, 0, s>>>(X, n, (int)d, ld, g_idx, kappa, C, Cb,   \
                                                                        delta, cnorm, k, labels_in, labels_out,  \
                                                                        best, st);                               \
    } while (0)
#define GK_ASB8G(NV, GS)                                                                                         \
    do {                                                                                                         \
        if (precision == 2)                                                                                      \
            GK_ASB8F(NV, GS, 0);                                                                                 \
        else if (lane_major && d4 == 32 * NV)                                                                    \
            GK_ASB8F(NV, GS, 2);                                                                                 \
        else                                                                                                     \
            GK_ASB8F(NV, GS, 1);                                                                                 \
    } while (0)
#define GK_ASB8(NV)                                                                                              \
    do {                                                                                                         \
        if (NV >= 8 || gw == 4)                                                                                  \
            GK_ASB8G(NV, 4);                                                                                     \
        else                                                                                                     \
            GK_ASB8G(NV, 8);                                                                                     \
    } while (0)
        if (d4 <= 32)
            GK_ASB8(1);
        else if (d4 <= 64)
            GK_ASB8(2);
        else if (d4 <= 128)
            GK_ASB8(4);
        else
            GK_ASB8(8);
#undef GK_ASB8
#undef GK_ASB8G
#undef GK_ASB8F
        done = true;
    }
    if constexpr (std::is_same_v<XT, float>) {  // tensor-core screening: FP32 samples only
        if (precision == 3 && vec4 && d4 <= 32 * 8) {
            k_shadow_bf16<<<(k + 7) / 8 < 152 * 16 ? (k + 7) / 8 : 152 * 16, 256, 0, s>>>(C, k, (int)d, Cb, delta,
                                                                                      cnorm);
            const bool tiles = members && assign_tc_supported(d, ld, X, C, kappa);
            if (tiles) {
                if ((e = launch_assign_tc(X, n, d, ld, g_idx, kappa, C, Cb, delta, cnorm, k, labels_in, members,
                                          sel_lab, sel_n, tile_flag, st, s)) != cudaSuccess)
                    return e;
            }
#define GK_ASGB(NV, T)                                                                                           \
    k_assign_rows_bf<NV, T><<<AS_BLOCKS, AS_WARPS * 32, 0, s>>>(X, n, (int)d, ld, g_idx, kappa, C, Cb, delta, k,   \
                                                                labels_in, labels_out, best,                        \
                                                                members, tile_flag, sel_lab, sel_n, st)
            if (tiles) {
                GK_ASGB(1, true);  // d <= 128 on the tensor-core path
            } else if (d4 <= 32) {
                GK_ASGB(1, false);
            } else if (d4 <= 64) {
                GK_ASGB(2, false);
            } else if (d4 <= 128) {
                GK_ASGB(4, false);
            } else {
                GK_ASGB(8, false);
            }
#undef GK_ASGB
            done = true;
        }
    }
    if (done) {
    } else if (vec4 && d4 <= 32 * 8) {
#define GK_ASGG(NV, GS)                                                                                          \
    do {                                                                                                         \
        if ((e = resident_grid(reinterpret_cast<const void *>(k_assign_rows<NV, XT, GS>), AS_WARPS * 32, 0,      \
                               &grid)) != cudaSuccess)                                                           \
            return e;                                                                                            \
        k_assign_rows<NV, XT, GS><<<grid, AS_WARPS * 32, 0, s>>>(X, n, (int)d, ld, g_idx, kappa, C, k, labels_in,  \
                                                                 labels_out, best, st);                          \
    } while (0)
#define GK_ASG(NV)                                                                                               \
    do {                                                                                                         \
        if (NV >= 8 || gw == 4)                                                                                  \
            GK_ASGG(NV, 4);                                                                                      \
        else                                                                                                     \
            GK_ASGG(NV, 8);                                                                                      \
    } while (0)
        if (d4 <= 32)
            GK_ASG(1);
        else if (d4 <= 64)
            GK_ASG(2);
        else if (d4 <= 128)
            GK_ASG(4);
        else
            GK_ASG(8);
#undef GK_ASG
#undef GK_ASGG
    } else {
        int dpad = (int)((d + 3) & ~3);
        size_t shm = sizeof(float) * (size_t)AS_WARPS * dpad + sizeof(int) * AS_WARPS * AS_QCAP;
        const int shm_max = (int)(sizeof(float) * (size_t)AS_WARPS * MAX_D + sizeof(int) * AS_WARPS * AS_QCAP);
        if (vec4) {
            if ((e = set_max_smem(reinterpret_cast<const void *>(k_assign<4, XT>), shm_max)) !=
                cudaSuccess)
                return e;
            k_assign<4, XT><<<AS_BLOCKS, AS_WARPS * 32, shm, s>>>(X, n, (int)d, ld, g_idx, kappa, C, k, labels_in,
                                                                labels_out, best, st);
        } else {
            if ((e = set_max_smem(reinterpret_cast<const void *>(k_assign<1, XT>), shm_max)) !=
                cudaSuccess)
                return e;
            k_assign<1, XT><<<AS_BLOCKS, AS_WARPS * 32, shm, s>>>(X, n, (int)d, ld, g_idx, kappa, C, k, labels_in,
                                                                labels_out, best, st);
        }
    }
    if (sum_d2 || n_changed) {
        k_assign_reduce<<<AS_BLOCKS, 256, 0, s>>>(best, labels_in, labels_out, n, blk_sum, blk_chg);
        k_assign_finish<<<1, 1024, 0, s>>>(blk_sum, blk_chg, AS_BLOCKS, sum_d2, n_changed);
    }
    return cudaGetLastError();
}

cudaError_t launch_assign(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                          int32_t kappa, const float *C, int32_t k, const int32_t *labels_in, int32_t *labels_out,
                          float *best_d2, double *sum_d2, int64_t *n_changed, void *scratch, DevStatus *st,
                          cudaStream_t s, int precision, const int32_t *members)
{
    if (bf16)
        return assign_t(static_cast<const __nv_bfloat16 *>(X), n, d, ld, g_idx, kappa, C, k, labels_in, labels_out,
                        best_d2, sum_d2, n_changed, scratch, st, s, precision, members);
    return assign_t(static_cast<const float *>(X), n, d, ld, g_idx, kappa, C, k, labels_in, labels_out, best_d2,
                    sum_d2, n_changed, scratch, st, s, precision, members);
}

}  // namespace gkm
