// Graph refinement inside clusters (Alg. 3) with the pair distances of a run
// taken from a Gram matrix computed on the tensor cores (tcgen05, BF16 inputs,
// FP32 accumulation in tensor memory), and the same results as the FP32 path.
//
// One CTA (8 warps) per run of <= 128 members.  The run's rows, centred on the
// run's first member, are converted to BF16 and staged in shared memory in the
// 128-byte swizzle layout (two 64-column K-blocks at a time); one thread issues
// the 128 x N x 16 MMAs of G = X' X'^T into tensor memory and commits them to
// an mbarrier.  Warps w and w + 4 then read TMEM lanes 32 (w % 4) .. + 31 (one
// row of G per thread, half of the columns each) and form
// d2(i, j) = n_i + n_j - 2 G_ij with n_i = ||x_i'||^2.
//
// Exactness: when every centred coordinate of the run is an integer of
// magnitude <= 255 and 2 d 255^2 < 2^24, every BF16 value, product and partial
// sum is an exact integer below 2^24, so d2 equals the FP32 sum of squared
// differences bit for bit (no rerank).  Otherwise a candidate is kept only if
// its Gram distance minus a rigorous error bound E_ij beats the row's kappa-th
// key, and its distance is then recomputed exactly in FP32 in the order of
// pair_d2_seq; the bound covers the BF16 rounding of both operands
// ((4u + 2u^2) ||x_i'|| ||x_j'||, u = 2^-8), FP32 accumulation and the final
// combination, so no pair that would enter the row is dropped.
// The merge into the graph rows is the one of the FP32 path (merge.cuh).
#include "common.cuh"
#include "merge.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace gkm {

constexpr int TC_M = 128;              // rows of the MMA tile (TMEM lanes)
constexpr int TC_KB = 64;              // BF16 elements per K-block (one 128-byte swizzle row)
constexpr int TC_KCH = 2;              // K-blocks staged per chunk
constexpr int TC_KB_BYTES = TC_M * 128;  // 16 KB per K-block
constexpr uint32_t TC_WAIT_ITERS = 1u << 22;

// TN: widest run handled (64 or 128).  The 64-wide instance uses 4 warps, a
// 64-column TMEM accumulator and a 64 x 65 distance tile, so more CTAs fit on
// an SM; the 128-wide one 8 warps and 128 columns.
template <int TN>
struct TcCfg {
    static constexpr int THREADS = TN == 64 ? 128 : 256;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int DS = TN + 1;  // stride of the distance tile (floats)
    // the staging area (K-blocks) and the distance tile share one region
    static constexpr size_t region = (size_t)TC_KCH * TC_KB_BYTES > sizeof(float) * TN * DS
                                         ? (size_t)TC_KCH * TC_KB_BYTES
                                         : sizeof(float) * TN * DS;
    static constexpr size_t fixed = region + sizeof(float) * TC_M /*norms*/ + sizeof(int) * TC_M /*ids*/ +
                                    64 /*barrier, tmem slot, flags*/;
    __host__ __device__ static size_t warp_bytes(int kappa)
    {
        return (sizeof(int) + sizeof(float)) * (size_t)(2 * kappa + TN) + 4 * sizeof(unsigned);
    }
    __host__ __device__ static size_t bytes(int kappa)
    {
        return 1024 /*alignment slack*/ + fixed + WARPS * warp_bytes(kappa);
    }
};

template <int TN>
__global__ void __launch_bounds__(TcCfg<TN>::THREADS) k_refine_tc(const float *__restrict__ X, int64_t n, int d,
                                                                  int64_t ld,
                                                          const int32_t *__restrict__ off,
                                                          const int32_t *__restrict__ mem,
                                                          const int32_t *__restrict__ run_off, int k, int kappa,
                                                          int cap, bool vec4, int32_t *__restrict__ g_idx,
                                                          float *__restrict__ g_dist, DevStatus *st)
{
    using CF = TcCfg<TN>;
    constexpr int TC_THREADS = CF::THREADS, TC_WARPS = CF::WARPS, TC_DS = CF::DS;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *stage = base;                                   // K-blocks, 1024-aligned
    float *dt = reinterpret_cast<float *>(base);                   // distance tile (after the MMAs)
    float *nrm = reinterpret_cast<float *>(base + CF::region);
    int *rid = reinterpret_cast<int *>(nrm + TC_M);
    uint64_t *bar = reinterpret_cast<uint64_t *>(rid + TC_M);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *flags = reinterpret_cast<int *>(tslot + 1);              // [0] not exact, [1] timeout
    unsigned char *wb = base + CF::fixed;

    const int tid = threadIdx.x, w = tid >> 5, lane = lane_id();
    unsigned char *wbase = wb + w * CF::warp_bytes(kappa);
    int *li = reinterpret_cast<int *>(wbase);
    float *lv = reinterpret_cast<float *>(li + kappa);
    int *ni = reinterpret_cast<int *>(lv + kappa);
    float *nv = reinterpret_cast<float *>(ni + kappa);
    int *bi = reinterpret_cast<int *>(nv + kappa);
    float *bv = reinterpret_cast<float *>(bi + TN);
    unsigned *dup = reinterpret_cast<unsigned *>(bv + TN);

    // this block's run (as in the FP32 kernel)
    const int run = blockIdx.x;
    if (run >= run_off[k])
        return;
    int lo = 0, hi = k;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (run_off[mid] <= run)
            lo = mid;
        else
            hi = mid;
    }
    const int r = lo;
    const int beg = off[r], m = off[r + 1] - beg;
    const int nc = (m + cap - 1) / cap, rbase = m / nc, rem = m % nc;
    const int c = run - run_off[r];
    const int s0 = c * rbase + min(c, rem), sz = rbase + (c < rem ? 1 : 0);
    // the 64-wide instance takes runs of <= 64 members, the 128-wide one runs of 65..128;
    // longer runs (max_cluster > 128) are handled by the FP32 kernel
    if (sz < 2 || sz > TN || (TN == 128 && sz <= 64))
        return;
    const int32_t *S = mem + beg + s0;
    const int N = (sz + 15) & ~15;

    if (w == 0) {
        tc::tmem_alloc(tslot, TN);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
        flags[0] = 0;
        flags[1] = 0;
    }
    for (int q = tid; q < TC_M; q += TC_THREADS) {
        int a = q < sz ? S[q] : -1;
        if (a >= n) {
            flag_error(st, GK_ERR_INVALID, (unsigned)r);
            a = -1;
        }
        rid[q] = a;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const int ref = rid[0] >= 0 ? rid[0] : 0;
    const float *xref = X + (int64_t)ref * ld;

    // ---- Gram matrix of the centred run, K-chunk by K-chunk ----
    bool inexact = false;
    uint32_t phase = 0;
    const uint32_t idesc = tc::idesc_bf16_f32(TC_M, N);
    const int kchunk = TC_KCH * TC_KB;
    for (int k0 = 0; k0 < d; k0 += kchunk) {
        // stage rows: warp w handles rows w, w + 8, ...; lane l covers 4 consecutive coordinates
#pragma unroll 4
        for (int row = w; row < TN; row += TC_WARPS) {
            const int a = rid[row];
            float part = 0.f;
            for (int kk = lane * 4; kk < kchunk; kk += 128) {
                const int t = k0 + kk;
                float v[4] = {0.f, 0.f, 0.f, 0.f};
                if (a >= 0) {
                    if (vec4 && t + 3 < d) {
                        const float4 xa = __ldg(reinterpret_cast<const float4 *>(X + (int64_t)a * ld + t));
                        const float4 xr = __ldg(reinterpret_cast<const float4 *>(xref + t));
                        v[0] = xa.x - xr.x;
                        v[1] = xa.y - xr.y;
                        v[2] = xa.z - xr.z;
                        v[3] = xa.w - xr.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; e++)
                            if (t + e < d)
                                v[e] = __ldg(X + (int64_t)a * ld + t + e) - __ldg(xref + t + e);
                    }
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        part = fmaf(v[e], v[e], part);
                        inexact |= !(v[e] == rintf(v[e]) && fabsf(v[e]) <= 255.f);
                    }
                }
                const int kb = kk / TC_KB, kin = kk % TC_KB;
                __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]);
                __nv_bfloat162 p1 = __floats2bfloat162_rn(v[2], v[3]);
                uint2 pk;
                pk.x = *reinterpret_cast<uint32_t *>(&p0);
                pk.y = *reinterpret_cast<uint32_t *>(&p1);
                *reinterpret_cast<uint2 *>(stage + kb * TC_KB_BYTES + tc::swz128_offset(row, kin)) = pk;
            }
            for (int o = 16; o > 0; o >>= 1)
                part += __shfl_xor_sync(FULL_MASK, part, o);
            if (lane == 0)
                nrm[row] = (k0 == 0 ? 0.f : nrm[row]) + part;
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const int nkb = min(TC_KCH, (d - k0 + TC_KB - 1) / TC_KB);
            for (int kb = 0; kb < nkb; kb++) {
                const uint32_t a_addr = tc::smem_addr(stage + kb * TC_KB_BYTES);
#pragma unroll
                for (int s = 0; s < TC_KB / 16; s++) {
                    const uint64_t desc = tc::desc_k128(a_addr + 32 * s);
                    tc::mma_bf16(taddr, desc, desc, idesc, (k0 > 0) || (kb > 0) || (s > 0));
                }
            }
            tc::mma_commit(bar);
        }
        __syncwarp();
        if (!tc::mbar_wait_bounded(bar, phase, TC_WAIT_ITERS)) {
            if (lane == 0)
                atomicOr(&flags[1], 1);
        }
        phase ^= 1u;
        tc::fence_after_sync();
        __syncthreads();  // the staging area may be rewritten only after every warp saw the MMAs complete
    }
    if (inexact)
        atomicOr(&flags[0], 1);
    __syncthreads();
    const bool timed_out = flags[1] != 0;
    if (timed_out && tid == 0)
        flag_error(st, GK_ERR_TIMEOUT, (unsigned)run);
    // integer run with |x| <= 255: exact only while 2 d 255^2 < 2^24
    const bool exact = flags[0] == 0 && 2.0 * d * 255.0 * 255.0 < 16777216.0;

    // ---- distances from the Gram matrix into the tile ----
    if (!timed_out && 32 * (w & 3) < TN) {
        const int quad = w & 3, half = w >> 2;
        const int i = 32 * quad + lane;
        const float ni_ = nrm[i];
        for (int c0 = 64 * half; c0 < min(N, 64 * half + 64); c0 += 32) {
            float g[32];
            tc::tmem_ld32(taddr + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0, g);
            tc::tmem_ld_wait();
            if (i < sz) {
#pragma unroll
                for (int q = 0; q < 32; q++) {
                    const int j = c0 + q;
                    if (j < sz)
                        dt[i * TC_DS + j] = (ni_ + nrm[j]) - 2.f * g[q];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();

    // ---- merge (with an exact FP32 rerank of the pairs inside the error bound) ----
    if (!timed_out) {
        const float u = 1.0f / 256.0f;
        const float c1 = 1.02f * (4.f * u + 2.f * u * u + 4.f * (d + 2) * 5.9604645e-8f);
        const float c2 = 1.02f * (d + 8) * 1.1920929e-7f;
        RowRegs cur, nxt;
        if (w < sz && rid[w] >= 0)
            load_row(cur, g_idx + (int64_t)rid[w] * kappa, g_dist + (int64_t)rid[w] * kappa, kappa);
        for (int row = w; row < sz; row += TC_WARPS) {
            const int i = rid[row];
            const int rn = row + TC_WARPS;
            if (rn < sz && rid[rn] >= 0)  // next row's list in flight during this merge
                load_row(nxt, g_idx + (int64_t)rid[rn] * kappa, g_dist + (int64_t)rid[rn] * kappa, kappa);
            if (i < 0) {
                cur = nxt;
                continue;
            }
            float *drow = dt + row * TC_DS;
            if (!exact) {
                const int uq = (kappa - 1) >> 5;
                const float src = uq == 0 ? cur.dv[0] : uq == 1 ? cur.dv[1] : uq == 2 ? cur.dv[2] : cur.dv[3];
                const float th = __shfl_sync(FULL_MASK, src, (kappa - 1) & 31);
                const float nr_i = nrm[row];
                const float *xi = X + (int64_t)i * ld;
                for (int cc = lane; cc < sz; cc += 32) {
                    const float approx = drow[cc];
                    const float e = c1 * sqrtf(nr_i * nrm[cc]) + c2 * (nr_i + nrm[cc]);
                    const int j = rid[cc];
                    float exact_d = __int_as_float(0x7f800000);
                    if (j >= 0 && j != i && approx - e <= th)
                        exact_d = vec4 ? pair_d2_seq4(xi, X + (int64_t)j * ld, d)
                                       : pair_d2_seq(xi, X + (int64_t)j * ld, d);
                    drow[cc] = exact_d;
                }
                __syncwarp();
            }
            merge_row(i, rid, drow, sz, kappa, cur, g_idx + (int64_t)i * kappa, g_dist + (int64_t)i * kappa, li,
                      lv, bi, bv, ni, nv, dup);
            cur = nxt;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0)
        tc::tmem_dealloc(taddr, TN);
}

cudaError_t launch_refine_tc(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                             const int32_t *members, const int32_t *run_off, int32_t k, int32_t kappa,
                             int32_t max_cluster, int64_t grid, int32_t *g_idx, float *g_dist, DevStatus *st,
                             cudaStream_t s)
{
    const size_t shm64 = TcCfg<64>::bytes(kappa), shm128 = TcCfg<128>::bytes(kappa);
    cudaError_t e = cudaFuncSetAttribute(k_refine_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm64);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_refine_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm128)) !=
        cudaSuccess)
        return e;
    const bool vec4 = (d % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    k_refine_tc<64><<<(unsigned)grid, TcCfg<64>::THREADS, shm64, s>>>(X, n, (int)d, ld, offsets, members, run_off, k,
                                                                      kappa, max_cluster, vec4, g_idx, g_dist, st);
    k_refine_tc<128><<<(unsigned)grid, TcCfg<128>::THREADS, shm128, s>>>(X, n, (int)d, ld, offsets, members, run_off,
                                                                         k, kappa, max_cluster, vec4, g_idx, g_dist,
                                                                         st);
    return cudaGetLastError();
}

}  // namespace gkm
