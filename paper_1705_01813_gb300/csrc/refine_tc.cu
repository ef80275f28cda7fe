// Graph refinement inside clusters (Alg. 3) with the pair distances of a run
// taken from a Gram matrix on the tensor cores (tcgen05, BF16 inputs, FP32
// accumulation in tensor memory), and the same graph as the FP32 path.
//
// Four kernels per refinement:
//
// k_refine_perm, one CTA per run of <= 128 members: the cluster-sorted copy.
// Row p of Xp is the sample at position p of the grouping (members[p]) in
// BF16: FP32 samples centred on their run's first member, BF16 samples as
// they are; rows padded with zeros to a multiple of 8 columns.  It also writes
// each row's FP32 squared norm (of the unrounded centred values) and per run
// two flags: a centred value that is not an integer of magnitude <= 255, and
// a value that BF16 rounded.
//
// k_refine_gram, one CTA (4 warps) per run: one thread loads the run's 128-row
// tile of Xp with the TMA engine (cp.async.bulk.tensor, 64-column boxes in the
// 128-byte swizzle layout the MMA descriptors expect; rows of the next runs
// and past the end come along and are ignored) and issues the 128 x N x 16
// MMAs of G = X' X'^T into tensor memory.  Thread t then owns TMEM lane t,
// i.e. row t of G, forms d2(t, j) = n_t + n_j - 2 G_tj (n = the squared
// norms) and appends to its graph row's candidate list every j that may enter
// the row: key (d2, id_j) below the row's kappa-th key.
// Exactness: when every staged coordinate of the run is an integer of
// magnitude <= 255 and 2 d 255^2 < 2^24, every BF16 value, product and partial
// sum is an exact integer below 2^24, so d2 equals the FP32 sum of squared
// differences bit for bit.  Otherwise a pair is kept when d2 - E_tj is not
// above the kappa-th distance, E_tj being a rigorous bound on the error of the
// Gram distance (BF16 rounding of both operands, (4u + 2u^2) |x_t'| |x_j'|
// with u = 2^-8, a term that vanishes when every staged coordinate is a BF16
// value already, as for BF16 samples; plus FP32 accumulation and combination),
// marked (recorded by its column in the run instead of its id), and the run is
// flagged.
//
// k_refine_exact, one CTA per flagged run: the run's FP32 rows are staged in
// shared memory once and every marked pair is recomputed exactly in the order
// of pair_d2_seq, in place.
//
// k_refine_merge, one warp per graph row that received candidates: the
// candidates are merged into the row as in the FP32 path (merge.cuh).  Rows
// that received nothing are not touched.
#include "assign_common.cuh"
#include "common.cuh"
#include "merge.cuh"
#include "tc.cuh"
#include "tmap.cuh"

#include <cuda_bf16.h>

#include <mutex>
#include <type_traits>

namespace gkm {

constexpr int TC_M = 128;                // rows of the MMA tile (TMEM lanes) and widest run
constexpr int TC_KB = 64;                // BF16 elements per K-block (one 128-byte swizzle row, one TMA box)
constexpr int TC_KCH = 2;                // K-blocks of the widest row (d <= 128)
constexpr int TC_KB_BYTES = TC_M * 128;  // 16 KB per K-block
constexpr int TC_THREADS = 128;          // one thread per TMEM lane
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_CAP = 128;              // candidate slots per graph row
constexpr uint32_t TC_WAIT_ITERS = 1u << 22;
constexpr unsigned TC_RERANK = 0x80000000u;  // candidate id flag: distance needs the exact recompute

constexpr size_t TC_STAGE = (size_t)TC_KCH * TC_KB_BYTES;
constexpr size_t TC_BUF = (size_t)2 * TC_M * 32 * sizeof(int);  // ids and distances of one 32-column chunk
static_assert(TC_BUF <= TC_STAGE, "the epilogue's candidate buffers reuse the staging area");
constexpr size_t TC_SMEM = 1024 /*alignment slack*/ + TC_STAGE + sizeof(float) * TC_M + sizeof(int) * TC_M * 3 + 64;

// Columns of a row of the cluster-sorted copy: d rounded up to 8 (16-byte rows for the tensor map).
static int64_t perm_cols(int64_t d) { return (d + 7) & ~int64_t(7); }

// Slot of entry m (< 32) of row r in the candidate buffers: rows of 32 words
// with the entry index xor-ed by r % 32, so the 32 rows of a warp writing
// their m-th entries, and a warp reading one row, touch 32 distinct banks.
__device__ __forceinline__ int buf_slot(int r, int m) { return r * 32 + (m ^ (r & 31)); }

// The run of block `run`: its cluster r, first member position p0 (in members / Xp) and size sz.
__device__ __forceinline__ void run_range(int run, const int32_t *__restrict__ off, const int32_t *__restrict__ run_off,
                                          const int32_t *__restrict__ run_cl, int cap, int *p0, int *sz, int *r)
{
    *r = run_cl[run];
    const int beg = off[*r], m = off[*r + 1] - beg;
    const int nc = (m + cap - 1) / cap, rbase = m / nc, rem = m % nc;
    const int c = run - run_off[*r];
    *p0 = beg + c * rbase + min(c, rem);
    *sz = rbase + (c < rem ? 1 : 0);
}

template <typename XT>
__global__ void __launch_bounds__(TC_THREADS) k_refine_perm(const XT *__restrict__ X, int64_t n, int d, int64_t ld,
                                                            const int32_t *__restrict__ off,
                                                            const int32_t *__restrict__ mem,
                                                            const int32_t *__restrict__ run_off,
                                                            const int32_t *__restrict__ run_cl, int k, int cap,
                                                            int dp, __nv_bfloat16 *__restrict__ Xp,
                                                            float *__restrict__ pnrm, int32_t *__restrict__ run_flags,
                                                            DevStatus *st)
{
    const int run = blockIdx.x;
    if (run >= run_off[k])
        return;
    int p0, sz, r;
    run_range(run, off, run_off, run_cl, cap, &p0, &sz, &r);
    if (sz < 2 || sz > TC_M)  // no pairs, or a run of the FP32 kernel
        return;
    const int tid = threadIdx.x, w = tid >> 5, lane = lane_id();
    // BF16 samples are copied as they are: their values, products and the Gram's accumulation carry no BF16
    // rounding (centring would round the differences)
    constexpr bool CENTRE = !std::is_same_v<XT, __nv_bfloat16>;
    int ref = mem[p0];
    ref = (unsigned)ref < (unsigned)n ? ref : -1;
    const bool vec4 = (d % 4 == 0) && (ld % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(XT))) == 0;
    bool inexact = false, lossy = false;
    for (int q = w; q < sz; q += TC_WARPS) {
        const int p = p0 + q;
        int a = mem[p];
        if ((unsigned)a >= (unsigned)n) {
            if (lane == 0)
                flag_error(st, GK_ERR_INVALID, (unsigned)r);
            a = -1;
        }
        float part = 0.f;
        for (int t = lane * 4; t < dp; t += 128) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (a >= 0 && t < d) {
                const XT *xa = X + (int64_t)a * ld + t;
                const XT *xr = X + (int64_t)(ref >= 0 ? ref : a) * ld + t;
                if (vec4) {
                    const float4 xv = ldx4<XT>(xa);
                    v[0] = xv.x, v[1] = xv.y, v[2] = xv.z, v[3] = xv.w;
                    if (CENTRE && ref >= 0) {
                        const float4 rv = ldx4<XT>(xr);
                        v[0] -= rv.x, v[1] -= rv.y, v[2] -= rv.z, v[3] -= rv.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++)
                        if (t + e < d)
                            v[e] = ldx(xa + e) - (CENTRE && ref >= 0 ? ldx(xr + e) : 0.f);
                }
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                part = fmaf(v[e], v[e], part);
                inexact |= !(v[e] == rintf(v[e]) && fabsf(v[e]) <= 255.f);
            }
            const __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0], v[1]), b1 = __floats2bfloat162_rn(v[2], v[3]);
            const float2 f0 = __bfloat1622float2(b0), f1 = __bfloat1622float2(b1);
            lossy |= f0.x != v[0] || f0.y != v[1] || f1.x != v[2] || f1.y != v[3];
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t *>(&b0);
            pk.y = *reinterpret_cast<const uint32_t *>(&b1);
            *reinterpret_cast<uint2 *>(Xp + (int64_t)p * dp + t) = pk;
        }
        part = warp_total(part);
        if (lane == 0)
            pnrm[p] = part;
    }
    const int any_inexact = __syncthreads_or(inexact ? 1 : 0), any_lossy = __syncthreads_or(lossy ? 1 : 0);
    if (tid == 0)
        run_flags[run] = (any_inexact ? 1 : 0) | (any_lossy ? 2 : 0);
}

__global__ void __launch_bounds__(TC_THREADS) k_refine_gram(const __grid_constant__ CUtensorMap tmap, int64_t n,
                                                            int d, const int32_t *__restrict__ off,
                                                            const int32_t *__restrict__ mem,
                                                            const int32_t *__restrict__ run_off,
                                                            const int32_t *__restrict__ run_cl, int k, int kappa,
                                                            int cap, const int32_t *__restrict__ g_idx,
                                                            const float *__restrict__ g_dist,
                                                            const float *__restrict__ pnrm,
                                                            const int32_t *__restrict__ run_flags,
                                                            int32_t *__restrict__ cand_id,
                                                            float *__restrict__ cand_d, int32_t *__restrict__ cand_n,
                                                            int32_t *__restrict__ run_tag, DevStatus *st)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *stage = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    float *nrm = reinterpret_cast<float *>(stage + TC_STAGE);
    int *rid = reinterpret_cast<int *>(nrm + TC_M);
    int *bcnt = rid + TC_M;   // candidates of each row in the current chunk
    int *btot = bcnt + TC_M;  // candidates of each row written so far
    uint64_t *bar = reinterpret_cast<uint64_t *>(btot + TC_M);  // [0] the tile's copies, [1] the MMAs
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, w = tid >> 5, lane = lane_id();

    const int run = blockIdx.x;
    if (run >= run_off[k])
        return;
    int p0, sz, r;
    run_range(run, off, run_off, run_cl, cap, &p0, &sz, &r);
    if (sz < 2 || sz > TC_M)  // longer runs (max_cluster > 128) go to the FP32 kernel
        return;
    const int N = (sz + 15) & ~15;
    const uint32_t ncols = sz <= 32 ? 32u : sz <= 64 ? 64u : 128u;
    const int nkb = (d + TC_KB - 1) / TC_KB;

    if (w == 0) {
        tc::tmem_alloc(tslot, ncols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
        // the run's rows p0 .. p0 + 127 of the cluster-sorted copy, one 64-column box per K-block
        tc::mbar_arrive_expect_tx(&bar[0], (uint32_t)(nkb * TC_KB_BYTES));
        for (int kb = 0; kb < nkb; kb++)
            tc::tma_load_2d(stage + kb * TC_KB_BYTES, &tmap, kb * TC_KB, p0, &bar[0]);
    }
    // this thread's graph row, its kappa-th key and its norm, while the tile is in flight
    int gi_row = tid < sz ? mem[p0 + tid] : -1;
    if (gi_row >= n) {
        flag_error(st, GK_ERR_INVALID, (unsigned)r);
        gi_row = -1;
    }
    rid[tid] = gi_row;
    nrm[tid] = tid < sz ? pnrm[p0 + tid] : 0.f;
    float thd = 0.f;
    int thi = 0;
    if (gi_row >= 0) {
        thd = __ldcg(g_dist + (int64_t)gi_row * kappa + kappa - 1);
        thi = __ldcg(g_idx + (int64_t)gi_row * kappa + kappa - 1);
    }
    const int rf = run_flags[run];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;

    // ---- the tile, then the Gram matrix of the (centred) run ----
    bool late = !tc::mbar_wait_bounded(&bar[0], 0, TC_WAIT_ITERS);
    if (__syncthreads_or(late ? 1 : 0)) {
        // the copies gave up: issue nothing, give them one more bounded wait, free the tensor memory
        if (tid == 0)
            flag_error(st, GK_ERR_TIMEOUT, (unsigned)run);
        tc::mbar_wait_bounded(&bar[0], 0, TC_WAIT_ITERS);
        tc::fence_before_sync();
        __syncthreads();
        if (w == 0)
            tc::tmem_dealloc(taddr, ncols);
        return;
    }
    if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t idesc = tc::idesc_bf16_f32(TC_M, N);
        for (int kb = 0; kb < nkb; kb++) {
            const uint32_t a_addr = tc::smem_addr(stage + kb * TC_KB_BYTES);
#pragma unroll
            for (int s = 0; s < TC_KB / 16; s++) {
                const uint64_t desc = tc::desc_k128(a_addr + 32 * s);
                tc::mma_bf16(taddr, desc, desc, idesc, (kb > 0) || (s > 0));
            }
        }
        tc::mma_commit(&bar[1]);
    }
    __syncwarp();
    late = !tc::mbar_wait_bounded(&bar[1], 0, TC_WAIT_ITERS);
    tc::fence_after_sync();
    if (__syncthreads_or(late ? 1 : 0)) {
        // the MMAs gave up: skip the epilogue, one more bounded wait before their tensor memory is freed
        if (tid == 0)
            flag_error(st, GK_ERR_TIMEOUT, (unsigned)run);
        tc::mbar_wait_bounded(&bar[1], 0, TC_WAIT_ITERS);
        tc::fence_before_sync();
        __syncthreads();
        if (w == 0)
            tc::tmem_dealloc(taddr, ncols);
        return;
    }
    // integer run with |x| <= 255: exact only while 2 d 255^2 < 2^24
    const bool exact = (rf & 1) == 0 && 2.0 * d * 255.0 * 255.0 < 16777216.0;
    if (tid == 0)
        run_tag[run] = exact ? 0 : 1;  // k_refine_exact recomputes the marked pairs of this run

    // ---- candidates of row tid (TMEM lane tid), 32 columns at a time ----
    // Each thread collects its row's candidates of the chunk in shared memory
    // (the staging area is free once the MMAs completed); then each warp writes
    // whole row segments to the global lists, so that the stores coalesce.
    int *bid = reinterpret_cast<int *>(stage);
    float *bdv = reinterpret_cast<float *>(bid + TC_M * 32);
    const bool rows_here = 32 * w < sz;  // warp-uniform
    const int row = tid;
    const float n_i = nrm[row];
    const float u = 1.0f / 256.0f;
    const float rnd = (rf & 2) != 0 ? 4.f * u + 2.f * u * u : 0.f;  // BF16 rounding of the operands
    // accumulation of G: exact products, each 16-deep step aligned to its largest term and truncated (an
    // error below 16 units of 2^-23 of the step's terms), over d / 16 steps, doubled by the factor 2 of
    // 2 G and once more as a margin
    const float c1 = 1.02f * (rnd + 8.f * (d + 2) * 5.9604645e-8f);
    const float c2 = 1.02f * (d + 8) * 1.1920929e-7f;
    btot[tid] = 0;
    for (int c0 = 0; c0 < N; c0 += 32) {
        int m = 0;
        if (rows_here) {
            float g[32];
            tc::tmem_ld32(taddr + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, g);
            tc::tmem_ld_wait();
            if (gi_row >= 0) {
#pragma unroll
                for (int q = 0; q < 32; q++) {
                    const int j = c0 + q;
                    if (j < sz && j != row) {
                        const int jid = rid[j];
                        const float d2 = (n_i + nrm[j]) - 2.f * g[q];
                        bool keep;
                        unsigned tag = 0;
                        if (exact) {
                            keep = key_less(d2, jid, thd, thi);
                        } else {
                            const float e = c1 * sqrtf(n_i * nrm[j]) + c2 * (n_i + nrm[j]);
                            keep = d2 - e <= thd;
                            tag = TC_RERANK;
                        }
                        if (keep && jid >= 0) {
                            // a marked pair records the run column of j (k_refine_exact writes the id back)
                            bid[buf_slot(row, m)] = tag ? (int)(TC_RERANK | (unsigned)j) : jid;
                            bdv[buf_slot(row, m)] = d2;
                            m++;
                        }
                    }
                }
            }
        }
        bcnt[tid] = m;
        __syncthreads();
        for (int r2 = w; r2 < sz; r2 += TC_WARPS) {
            const int mr = bcnt[r2], g2 = rid[r2];
            if (mr == 0 || g2 < 0)
                continue;
            const int base = btot[r2];
            if (lane < mr) {
                cand_id[(int64_t)g2 * TC_CAP + base + lane] = bid[buf_slot(r2, lane)];
                cand_d[(int64_t)g2 * TC_CAP + base + lane] = bdv[buf_slot(r2, lane)];
            }
            __syncwarp();
            if (lane == 0)
                btot[r2] = base + mr;
        }
        __syncthreads();
    }
    if (rows_here && gi_row >= 0)
        cand_n[gi_row] = btot[tid];
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0)
        tc::tmem_dealloc(taddr, ncols);
}

// Exact distances of the marked candidates of an inexact run: one CTA per run
// stages the run's rows in FP32 in shared memory (row stride d + 1 words) and
// the threads share out all (row, candidate) pairs of the run; each marked
// pair (t, column c) is recomputed by one thread in the order of pair_d2_seq
// and written back in place with the id of column c.  Runs the Gram kernel
// found exact return at once.
constexpr int EX_THREADS = TC_M;

template <typename XT>
__global__ void __launch_bounds__(EX_THREADS) k_refine_exact(const XT *__restrict__ X, int64_t n, int d,
                                                             int64_t ld, const int32_t *__restrict__ off,
                                                             const int32_t *__restrict__ mem,
                                                             const int32_t *__restrict__ run_off,
                                                             const int32_t *__restrict__ run_cl, int k, int cap,
                                                             const int32_t *__restrict__ run_tag,
                                                             int32_t *__restrict__ cand_id,
                                                             float *__restrict__ cand_d,
                                                             const int32_t *__restrict__ cand_n, DevStatus *st)
{
    extern __shared__ float xs[];  // [sz][d + 1], d <= 128
    __shared__ int rid[TC_M], pre[TC_M + 1], wsum[EX_THREADS / 32];
    const int run = blockIdx.x;
    if (run >= run_off[k] || run_tag[run] == 0)
        return;
    const int r = run_cl[run];
    const int beg = off[r], m = off[r + 1] - beg;
    const int nc = (m + cap - 1) / cap, rbase = m / nc, rem = m % nc;
    const int c = run - run_off[r];
    const int s0 = c * rbase + min(c, rem), sz = rbase + (c < rem ? 1 : 0);
    if (sz < 2 || sz > TC_M)
        return;
    const int tid = threadIdx.x, w = tid >> 5, lane = lane_id();
    const int ds = d + 1;
    int cnt = 0;
    if (tid < sz) {
        const int a = mem[beg + s0 + tid];
        rid[tid] = (a >= 0 && a < n) ? a : -1;
        cnt = rid[tid] >= 0 ? cand_n[rid[tid]] : 0;
    }
    // exclusive prefix of the rows' candidate counts
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o)
            incl += v;
    }
    if (lane == 31)
        wsum[w] = incl;
    __syncthreads();
    int base = 0;
    for (int q = 0; q < w; q++)
        base += wsum[q];
    pre[tid] = base + incl - cnt;
    if (tid == EX_THREADS - 1)
        pre[EX_THREADS] = base + incl;
#pragma unroll 4
    for (int row = w; row < sz; row += EX_THREADS / 32) {
        const int a = rid[row];
        for (int t = lane; t < d; t += 32)
            xs[row * ds + t] = a >= 0 ? ldx(X + (int64_t)a * ld + t) : 0.f;
    }
    __syncthreads();  // the staged rows and the prefix pre[] (pre[EX_THREADS]: the run's pair count)
    const int total = pre[EX_THREADS];
    for (int p = tid; p < total; p += EX_THREADS) {
        int lo = 0, hi = sz;  // the row of pair p: last row with pre[row] <= p
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pre[mid] <= p)
                lo = mid;
            else
                hi = mid;
        }
        const int row = lo, q = p - pre[row];
        const int64_t slot = (int64_t)rid[row] * TC_CAP + q;
        const unsigned raw = (unsigned)cand_id[slot];
        if (!(raw & TC_RERANK))
            continue;
        const int col = (int)(raw & ~TC_RERANK);
        if (col >= sz || rid[col] < 0) {
            flag_error(st, GK_ERR_INVALID, (unsigned)r);
            continue;
        }
        const float *xa = xs + row * ds, *xb = xs + col * ds;
        float acc = 0.f;
        for (int t = 0; t < d; t++) {
            const float e = xa[t] - xb[t];
            acc = fmaf(e, e, acc);
        }
        cand_d[slot] = acc;
        cand_id[slot] = rid[col];
    }
}

// One warp per graph row that received candidates (all exact by now): the
// merge of the FP32 path.  Candidate ids arrive in ascending order.
constexpr int MG_WARPS = 8;

// per warp: candidate keys (TC_CAP), row and merged-row keys (kappa each), candidate ids and distances, dup bits
__host__ __device__ inline size_t merge_warp_bytes(int kappa)
{
    return sizeof(uint64_t) * (size_t)(TC_CAP + 2 * kappa) + (sizeof(int) + sizeof(float)) * TC_CAP + 16;
}

__global__ void __launch_bounds__(MG_WARPS * 32) k_refine_merge(int64_t n, int kappa,
                                                                const int32_t *__restrict__ cand_id,
                                                                const float *__restrict__ cand_d,
                                                                const int32_t *__restrict__ cand_n,
                                                                int32_t *__restrict__ g_idx,
                                                                float *__restrict__ g_dist)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, lane = lane_id();
    unsigned char *wb = smem_raw + (size_t)w * merge_warp_bytes(kappa);
    uint64_t *bk = reinterpret_cast<uint64_t *>(wb);
    uint64_t *rk = bk + TC_CAP;
    uint64_t *nk = rk + kappa;
    int *cid = reinterpret_cast<int *>(nk + kappa);
    float *cdv = reinterpret_cast<float *>(cid + TC_CAP);
    unsigned *dup = reinterpret_cast<unsigned *>(cdv + TC_CAP);
    for (int64_t i = (int64_t)blockIdx.x * MG_WARPS + w; i < n; i += (int64_t)gridDim.x * MG_WARPS) {
        const int cnt = cand_n[i];
        if (cnt == 0)
            continue;
        RowRegs cur;
        load_row(cur, g_idx + i * kappa, g_dist + i * kappa, kappa);
        for (int q = lane; q < cnt; q += 32) {
            cid[q] = (int)((unsigned)__ldcg(cand_id + i * TC_CAP + q) & ~TC_RERANK);
            cdv[q] = __ldcg(cand_d + i * TC_CAP + q);
        }
        __syncwarp();
        merge_row((int)i, cid, cdv, cnt, kappa, cur, g_idx + i * kappa, g_dist + i * kappa, rk, bk, nk, dup);
        __syncwarp();
    }
}

// candidate ids and distances (n x TC_CAP each), counts (n), run flags (at most k + n / 2 + 1 runs)
static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// candidate ids and distances (n x TC_CAP each), counts (n), run tags and run flags (at most k + n / 2 + 1 runs
// each), and for 64 <= d <= 128 the cluster-sorted BF16 copy (n x perm_cols(d)) with its row norms (n)
size_t refine_tc_scratch_bytes(int64_t n, int32_t k, int64_t d)
{
    const size_t a = al256((size_t)n * TC_CAP * sizeof(int32_t));
    const size_t c = al256((size_t)n * sizeof(int32_t));
    const size_t t = al256((size_t)(k + n / 2 + 1) * sizeof(int32_t));
    const size_t perm = (d >= 64 && d <= 128) ? al256((size_t)n * (size_t)perm_cols(d) * 2) + al256((size_t)n * 4) : 0;
    return 2 * a + c + 2 * t + perm;
}

// cuTensorMapEncodeTiled, from the CUDA driver through the runtime (no link against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t encode_tiled(EncodeTiledFn *fn)
{
    static std::once_flag once;
    static void *ptr = nullptr;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q);
        if (err == cudaSuccess && (q != cudaDriverEntryPointSuccess || !ptr))
            err = cudaErrorNotSupported;
    });
    *fn = reinterpret_cast<EncodeTiledFn>(ptr);
    return err;
}

cudaError_t bf16_tensor_map(CUtensorMap *tm, const void *base, int64_t cols, int64_t rows, int64_t row_elems,
                            uint32_t box_cols, uint32_t box_rows)
{
    EncodeTiledFn fn = nullptr;
    cudaError_t e = encode_tiled(&fn);
    if (e != cudaSuccess)
        return e;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_elems * 2};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of the cluster-sorted copy: n rows of dp BF16 (row stride dp * 2 bytes, a multiple of 16), boxes of
// 64 columns x 128 rows in the 128-byte swizzle layout, rows past n read as zeros.
static cudaError_t perm_tensor_map(CUtensorMap *tm, const __nv_bfloat16 *Xp, int64_t n, int64_t dp)
{
    return bf16_tensor_map(tm, Xp, dp, n, dp, TC_KB, TC_M);
}

template <typename XT>
static cudaError_t refine_tc_t(const XT *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                               const int32_t *members, const int32_t *run_off, const int32_t *run_cl, int32_t k,
                               int32_t kappa, int32_t max_cluster, int64_t grid, int32_t *g_idx, float *g_dist,
                               void *scratch, DevStatus *st, cudaStream_t s)
{
    const size_t a = al256((size_t)n * TC_CAP * sizeof(int32_t));
    const size_t t = al256((size_t)(k + n / 2 + 1) * sizeof(int32_t));
    char *sp = static_cast<char *>(scratch);
    int32_t *cand_id = reinterpret_cast<int32_t *>(sp);
    float *cand_d = reinterpret_cast<float *>(sp + a);
    int32_t *cand_n = reinterpret_cast<int32_t *>(sp + 2 * a);
    int32_t *run_tag = reinterpret_cast<int32_t *>(sp + 2 * a + al256((size_t)n * 4));
    int32_t *run_flags = reinterpret_cast<int32_t *>(sp + 2 * a + al256((size_t)n * 4) + t);
    __nv_bfloat16 *Xp = reinterpret_cast<__nv_bfloat16 *>(sp + 2 * a + al256((size_t)n * 4) + 2 * t);
    const int64_t dp = perm_cols(d);
    float *pnrm = reinterpret_cast<float *>(reinterpret_cast<char *>(Xp) + al256((size_t)n * (size_t)dp * 2));
    CUtensorMap tmap;
    cudaError_t e = perm_tensor_map(&tmap, Xp, n, dp);
    if (e != cudaSuccess)
        return e;
    if ((e = set_max_smem(reinterpret_cast<const void *>(k_refine_gram), (int)TC_SMEM)) != cudaSuccess)
        return e;
    const size_t shm_exact = sizeof(float) * (size_t)TC_M * (size_t)(d + 1);  // d <= 128 on this path
    if ((e = set_max_smem(reinterpret_cast<const void *>(k_refine_exact<XT>),
                          (int)(sizeof(float) * TC_M * (128 + 1)))) != cudaSuccess)
        return e;
    const size_t shm_merge = MG_WARPS * merge_warp_bytes(kappa);
    if ((e = set_max_smem(reinterpret_cast<const void *>(k_refine_merge),
                          (int)(MG_WARPS * merge_warp_bytes(MAX_KAPPA)))) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(cand_n, 0, sizeof(int32_t) * (size_t)n, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(run_tag, 0, sizeof(int32_t) * (size_t)grid, s)) != cudaSuccess)
        return e;
    k_refine_perm<XT><<<(unsigned)grid, TC_THREADS, 0, s>>>(X, n, (int)d, ld, offsets, members, run_off, run_cl, k,
                                                            max_cluster, (int)dp, Xp, pnrm, run_flags, st);
    k_refine_gram<<<(unsigned)grid, TC_THREADS, TC_SMEM, s>>>(tmap, n, (int)d, offsets, members, run_off, run_cl, k,
                                                              kappa, max_cluster, g_idx, g_dist, pnrm, run_flags,
                                                              cand_id, cand_d, cand_n, run_tag, st);
    k_refine_exact<XT><<<(unsigned)grid, EX_THREADS, shm_exact, s>>>(X, n, (int)d, ld, offsets, members, run_off, run_cl,
                                                                 k, max_cluster, run_tag, cand_id, cand_d, cand_n,
                                                                 st);
    int64_t mblocks = (n + MG_WARPS - 1) / MG_WARPS;
    if (mblocks > 152 * 64)
        mblocks = 152 * 64;
    k_refine_merge<<<(unsigned)mblocks, MG_WARPS * 32, shm_merge, s>>>(n, kappa, cand_id, cand_d, cand_n, g_idx,
                                                                        g_dist);
    return cudaGetLastError();
}

cudaError_t launch_refine_tc(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                             const int32_t *members, const int32_t *run_off, const int32_t *run_cl, int32_t k,
                             int32_t kappa, int32_t max_cluster, int64_t grid, int32_t *g_idx, float *g_dist,
                             void *scratch, DevStatus *st, cudaStream_t s)
{
    if (bf16)
        return refine_tc_t(static_cast<const __nv_bfloat16 *>(X), n, d, ld, offsets, members, run_off, run_cl, k,
                           kappa, max_cluster, grid, g_idx, g_dist, scratch, st, s);
    return refine_tc_t(static_cast<const float *>(X), n, d, ld, offsets, members, run_off, run_cl, k, kappa,
                       max_cluster, grid, g_idx, g_dist, scratch, st, s);
}

}  // namespace gkm
