// Two-means tree (Alg. 1, Sec. 3.2): k clusters by repeated bisection of the
// largest cluster into two halves of equal size.
//
// Every bisection halves a cluster (half u takes ceil(m/2) members), so the
// sizes in the tree depend on n and k only: the clusters of depth L have
// floor(n / 2^L) or that plus one members, whole depths are split before the
// next depth starts (a child is never larger than a cluster left at its
// parent's depth, and the shallower cluster goes first among equal sizes), and
// when k is not a power of two the last depth splits its larger clusters
// first, leftmost first.  The kernels therefore run one depth at a time over
// all of its clusters at once.  A cluster is a range [off, off + m) of a
// permutation of the samples; the permutation keeps each cluster's members in
// ascending id, and cluster j of depth L has the range that the bits of j
// (most significant first, 0 = u) pick out from the root.
//
// One bisection (each step over every cluster of the depth):
//   seeds    the two members with the smallest (draw(seed ^ TREE, L * 2^32 + id), id)
//   iters x  Lloyd 2-means: a member joins u when d(x, c_u) <= d(x, c_v), then
//            each centre becomes the FP32 rounding of the FP64 mean of its half
//            (an empty half keeps its centre)
//   keys     (d(x, c_u) - d(x, c_v) in FP32, id) as one ordered 64-bit word
//   select   the ceil(m/2)-th smallest key of the cluster (radix select)
//   split    members with a key up to it form u, the rest v, each in the
//            order they had (a stable partition: ascending id again)
// Distances are FP32 with one accumulator over ascending coordinates and one
// fused multiply-add per step, the decisions' precision.  Clusters are
// numbered left to right at the end.
#include <algorithm>

#include "common.cuh"

namespace gkm {
namespace {

constexpr uint64_t TAG_TREE = 0x5452454500000000ull;  // "TREE"
constexpr int TR_THREADS = 128;                       // pass kernel: one member per thread at a time
constexpr int TR_STAGE = 64;                          // coordinates staged per round
constexpr int TR_PITCH = TR_STAGE + 1;                // padded row of the stage (conflict-free column reads)
constexpr int64_t TR_CHUNK = 512;                     // members per chunk block; larger clusters take several
constexpr int SEL_THREADS = 256;
static_assert(TR_THREADS == 2 * TR_STAGE, "the sums give each thread one coordinate of one half");

// Range of cluster j of depth L: the bits of j from the most significant, 0 = u (the left ceil(m/2)).
__device__ __forceinline__ void seg_geom(int64_t n, int L, int64_t j, int64_t &off, int64_t &m)
{
    off = 0;
    m = n;
    for (int b = L - 1; b >= 0; b--) {
        const int64_t h = (m + 1) >> 1;
        if ((j >> b) & 1) {
            off += h;
            m -= h;
        } else {
            m = h;
        }
    }
}

// Order-preserving map of an FP32 value to an unsigned word.
__device__ __forceinline__ uint32_t f32_order(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ bool hk_less(uint64_t ha, int ia, uint64_t hb, int ib)
{
    return ha < hb || (ha == hb && ia < ib);
}

// (h1, i1) <= (h2, i2) are the two smallest keys seen; merge another such pair (g1, j1) <= (g2, j2).
__device__ __forceinline__ void top2_merge(uint64_t &h1, int &i1, uint64_t &h2, int &i2, uint64_t g1, int j1,
                                           uint64_t g2, int j2)
{
    if (hk_less(g1, j1, h1, i1)) {  // the other pair's first wins; the second is the smaller of h1 and g2
        if (hk_less(h1, i1, g2, j2)) {
            h2 = h1;
            i2 = i1;
        } else {
            h2 = g2;
            i2 = j2;
        }
        h1 = g1;
        i1 = j1;
    } else if (hk_less(g1, j1, h2, i2)) {
        h2 = g1;
        i2 = j1;
    }
}

// Radix selection step, one full warp: over a 256-bin histogram, the digit whose cumulative count first exceeds
// rank and the number of keys below that digit (lane q reads bins 8q .. 8q + 7).  The caller guarantees that
// the bins hold more than rank keys.
__device__ __forceinline__ void warp_pick(const unsigned *hist, int64_t rank, int &digit, int64_t &below)
{
    const int lane = threadIdx.x & 31;
    unsigned own = 0;
    for (int q = 0; q < 8; q++)
        own += hist[8 * lane + q];
    unsigned incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o)
            incl += v;
    }
    const unsigned hit = __ballot_sync(FULL_MASK, (int64_t)incl > rank);
    const int first = hit ? __ffs(hit) - 1 : 31;
    int dg = 8 * lane + 7;
    int64_t base = 0;
    if (lane == first) {
        base = incl - own;
        for (int q = 0; q < 8; q++) {
            const unsigned h = hist[8 * lane + q];
            if (base + (int64_t)h > rank) {
                dg = 8 * lane + q;
                break;
            }
            base += h;
        }
    }
    digit = __shfl_sync(FULL_MASK, dg, first);
    below = __shfl_sync(FULL_MASK, base, first);
}

__global__ void k_tree_iota(int32_t *perm, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (int32_t)i;
}

// Last, partial depth L: which of its S = 2^L clusters split (r of them, the larger first, then the leftmost) and
// how many split before each.  One block.
__global__ void __launch_bounds__(1024) k_tree_plan(int64_t n, int L, int64_t r, int32_t *spl, int32_t *pre)
{
    __shared__ int wsum[32];
    const int64_t S = (int64_t)1 << L;
    const int64_t a = n >> L;
    const int64_t r1 = min(r, n - a * S);  // larger clusters (a + 1 members) split
    const int64_t r0 = r - r1;             // clusters of a members split
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < S; t0 += blockDim.x) {
        const int64_t j = t0 + threadIdx.x;
        bool big = false;
        if (j < S) {
            int64_t off, m;
            seg_geom(n, L, j, off, m);
            big = m == a + 1;
        }
        const unsigned bal = __ballot_sync(FULL_MASK, big);
        if (lane == 0)
            wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            before += w < warp ? wsum[w] : 0;
            total += wsum[w];
        }
        const int64_t rank1 = carry + before + __popc(bal & lanemask_lt());
        if (j < S) {
            const int64_t rank0 = j - rank1;
            spl[j] = big ? (rank1 < r1) : (rank0 < r0);
            pre[j] = (int32_t)(min(rank1, r1) + min(rank0, r0));
        }
        carry += total;
        __syncthreads();
    }
}

// Chunk c of cluster j: C chunks of nearly equal length over the cluster's range.
__device__ __forceinline__ void chunk_range(int64_t off, int64_t m, int64_t C, int64_t c, int64_t &b, int64_t &e)
{
    b = off + c * m / C;
    e = off + (c + 1) * m / C;
}

struct Top2 {
    uint64_t h1, h2;
    int32_t i1, i2;
};

// Seeds, first step: the two members of smallest (draw, id) in every chunk of a splitting cluster.
__global__ void __launch_bounds__(SEL_THREADS) k_tree_seed_part(int64_t n, int L, int64_t C,
                                                                 const int32_t *__restrict__ perm,
                                                                 const int32_t *__restrict__ spl, uint64_t seed,
                                                                 Top2 *__restrict__ part)
{
    __shared__ Top2 sw[SEL_THREADS / 32];
    const int64_t j = blockIdx.x / C, c = blockIdx.x % C;
    if (spl && !spl[j])
        return;
    int64_t off, m, b, e;
    seg_geom(n, L, j, off, m);
    chunk_range(off, m, C, c, b, e);
    const uint64_t key = seed ^ TAG_TREE;
    uint64_t h1 = ~0ull, h2 = ~0ull;
    int i1 = INT32_MAX, i2 = INT32_MAX;
    for (int64_t p = b + threadIdx.x; p < e; p += SEL_THREADS) {
        const int id = perm[p];
        top2_merge(h1, i1, h2, i2, sm64_draw(key, ((uint64_t)(uint32_t)L << 32) | (uint32_t)id), id, ~0ull,
                   INT32_MAX);
    }
    for (int o = 16; o > 0; o >>= 1)
        top2_merge(h1, i1, h2, i2, __shfl_xor_sync(FULL_MASK, h1, o), __shfl_xor_sync(FULL_MASK, i1, o),
                   __shfl_xor_sync(FULL_MASK, h2, o), __shfl_xor_sync(FULL_MASK, i2, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        sw[warp] = Top2{h1, h2, i1, i2};
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < SEL_THREADS / 32; w++)
            top2_merge(h1, i1, h2, i2, sw[w].h1, sw[w].i1, sw[w].h2, sw[w].i2);
        part[blockIdx.x] = Top2{h1, h2, i1, i2};
    }
}

// Seeds, second step: merge the chunks' pairs; the two winners' rows become the starting centres c_u, c_v
// (cen: 2 x d floats per cluster).
template <typename XT>
__global__ void __launch_bounds__(TR_THREADS) k_tree_seed_final(const XT *__restrict__ X, int64_t n, int d,
                                                                 int64_t ld, int64_t C,
                                                                 const int32_t *__restrict__ spl,
                                                                 const Top2 *__restrict__ part,
                                                                 float *__restrict__ cen, DevStatus *st)
{
    __shared__ int s_id[2];
    const int64_t j = blockIdx.x;
    if (spl && !spl[j])
        return;
    if (threadIdx.x < 32) {
        uint64_t h1 = ~0ull, h2 = ~0ull;
        int i1 = INT32_MAX, i2 = INT32_MAX;
        for (int64_t c = threadIdx.x; c < C; c += 32) {
            const Top2 t = part[j * C + c];
            top2_merge(h1, i1, h2, i2, t.h1, t.i1, t.h2, t.i2);
        }
        for (int o = 16; o > 0; o >>= 1)
            top2_merge(h1, i1, h2, i2, __shfl_xor_sync(FULL_MASK, h1, o), __shfl_xor_sync(FULL_MASK, i1, o),
                       __shfl_xor_sync(FULL_MASK, h2, o), __shfl_xor_sync(FULL_MASK, i2, o));
        if (threadIdx.x == 0) {
            if ((unsigned)i1 >= (unsigned)n || (unsigned)i2 >= (unsigned)n) {
                flag_error(st, GK_ERR_INVALID, (unsigned)j);
                i1 = i2 = 0;
            }
            s_id[0] = i1;
            s_id[1] = i2;
        }
    }
    __syncthreads();
    const XT *xa = X + (int64_t)s_id[0] * ld, *xb = X + (int64_t)s_id[1] * ld;
    float *cj = cen + j * 2 * (int64_t)d;
    for (int t = threadIdx.x; t < d; t += TR_THREADS) {
        cj[t] = ldx(xa + t);
        cj[d + t] = ldx(xb + t);
    }
}

// The coordinates t0 .. t0 + tw - 1 of the block's TR_THREADS member rows into the stage: warp w loads rows
// w, w + 4, ..., one coalesced load per 32 coordinates.
template <typename XT>
__device__ __forceinline__ void stage_rows(const XT *__restrict__ X, int64_t ld, const int *sid, int t0, int tw,
                                           float *stage, int warp, int lane)
{
    for (int r = warp; r < TR_THREADS; r += TR_THREADS / 32) {
        const XT *row = X + (int64_t)sid[r] * ld + t0;
        for (int q = lane; q < tw; q += 32)
            stage[r * TR_PITCH + q] = ldx(row + q);
    }
}

// Dynamic shared memory of the pass kernel: FP64 sums of both halves, both centres, the staged rows, the block's
// member ids and halves.
__host__ __device__ constexpr size_t pass_smem(int d)
{
    return (size_t)16 * d + (size_t)8 * d + sizeof(float) * TR_THREADS * TR_PITCH + 2 * sizeof(int) * TR_THREADS;
}

// One pass over the members of every splitting cluster of depth L, C chunks per cluster (grid S x C).  Each thread
// takes one member at a time: the rows of the block's 128 members are staged 64 coordinates at a time and each
// thread sums its member's two distances in the canonical FP32 order.
//   KEYS = false (a Lloyd iteration): the member joins u when d_u <= d_v and its row is added, in FP64 and in
//     member order, to its half's sums (a second staging of the group's rows; one thread per coordinate and
//     half keeps each sum); with one chunk the block writes the new centres, otherwise its sums and counts go
//     to part (2d + 2 doubles per chunk) for k_tree_reduce.
//   KEYS = true: keys[p] = (order(d_u - d_v) << 32) | id.
template <typename XT, bool KEYS>
__global__ void __launch_bounds__(TR_THREADS) k_tree_pass(const XT *__restrict__ X, int64_t n, int d, int64_t ld,
                                                          int L, int64_t C, const int32_t *__restrict__ perm,
                                                          const int32_t *__restrict__ spl, float *__restrict__ cen,
                                                          double *__restrict__ part, uint64_t *__restrict__ keys,
                                                          DevStatus *st)
{
    extern __shared__ __align__(16) unsigned char tr_smem[];
    double *acc = reinterpret_cast<double *>(tr_smem);              // [2][d]
    float *cuv = reinterpret_cast<float *>(acc + 2 * (size_t)d);    // [2][d]
    float *stage = cuv + 2 * (size_t)d;                             // [TR_THREADS][TR_PITCH]
    int *sid = reinterpret_cast<int *>(stage + TR_THREADS * TR_PITCH);
    int *shalf = sid + TR_THREADS;
    const int64_t j = blockIdx.x / C, c = blockIdx.x % C;
    if (spl && !spl[j])
        return;
    int64_t off, m, b, e;
    seg_geom(n, L, j, off, m);
    chunk_range(off, m, C, c, b, e);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *cj = cen + j * 2 * (int64_t)d;
    for (int t = tid; t < 2 * d; t += TR_THREADS) {
        cuv[t] = cj[t];
        if (!KEYS)
            acc[t] = 0.0;
    }
    __syncthreads();
    int64_t cnt_u = 0, cnt_v = 0;
    for (int64_t g = b; g < e; g += TR_THREADS) {
        const int64_t p = g + tid;
        const bool valid = p < e;
        int id = perm[valid ? p : b];
        if ((unsigned)id >= (unsigned)n) {
            flag_error(st, GK_ERR_INVALID, (unsigned)j);
            id = 0;
        }
        sid[tid] = id;
        float du = 0.f, dv = 0.f;
        for (int t0 = 0; t0 < d; t0 += TR_STAGE) {
            const int tw = min(TR_STAGE, d - t0);
            __syncthreads();  // sid written; the previous round's stage consumed
            stage_rows(X, ld, sid, t0, tw, stage, warp, lane);
            __syncthreads();
            const float *xs = stage + tid * TR_PITCH;
            for (int tt = 0; tt < tw; tt++) {
                const float x = xs[tt];
                const float eu = __fsub_rn(x, cuv[t0 + tt]);
                const float ev = __fsub_rn(x, cuv[d + t0 + tt]);
                du = __fmaf_rn(eu, eu, du);
                dv = __fmaf_rn(ev, ev, dv);
            }
        }
        if (KEYS) {
            if (valid) {
                const float dk = __fsub_rn(du, dv);
                if (!isfinite(dk))
                    flag_error(st, GK_ERR_NUMERIC, (unsigned)id);
                keys[p] = ((uint64_t)f32_order(dk) << 32) | (uint32_t)id;
            }
        } else {
            // the group's rows are staged again, 64 coordinates at a time; thread (c, h) adds coordinate c of the
            // members of half h in member order (ascending id within the cluster)
            shalf[tid] = valid ? (du <= dv ? 0 : 1) : 2;
            const int gn = (int)min((int64_t)TR_THREADS, e - g);
            for (int t0 = 0; t0 < d; t0 += TR_STAGE) {
                const int tw = min(TR_STAGE, d - t0);
                __syncthreads();  // shalf written; the previous round's stage consumed
                stage_rows(X, ld, sid, t0, tw, stage, warp, lane);
                __syncthreads();
                const int hh = tid / TR_STAGE, cc = tid % TR_STAGE;  // warps 0-1: half u, 2-3: half v
                if (cc < tw) {
                    double sum = acc[(size_t)hh * d + t0 + cc];
                    for (int r = 0; r < gn; r++)
                        if (shalf[r] == hh)
                            sum += widen(stage[r * TR_PITCH + cc]);
                    acc[(size_t)hh * d + t0 + cc] = sum;
                }
            }
            for (int r = 0; r < gn; r++) {
                cnt_u += shalf[r] == 0;
                cnt_v += shalf[r] == 1;
            }
        }
        __syncthreads();  // sid and shalf are rewritten by the next group
    }
    if (KEYS)
        return;
    if (C == 1) {
        for (int t = tid; t < d; t += TR_THREADS) {
            if (cnt_u)
                cj[t] = (float)(acc[t] / (double)cnt_u);
            if (cnt_v)
                cj[d + t] = (float)(acc[d + t] / (double)cnt_v);
        }
    } else {
        double *pc = part + blockIdx.x * (2 * (int64_t)d + 2);
        for (int t = tid; t < 2 * d; t += TR_THREADS)
            pc[t] = acc[t];
        if (tid == 0) {
            pc[2 * d] = (double)cnt_u;
            pc[2 * d + 1] = (double)cnt_v;
        }
    }
}

// Centres of the clusters split over several chunks: the chunks' FP64 sums added in chunk order.
__global__ void __launch_bounds__(TR_THREADS) k_tree_reduce(int d, int64_t C, const int32_t *__restrict__ spl,
                                                            float *__restrict__ cen, const double *__restrict__ part)
{
    const int64_t j = blockIdx.x;
    if (spl && !spl[j])
        return;
    const double *p0 = part + j * C * (2 * (int64_t)d + 2);
    double nu = 0.0, nv = 0.0;
    for (int64_t c = 0; c < C; c++) {
        nu += p0[c * (2 * (int64_t)d + 2) + 2 * d];
        nv += p0[c * (2 * (int64_t)d + 2) + 2 * d + 1];
    }
    float *cj = cen + j * 2 * (int64_t)d;
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
        double su = 0.0, sv = 0.0;
        for (int64_t c = 0; c < C; c++) {
            su += p0[c * (2 * (int64_t)d + 2) + t];
            sv += p0[c * (2 * (int64_t)d + 2) + d + t];
        }
        if (nu > 0.0)
            cj[t] = (float)(su / nu);
        if (nv > 0.0)
            cj[d + t] = (float)(sv / nv);
    }
}


// The ceil(m/2)-th smallest key of every splitting cluster (keys are distinct: they end in the member's id), by
// radix selection over 8-bit digits from the most significant.  Clusters of one chunk: one block each.
__global__ void __launch_bounds__(SEL_THREADS) k_tree_select(int64_t n, int L, const int32_t *__restrict__ spl,
                                                             const uint64_t *__restrict__ keys,
                                                             uint64_t *__restrict__ thr)
{
    __shared__ unsigned hist[256];
    __shared__ uint64_t s_prefix;
    __shared__ int64_t s_rank;
    const int64_t j = blockIdx.x;
    if (spl && !spl[j])
        return;
    int64_t off, m;
    seg_geom(n, L, j, off, m);
    const int tid = threadIdx.x;
    uint64_t prefix = 0, mask = 0;
    int64_t rank = (m + 1) / 2 - 1;  // among the keys that match the prefix so far
    for (int shift = 56; shift >= 0; shift -= 8) {
        hist[tid] = 0;  // SEL_THREADS == 256 bins
        __syncthreads();
        for (int64_t p = off + tid; p < off + m; p += SEL_THREADS) {
            const uint64_t k = keys[p];
            if ((k & mask) == prefix)
                atomicAdd(&hist[(k >> shift) & 255], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            int dg;
            int64_t below;
            warp_pick(hist, rank, dg, below);
            if (tid == 0) {
                s_prefix = prefix | ((uint64_t)dg << shift);
                s_rank = rank - below;
            }
        }
        __syncthreads();
        prefix = s_prefix;
        rank = s_rank;
        mask |= (uint64_t)255 << shift;
    }
    if (tid == 0)
        thr[j] = prefix;
}

// The same selection for clusters of several chunks, one digit at a time: k_tree_sel_init, then per digit
// k_tree_hist (every chunk adds its histogram of the keys that match the prefix) and k_tree_digit (one warp per
// cluster picks the digit and clears the histogram).  thr holds the prefix, srank the rank within it.
__global__ void __launch_bounds__(SEL_THREADS) k_tree_sel_init(int64_t n, int L, const int32_t *__restrict__ spl,
                                                               uint64_t *__restrict__ thr, int64_t *__restrict__ srank,
                                                               unsigned *__restrict__ ghist)
{
    const int64_t j = blockIdx.x;
    if (spl && !spl[j])
        return;
    int64_t off, m;
    seg_geom(n, L, j, off, m);
    ghist[j * 256 + threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        thr[j] = 0;
        srank[j] = (m + 1) / 2 - 1;
    }
}

__global__ void __launch_bounds__(SEL_THREADS) k_tree_hist(int64_t n, int L, int64_t C, int shift,
                                                           const int32_t *__restrict__ spl,
                                                           const uint64_t *__restrict__ keys,
                                                           const uint64_t *__restrict__ thr,
                                                           unsigned *__restrict__ ghist)
{
    __shared__ unsigned hist[256];
    const int64_t j = blockIdx.x / C, c = blockIdx.x % C;
    if (spl && !spl[j])
        return;
    int64_t off, m, b, e;
    seg_geom(n, L, j, off, m);
    chunk_range(off, m, C, c, b, e);
    const uint64_t prefix = thr[j];
    const uint64_t mask = shift == 56 ? 0ull : ~0ull << (shift + 8);
    hist[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t p = b + threadIdx.x; p < e; p += SEL_THREADS) {
        const uint64_t k = keys[p];
        if ((k & mask) == prefix)
            atomicAdd(&hist[(k >> shift) & 255], 1u);
    }
    __syncthreads();
    if (hist[threadIdx.x])
        atomicAdd(&ghist[j * 256 + threadIdx.x], hist[threadIdx.x]);
}

__global__ void __launch_bounds__(32) k_tree_digit(int shift, const int32_t *__restrict__ spl,
                                                   uint64_t *__restrict__ thr, int64_t *__restrict__ srank,
                                                   unsigned *__restrict__ ghist)
{
    const int64_t j = blockIdx.x;
    if (spl && !spl[j])
        return;
    unsigned *h = ghist + j * 256;
    int dg;
    int64_t below;
    const int64_t rank = srank[j];
    warp_pick(h, rank, dg, below);
    __syncwarp();
    for (int q = 0; q < 8; q++)
        h[8 * threadIdx.x + q] = 0;
    if (threadIdx.x == 0) {
        thr[j] |= (uint64_t)dg << shift;
        srank[j] = rank - below;
    }
}

// Members with key <= thr[j] (half u) in every chunk of a cluster of several chunks, and their exclusive scan
// over the cluster's chunks (one warp per cluster): where each chunk's u and v members start.
__global__ void __launch_bounds__(SEL_THREADS) k_tree_count(int64_t n, int L, int64_t C,
                                                            const int32_t *__restrict__ spl,
                                                            const uint64_t *__restrict__ keys,
                                                            const uint64_t *__restrict__ thr,
                                                            int32_t *__restrict__ ccount)
{
    __shared__ int wsum[SEL_THREADS / 32];
    const int64_t j = blockIdx.x / C, c = blockIdx.x % C;
    if (spl && !spl[j])
        return;
    int64_t off, m, b, e;
    seg_geom(n, L, j, off, m);
    chunk_range(off, m, C, c, b, e);
    const uint64_t T = thr[j];
    int cnt = 0;
    for (int64_t p = b + threadIdx.x; p < e; p += SEL_THREADS)
        cnt += keys[p] <= T;
    for (int o = 16; o > 0; o >>= 1)
        cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
    if ((threadIdx.x & 31) == 0)
        wsum[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < SEL_THREADS / 32; w++)
            t += wsum[w];
        ccount[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(32) k_tree_cscan(int64_t C, const int32_t *__restrict__ spl,
                                                   const int32_t *__restrict__ ccount, int32_t *__restrict__ cbase)
{
    const int64_t j = blockIdx.x;
    if (spl && !spl[j])
        return;
    const int lane = threadIdx.x;
    int carry = 0;
    for (int64_t c0 = 0; c0 < C; c0 += 32) {
        const int64_t c = c0 + lane;
        const int v = c < C ? ccount[j * C + c] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o)
                incl += u;
        }
        if (c < C)
            cbase[j * C + c] = carry + incl - v;
        carry += __shfl_sync(FULL_MASK, incl, 31);
    }
}

// Stable partition of every cluster of depth L, chunk by chunk: the members with key <= thr[j] to the left
// ceil(m/2) positions, the others after them, each in their previous order (cbase: where the chunk's u members
// start among the cluster's, NULL for clusters of one chunk); clusters that do not split are copied.
__global__ void __launch_bounds__(SEL_THREADS) k_tree_split(int64_t n, int L, int64_t C,
                                                            const int32_t *__restrict__ spl,
                                                            const uint64_t *__restrict__ keys,
                                                            const uint64_t *__restrict__ thr,
                                                            const int32_t *__restrict__ cbase,
                                                            const int32_t *__restrict__ perm_in,
                                                            int32_t *__restrict__ perm_out, DevStatus *st)
{
    __shared__ int wsum[SEL_THREADS / 32];
    const int64_t j = blockIdx.x / C, c = blockIdx.x % C;
    int64_t off, m, b, e;
    seg_geom(n, L, j, off, m);
    chunk_range(off, m, C, c, b, e);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (spl && !spl[j]) {
        for (int64_t p = b + tid; p < e; p += SEL_THREADS)
            perm_out[p] = perm_in[p];
        return;
    }
    const uint64_t T = thr[j];
    const int64_t h = (m + 1) / 2;
    int64_t bu = cbase ? cbase[blockIdx.x] : 0;
    int64_t bv = (b - off) - bu;
    for (int64_t t0 = b; t0 < e; t0 += SEL_THREADS) {
        const int64_t p = t0 + tid;
        const bool valid = p < e;
        const uint64_t k = valid ? keys[p] : 0;
        const bool f = valid && k <= T;
        const unsigned bal = __ballot_sync(FULL_MASK, f);
        if (lane == 0)
            wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < SEL_THREADS / 32; w++) {
            before += w < warp ? wsum[w] : 0;
            total += wsum[w];
        }
        const int64_t ru = before + __popc(bal & lanemask_lt());  // u members before this one in the tile
        if (valid) {
            const int64_t dst = f ? off + bu + ru : off + h + bv + (tid - ru);
            if (dst >= off && dst < off + m)
                perm_out[dst] = (int32_t)(uint32_t)k;
            else
                flag_error(st, GK_ERR_INVALID, (unsigned)j);
        }
        const int64_t nvalid = min((int64_t)SEL_THREADS, e - t0);
        bu += total;
        bv += nvalid - total;
        __syncthreads();
    }
}

// Labels: clusters numbered left to right.  Cluster j of the last depth L keeps number j + pre[j], or, when it
// splits (spl[j]), its halves take j + pre[j] and j + pre[j] + 1.  With spl == NULL the depth is complete.
__global__ void __launch_bounds__(SEL_THREADS) k_tree_label(int64_t n, int L, int64_t C,
                                                            const int32_t *__restrict__ spl,
                                                            const int32_t *__restrict__ pre,
                                                            const int32_t *__restrict__ perm,
                                                            int32_t *__restrict__ labels)
{
    const int64_t j = blockIdx.x / C, c = blockIdx.x % C;
    int64_t off, m, b, e;
    seg_geom(n, L, j, off, m);
    chunk_range(off, m, C, c, b, e);
    const bool split = spl && spl[j];
    const int32_t base = (int32_t)j + (spl ? pre[j] : 0);
    const int64_t h = (m + 1) / 2;
    for (int64_t p = b + threadIdx.x; p < e; p += SEL_THREADS) {
        const int id = perm[p];
        if ((unsigned)id < (unsigned)n)
            labels[id] = base + (split && p - off >= h ? 1 : 0);
    }
}

// Depth L such that 2^L <= k < 2^(L + 1): depths 0 .. L - 1 split completely, depth L splits k - 2^L clusters.
int tree_depth(int32_t k)
{
    int L = 0;
    while (((int64_t)2 << L) <= (int64_t)k)
        L++;
    return L;
}

// Pass blocks per cluster at depth L: clusters of up to TR_CHUNK members take one.
int64_t tree_chunks(int64_t n, int L)
{
    const int64_t a1 = (n >> L) + 1;
    return std::max<int64_t>(1, (a1 + TR_CHUNK - 1) / TR_CHUNK);
}

struct TreeBufs {
    int32_t *perm_a, *perm_b, *spl, *pre, *ccount, *cbase;
    uint64_t *keys, *thr;
    int64_t *srank;
    unsigned *ghist;
    Top2 *seeds;
    float *cen;
    double *part;
    size_t bytes;
};

TreeBufs tree_carve(void *scratch, int64_t n, int64_t d, int32_t k)
{
    Carver cv{static_cast<char *>(scratch), 0, 0};
    const int Lf = tree_depth(k);
    const int64_t S = (int64_t)1 << Lf;
    int64_t part = 1, chunks = 1, multi = 1;  // doubles of partial sums; chunk blocks; clusters of several chunks
    for (int L = 0; L <= Lf; L++) {
        const int64_t C = tree_chunks(n, L);
        chunks = std::max(chunks, ((int64_t)1 << L) * C);
        if (C > 1) {
            part = std::max(part, ((int64_t)1 << L) * C * (2 * d + 2));
            multi = std::max(multi, (int64_t)1 << L);
        }
    }
    TreeBufs B{};
    B.perm_a = cv.take<int32_t>((size_t)n);
    B.perm_b = cv.take<int32_t>((size_t)n);
    B.keys = cv.take<uint64_t>((size_t)n);
    B.cen = cv.take<float>((size_t)S * 2 * (size_t)d);
    B.thr = cv.take<uint64_t>((size_t)S);
    B.srank = cv.take<int64_t>((size_t)S);
    B.spl = cv.take<int32_t>((size_t)S);
    B.pre = cv.take<int32_t>((size_t)S);
    B.seeds = cv.take<Top2>((size_t)chunks);
    B.ccount = cv.take<int32_t>((size_t)chunks);
    B.cbase = cv.take<int32_t>((size_t)chunks);
    B.ghist = cv.take<unsigned>((size_t)multi * 256);
    B.part = cv.take<double>((size_t)part);
    B.bytes = cv.off;
    return B;
}

// Per depth L (S clusters, C chunk blocks per cluster; spl = NULL when every cluster splits):
//   seeds (2 launches), iters x {pass, reduce if C > 1}, keys pass, select (1 launch, or 17 when C > 1),
//   split (1 launch, or 3 when C > 1).
template <typename XT>
cudaError_t tree_run(const XT *X, int64_t n, int d, int64_t ld, int32_t k, int32_t iters, uint64_t seed,
                     int32_t *labels, const TreeBufs &B, DevStatus *st, cudaStream_t s)
{
    cudaError_t e;
    if ((e = set_max_smem((const void *)k_tree_pass<XT, false>, (int)pass_smem(MAX_D))) != cudaSuccess ||
        (e = set_max_smem((const void *)k_tree_pass<XT, true>, (int)pass_smem(MAX_D))) != cudaSuccess)
        return e;
    const size_t smem = pass_smem(d);
    k_tree_iota<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(B.perm_a, n);
    const int Lf = tree_depth(k);
    const int64_t r = (int64_t)k - ((int64_t)1 << Lf);
    int32_t *cur = B.perm_a, *nxt = B.perm_b;
    for (int L = 0; L <= Lf; L++) {
        const int32_t *spl = nullptr;
        const int64_t S = (int64_t)1 << L;
        if (L == Lf) {
            if (r == 0)
                break;
            k_tree_plan<<<1, 1024, 0, s>>>(n, L, r, B.spl, B.pre);
            spl = B.spl;
        }
        const int64_t C = tree_chunks(n, L);
        const unsigned SC = (unsigned)(S * C);
        k_tree_seed_part<<<SC, SEL_THREADS, 0, s>>>(n, L, C, cur, spl, seed, B.seeds);
        k_tree_seed_final<XT><<<(unsigned)S, TR_THREADS, 0, s>>>(X, n, d, ld, C, spl, B.seeds, B.cen, st);
        for (int it = 0; it < iters; it++) {
            k_tree_pass<XT, false><<<SC, TR_THREADS, smem, s>>>(X, n, d, ld, L, C, cur, spl, B.cen, B.part, B.keys,
                                                                st);
            if (C > 1)
                k_tree_reduce<<<(unsigned)S, TR_THREADS, 0, s>>>(d, C, spl, B.cen, B.part);
        }
        k_tree_pass<XT, true><<<SC, TR_THREADS, smem, s>>>(X, n, d, ld, L, C, cur, spl, B.cen, B.part, B.keys, st);
        if (C == 1) {
            k_tree_select<<<(unsigned)S, SEL_THREADS, 0, s>>>(n, L, spl, B.keys, B.thr);
            k_tree_split<<<SC, SEL_THREADS, 0, s>>>(n, L, C, spl, B.keys, B.thr, nullptr, cur, nxt, st);
        } else {
            k_tree_sel_init<<<(unsigned)S, SEL_THREADS, 0, s>>>(n, L, spl, B.thr, B.srank, B.ghist);
            for (int shift = 56; shift >= 0; shift -= 8) {
                k_tree_hist<<<SC, SEL_THREADS, 0, s>>>(n, L, C, shift, spl, B.keys, B.thr, B.ghist);
                k_tree_digit<<<(unsigned)S, 32, 0, s>>>(shift, spl, B.thr, B.srank, B.ghist);
            }
            k_tree_count<<<SC, SEL_THREADS, 0, s>>>(n, L, C, spl, B.keys, B.thr, B.ccount);
            k_tree_cscan<<<(unsigned)S, 32, 0, s>>>(C, spl, B.ccount, B.cbase);
            k_tree_split<<<SC, SEL_THREADS, 0, s>>>(n, L, C, spl, B.keys, B.thr, B.cbase, cur, nxt, st);
        }
        std::swap(cur, nxt);
    }
    const int64_t Cf = tree_chunks(n, Lf);
    k_tree_label<<<(unsigned)(((int64_t)1 << Lf) * Cf), SEL_THREADS, 0, s>>>(n, Lf, Cf, r > 0 ? B.spl : nullptr,
                                                                             B.pre, cur, labels);
    return cudaGetLastError();
}

}  // namespace

size_t tree_scratch_bytes(int64_t n, int64_t d, int32_t k) { return tree_carve(nullptr, n, d, k).bytes; }

cudaError_t launch_tree(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t k, int32_t iters,
                        uint64_t seed, int32_t *labels, void *scratch, DevStatus *st, cudaStream_t s)
{
    const TreeBufs B = tree_carve(scratch, n, d, k);
    if (bf16)
        return tree_run(static_cast<const __nv_bfloat16 *>(X), n, (int)d, ld, k, iters, seed, labels, B, st, s);
    return tree_run(static_cast<const float *>(X), n, (int)d, ld, k, iters, seed, labels, B, st, s);
}

}  // namespace gkm
