// Seeded initial state: random labels and the random initial KNN graph
// (Alg. 3 starts from a graph of random neighbour lists).  Random numbers come from the
// SplitMix64 generator used as a counter-based function (common.cuh).
#include "common.cuh"
#include "merge.cuh"
#include "tc.cuh"

namespace gkm {

__global__ void k_init_labels(int64_t n, int32_t k, uint64_t key, int32_t off, int32_t *__restrict__ labels)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        labels[i] = (int32_t)(sm64_draw(key, (uint64_t)i) % (uint64_t)k) + off;
}

cudaError_t launch_init_labels(int64_t n, int32_t k, uint64_t seed, int32_t *labels, cudaStream_t s,
                               int32_t label_offset)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64)
        blocks = 152 * 64;
    if (blocks < 1)
        blocks = 1;
    k_init_labels<<<(unsigned)blocks, 256, 0, s>>>(n, k, seed ^ TAG_LABELS, label_offset, labels);
    return cudaGetLastError();
}

// One warp per row.  Attempts a = base + lane are drawn 32 at a time and
// accepted in attempt order: a draw is kept when it is not the row itself, not
// already in the row, and the first of its value among this batch; only the
// first kappa - got kept draws are used, which is exactly the sequential
// rejection rule.  Each lane then computes the FP32 distance of one neighbour
// (pair_d2_seq), and the row is sorted by (distance, id) by ranking.
constexpr int IG_WARPS = 4;
constexpr int IG_DC_BYTES = 512;  // bytes of a row staged per step (vector path)

// Coordinates staged per step: 128 FP32 or 256 BF16 values (one 512-byte bulk copy per row).
template <typename XT>
__host__ __device__ constexpr int ig_dc() { return IG_DC_BYTES / (int)sizeof(XT); }
constexpr uint32_t IG_WAIT_ITERS = 1u << 22;

// Rows staged per batch: kappa cut into equal batches of at most 32.
__host__ __device__ inline int ig_batch(int kappa)
{
    const int nb = (kappa + 31) / 32;
    return (kappa + nb - 1) / nb;
}

// Staged row stride in elements: ig_dc() plus 16 bytes, so that the 32 lanes
// reading their own rows 16 bytes at a time hit distinct banks.
template <typename XT>
__host__ __device__ constexpr int ig_stride() { return ig_dc<XT>() + 16 / (int)sizeof(XT); }

// Dynamic shared memory per warp: on the vector path a batch of rows; on both
// paths at least the kappa 8-byte keys of the rank sort (they reuse the area).
// Kernel and launcher both size the warp areas with this.
template <typename XT>
__host__ __device__ inline size_t ig_warp_bytes(int kappa, bool vec)
{
    size_t b = vec ? sizeof(XT) * (size_t)ig_batch(kappa) * ig_stride<XT>() : 0;
    if (b < sizeof(uint64_t) * (size_t)kappa)
        b = sizeof(uint64_t) * (size_t)kappa;
    return (b + 15) & ~size_t(15);
}

// Exact a mod n for 0 < n < 2^32 with minv = floor((2^64 - 1) / n): the
// quotient estimate q = floor(a minv / 2^64) lies in [floor(a/n) - 2, floor(a/n)],
// so at most two subtractions finish the remainder (Barrett reduction).
__device__ __forceinline__ uint64_t mod_n(uint64_t a, uint64_t n, uint64_t minv)
{
    const uint64_t q = __umul64hi(a, minv);
    uint64_t r = a - q * n;
    if (r >= n)
        r -= n;
    if (r >= n)
        r -= n;
    return r;
}

// 16 bytes of elements as floats: from shared memory (SHARED) or through L1.
template <typename XT, bool SHARED>
__device__ __forceinline__ void ld16(const XT *p, float (&v)[16 / sizeof(XT)])
{
    const uint4 q = SHARED ? *reinterpret_cast<const uint4 *>(p) : __ldg(reinterpret_cast<const uint4 *>(p));
    if constexpr (sizeof(XT) == 4) {
        v[0] = __uint_as_float(q.x);
        v[1] = __uint_as_float(q.y);
        v[2] = __uint_as_float(q.z);
        v[3] = __uint_as_float(q.w);
    } else {
        const float4 a = bf16x4_to_float4(make_uint2(q.x, q.y)), b = bf16x4_to_float4(make_uint2(q.z, q.w));
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    }
}

template <typename XT>
__global__ void __launch_bounds__(IG_WARPS * 32, 4) k_init_graph(const XT *__restrict__ X, int64_t n, int d,
                                                              int64_t ld, int kappa, uint64_t key, uint64_t minv,
                                                              int32_t id_off, int32_t *__restrict__ g_idx,
                                                              float *__restrict__ g_dist, DevStatus *st, bool vec)
{
    constexpr int RS = ig_stride<XT>(), E = 16 / (int)sizeof(XT);
    __shared__ int s_idx[IG_WARPS][MAX_KAPPA];
    __shared__ uint64_t s_bar[IG_WARPS];
    // dynamic: per warp one batch of staged rows; after the distances, the row's keys
    extern __shared__ __align__(16) float s_dyn[];
    const int w = threadIdx.x >> 5, lane = lane_id();
    int *ridx = s_idx[w];
    const int B = ig_batch(kappa);
    XT *rows =
        reinterpret_cast<XT *>(reinterpret_cast<unsigned char *>(s_dyn) + (size_t)w * ig_warp_bytes<XT>(kappa, vec));
    uint64_t *rkey = reinterpret_cast<uint64_t *>(rows);
    uint64_t *bar = s_bar + w;
    if (lane == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    for (int64_t i = blockIdx.x * (int64_t)IG_WARPS + w; i < n; i += (int64_t)gridDim.x * IG_WARPS) {
        int got = 0;
        for (uint64_t a0 = 0; got < kappa; a0 += 32) {
            if (a0 >= (1ull << 31)) {  // cannot happen for kappa < n; bounded all the same
                if (lane == 0)
                    flag_error(st, GK_ERR_TIMEOUT, (unsigned)i);
                for (int q = got + lane; q < kappa; q += 32)
                    ridx[q] = (int)((i + 1 + q) % n);
                got = kappa;
                __syncwarp();
                break;
            }
            uint64_t a = a0 + (uint64_t)lane;
            int64_t j = (int64_t)mod_n(sm64_draw(key, ((uint64_t)i << 32) | a), (uint64_t)n, minv);
            unsigned peers = __match_any_sync(FULL_MASK, (unsigned long long)j);
            bool ok = (j != i) && ((peers & lanemask_lt()) == 0u);
            if (ok)
                for (int q = 0; q < got; q++)
                    if (ridx[q] == (int)j) {
                        ok = false;
                        break;
                    }
            unsigned oks = __ballot_sync(FULL_MASK, ok);
            int pos = got + __popc(oks & lanemask_lt());
            __syncwarp();
            if (ok && pos < kappa)
                ridx[pos] = (int)j;
            got = min(kappa, got + __popc(oks));
            __syncwarp();
        }
        const XT *xi = X + i * ld;
        float dist[(MAX_KAPPA + 31) / 32];  // distance of neighbour b0 + lane of batch b (lane < batch size)
        if (vec) {
            // A batch's neighbour rows are copied to shared memory by the TMA engine
            // (one bulk copy per row, issued by the row's lane, counted on the warp's
            // mbarrier); lane q then sums its row's squared differences in ascending
            // coordinate order (the order of pair_d2_seq), x_i coming through L1.
            for (int b0 = 0, bi = 0; b0 < kappa; b0 += B, bi++) {
                const int nb = min(B, kappa - b0);
                float acc = 0.f;
                for (int t0 = 0; t0 < d; t0 += ig_dc<XT>()) {
                    const int dc = min(ig_dc<XT>(), d - t0);
                    const uint32_t bytes = (uint32_t)(dc * (int)sizeof(XT));
                    __syncwarp();                 // the previous rows are no longer read
                    tc::fence_proxy_async_smem();  // ... before the async proxy rewrites them
                    if (lane == 0)
                        tc::mbar_arrive_expect_tx(bar, (uint32_t)nb * bytes);
                    __syncwarp();
                    if (lane < nb)
                        tc::bulk_g2s(rows + lane * RS, X + (int64_t)ridx[b0 + lane] * ld + t0, bytes, bar);
                    const bool ok = __all_sync(FULL_MASK, tc::mbar_wait_bounded(bar, phase, IG_WAIT_ITERS));
                    phase ^= 1u;
                    if (!ok) {  // the copies did not complete: report, give them one more bounded wait, stop
                        if (lane == 0)
                            flag_error(st, GK_ERR_TIMEOUT, (unsigned)i);
                        tc::mbar_wait_bounded(bar, phase ^ 1u, IG_WAIT_ITERS);
                        return;
                    }
                    if (lane < nb) {
                        const XT *xa = xi + t0, *xb = rows + lane * RS;
                        auto part = [&](int t) {
                            float va[E], vb[E];
                            ld16<XT, false>(xa + t, va);
                            ld16<XT, true>(xb + t, vb);
#pragma unroll
                            for (int e = 0; e < E; e++) {
                                const float df = va[e] - vb[e];
                                acc = fmaf(df, df, acc);
                            }
                        };
                        if (dc == ig_dc<XT>()) {  // a full chunk, unrolled: the next loads overlap this FMA chain
#pragma unroll 4
                            for (int t = 0; t < ig_dc<XT>(); t += E)
                                part(t);
                        } else {
                            for (int t = 0; t < dc; t += E)
                                part(t);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < (MAX_KAPPA + 31) / 32; q++)
                    if (q == bi)
                        dist[q] = acc;
            }
        } else {
            for (int b0 = 0, bi = 0; b0 < kappa; b0 += B, bi++) {
                const float acc = lane < min(B, kappa - b0) ? pair_d2_seq(xi, X + (int64_t)ridx[b0 + lane] * ld, d) : 0.f;
#pragma unroll
                for (int q = 0; q < (MAX_KAPPA + 31) / 32; q++)
                    if (q == bi)
                        dist[q] = acc;
            }
        }
        __syncwarp();
        // rank sort on packed (distance, id) keys: ids in a row are distinct, so keys are
#pragma unroll
        for (int q = 0; q < (MAX_KAPPA + 31) / 32; q++) {
            const int e = q * B + lane;
            if (lane < B && e < kappa)
                rkey[e] = pack_key(dist[q], ridx[e]);
        }
        __syncwarp();
        const int64_t out = i * (int64_t)kappa;
        for (int q = lane; q < kappa; q += 32) {
            const uint64_t kq = rkey[q];
            int r = 0;
            for (int p = 0; p < kappa; p++)
                r += rkey[p] < kq ? 1 : 0;
            g_idx[out + r] = key_id(kq) + id_off;
            g_dist[out + r] = key_dist(kq);
        }
        __syncwarp();
    }
}

template <typename XT>
static cudaError_t init_graph_t(const XT *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed,
                                int32_t *g_idx, float *g_dist, DevStatus *st, cudaStream_t s, int32_t id_offset)
{
    int64_t blocks = (n + IG_WARPS - 1) / IG_WARPS;
    if (blocks > 152 * 64)
        blocks = 152 * 64;
    // bulk copies of row chunks need 16-byte aligned rows and chunk sizes
    const bool vec = (d * (int64_t)sizeof(XT)) % 16 == 0 && (ld * (int64_t)sizeof(XT)) % 16 == 0 &&
                     (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    const size_t shm = IG_WARPS * ig_warp_bytes<XT>(kappa, vec);
    cudaError_t e = set_max_smem(reinterpret_cast<const void *>(k_init_graph<XT>),
                                 (int)(IG_WARPS * ig_warp_bytes<XT>(MAX_KAPPA, true)));
    if (e != cudaSuccess)
        return e;
    const uint64_t minv = ~0ull / (uint64_t)n;
    k_init_graph<XT><<<(unsigned)blocks, IG_WARPS * 32, shm, s>>>(X, n, (int)d, ld, kappa, seed ^ TAG_GRAPH, minv,
                                                               id_offset, g_idx, g_dist, st, vec);
    return cudaGetLastError();
}

cudaError_t launch_init_graph(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t kappa,
                              uint64_t seed, int32_t *g_idx, float *g_dist, DevStatus *st, cudaStream_t s,
                              int32_t id_offset)
{
    if (bf16)
        return init_graph_t(static_cast<const __nv_bfloat16 *>(X), n, d, ld, kappa, seed, g_idx, g_dist, st, s,
                            id_offset);
    return init_graph_t(static_cast<const float *>(X), n, d, ld, kappa, seed, g_idx, g_dist, st, s, id_offset);
}

}  // namespace gkm
