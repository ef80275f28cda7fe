// Seeded initial state: random labels and the random initial KNN graph
// (Alg. 3 starts from a graph of random neighbour lists).  Random numbers come from the
// SplitMix64 generator used as a counter-based function (common.cuh).
#include "common.cuh"

namespace gkm {

__global__ void k_init_labels(int64_t n, int32_t k, uint64_t key, int32_t *__restrict__ labels)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        labels[i] = (int32_t)(sm64_draw(key, (uint64_t)i) % (uint64_t)k);
}

cudaError_t launch_init_labels(int64_t n, int32_t k, uint64_t seed, int32_t *labels, cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64)
        blocks = 152 * 64;
    if (blocks < 1)
        blocks = 1;
    k_init_labels<<<(unsigned)blocks, 256, 0, s>>>(n, k, seed ^ TAG_LABELS, labels);
    return cudaGetLastError();
}

// One warp per row.  Attempts a = base + lane are drawn 32 at a time and
// accepted in attempt order: a draw is kept when it is not the row itself, not
// already in the row, and the first of its value among this batch; only the
// first kappa - got kept draws are used, which is exactly the sequential
// rejection rule.  Each lane then computes the FP32 distance of one neighbour
// (pair_d2_seq), and the row is sorted by (distance, id) by ranking.
constexpr int IG_WARPS = 4;
constexpr int IG_DC = 128;  // coordinates staged per step (vector path)

__global__ void __launch_bounds__(IG_WARPS * 32) k_init_graph(const float *__restrict__ X, int64_t n, int d,
                                                              int64_t ld, int kappa, uint64_t key,
                                                              int32_t *__restrict__ g_idx,
                                                              float *__restrict__ g_dist, DevStatus *st,
                                                              bool vec4)
{
    __shared__ int s_idx[IG_WARPS][MAX_KAPPA];
    __shared__ float s_dist[IG_WARPS][MAX_KAPPA];
    // dynamic: per warp IG_DC floats of x_i, then 32 staged rows of IG_DC + 4 floats
    extern __shared__ __align__(16) float s_dyn[];
    const int w = threadIdx.x >> 5, lane = lane_id();
    int *ridx = s_idx[w];
    float *rdist = s_dist[w];
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
            int64_t j = (int64_t)(sm64_draw(key, ((uint64_t)i << 32) | a) % (uint64_t)n);
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
        const float *xi = X + i * ld;
        if (vec4) {
            // neighbour rows staged 32 at a time, IG_DC coordinates at a time, with
            // one coalesced 16-byte load per lane and row; lane q then sums its
            // row's squared differences in ascending coordinate order (the order
            // of pair_d2_seq) from shared memory
            float *xs = s_dyn + w * (IG_DC + 32 * (IG_DC + 4));
            float *rows = xs + IG_DC;
            for (int b0 = 0; b0 < kappa; b0 += 32) {
                const int nb = min(32, kappa - b0);
                float acc = 0.f;
                for (int t0 = 0; t0 < d; t0 += IG_DC) {
                    const int dc = min(IG_DC, d - t0);
                    __syncwarp();
                    for (int t = lane * 4; t < dc; t += 128)
                        *reinterpret_cast<float4 *>(xs + t) = *reinterpret_cast<const float4 *>(xi + t0 + t);
                    // every row of the batch in flight at once (asynchronous copies to shared memory)
                    for (int q = 0; q < nb; q++) {
                        const float *src = X + (int64_t)ridx[b0 + q] * ld + t0;
                        for (int t = lane * 4; t < dc; t += 128)
                            cp_async16(rows + q * (IG_DC + 4) + t, src + t);
                    }
                    cp_async_wait_all();
                    __syncwarp();
                    if (lane < nb) {
                        const float *myrow = rows + lane * (IG_DC + 4);
                        for (int t = 0; t < dc; t += 4) {
                            float4 a = *reinterpret_cast<const float4 *>(xs + t);
                            float4 b = *reinterpret_cast<const float4 *>(myrow + t);
                            float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
                            acc = fmaf(e0, e0, acc);
                            acc = fmaf(e1, e1, acc);
                            acc = fmaf(e2, e2, acc);
                            acc = fmaf(e3, e3, acc);
                        }
                    }
                }
                if (lane < nb)
                    rdist[b0 + lane] = acc;
            }
        } else {
            for (int q = lane; q < kappa; q += 32)
                rdist[q] = pair_d2_seq(xi, X + (int64_t)ridx[q] * ld, d);
        }
        __syncwarp();
        // rank sort: ids in a row are distinct, so keys are distinct
        int64_t out = i * (int64_t)kappa;
        for (int q = lane; q < kappa; q += 32) {
            float dq = rdist[q];
            int iq = ridx[q];
            int r = 0;
            for (int p = 0; p < kappa; p++)
                r += key_less(rdist[p], ridx[p], dq, iq) ? 1 : 0;
            g_idx[out + r] = iq;
            g_dist[out + r] = dq;
        }
        __syncwarp();
    }
}

cudaError_t launch_init_graph(const float *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed,
                              int32_t *g_idx, float *g_dist, DevStatus *st, cudaStream_t s)
{
    int64_t blocks = (n + IG_WARPS - 1) / IG_WARPS;
    if (blocks > 152 * 64)
        blocks = 152 * 64;
    const bool vec4 = (d % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const size_t shm = vec4 ? sizeof(float) * IG_WARPS * (IG_DC + 32 * (IG_DC + 4)) : 0;
    if (shm) {
        cudaError_t e = cudaFuncSetAttribute(k_init_graph, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess)
            return e;
    }
    k_init_graph<<<(unsigned)blocks, IG_WARPS * 32, shm, s>>>(X, n, (int)d, ld, kappa, seed ^ TAG_GRAPH, g_idx,
                                                           g_dist, st, vec4);
    return cudaGetLastError();
}

}  // namespace gkm
