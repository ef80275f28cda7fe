// Top-1 recall of a KNN graph, estimated on sampled queries (Sec. 5: the
// recall of the top-1 neighbour, taken over randomly chosen samples where the
// full ground truth is too costly).  For each query q its exact nearest
// neighbour is found by brute force over all n samples, pair distances in the
// canonical FP32 order (tiles.cuh) and ties by the smaller id (the graph's key
// order); the query is a hit when that neighbour is the first entry of q's
// graph row.  With exact distances in rows sorted by key, the true neighbour
// is in a row exactly when it is its first entry, so this is also the
// fraction of queries whose row holds their nearest neighbour.
//
// k_nn_tiles: block (b, s) takes the 64 queries of query block b and the
// samples of slice s, 64 at a time, as 64 x 64 distance tiles; each warp keeps
// the smallest (distance, id) key of eight queries over the slice.
// k_nn_finish: per query the smallest key over the slices, the hit test, and
// the count of hits.
#include "common.cuh"
#include "merge.cuh"
#include "tiles.cuh"

#include <cuda_bf16.h>

namespace gkm {

constexpr int NN_T = 64;                                       // queries and samples per tile
constexpr size_t NN_SMEM = RefineTile<NN_T>::fixed_bytes + sizeof(uint64_t) * NN_T;

static int64_t nn_qblocks(int32_t m) { return ((int64_t)m + NN_T - 1) / NN_T; }

// slices of the samples per query block: about three blocks per SM in all
int recall_slices(int64_t n, int32_t m)
{
    const int64_t tiles = (n + NN_T - 1) / NN_T;
    int64_t s = (152 * 3 + nn_qblocks(m) - 1) / nn_qblocks(m);
    s = s < 1 ? 1 : s;
    return (int)(s > tiles ? tiles : s);
}

size_t recall_scratch_bytes(int64_t n, int32_t m)
{
    return (((size_t)m * (size_t)recall_slices(n, m) * sizeof(uint64_t)) + 255) & ~size_t(255);
}

template <typename XT>
__global__ void __launch_bounds__(RF_THREADS) k_nn_tiles(const XT *__restrict__ X, int64_t n, int d, int64_t ld,
                                                        const int32_t *__restrict__ queries, int m, int slices,
                                                        uint64_t *__restrict__ part, DevStatus *st)
{
    using TL = RefineTile<NN_T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *xr = reinterpret_cast<float *>(smem_raw);  // staging buffers of the pair tiles (tiles.cuh)
    float *dt = xr;  // aliases the staging buffers
    constexpr size_t span = TL::stage_floats > TL::tile_floats ? TL::stage_floats : TL::tile_floats;
    int *rid = reinterpret_cast<int *>(xr + span);
    int *cid = rid + NN_T;
    uint64_t *best = reinterpret_cast<uint64_t *>(cid + NN_T);
    const int tid = threadIdx.x, w = tid >> 5, lane = lane_id();
    const int q0 = blockIdx.x * NN_T, nr = min(NN_T, m - q0);
    const int64_t tiles = (n + NN_T - 1) / NN_T;
    const int64_t t_lo = tiles * blockIdx.y / slices, t_hi = tiles * (blockIdx.y + 1) / slices;
    if (tid < NN_T) {
        int q = tid < nr ? queries[q0 + tid] : -1;
        if (q >= n) {
            flag_error(st, GK_ERR_INVALID, (unsigned)(q0 + tid));
            q = -1;
        }
        rid[tid] = q;
        best[tid] = ~0ull;
    }
    for (int64_t t = t_lo; t < t_hi; t++) {
        const int64_t j0 = t * NN_T;
        __syncthreads();  // the previous tile's distances are read
        if (tid < NN_T)
            cid[tid] = j0 + tid < n ? (int)(j0 + tid) : -1;
        __syncthreads();
        tile_distances<NN_T, false, false>(X, d, ld, rid, cid, nr, xr, dt);
        __syncthreads();
        // warp w: queries w, w + 8, ..., the smallest key of the tile's samples other than the query
        for (int row = w; row < nr; row += RF_WARPS) {
            const int q = rid[row];
            uint64_t kmin = ~0ull;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int c = lane + 32 * h, j = cid[c];
                if (j >= 0 && j != q)
                    kmin = min(kmin, pack_key(dt[row * TL::DS + c], j));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                kmin = min(kmin, (uint64_t)__shfl_xor_sync(FULL_MASK, (unsigned long long)kmin, o));
            if (lane == 0 && kmin < best[row])
                best[row] = kmin;
        }
    }
    __syncthreads();
    if (tid < nr)
        part[(int64_t)(q0 + tid) * slices + blockIdx.y] = best[tid];
}

__global__ void k_nn_finish(const uint64_t *__restrict__ part, int m, int slices, const int32_t *__restrict__ queries,
                            int64_t n, const int32_t *__restrict__ g_idx, int kappa, int32_t *__restrict__ nn_idx,
                            float *__restrict__ nn_dist, unsigned long long *__restrict__ hits)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m)
        return;
    uint64_t k = ~0ull;
    for (int s = 0; s < slices; s++)
        k = min(k, part[(int64_t)q * slices + s]);
    const int qi = queries[q];
    const bool found = k != ~0ull && qi >= 0 && qi < n;
    const int id = found ? key_id(k) : -1;
    if (nn_idx)
        nn_idx[q] = id;
    if (nn_dist)
        nn_dist[q] = found ? key_dist(k) : __int_as_float(0x7f800000);
    if (found && __ldg(g_idx + (int64_t)qi * kappa) == id)
        atomicAdd(hits, 1ull);
}

template <typename XT>
static cudaError_t recall_t(const XT *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                            const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist, int64_t *hits,
                            void *scratch, DevStatus *st, cudaStream_t s)
{
    cudaError_t e = set_max_smem(reinterpret_cast<const void *>(k_nn_tiles<XT>), (int)NN_SMEM);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(hits, 0, sizeof(int64_t), s)) != cudaSuccess)
        return e;
    const int slices = recall_slices(n, m);
    uint64_t *part = static_cast<uint64_t *>(scratch);
    const dim3 grid((unsigned)nn_qblocks(m), (unsigned)slices);
    k_nn_tiles<XT><<<grid, RF_THREADS, NN_SMEM, s>>>(X, n, (int)d, ld, queries, m, slices, part, st);
    k_nn_finish<<<(m + 255) / 256, 256, 0, s>>>(part, m, slices, queries, n, g_idx, kappa, nn_idx, nn_dist,
                                                 reinterpret_cast<unsigned long long *>(hits));
    return cudaGetLastError();
}

cudaError_t launch_recall(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                          int32_t kappa, const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist,
                          int64_t *hits, void *scratch, DevStatus *st, cudaStream_t s)
{
    if (bf16)
        return recall_t(static_cast<const __nv_bfloat16 *>(X), n, d, ld, g_idx, kappa, queries, m, nn_idx, nn_dist,
                        hits, scratch, st, s);
    return recall_t(static_cast<const float *>(X), n, d, ld, g_idx, kappa, queries, m, nn_idx, nn_dist, hits, scratch,
                    st, s);
}

}  // namespace gkm
