// Grouping of samples by cluster label: the cluster set S of Alg. 1/3 as a
// CSR (offsets[k + 1], members[n]) with the members of each cluster in
// ascending sample id.  Built as a stable LSD radix sort of the labels
// (8-bit digits, as many passes as k - 1 has bytes) whose values are the
// sample ids, plus a label histogram and an exclusive scan for the offsets.
#include "common.cuh"

namespace gkm {

// --------------------------------------------------------------------------
// Exclusive scan of int32 (three phases: block sums, scan of the block sums
// in one block, block-local scans with the block's offset).
// --------------------------------------------------------------------------
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 16;
constexpr int SC_CHUNK = SC_THREADS * SC_ITEMS;  // 4096
constexpr int SC_MAX_BLOCKS = 4096;              // one block scans the partials in chunks

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= o)
            v += u;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
template <int THREADS>
__device__ __forceinline__ int block_excl_scan(int v, int *total)
{
    __shared__ int s_warp[THREADS / 32];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31)
        s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < THREADS / 32 ? s_warp[lane] : 0;
        int ti = warp_incl_scan(t);
        if (lane < THREADS / 32)
            s_warp[lane] = ti - t;
        if (lane == THREADS / 32 - 1)
            *total = ti;  // caller passes shared memory
    }
    __syncthreads();
    int r = s_warp[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const int32_t *__restrict__ in, int64_t count,
                                                            int32_t *__restrict__ partial)
{
    int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
    int s = 0;
    for (int q = 0; q < SC_ITEMS; q++) {
        int64_t e = base + (int64_t)q * SC_THREADS + threadIdx.x;
        if (e < count)
            s += in[e];
    }
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(FULL_MASK, s, o);
    __shared__ int s_w[SC_THREADS / 32];
    if (lane_id() == 0)
        s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < SC_THREADS / 32; w++)
            t += s_w[w];
        partial[blockIdx.x] = t;
    }
}

// One block: exclusive scan of nb partials in place; out_total receives the sum.
__global__ void __launch_bounds__(1024) k_scan_partials(int32_t *__restrict__ partial, int nb,
                                                        int32_t *__restrict__ out_total)
{
    __shared__ int s_total;
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int b = b0 + threadIdx.x;
        int v = b < nb ? partial[b] : 0;
        int ex = block_excl_scan<1024>(v, &s_total);
        if (b < nb)
            partial[b] = carry + ex;
        carry += s_total;
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *out_total = carry;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_down(const int32_t *__restrict__ in, int64_t count,
                                                          const int32_t *__restrict__ partial,
                                                          int32_t *__restrict__ out)
{
    __shared__ int s_total;
    int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS];
    int s = 0;
#pragma unroll
    for (int q = 0; q < SC_ITEMS; q++) {
        int64_t e = base + q;
        v[q] = e < count ? in[e] : 0;
        s += v[q];
    }
    int ex = block_excl_scan<SC_THREADS>(s, &s_total) + partial[blockIdx.x];
#pragma unroll
    for (int q = 0; q < SC_ITEMS; q++) {
        int64_t e = base + q;
        if (e < count)
            out[e] = ex;
        ex += v[q];
    }
}

size_t scan_scratch_bytes(int64_t count)
{
    int64_t nb = (count + SC_CHUNK - 1) / SC_CHUNK;
    return (size_t)((nb + 1) * sizeof(int32_t) + 255) & ~size_t(255);
}

cudaError_t launch_scan(const int32_t *in, int32_t *out, int64_t count, void *scratch, cudaStream_t s)
{
    int64_t nb = (count + SC_CHUNK - 1) / SC_CHUNK;
    if (nb < 1)
        nb = 1;
    if (nb > SC_MAX_BLOCKS * 1024)
        return cudaErrorInvalidValue;
    int32_t *partial = static_cast<int32_t *>(scratch);
    k_scan_reduce<<<(unsigned)nb, SC_THREADS, 0, s>>>(in, count, partial);
    k_scan_partials<<<1, 1024, 0, s>>>(partial, (int)nb, out + count);
    k_scan_down<<<(unsigned)nb, SC_THREADS, 0, s>>>(in, count, partial, out);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Label histogram (cluster sizes n_r), with the range check of the labels.
// --------------------------------------------------------------------------
__global__ void k_label_count(const int32_t *__restrict__ labels, int64_t n, int32_t k, int32_t *__restrict__ counts,
                              DevStatus *st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = labels[i];
        if ((unsigned)r >= (unsigned)k) {
            flag_error(st, GK_ERR_INVALID, (unsigned)i);
            continue;
        }
        atomicAdd(&counts[r], 1);
    }
}

// --------------------------------------------------------------------------
// Stable LSD radix sort passes over 8-bit digits of the label.
// A tile of RS_TILE consecutive elements is owned by one block; inside it warp
// w owns the RS_ITEMS * 32 consecutive elements starting at w * RS_ITEMS * 32
// and walks them 32 at a time, so rank order inside a tile is element order.
// --------------------------------------------------------------------------
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__device__ __forceinline__ int digit_of(int32_t key, int shift) { return (int)(((uint32_t)key >> shift) & (RADIX - 1)); }

// The sort key of a label: a label outside [0, k) sorts as k, after every
// cluster, so that it cannot shift the member ranges of the valid clusters
// (the label count leaves it out of every cluster and records it in the status
// word).  The passes cover the bits of k itself for this reason.
__device__ __forceinline__ int32_t sort_key(int32_t label, int32_t k)
{
    return (uint32_t)label < (uint32_t)k ? label : k;
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const int32_t *__restrict__ keys, int64_t n, int32_t k,
                                                           int shift, int32_t *__restrict__ tile_hist, int ntiles)
{
    __shared__ int h[RADIX];
    for (int b = threadIdx.x; b < RADIX; b += RS_THREADS)
        h[b] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int q = threadIdx.x; q < RS_TILE; q += RS_THREADS) {
        int64_t e = base + q;
        if (e < n)
            atomicAdd(&h[digit_of(sort_key(keys[e], k), shift)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < RADIX; b += RS_THREADS)
        tile_hist[(int64_t)b * ntiles + blockIdx.x] = h[b];
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const int32_t *__restrict__ keys_in,
                                                              const int32_t *__restrict__ vals_in, int64_t n,
                                                              int32_t k, int shift,
                                                              const int32_t *__restrict__ tile_off,
                                                              int ntiles, int32_t *__restrict__ keys_out,
                                                              int32_t *__restrict__ vals_out)
{
    __shared__ int whist[RS_WARPS][RADIX];
    for (int b = threadIdx.x; b < RS_WARPS * RADIX; b += RS_THREADS)
        (&whist[0][0])[b] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (RS_ITEMS * 32);
    int key[RS_ITEMS], val[RS_ITEMS], dig[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        int64_t e = wbase + r * 32 + lane;
        bool valid = e < n;
        key[r] = valid ? sort_key(keys_in[e], k) : 0;
        val[r] = valid ? (vals_in ? vals_in[e] : (int)e) : 0;
        int dg = valid ? digit_of(key[r], shift) : RADIX;
        dig[r] = dg;
        unsigned peers = __match_any_sync(FULL_MASK, dg);
        int base = dg < RADIX ? whist[w][dg] : 0;
        rank[r] = base + __popc(peers & lanemask_lt());
        __syncwarp();
        if (dg < RADIX && (peers & lanemask_lt()) == 0u)
            whist[w][dg] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int b = threadIdx.x; b < RADIX; b += RS_THREADS) {
        int run = 0;
        for (int q = 0; q < RS_WARPS; q++) {
            int t = whist[q][b];
            whist[q][b] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        int dg = dig[r];
        if (dg < RADIX) {
            int pos = tile_off[(int64_t)dg * ntiles + blockIdx.x] + whist[w][dg] + rank[r];
            if (keys_out)
                keys_out[pos] = key[r];
            vals_out[pos] = val[r];
        }
    }
}

// 8-bit passes that cover every sort key 0..k (k: the key of an out-of-range label)
static int radix_passes(int32_t k)
{
    uint32_t top = (uint32_t)k;
    int bits = 0;
    while (top) {
        bits++;
        top >>= 1;
    }
    return (bits + RADIX_BITS - 1) / RADIX_BITS;
}

size_t group_scratch_bytes(int64_t n, int32_t k)
{
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    int64_t hist = (int64_t)RADIX * ntiles;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += (bytes + 255) & ~size_t(255); };
    add(sizeof(int32_t) * (size_t)k);           // counts (when the caller keeps none)
    add(sizeof(int32_t) * (size_t)n * 4);        // keys / values, two buffers each
    add(sizeof(int32_t) * (size_t)(hist + 1));   // tile histogram, scanned in place
    size_t sc = scan_scratch_bytes(hist > (int64_t)k ? hist : (int64_t)k);
    add(sc);
    return b;
}

cudaError_t launch_group(const int32_t *labels, int64_t n, int32_t k, int32_t *offsets, int32_t *members,
                         int32_t *counts_out, void *scratch, DevStatus *st, cudaStream_t s)
{
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    int64_t hist = (int64_t)RADIX * ntiles;
    Carver cv{static_cast<char *>(scratch), 0, 0};
    int32_t *counts_tmp = cv.take<int32_t>((size_t)k);
    int32_t *kbuf0 = cv.take<int32_t>((size_t)n);
    int32_t *kbuf1 = cv.take<int32_t>((size_t)n);
    int32_t *vbuf0 = cv.take<int32_t>((size_t)n);
    int32_t *vbuf1 = cv.take<int32_t>((size_t)n);
    int32_t *thist = cv.take<int32_t>((size_t)(hist + 1));
    void *sc = cv.take<char>(scan_scratch_bytes(hist > (int64_t)k ? hist : (int64_t)k));
    int32_t *counts = counts_out ? counts_out : counts_tmp;
    cudaError_t e;

    // cluster sizes and offsets
    if ((e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)k, s)) != cudaSuccess)
        return e;
    {
        int64_t blocks = (n + 255) / 256;
        if (blocks > 152 * 16)
            blocks = 152 * 16;
        k_label_count<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(labels, n, k, counts, st);
    }
    if ((e = launch_scan(counts, offsets, k, sc, s)) != cudaSuccess)
        return e;

    // members: stable sort of ids by label
    const int passes = radix_passes(k);  // at least one (k >= 1)
    const int32_t *kin = labels;
    const int32_t *vin = nullptr;
    for (int p = 0; p < passes; p++) {
        bool last = p == passes - 1;
        int32_t *kout = last ? nullptr : (p & 1 ? kbuf1 : kbuf0);
        int32_t *vout = last ? members : (p & 1 ? vbuf1 : vbuf0);
        int shift = p * RADIX_BITS;
        k_radix_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(kin, n, k, shift, thist, (int)ntiles);
        if ((e = launch_scan(thist, thist, hist, sc, s)) != cudaSuccess)
            return e;
        k_radix_scatter<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(kin, vin, n, k, shift, thist, (int)ntiles, kout,
                                                                vout);
        kin = kout;
        vin = vout;
    }
    return cudaGetLastError();
}

}  // namespace gkm
