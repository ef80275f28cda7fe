// Graph refinement inside clusters (Alg. 3: every pair of samples that share
// a cluster is compared, and the pair's distance updates both samples' rows),
// exact FP32.
//
// A cluster of m members (CSR, ascending id) larger than max_cluster is cut
// into ceil(m / max_cluster) runs of consecutive members whose sizes differ by
// at most one; pairs are formed inside a run only.  One block per cluster (the
// hardware hands clusters to SMs as blocks finish, which balances uneven
// cluster sizes).  Two instances of the kernel run back to back: a 64-wide
// tile for clusters whose runs hold at most 64 members (the common case, small
// shared memory, several blocks per SM) and a 128-wide tile for the others.
// A run is covered by T x T tiles (rows x columns of the run); for each tile
// the block stages 32 coordinates of the row and column samples at a time in
// shared memory and every thread accumulates a (T/16) x (T/16) set of pair
// distances (rows ty + 16 a, columns tx + 16 b) with one accumulator in
// ascending coordinate order (the order of pair_d2_seq), so a pair's distance
// has the same bits here, in the initial graph and in any later round.  Each
// warp then merges the tile's candidates into the graph rows of its rows:
// candidates that beat the row's kappa-th key and are not already in the row
// are compacted, ranked among themselves, located in the row by binary
// search, and the kappa smallest keys of the union are written back.  Every
// row belongs to exactly one run per refinement, so blocks never write the
// same row.
#include "common.cuh"

namespace gkm {

constexpr int RF_THREADS = 256;
constexpr int RF_WARPS = RF_THREADS / 32;
constexpr int RF_DK = 32;  // coordinates staged per step

template <int T>
struct RefineTile {
    static constexpr int XS = T + 1;  // padded stride of the staged coordinates
    static constexpr int DS = T + 1;  // padded stride of the distance tile
    static constexpr int Q = T / 16;  // pairs per thread along each axis
    // the distance tile reuses the staging buffers (written after the last stage)
    static constexpr size_t stage_floats = 2 * RF_DK * XS;
    static constexpr size_t tile_floats = (size_t)T * DS;
    static constexpr size_t fixed_bytes =
        sizeof(float) * (stage_floats > tile_floats ? stage_floats : tile_floats) + sizeof(int) * 2 * T;
    // per warp: row list (kappa ids + dists), candidates (T), new row (kappa)
    __host__ __device__ static size_t warp_bytes(int kappa)
    {
        return (sizeof(int) + sizeof(float)) * (size_t)(2 * kappa + T) + 4 * sizeof(unsigned);
    }
    __host__ __device__ static size_t smem_bytes(int kappa) { return fixed_bytes + RF_WARPS * warp_bytes(kappa); }
};

// Number of keys of (v, id)[0..len) smaller than (kv, kj); the array is sorted.
__device__ __forceinline__ int lower_rank(const float *v, const int *id, int len, float kv, int kj)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (key_less(v[mid], id[mid], kv, kj))
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Merge the candidates (ids cid[0..ncol), ascending; distances drow[0..ncol))
// into graph row i (kappa sorted keys at gi / gd).  Warp-cooperative.
// Candidates already in the row are found by a binary search of each row id
// among the (sorted) candidate ids and masked out; the others that beat the
// row's kappa-th key are ranked among themselves and placed by rank.
__device__ void merge_row(int i, const int *__restrict__ cid, const float *__restrict__ drow, int ncol, int kappa,
                          int32_t *__restrict__ gi, float *__restrict__ gd, int *li, float *lv, int *bi, float *bv,
                          int *ni, float *nv, unsigned *dup)
{
    const int lane = lane_id();
    if (lane < 4)
        dup[lane] = 0u;
    __syncwarp();
    for (int q = lane; q < kappa; q += 32) {
        const int j = gi[q];
        li[q] = j;
        lv[q] = gd[q];
        int lo = 0, hi = ncol;  // first candidate id >= j
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (cid[mid] < j)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo < ncol && cid[lo] == j)
            atomicOr(&dup[lo >> 5], 1u << (lo & 31));
    }
    __syncwarp();
    const float td = lv[kappa - 1];
    const int ti = li[kappa - 1];
    // candidates that would enter the row and are not in it yet
    int ns = 0;
    for (int c0 = 0; c0 < ncol; c0 += 32) {
        const int c = c0 + lane;
        bool ok = c < ncol;
        const int j = ok ? cid[c] : -1;
        const float dv = ok ? drow[c] : 0.f;
        ok = ok && j != i && ((dup[c0 >> 5] >> lane) & 1u) == 0u && key_less(dv, j, td, ti);
        const unsigned bal = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            const int p = ns + __popc(bal & lanemask_lt());
            bi[p] = j;
            bv[p] = dv;
        }
        ns += __popc(bal);
    }
    __syncwarp();
    if (ns == 0)
        return;
    // rank the candidates among themselves (keys are distinct: ids differ)
    int rk[4];
    float kvs[4];
    int kjs[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int b = lane + 32 * u;
        rk[u] = -1;
        if (b < ns) {
            kvs[u] = bv[b];
            kjs[u] = bi[b];
            int r = 0;
            for (int q = 0; q < ns; q++)
                r += key_less(bv[q], bi[q], kvs[u], kjs[u]) ? 1 : 0;
            rk[u] = r;
        }
    }
    __syncwarp();
    // place the sorted candidates in bi / bv, then merge with the row
#pragma unroll
    for (int u = 0; u < 4; u++) {
        if (rk[u] >= 0) {
            bi[rk[u]] = kjs[u];
            bv[rk[u]] = kvs[u];
        }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; u++) {
        if (rk[u] >= 0) {
            const int pos = rk[u] + lower_rank(lv, li, kappa, kvs[u], kjs[u]);
            if (pos < kappa) {
                ni[pos] = kjs[u];
                nv[pos] = kvs[u];
            }
        }
    }
    for (int a = lane; a < kappa; a += 32) {
        const float kv = lv[a];
        const int kj = li[a];
        const int pos = a + lower_rank(bv, bi, ns, kv, kj);
        if (pos < kappa) {
            ni[pos] = kj;
            nv[pos] = kv;
        }
    }
    __syncwarp();
    for (int q = lane; q < kappa; q += 32) {
        gi[q] = ni[q];
        gd[q] = nv[q];
    }
    __syncwarp();
}

// Runs of each cluster: ceil(m / cap) for m >= 2, else none.
__global__ void k_count_runs(const int32_t *__restrict__ off, int k, int cap, int32_t *__restrict__ nruns)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) {
        int m = off[r + 1] - off[r];
        nruns[r] = m >= 2 ? (m + cap - 1) / cap : 0;
    }
}

template <int T>
__global__ void __launch_bounds__(RF_THREADS) k_refine(const float *__restrict__ X, int64_t n, int d, int64_t ld,
                                                       const int32_t *__restrict__ off,
                                                       const int32_t *__restrict__ mem,
                                                       const int32_t *__restrict__ run_off, int k, int kappa,
                                                       int cap, int lo_run, int32_t *__restrict__ g_idx,
                                                       float *__restrict__ g_dist, DevStatus *st)
{
    using TL = RefineTile<T>;
    constexpr int XS = TL::XS, DS = TL::DS, Q = TL::Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *xr = reinterpret_cast<float *>(smem_raw);
    float *xc = xr + RF_DK * XS;
    float *dt = xr;  // aliases the staging buffers
    constexpr size_t span = TL::stage_floats > TL::tile_floats ? TL::stage_floats : TL::tile_floats;
    int *rid = reinterpret_cast<int *>(xr + span);
    int *cid = rid + T;
    const int tid = threadIdx.x, w = tid >> 5;
    unsigned char *wbase = reinterpret_cast<unsigned char *>(cid + T) + w * TL::warp_bytes(kappa);
    int *li = reinterpret_cast<int *>(wbase);
    float *lv = reinterpret_cast<float *>(li + kappa);
    int *ni = reinterpret_cast<int *>(lv + kappa);
    float *nv = reinterpret_cast<float *>(ni + kappa);
    int *bi = reinterpret_cast<int *>(nv + kappa);
    float *bv = reinterpret_cast<float *>(bi + T);
    unsigned *dup = reinterpret_cast<unsigned *>(bv + T);
    const int ty = tid >> 4, tx = tid & 15;

    // block `run` handles that run: find its cluster r, run_off[r] <= run < run_off[r + 1]
    const int run = blockIdx.x;
    if (run >= run_off[k])
        return;
    int lo = 0, hi = k;  // last r with run_off[r] <= run
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (run_off[mid] <= run)
            lo = mid;
        else
            hi = mid;
    }
    const int r = lo;
    const int beg = off[r], m = off[r + 1] - beg;
    const int nc = (m + cap - 1) / cap, base = m / nc, rem = m % nc;
    const int c = run - run_off[r];
    const int s0 = c * base + min(c, rem), sz = base + (c < rem ? 1 : 0);
    // the 64-wide instance (lo_run = 0) takes runs of <= 64 members, the
    // 128-wide instance (lo_run = 64) all longer runs
    const bool mine = lo_run == 0 ? sz <= T : sz > lo_run;
    if (!mine || sz < 2)
        return;
    {
        const int32_t *S = mem + beg + s0;
        for (int rb = 0; rb < sz; rb += T) {
            const int nr = min(T, sz - rb);
            for (int cb = 0; cb < sz; cb += T) {
                const int ncl = min(T, sz - cb);
                const bool same = rb == cb;
                __syncthreads();
                for (int q = tid; q < T; q += RF_THREADS) {
                    int a = q < nr ? S[rb + q] : -1;
                    int b = q < ncl ? S[cb + q] : -1;
                    if (a >= n || b >= n) {  // corrupt grouping: record, skip the sample
                        flag_error(st, GK_ERR_INVALID, (unsigned)r);
                        a = a >= n ? -1 : a;
                        b = b >= n ? -1 : b;
                    }
                    rid[q] = a;
                    cid[q] = b;
                }
                __syncthreads();
                const int nqr = (nr + 15) >> 4, nqc = (ncl + 15) >> 4;
                const float *xcs = same ? xr : xc;
                float acc[Q][Q];
#pragma unroll
                for (int a = 0; a < Q; a++)
#pragma unroll
                    for (int b = 0; b < Q; b++)
                        acc[a][b] = 0.f;
                for (int t0 = 0; t0 < d; t0 += RF_DK) {
                    // stage coordinates t0 .. t0+31 of the row (and column) samples, zero padded
                    for (int e = tid; e < T * RF_DK; e += RF_THREADS) {
                        int row = e / RF_DK, tt = e % RF_DK;
                        int t = t0 + tt;
                        int a = rid[row];
                        xr[tt * XS + row] = (a >= 0 && t < d) ? __ldg(X + (int64_t)a * ld + t) : 0.f;
                        if (!same) {
                            int b = cid[row];
                            xc[tt * XS + row] = (b >= 0 && t < d) ? __ldg(X + (int64_t)b * ld + t) : 0.f;
                        }
                    }
                    __syncthreads();
                    const int tmax = min(RF_DK, d - t0);
                    for (int tt = 0; tt < tmax; tt++) {
                        float vr[Q], vc[Q];
#pragma unroll
                        for (int q = 0; q < Q; q++) {
                            vr[q] = xr[tt * XS + ty + 16 * q];
                            vc[q] = xcs[tt * XS + tx + 16 * q];
                        }
#pragma unroll
                        for (int a = 0; a < Q; a++) {
                            if (a < nqr) {
#pragma unroll
                                for (int b = 0; b < Q; b++) {
                                    if (b < nqc) {
                                        float diff = vr[a] - vc[b];
                                        acc[a][b] = fmaf(diff, diff, acc[a][b]);
                                    }
                                }
                            }
                        }
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int a = 0; a < Q; a++)
#pragma unroll
                    for (int b = 0; b < Q; b++)
                        dt[(ty + 16 * a) * DS + tx + 16 * b] = acc[a][b];
                __syncthreads();
                for (int row = w; row < nr; row += RF_WARPS) {
                    int i = rid[row];
                    if (i < 0)
                        continue;
                    merge_row(i, cid, dt + row * DS, ncl, kappa, g_idx + (int64_t)i * kappa,
                              g_dist + (int64_t)i * kappa, li, lv, bi, bv, ni, nv, dup);
                }
            }
        }
    }
}

size_t refine_scratch_bytes(int32_t k)
{
    return ((size_t)(2 * (k + 1)) * sizeof(int32_t) + 255) / 256 * 256 + scan_scratch_bytes(k);
}

cudaError_t launch_refine(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster, int32_t *g_idx,
                          float *g_dist, void *scratch, DevStatus *st, cudaStream_t s)
{
    int32_t *nruns = static_cast<int32_t *>(scratch);
    int32_t *run_off = nruns + (k + 1);
    void *sc = static_cast<char *>(scratch) + ((size_t)(2 * (k + 1)) * sizeof(int32_t) + 255) / 256 * 256;
    size_t shm64 = RefineTile<64>::smem_bytes(kappa), shm128 = RefineTile<128>::smem_bytes(kappa);
    cudaError_t e = cudaFuncSetAttribute(k_refine<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm64);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_refine<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm128)) !=
        cudaSuccess)
        return e;
    k_count_runs<<<(k + 255) / 256 < 1024 ? (k + 255) / 256 : 1024, 256, 0, s>>>(offsets, k, max_cluster, nruns);
    if ((e = launch_scan(nruns, run_off, k, sc, s)) != cudaSuccess)
        return e;
    // an upper bound of the number of runs: sum over clusters of (m / cap + 1)
    const int64_t grid = (int64_t)k + n / max_cluster + 1;
    // runs of <= 64 members, then the longer runs (up to 128 per tile, longer runs in tiles)
    k_refine<64><<<(unsigned)grid, RF_THREADS, shm64, s>>>(X, n, (int)d, ld, offsets, members, run_off, k, kappa,
                                                           max_cluster, 0, g_idx, g_dist, st);
    k_refine<128><<<(unsigned)grid, RF_THREADS, shm128, s>>>(X, n, (int)d, ld, offsets, members, run_off, k, kappa,
                                                             max_cluster, 64, g_idx, g_dist, st);
    return cudaGetLastError();
}

}  // namespace gkm
