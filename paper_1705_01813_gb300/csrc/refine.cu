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
// shared memory (the row samples twice over, as broadcast pairs) and every
// thread accumulates the pair distances of Q = T/16 consecutive rows and Q
// consecutive columns, two columns at a time in packed FP32x2 FMAs (the
// difference as fma(y, -1, x), then fma(e, e, acc): per pair the operations of
// pair_d2_seq), with one accumulator in ascending coordinate order, so a
// pair's distance has the same bits here, in the initial graph and in any
// later round.  Each
// warp then merges the tile's candidates into the graph rows of its rows:
// candidates that beat the row's kappa-th key and are not already in the row
// are compacted, ranked among themselves, located in the row by binary
// search (all on 64-bit packed keys), and the kappa smallest keys of the union
// are written back.  Every
// row belongs to exactly one run per refinement, so blocks never write the
// same row.
#include "common.cuh"
#include "merge.cuh"
#include "tiles.cuh"

#include <type_traits>

namespace gkm {

// Cluster of every run: run_cl[run_off[r] + c] = r for c < nruns[r].
__global__ void k_run_clusters(const int32_t *__restrict__ run_off, int k, int32_t *__restrict__ run_cl)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x)
        for (int q = run_off[r]; q < run_off[r + 1]; q++)
            run_cl[q] = r;
}

// Runs of each cluster: ceil(m / cap) for m >= 2, else none.
__global__ void k_count_runs(const int32_t *__restrict__ off, int k, int cap, int32_t *__restrict__ nruns)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) {
        int m = off[r + 1] - off[r];
        nruns[r] = m >= 2 ? (m + cap - 1) / cap : 0;
    }
}

template <int T, typename XT, bool VEC>
__global__ void __launch_bounds__(RF_THREADS, T == 64 ? 3 : 2) k_refine(const XT *__restrict__ X, int64_t n, int d, int64_t ld,
                                                       const int32_t *__restrict__ off,
                                                       const int32_t *__restrict__ mem,
                                                       const int32_t *__restrict__ run_off,
                                                       const int32_t *__restrict__ run_cl, int k, int kappa,
                                                       int cap, int lo_run, int32_t *__restrict__ g_idx,
                                                       float *__restrict__ g_dist, DevStatus *st)
{
    using TL = RefineTile<T>;
    constexpr int DS = TL::DS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *xr = reinterpret_cast<float *>(smem_raw);  // staging buffers of the pair tiles (tiles.cuh)
    float *dt = xr;  // aliases the staging buffers
    constexpr size_t span = TL::stage_floats > TL::tile_floats ? TL::stage_floats : TL::tile_floats;
    int *rid = reinterpret_cast<int *>(xr + span);
    int *cid = rid + T;
    const int tid = threadIdx.x, w = tid >> 5;
    unsigned char *wbase = reinterpret_cast<unsigned char *>(cid + T) + w * TL::warp_bytes(kappa);
    uint64_t *rk = reinterpret_cast<uint64_t *>(wbase);
    uint64_t *nk = rk + kappa;
    uint64_t *bk = nk + kappa;
    unsigned *dup = reinterpret_cast<unsigned *>(bk + T);

    // block `run` handles that run: find its cluster r, run_off[r] <= run < run_off[r + 1]
    const int run = blockIdx.x;
    if (run >= run_off[k])
        return;
    const int r = run_cl[run];
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
                if (same)
                    tile_distances<T, true, VEC>(X, d, ld, rid, cid, nr, xr, dt);
                else
                    tile_distances<T, false, VEC>(X, d, ld, rid, cid, nr, xr, dt);
                __syncthreads();
                RowRegs cur, nxt;
                if (w < nr && rid[w] >= 0)
                    load_row(cur, g_idx + (int64_t)rid[w] * kappa, g_dist + (int64_t)rid[w] * kappa, kappa);
                for (int row = w; row < nr; row += RF_WARPS) {
                    const int i = rid[row];
                    const int rn = row + RF_WARPS;
                    if (rn < nr && rid[rn] >= 0)  // next row's list in flight during this merge
                        load_row(nxt, g_idx + (int64_t)rid[rn] * kappa, g_dist + (int64_t)rid[rn] * kappa, kappa);
                    if (i >= 0)
                        merge_row(i, cid, dt + row * DS, ncl, kappa, cur, g_idx + (int64_t)i * kappa,
                                  g_dist + (int64_t)i * kappa, rk, bk, nk, dup);
                    cur = nxt;
                }
            }
        }
    }
}

// Runs of at most 64 members, warp-specialised: a persistent block takes runs blockIdx.x, + gridDim.x, ...; five
// of its nine warps (the compute group, WS_NC threads, rotated over the block's warps by blockIdx.x so that the
// blocks of an SM spread them over its four schedulers) stage and compute a run's pair tile while the other four
// merge the previous run's rows.  The two hand the distance tile over through named barriers: FULL (the compute group
// arrives when the tile and the run's ids are written, the merge warps wait) and EMPTY (the merge warps arrive
// when they no longer read it, the compute group waits before writing the next one).  Both sides walk the same
// runs with the same skips, so the barriers pair up: per run one FULL and one EMPTY phase, plus the EMPTY phase
// the merge warps open before the first run and the compute group closes after the last.  Pair arithmetic,
// merge order and results are those of k_refine<64>.
constexpr int WS_NC = 160;  // compute group: 5 warps, covers the 136 pair blocks of a 64-row triangle
constexpr int WS_NM = 4;    // merge warps
constexpr int WS_THREADS = WS_NC + 32 * WS_NM;
constexpr int WS_BAR_C = 1, WS_BAR_FULL = 2, WS_BAR_EMPTY = 3;

// dynamic shared memory: two stage buffers, the distance tile, the run ids of two runs, the merge warps' buffers
__host__ __device__ inline size_t refine_ws_smem_bytes(int kappa)
{
    using TL = RefineTile<64>;
    return sizeof(float) * (TL::stage_floats + TL::tile_floats) + sizeof(int) * 2 * 64 + WS_NM * TL::warp_bytes(kappa);
}

template <typename XT, bool VEC>
__global__ void __launch_bounds__(WS_THREADS, 3) k_refine_ws(const XT *__restrict__ X, int64_t n, int d, int64_t ld,
                                                             const int32_t *__restrict__ off,
                                                             const int32_t *__restrict__ mem,
                                                             const int32_t *__restrict__ run_off,
                                                             const int32_t *__restrict__ run_cl, int k, int kappa,
                                                             int cap, int32_t *__restrict__ g_idx,
                                                             float *__restrict__ g_dist, DevStatus *st)
{
    constexpr int T = 64;
    using TL = RefineTile<T>;
    constexpr int DS = TL::DS, Q = TL::Q;
    constexpr int WARPS = WS_THREADS / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *stage = reinterpret_cast<float *>(smem_raw);
    float *dt = stage + TL::stage_floats;
    int *rids = reinterpret_cast<int *>(dt + TL::tile_floats);  // [2][T]: the ids of runs j and j + 1
    unsigned char *mbase = reinterpret_cast<unsigned char *>(rids + 2 * T);
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int rr = (w + WARPS - (int)(blockIdx.x & 3)) % WARPS;  // 0 .. 4: compute group, 5 .. 8: merge warps
    const int nruns = run_off[k];
    // run `run`: its cluster, first member (in mem) and size, as k_refine cuts clusters into runs
    auto geometry = [&](int run, int &r, int &first, int &sz) {
        r = run_cl[run];
        const int beg = off[r], m = off[r + 1] - beg;
        const int nc = (m + cap - 1) / cap, base = m / nc, rem = m % nc;
        const int c = run - run_off[r];
        first = beg + c * base + min(c, rem);
        sz = base + (c < rem ? 1 : 0);
    };
    if (rr < 5) {
        // ---- compute group ----
        const int ct = rr * 32 + lane;
        int j = 0;
        for (int run = blockIdx.x; run < nruns; run += gridDim.x) {
            int r, first, sz;
            geometry(run, r, first, sz);
            if (sz < 2 || sz > T)
                continue;  // a run of the 128-wide kernel, or no pairs: skipped alike by the merge warps
            int *rid = rids + (j & 1) * T;
            if (ct < T) {
                int a = ct < sz ? mem[first + ct] : -1;
                if (a >= n) {  // corrupt grouping: record, skip the sample
                    flag_error(st, GK_ERR_INVALID, (unsigned)r);
                    a = -1;
                }
                rid[ct] = a;  // the merges of run j - 2, which read this slot, ended before EMPTY of run j - 1
            }
            bar_sync(WS_BAR_C, WS_NC);
            float2 acc[Q][Q / 2];
            int by, bx;
            const bool live = tile_distances_group<WS_NC, VEC>(X, d, ld, rid, sz, stage, ct, WS_BAR_C, acc, by, bx);
            bar_sync(WS_BAR_EMPTY, WS_THREADS);  // the merge warps no longer read the distance tile
            if (live) {
#pragma unroll
                for (int a = 0; a < Q; a++)
#pragma unroll
                    for (int b = 0; b < Q / 2; b++) {
                        dt[(Q * by + a) * DS + Q * bx + 2 * b] = acc[a][b].x;
                        dt[(Q * by + a) * DS + Q * bx + 2 * b + 1] = acc[a][b].y;
                        if (by != bx) {
                            dt[(Q * bx + 2 * b) * DS + Q * by + a] = acc[a][b].x;
                            dt[(Q * bx + 2 * b + 1) * DS + Q * by + a] = acc[a][b].y;
                        }
                    }
            }
            __threadfence_block();
            bar_arrive(WS_BAR_FULL, WS_THREADS);  // this run's ids and distance tile are in place
            j++;
        }
        bar_sync(WS_BAR_EMPTY, WS_THREADS);  // the merge warps' arrival after the last run
    } else {
        // ---- merge warps ----
        const int mw = rr - 5;
        unsigned char *wb = mbase + mw * TL::warp_bytes(kappa);
        uint64_t *rk = reinterpret_cast<uint64_t *>(wb);
        uint64_t *nk = rk + kappa;
        uint64_t *bk = nk + kappa;
        unsigned *dup = reinterpret_cast<unsigned *>(bk + T);
        bar_arrive(WS_BAR_EMPTY, WS_THREADS);  // the distance tile starts free
        int j = 0;
        for (int run = blockIdx.x; run < nruns; run += gridDim.x) {
            int r, first, sz;
            geometry(run, r, first, sz);
            if (sz < 2 || sz > T)
                continue;
            const int *rid = rids + (j & 1) * T;
            bar_sync(WS_BAR_FULL, WS_THREADS);  // run j's ids and distances
            RowRegs cur, nxt;
            if (mw < sz && rid[mw] >= 0)
                load_row(cur, g_idx + (int64_t)rid[mw] * kappa, g_dist + (int64_t)rid[mw] * kappa, kappa);
            for (int row = mw; row < sz; row += WS_NM) {
                const int i = rid[row];
                const int rn = row + WS_NM;
                if (rn < sz && rid[rn] >= 0)  // next row's list in flight during this merge
                    load_row(nxt, g_idx + (int64_t)rid[rn] * kappa, g_dist + (int64_t)rid[rn] * kappa, kappa);
                if (i >= 0)
                    merge_row(i, rid, dt + row * DS, sz, kappa, cur, g_idx + (int64_t)i * kappa,
                              g_dist + (int64_t)i * kappa, rk, bk, nk, dup);
                cur = nxt;
            }
            __threadfence_block();
            bar_arrive(WS_BAR_EMPTY, WS_THREADS);  // done with the distance tile and this slot of ids
            j++;
        }
    }
}

static size_t run_bytes(int32_t k) { return ((size_t)(2 * (k + 1)) * sizeof(int32_t) + 255) / 256 * 256; }
// runs per refinement are at most k + n / max_cluster (max_cluster >= 2)
static size_t run_cl_bytes(int64_t n, int32_t k) { return ((size_t)(k + n / 2 + 1) * sizeof(int32_t) + 255) / 256 * 256; }

size_t refine_scratch_bytes(int64_t n, int32_t k, int64_t d)
{
    return run_bytes(k) + run_cl_bytes(n, k) + scan_scratch_bytes(k) + refine_tc_scratch_bytes(n, k, d);
}

template <typename XT, bool VEC>
static cudaError_t refine_tv(const XT *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                            const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster, int32_t *g_idx,
                            float *g_dist, void *scratch, DevStatus *st, cudaStream_t s, int precision)
{
    int32_t *nruns = static_cast<int32_t *>(scratch);
    int32_t *run_off = nruns + (k + 1);
    int32_t *run_cl = reinterpret_cast<int32_t *>(static_cast<char *>(scratch) + run_bytes(k));
    void *sc = static_cast<char *>(scratch) + run_bytes(k) + run_cl_bytes(n, k);
    void *tc_scratch = static_cast<char *>(sc) + scan_scratch_bytes(k);
    const size_t shm64 = RefineTile<64>::smem_bytes(kappa), shm128 = RefineTile<128>::smem_bytes(kappa),
                 shm_ws = refine_ws_smem_bytes(kappa);
    cudaError_t e;
    if constexpr (VEC)
        e = set_max_smem(reinterpret_cast<const void *>(k_refine_ws<XT, VEC>), (int)refine_ws_smem_bytes(MAX_KAPPA));
    else
        e = set_max_smem(reinterpret_cast<const void *>(k_refine<64, XT, VEC>),
                         (int)RefineTile<64>::smem_bytes(MAX_KAPPA));
    if (e != cudaSuccess)
        return e;
    if ((e = set_max_smem(reinterpret_cast<const void *>(k_refine<128, XT, VEC>),
                          (int)RefineTile<128>::smem_bytes(MAX_KAPPA))) != cudaSuccess)
        return e;
    k_count_runs<<<(k + 255) / 256 < 1024 ? (k + 255) / 256 : 1024, 256, 0, s>>>(offsets, k, max_cluster, nruns);
    if ((e = launch_scan(nruns, run_off, k, sc, s)) != cudaSuccess)
        return e;
    k_run_clusters<<<(k + 255) / 256 < 1024 ? (k + 255) / 256 : 1024, 256, 0, s>>>(run_off, k, run_cl);
    // an upper bound of the number of runs: sum over clusters of (m / cap + 1)
    const int64_t grid = (int64_t)k + n / max_cluster + 1;
    // The tensor-core path for 64 <= d <= 128.  Its Gram is exact only for integer data with 2 d 255^2 < 2^24
    // (d <= 128), and wider rows made the recompute of every kept pair dearer than the FP32 tile kernels
    // (1M x 960 FP32: 91 ms against 25 ms per call; 10M x 512 BF16 unit vectors, whose Gram carries no BF16
    // rounding but of whose pairs about 45% may enter a row in every round: 106 ms against 86 ms); for d < 64 the
    // tile kernels'
    // cost, proportional to d, is below the fixed per-run cost of the Gram path (20k x 32: 0.18 ms against
    // 0.12 ms per call).
    if (precision >= 1 && d >= 64 && d <= 128) {
        // tensor-core Gram for runs of <= 128 members, the FP32 kernel for longer runs
        constexpr bool bf16 = std::is_same_v<XT, __nv_bfloat16>;
        if ((e = launch_refine_tc(X, bf16, n, d, ld, offsets, members, run_off, run_cl, k, kappa, max_cluster, grid,
                                  g_idx, g_dist, tc_scratch, st, s)) != cudaSuccess)
            return e;
        if (max_cluster > 128)
            k_refine<128, XT, VEC><<<(unsigned)grid, RF_THREADS, shm128, s>>>(X, n, (int)d, ld, offsets, members, run_off,
                                                                     run_cl, k, kappa, max_cluster, 128, g_idx,
                                                                     g_dist, st);
        return cudaGetLastError();
    }
    // runs of <= 64 members, then the longer runs (up to 128 per tile, longer runs in tiles).  Rows staged by
    // 16-byte loads take the persistent warp-specialised kernel (one wave of blocks; 10M x 512 BF16: 32.0 ->
    // 31.3 ms per call, 98 -> 75 ms for runs of about ten); rows staged element by element keep the block per
    // run, where five warps' share of the element loads made the specialised form slower (1M x 960 FP32: 7.6
    // against 7.7 ms; 1M x 128 FP32: 3.7 against 3.9 ms)
    if constexpr (VEC) {
        int wgrid = 0;
        if ((e = resident_grid(reinterpret_cast<const void *>(k_refine_ws<XT, VEC>), WS_THREADS, shm_ws, &wgrid)) !=
            cudaSuccess)
            return e;
        k_refine_ws<XT, VEC><<<(unsigned)(grid < wgrid ? grid : wgrid), WS_THREADS, shm_ws, s>>>(
            X, n, (int)d, ld, offsets, members, run_off, run_cl, k, kappa, max_cluster, g_idx, g_dist, st);
    } else {
        (void)shm_ws;
        k_refine<64, XT, VEC><<<(unsigned)grid, RF_THREADS, shm64, s>>>(X, n, (int)d, ld, offsets, members, run_off,
                                                                        run_cl, k, kappa, max_cluster, 0, g_idx,
                                                                        g_dist, st);
    }
    k_refine<128, XT, VEC><<<(unsigned)grid, RF_THREADS, shm128, s>>>(X, n, (int)d, ld, offsets, members, run_off, run_cl, k,
                                                             kappa, max_cluster, 64, g_idx, g_dist, st);
    return cudaGetLastError();
}

// the tile kernels with 16-byte stage loads where the rows allow them, for BF16 rows (eight elements per load
// instead of one 2-byte load each; FP32 rows keep the element loads, whose kernel uses fewer registers)
template <typename XT>
static cudaError_t refine_t(const XT *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                            const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster, int32_t *g_idx,
                            float *g_dist, void *scratch, DevStatus *st, cudaStream_t s, int precision)
{
    if (std::is_same_v<XT, __nv_bfloat16> && tile_vec16(X, (int)d, ld))
        return refine_tv<XT, true>(X, n, d, ld, offsets, members, k, kappa, max_cluster, g_idx, g_dist, scratch, st, s,
                                   precision);
    return refine_tv<XT, false>(X, n, d, ld, offsets, members, k, kappa, max_cluster, g_idx, g_dist, scratch, st, s,
                                precision);
}

cudaError_t launch_refine(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster, int32_t *g_idx,
                          float *g_dist, void *scratch, DevStatus *st, cudaStream_t s, int precision)
{
    if (bf16)
        return refine_t(static_cast<const __nv_bfloat16 *>(X), n, d, ld, offsets, members, k, kappa, max_cluster,
                        g_idx, g_dist, scratch, st, s, precision);
    return refine_t(static_cast<const float *>(X), n, d, ld, offsets, members, k, kappa, max_cluster, g_idx, g_dist,
                    scratch, st, s, precision);
}

}  // namespace gkm
