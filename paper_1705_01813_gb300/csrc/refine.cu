// Graph refinement inside clusters (Alg. 3: every pair of samples that share
// a cluster is compared, and the pair's distance updates both samples' rows),
// exact FP32.
//
// A cluster of m members (CSR, ascending id) larger than max_cluster is cut
// into ceil(m / max_cluster) runs of consecutive members whose sizes differ by
// at most one; pairs are formed inside a run only.  One block per cluster
// walks its runs; a run is covered by 128 x 128 tiles (rows x columns of the
// run).  For each tile the block stages 32 coordinates of the 128 row samples
// and the 128 column samples in shared memory at a time and every thread
// accumulates an 8 x 8 set of pair distances (rows ty + 16 q, columns
// tx + 16 q') with the one-accumulator, ascending-coordinate order of
// pair_d2_seq, so that a pair's distance has the same bits here, in the
// initial graph and in any later round.  Each warp then merges the tile's
// candidates into the graph rows of its rows: candidates that beat the row's
// kappa-th key and are not already in the row are compacted, and the new row
// is the kappa smallest keys of the union, placed by rank.  Every row belongs
// to exactly one run per refinement, so blocks never write the same row.
#include "common.cuh"

namespace gkm {

constexpr int RF_THREADS = 256;
constexpr int RF_WARPS = RF_THREADS / 32;
constexpr int RF_T = 128;     // tile edge (rows and columns of a run per tile)
constexpr int RF_DK = 32;     // coordinates staged per step
constexpr int RF_XS = RF_T + 1;   // padded stride of the staged coordinates
constexpr int RF_DS = RF_T + 1;   // padded stride of the distance tile

struct RefineSmem {
    float xr[RF_DK * RF_XS];
    float xc[RF_DK * RF_XS];
    float dt[RF_T * RF_DS];
    int rid[RF_T];
    int cid[RF_T];
    int li[RF_WARPS][MAX_KAPPA];
    float lv[RF_WARPS][MAX_KAPPA];
    int bi[RF_WARPS][RF_T];
    float bv[RF_WARPS][RF_T];
    int ni[RF_WARPS][MAX_KAPPA];
    float nv[RF_WARPS][MAX_KAPPA];
};

// Merge the candidates (cand ids cid[0..ncol), distances drow[0..ncol)) into
// graph row i.  Warp-cooperative.
__device__ void merge_row(int i, const int *__restrict__ cid, const float *__restrict__ drow, int ncol, int kappa,
                          int32_t *__restrict__ gi, float *__restrict__ gd, int *li, float *lv, int *bi, float *bv,
                          int *ni, float *nv)
{
    const int lane = lane_id();
    for (int q = lane; q < kappa; q += 32) {
        li[q] = gi[q];
        lv[q] = gd[q];
    }
    __syncwarp();
    const float td = lv[kappa - 1];
    const int ti = li[kappa - 1];
    int ns = 0;
    for (int c0 = 0; c0 < ncol; c0 += 32) {
        int c = c0 + lane;
        bool ok = c < ncol;
        int j = ok ? cid[c] : -1;
        float dv = ok ? drow[c] : 0.f;
        ok = ok && j != i && key_less(dv, j, td, ti);
        if (ok)
            for (int q = 0; q < kappa; q++)
                if (li[q] == j) {
                    ok = false;
                    break;
                }
        unsigned bal = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            int p = ns + __popc(bal & lanemask_lt());
            bi[p] = j;
            bv[p] = dv;
        }
        ns += __popc(bal);
    }
    __syncwarp();
    if (ns == 0)
        return;
    for (int b = lane; b < ns; b += 32) {
        float kv = bv[b];
        int kj = bi[b];
        int pos = 0;
        for (int q = 0; q < kappa; q++)
            pos += key_less(lv[q], li[q], kv, kj) ? 1 : 0;
        for (int q = 0; q < ns; q++)
            pos += key_less(bv[q], bi[q], kv, kj) ? 1 : 0;
        if (pos < kappa) {
            ni[pos] = kj;
            nv[pos] = kv;
        }
    }
    for (int a = lane; a < kappa; a += 32) {
        float kv = lv[a];
        int kj = li[a];
        int pos = a;
        for (int q = 0; q < ns; q++)
            pos += key_less(bv[q], bi[q], kv, kj) ? 1 : 0;
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

__global__ void __launch_bounds__(RF_THREADS) k_refine(const float *__restrict__ X, int64_t n, int d, int64_t ld,
                                                       const int32_t *__restrict__ off,
                                                       const int32_t *__restrict__ mem, int k, int kappa, int cap,
                                                       int32_t *__restrict__ g_idx, float *__restrict__ g_dist,
                                                       DevStatus *st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RefineSmem &sm = *reinterpret_cast<RefineSmem *>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;

    for (int r = blockIdx.x; r < k; r += gridDim.x) {
        const int beg = off[r], m = off[r + 1] - beg;
        if (m < 2)
            continue;
        const int nc = (m + cap - 1) / cap, base = m / nc, rem = m % nc;
        for (int c = 0; c < nc; c++) {
            const int s0 = c * base + min(c, rem), sz = base + (c < rem ? 1 : 0);
            if (sz < 2)
                continue;
            const int32_t *S = mem + beg + s0;
            for (int rb = 0; rb < sz; rb += RF_T) {
                const int nr = min(RF_T, sz - rb);
                for (int cb = 0; cb < sz; cb += RF_T) {
                    const int ncl = min(RF_T, sz - cb);
                    __syncthreads();
                    for (int q = tid; q < RF_T; q += RF_THREADS) {
                        int a = q < nr ? S[rb + q] : -1;
                        int b = q < ncl ? S[cb + q] : -1;
                        if ((a >= 0 && a >= n) || (b >= 0 && b >= n)) {  // corrupt grouping: record, skip the pair
                            flag_error(st, GK_ERR_INVALID, (unsigned)r);
                            a = a >= n ? -1 : a;
                            b = b >= n ? -1 : b;
                        }
                        sm.rid[q] = a;
                        sm.cid[q] = b;
                    }
                    __syncthreads();
                    const int nqr = (nr + 15) >> 4, nqc = (ncl + 15) >> 4;
                    float acc[8][8];
#pragma unroll
                    for (int a = 0; a < 8; a++)
#pragma unroll
                        for (int b = 0; b < 8; b++)
                            acc[a][b] = 0.f;
                    for (int t0 = 0; t0 < d; t0 += RF_DK) {
                        // stage coordinates t0 .. t0+31 of the row and column samples (zero padded)
                        for (int e = tid; e < RF_T * RF_DK; e += RF_THREADS) {
                            int row = e / RF_DK, tt = e % RF_DK;
                            int t = t0 + tt;
                            int a = sm.rid[row], b = sm.cid[row];
                            sm.xr[tt * RF_XS + row] = (a >= 0 && t < d) ? X[(int64_t)a * ld + t] : 0.f;
                            sm.xc[tt * RF_XS + row] = (b >= 0 && t < d) ? X[(int64_t)b * ld + t] : 0.f;
                        }
                        __syncthreads();
                        const int tmax = min(RF_DK, d - t0);
                        for (int tt = 0; tt < tmax; tt++) {
                            float xr[8], xc[8];
#pragma unroll
                            for (int q = 0; q < 8; q++) {
                                xr[q] = sm.xr[tt * RF_XS + ty + 16 * q];
                                xc[q] = sm.xc[tt * RF_XS + tx + 16 * q];
                            }
#pragma unroll
                            for (int a = 0; a < 8; a++) {
                                if (a < nqr) {
#pragma unroll
                                    for (int b = 0; b < 8; b++) {
                                        float diff = xr[a] - xc[b];
                                        acc[a][b] = fmaf(diff, diff, acc[a][b]);
                                    }
                                }
                            }
                        }
                        __syncthreads();
                    }
                    (void)nqc;
#pragma unroll
                    for (int a = 0; a < 8; a++)
#pragma unroll
                        for (int b = 0; b < 8; b++)
                            sm.dt[(ty + 16 * a) * RF_DS + tx + 16 * b] = acc[a][b];
                    __syncthreads();
                    for (int row = w; row < nr; row += RF_WARPS) {
                        int i = sm.rid[row];
                        if (i < 0)
                            continue;
                        merge_row(i, sm.cid, sm.dt + row * RF_DS, ncl, kappa, g_idx + (int64_t)i * kappa,
                                  g_dist + (int64_t)i * kappa, sm.li[w], sm.lv[w], sm.bi[w], sm.bv[w], sm.ni[w],
                                  sm.nv[w]);
                    }
                }
            }
        }
    }
}

cudaError_t launch_refine(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster, int32_t *g_idx,
                          float *g_dist, DevStatus *st, cudaStream_t s)
{
    size_t shm = sizeof(RefineSmem);
    cudaError_t e = cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess)
        return e;
    int blocks = k < 152 * 8 ? k : 152 * 8;
    if (blocks < 1)
        blocks = 1;
    k_refine<<<blocks, RF_THREADS, shm, s>>>(X, n, (int)d, ld, offsets, members, k, kappa, max_cluster, g_idx, g_dist,
                                             st);
    return cudaGetLastError();
}

}  // namespace gkm
