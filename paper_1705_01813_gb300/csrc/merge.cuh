// Top-kappa merge of one graph row with a tile of candidates (Alg. 3: a
// compared pair updates the row), shared by the SIMT and tensor-core
// refinement kernels.
#pragma once

#include "common.cuh"

namespace gkm {

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

// A graph row's kappa keys held in registers (lane l owns entries l, l + 32,
// l + 64, l + 96), so that the next row's list can be loaded while the
// current row is merged.
struct RowRegs {
    int id[4];
    float dv[4];
};

__device__ __forceinline__ void load_row(RowRegs &r, const int32_t *__restrict__ gi, const float *__restrict__ gd,
                                         int kappa)
{
    const int lane = lane_id();
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int q = lane + 32 * u;
        if (q < kappa) {
            r.id[u] = __ldcg(gi + q);
            r.dv[u] = __ldcg(gd + q);
        }
    }
}

// Merge the candidates (ids cid[0..ncol), ascending; distances drow[0..ncol))
// into graph row i, whose current kappa sorted keys are in `cur`; the merged
// row is written to gi / gd when it changes.  Warp-cooperative.  Candidates
// already in the row are found by a binary search of each row id among the
// (sorted) candidate ids and masked out; the others that beat the row's
// kappa-th key are ranked among themselves and placed by rank.
__device__ __forceinline__ void merge_row(int i, const int *__restrict__ cid, const float *__restrict__ drow,
                                          int ncol, int kappa, const RowRegs &cur, int32_t *__restrict__ gi,
                                          float *__restrict__ gd, int *li, float *lv, int *bi, float *bv, int *ni,
                                          float *nv, unsigned *dup)
{
    const int lane = lane_id();
    if (lane < 4)
        dup[lane] = 0u;
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int q = lane + 32 * u;
        if (q < kappa) {
            const int j = cur.id[u];
            li[q] = j;
            lv[q] = cur.dv[u];
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

}  // namespace gkm
