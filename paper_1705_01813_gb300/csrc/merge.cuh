// Top-kappa merge of one graph row with a tile of candidates (Alg. 3: a
// compared pair updates the row), shared by the SIMT and tensor-core
// refinement kernels.
#pragma once

#include "common.cuh"

namespace gkm {

// A (distance, id) key packed in 64 bits so that one unsigned comparison
// orders keys as key_less does: the distance's bits mapped to an unsigned
// integer of the same order (sign bit set for non-negative values, all bits
// inverted for negative ones; -0 is first made +0, which compares equal to
// it) in the high word, the id (non-negative) in the low word.
__device__ __forceinline__ uint64_t pack_key(float dv, int id)
{
    const unsigned b = __float_as_uint(dv + 0.0f);
    const unsigned o = b ^ ((unsigned)((int)b >> 31) | 0x80000000u);
    return ((uint64_t)o << 32) | (uint32_t)id;
}

__device__ __forceinline__ float key_dist(uint64_t key)
{
    const unsigned o = (unsigned)(key >> 32);
    return __uint_as_float((o & 0x80000000u) ? (o ^ 0x80000000u) : ~o);
}

__device__ __forceinline__ int key_id(uint64_t key) { return (int)(uint32_t)key; }

// Number of keys of the sorted k[0..len) smaller than key.
__device__ __forceinline__ int lower_rank(const uint64_t *k, int len, uint64_t key)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (k[mid] < key)
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
// row is written to gi / gd when it changes.  Warp-cooperative, on packed
// keys; per-warp shared buffers rk, nk (kappa keys each), bk (ncol keys) and
// dup (ncol bits).  Candidates already in the row are found by a binary
// search of each row id among the (sorted) candidate ids and masked out; the
// others that beat the row's kappa-th key are ranked among themselves and
// placed by rank plus their position in the row.
__device__ __forceinline__ void merge_row(int i, const int *__restrict__ cid, const float *__restrict__ drow,
                                          int ncol, int kappa, const RowRegs &cur, int32_t *__restrict__ gi,
                                          float *__restrict__ gd, uint64_t *rk, uint64_t *bk, uint64_t *nk,
                                          unsigned *dup)
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
            rk[q] = pack_key(cur.dv[u], j);
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
    const uint64_t th = rk[kappa - 1];
    // candidates that would enter the row and are not in it yet
    int ns = 0;
    for (int c0 = 0; c0 < ncol; c0 += 32) {
        const int c = c0 + lane;
        bool ok = c < ncol;
        const int j = ok ? cid[c] : -1;
        const uint64_t key = ok ? pack_key(drow[c], j) : ~0ull;
        ok = ok && j != i && ((dup[c0 >> 5] >> lane) & 1u) == 0u && key < th;
        const unsigned bal = __ballot_sync(FULL_MASK, ok);
        if (ok)
            bk[ns + __popc(bal & lanemask_lt())] = key;
        ns += __popc(bal);
    }
    __syncwarp();
    if (ns == 0)
        return;
    // rank the candidates among themselves (keys are distinct: ids differ)
    int rnk[4];
    uint64_t kb[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int b = lane + 32 * u;
        rnk[u] = -1;
        if (b < ns) {
            kb[u] = bk[b];
            int r = 0;
            for (int q = 0; q < ns; q++)
                r += bk[q] < kb[u] ? 1 : 0;
            rnk[u] = r;
        }
    }
    __syncwarp();
    // sorted candidates in bk, then each key's slot in the merged row
#pragma unroll
    for (int u = 0; u < 4; u++)
        if (rnk[u] >= 0)
            bk[rnk[u]] = kb[u];
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; u++) {
        if (rnk[u] >= 0) {
            const int pos = rnk[u] + lower_rank(rk, kappa, kb[u]);
            if (pos < kappa)
                nk[pos] = kb[u];
        }
    }
    for (int a = lane; a < kappa; a += 32) {
        const uint64_t key = rk[a];
        const int pos = a + lower_rank(bk, ns, key);
        if (pos < kappa)
            nk[pos] = key;
    }
    __syncwarp();
    for (int q = lane; q < kappa; q += 32) {
        const uint64_t key = nk[q];
        gi[q] = key_id(key);
        gd[q] = key_dist(key);
    }
    __syncwarp();
}

}  // namespace gkm
