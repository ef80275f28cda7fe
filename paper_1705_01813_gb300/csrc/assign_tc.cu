// Graph-guided assignment (Alg. 2 candidate loop with the closest-centroid
// rule of Sec. 4.2) with the candidate distances screened on the tensor
// cores, and the FP32 path's results bit for bit.
//
// One CTA (4 warps) per tile of 128 consecutive samples in the order of the
// grouping of the input labels (samples of one cluster are adjacent, so their
// candidate sets overlap).  Each thread gathers its sample's candidate labels
// (own label and the labels of its kappa graph neighbours) and inserts them in
// a shared hash table; the union U of the tile (at most AT_UMAX labels, else
// the tile is left to the SIMT kernel) gets dense column numbers in slot
// order, and every sample a bit mask over U.  The samples (BF16) form the A
// operand, the centroids of U (from the BF16 copy) the B operand, 128 columns
// at a time; tcgen05 MMAs accumulate x.c in tensor memory.  Thread t owns TMEM
// lane t (its sample): approx = |x|^2 + |c|^2 - 2 x~.c~ for its own candidate
// columns only, with a rigorous bound E on |approx - D|, D being the FP32
// path's distance (BF16 rounding of both operands (4u + 2u^2)|x||c|, u = 2^-8,
// FP32 accumulation and norms, and the FP32 path's own rounding).  The labels
// of every candidate whose approx - E is not above the smallest approx + E
// (at most AT_SEL of them, else the sample is marked) are written out; the
// SIMT kernel then recomputes exactly those with the FP32 path's lane partials
// and reduction tree, so the argmin over (distance, label) and its distance
// are the FP32 path's.
#include "assign_common.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace gkm {

constexpr int AT_TILE = 128;               // samples per tile (TMEM lanes)
constexpr int AT_THREADS = 128;
constexpr int AT_WARPS = AT_THREADS / 32;
constexpr int AT_UMAX = 1024;              // largest candidate union screened on the tensor cores
constexpr int AT_HASH = 2048;              // hash slots (power of two)
constexpr int AT_NCH = 128;                // union columns per MMA chunk
constexpr int AT_KB = 64;                  // BF16 per K-block (128-byte swizzle row)
constexpr int AT_NKB = 2;                  // K-blocks: d <= 128
constexpr int AT_KB_BYTES = AT_TILE * 128; // 16 KB
constexpr int AT_SEL = 8;                  // screened candidates kept per sample (AS_SEL in assign.cu)
constexpr int AT_MW = AT_UMAX / 32;        // mask words per sample
constexpr int AT_VS = 33;                  // stride of the per-thread value rows
constexpr uint32_t AT_WAIT_ITERS = 1u << 22;

struct AtSmem {
    static constexpr size_t opA = (size_t)AT_NKB * AT_KB_BYTES;       // samples
    static constexpr size_t opB = (size_t)AT_NKB * AT_KB_BYTES;       // centroid chunk / label scratch / values
    static constexpr size_t hash = (size_t)AT_HASH * 2 * sizeof(int);  // keys, columns
    static constexpr size_t ulab = (size_t)AT_UMAX * sizeof(int);
    static constexpr size_t mask = (size_t)AT_TILE * AT_MW * sizeof(unsigned);
    static constexpr size_t misc = (size_t)AT_TILE * (2 * sizeof(float) + sizeof(int)) + 64;
    static constexpr size_t bytes = 1024 + opA + opB + hash + ulab + mask + misc;
};

__device__ __forceinline__ uint32_t at_hash(int v) { return ((uint32_t)v * 0x9E3779B1u) >> (32 - 11); }

// Look a label up (present by construction); returns its slot.
__device__ __forceinline__ int at_find(const int *hkey, int lab)
{
    uint32_t h = at_hash(lab);
    for (int probe = 0; probe < AT_HASH; probe++) {
        if (hkey[h] == lab)
            return (int)h;
        h = (h + 1) & (AT_HASH - 1);
    }
    return -1;
}

__global__ void __launch_bounds__(AT_THREADS) k_assign_tc(const float *__restrict__ X, int64_t n, int d, int64_t ld,
                                                          const int32_t *__restrict__ G, int kappa,
                                                          const float *__restrict__ C,
                                                          const __nv_bfloat16 *__restrict__ Cb,
                                                          const float *__restrict__ delta,
                                                          const float *__restrict__ cnorm, int k,
                                                          const int32_t *__restrict__ Lin,
                                                          const int32_t *__restrict__ members,
                                                          int32_t *__restrict__ sel_lab, int32_t *__restrict__ sel_n,
                                                          int32_t *__restrict__ tile_fallback, DevStatus *st)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *opA = base;
    unsigned char *opB = opA + AtSmem::opA;
    int *hkey = reinterpret_cast<int *>(opB + AtSmem::opB);
    int *hcol = hkey + AT_HASH;
    int *ulab = hcol + AT_HASH;
    unsigned *mask = reinterpret_cast<unsigned *>(ulab + AT_UMAX);
    float *xn = reinterpret_cast<float *>(mask + AT_TILE * AT_MW);
    float *cn = xn + AT_TILE;
    int *sid = reinterpret_cast<int *>(cn + AT_TILE);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sid + AT_TILE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *sh = reinterpret_cast<int *>(tslot + 1);  // [0] union size, [1] overflow, [2] timeout, [3] scan total
    int *labs = reinterpret_cast<int *>(opB);      // [AT_TILE][kappa + 1] during the gather
    float *vals = reinterpret_cast<float *>(opB);  // [AT_TILE][AT_VS] during the screening

    const int tid = threadIdx.x, w = tid >> 5, lane = lane_id();
    const int64_t p0 = (int64_t)blockIdx.x * AT_TILE;
    const int ns = (int)((n - p0) < AT_TILE ? (n - p0) : AT_TILE);
    const int lsz = kappa + 1;

    if (w == 0) {
        tc::tmem_alloc(tslot, AT_NCH);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
        sh[0] = 0;
        sh[1] = 0;
        sh[2] = 0;
        sh[3] = 0;
    }
    for (int q = tid; q < AT_HASH; q += AT_THREADS)
        hkey[q] = -1;
    for (int q = tid; q < AT_TILE * AT_MW; q += AT_THREADS)
        mask[q] = 0u;
    sid[tid] = tid < ns ? members[p0 + tid] : -1;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;

    // ---- 1. candidate labels of each sample, union in the hash table ----
    {
        const int i = sid[tid];
        int *my = labs + tid * lsz;
        if (i >= 0 && i < n) {
            const int own = Lin[i];
            for (int c = 0; c < lsz; c++) {
                int lab = -1;
                if (c == 0) {
                    lab = own;
                } else {
                    const int nb = __ldg(G + (int64_t)i * kappa + (c - 1));
                    if ((unsigned)nb < (unsigned)n)
                        lab = Lin[nb];
                    else
                        flag_error(st, GK_ERR_INVALID, (unsigned)i);
                }
                if ((unsigned)lab >= (unsigned)k) {
                    if (c > 0 || lab != -1)
                        flag_error(st, GK_ERR_INVALID, (unsigned)i);
                    lab = -1;
                }
                my[c] = lab;
                if (lab >= 0 && !sh[1]) {
                    uint32_t h = at_hash(lab);
                    int probe = 0;
                    for (; probe < AT_HASH; probe++) {
                        const int prev = atomicCAS(&hkey[h], -1, lab);
                        if (prev == -1) {
                            if (atomicAdd(&sh[0], 1) >= AT_UMAX)
                                sh[1] = 1;
                            break;
                        }
                        if (prev == lab)
                            break;
                        h = (h + 1) & (AT_HASH - 1);
                    }
                    if (probe == AT_HASH)
                        sh[1] = 1;
                }
            }
        } else {
            for (int c = 0; c < lsz; c++)
                my[c] = -1;
        }
    }
    __syncthreads();
    const bool overflow = sh[1] != 0;
    if (overflow) {
        if (tid == 0)
            tile_fallback[blockIdx.x] = 1;
    } else {
        // ---- 2. dense union columns in slot order (deterministic) ----
        constexpr int PER = AT_HASH / AT_THREADS;
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < PER; q++)
            cnt += hkey[tid * PER + q] >= 0 ? 1 : 0;
        // block exclusive scan of cnt
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o)
                incl += v;
        }
        __shared__ int wsum[AT_WARPS];
        if (lane == 31)
            wsum[w] = incl;
        __syncthreads();
        int woff = 0;
        for (int q = 0; q < w; q++)
            woff += wsum[q];
        int col = woff + incl - cnt;
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int slot = tid * PER + q;
            const int key = hkey[slot];
            if (key >= 0) {
                hcol[slot] = col;
                ulab[col] = key;
                col++;
            }
        }
        if (tid == AT_THREADS - 1)
            sh[3] = woff + incl;
        __syncthreads();
        // ---- 3. each sample's candidate mask over the union ----
        {
            const int *my = labs + tid * lsz;
            unsigned *mrow = mask + tid * AT_MW;
            for (int c = 0; c < lsz; c++) {
                const int lab = my[c];
                if (lab >= 0) {
                    const int slot = at_find(hkey, lab);
                    if (slot >= 0) {
                        const int cc = hcol[slot];
                        mrow[cc >> 5] |= 1u << (cc & 31);
                    }
                }
            }
        }
    }
    __syncthreads();  // labels scratch (opB) is free from here on
    const int nu = sh[3];

    float best_up = __int_as_float(0x7f800000);
    int sel_col[AT_SEL];
    float sel_lo[AT_SEL];
    int nsel = 0;
    bool sel_over = false;
    bool timed_out = false;
    if (!overflow) {
        // ---- 4. A operand: the tile's samples in BF16, and their FP32 squared norms ----
        for (int row = w; row < AT_TILE; row += AT_WARPS) {
            const int i = sid[row];
            float part = 0.f;
            const int kk = lane * 4;  // d <= 128: one 4-element group per lane
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i >= 0 && kk < d)
                v = __ldg(reinterpret_cast<const float4 *>(X + (int64_t)i * ld) + lane);
            part = fmaf(v.x, v.x, part);
            part = fmaf(v.y, v.y, part);
            part = fmaf(v.z, v.z, part);
            part = fmaf(v.w, v.w, part);
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(v.x, v.y), p1 = __floats2bfloat162_rn(v.z, v.w);
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t *>(&p0);
            pk.y = *reinterpret_cast<const uint32_t *>(&p1);
            *reinterpret_cast<uint2 *>(opA + (kk / AT_KB) * AT_KB_BYTES + tc::swz128_offset(row, kk % AT_KB)) = pk;
            for (int o = 16; o > 0; o >>= 1)
                part += __shfl_xor_sync(FULL_MASK, part, o);
            if (lane == 0)
                xn[row] = part;
        }
        __syncthreads();
        const float x2 = xn[tid];
        const float u = 1.0f / 256.0f;
        const float c1 = 1.05f * (4.f * u + 2.f * u * u + 4.f * (d + 2) * 1.1920929e-7f);
        const float c2 = 1.05f * 4.f * (d + 2) * 1.1920929e-7f;
        const float gp = (d + 8) * 1.1920929e-7f;
        const unsigned *mrow = mask + tid * AT_MW;
        uint32_t phase = 0;
        const int nkb = (d + AT_KB - 1) / AT_KB;
        for (int c0 = 0; c0 < nu; c0 += AT_NCH) {
            const int nch = min(AT_NCH, nu - c0);
            const int N = (nch + 15) & ~15;
            // ---- 5. B operand: the chunk's centroids from the BF16 copy ----
            for (int row = w; row < N; row += AT_WARPS) {
                const int kk = lane * 4;
                uint2 pk = make_uint2(0u, 0u);
                if (row < nch && kk < d) {
                    const int r = ulab[c0 + row];
                    pk = __ldg(reinterpret_cast<const uint2 *>(Cb + (int64_t)r * d) + lane);
                }
                *reinterpret_cast<uint2 *>(opB + (kk / AT_KB) * AT_KB_BYTES + tc::swz128_offset(row, kk % AT_KB)) =
                    pk;
            }
            if (tid < nch)
                cn[tid] = cnorm[ulab[c0 + tid]];
            tc::fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t idesc = tc::idesc_bf16_f32(AT_TILE, N);
                for (int kb = 0; kb < nkb; kb++) {
                    const uint32_t a_addr = tc::smem_addr(opA + kb * AT_KB_BYTES);
                    const uint32_t b_addr = tc::smem_addr(opB + kb * AT_KB_BYTES);
#pragma unroll
                    for (int s = 0; s < AT_KB / 16; s++)
                        tc::mma_bf16(taddr, tc::desc_k128(a_addr + 32 * s), tc::desc_k128(b_addr + 32 * s), idesc,
                                     (kb > 0) || (s > 0));
                }
                tc::mma_commit(bar);
            }
            __syncwarp();
            const bool late = !tc::mbar_wait_bounded(bar, phase, AT_WAIT_ITERS);
            phase ^= 1u;
            tc::fence_after_sync();
            // every thread saw the MMAs complete (opB may now hold values); a timeout is block-wide
            timed_out = __syncthreads_or(late ? 1 : 0) != 0;
            if (timed_out)
                break;  // stage and issue nothing more: the abandoned MMAs may still read opB
            // ---- 6. screening of this thread's own candidate columns ----
            {
                float *vrow = vals + tid * AT_VS;
                for (int s0 = 0; s0 < N; s0 += 32) {
                    float g[32];
                    tc::tmem_ld32(taddr + ((uint32_t)(32 * w) << 16) + (uint32_t)s0, g);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 32; q++)
                        vrow[q] = g[q];
                    unsigned m = mrow[(c0 + s0) >> 5];
                    const int lim = nch - s0;
                    if (lim < 32)
                        m &= lim <= 0 ? 0u : (0xffffffffu >> (32 - lim));
                    while (m) {
                        const int q = __ffs(m) - 1;
                        m &= m - 1;
                        const float c2n = cn[s0 + q];
                        const float approx = (x2 + c2n) - 2.f * vrow[q];
                        const float xc = sqrtf(x2 * c2n);
                        const float e = c1 * xc + c2 * (x2 + c2n) + gp * fabsf(approx) + 1e-30f;
                        const float lo_v = approx - e, up_v = approx + e;
                        best_up = fminf(best_up, up_v);
                        if (lo_v <= best_up) {
                            if (nsel < AT_SEL) {
                                sel_col[nsel] = c0 + s0 + q;
                                sel_lo[nsel] = lo_v;
                                nsel++;
                            } else {
                                // keep the list to the candidates still in range, else recompute all
                                int kept = 0;
#pragma unroll
                                for (int z = 0; z < AT_SEL; z++)
                                    if (sel_lo[z] <= best_up) {
                                        sel_col[kept] = sel_col[z];
                                        sel_lo[kept] = sel_lo[z];
                                        kept++;
                                    }
                                if (kept < AT_SEL) {
                                    nsel = kept;
                                    sel_col[nsel] = c0 + s0 + q;
                                    sel_lo[nsel] = lo_v;
                                    nsel++;
                                } else {
                                    nsel = kept;
                                    sel_over = true;
                                }
                            }
                        }
                    }
                }
            }
            __syncthreads();  // values read, opB free for the next chunk
        }
        if (timed_out) {
            if (tid == 0)
                flag_error(st, GK_ERR_TIMEOUT, blockIdx.x);
            // one more bounded wait for the abandoned MMAs before their tensor memory is freed below
            tc::mbar_wait_bounded(bar, phase ^ 1u, AT_WAIT_ITERS);
        }
    }

    // ---- 7. the screened candidates of each sample, for the exact pass ----
    if (!overflow && !timed_out && tid < ns) {
        const int i = sid[tid];
        if (i >= 0) {
            int cnt = 0;
            int32_t *out = sel_lab + (int64_t)i * AT_SEL;
            if (!sel_over) {
#pragma unroll
                for (int z = 0; z < AT_SEL; z++)
                    if (z < nsel && sel_lo[z] <= best_up)
                        out[cnt++] = ulab[sel_col[z]];
            }
            sel_n[i] = sel_over ? -1 : cnt;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0)
        tc::tmem_dealloc(taddr, AT_NCH);
}

bool assign_tc_supported(int64_t d, int64_t ld, const float *X, const float *C, int32_t kappa)
{
    return d % 4 == 0 && d <= 128 && ld % 4 == 0 && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
           ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && kappa + 1 <= (int)(AtSmem::opB / (AT_TILE * sizeof(int)));
}

cudaError_t launch_assign_tc(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                             const float *C, const __nv_bfloat16 *Cb, const float *delta, const float *cnorm,
                             int32_t k, const int32_t *labels_in, const int32_t *members, int32_t *sel_lab,
                             int32_t *sel_n, int32_t *tile_fallback, DevStatus *st, cudaStream_t s)
{
    const int64_t tiles = (n + AT_TILE - 1) / AT_TILE;
    cudaError_t e = cudaMemsetAsync(tile_fallback, 0, sizeof(int32_t) * (size_t)tiles, s);
    if (e != cudaSuccess)
        return e;
    if ((e = set_max_smem(reinterpret_cast<const void *>(k_assign_tc), (int)AtSmem::bytes)) !=
        cudaSuccess)
        return e;
    k_assign_tc<<<(unsigned)tiles, AT_THREADS, AtSmem::bytes, s>>>(X, n, (int)d, ld, g_idx, kappa, C, Cb, delta,
                                                                   cnorm, k, labels_in, members, sel_lab, sel_n,
                                                                   tile_fallback, st);
    return cudaGetLastError();
}

}  // namespace gkm
