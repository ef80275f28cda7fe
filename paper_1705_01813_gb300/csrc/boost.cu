// Boost form of GK-means (Sec. 3.1 Eq. 2 and Eq. 3; the move step of Alg. 2,
// Sec. 4.2).  State per cluster r: the composite vector D_r (FP64, the sum of
// its members, Eq. 2), its size n_r and S_r = D_r'D_r.  Alg. 2 visits samples
// one at a time; sample i in cluster u looks at the clusters of its kappa
// neighbours and moves to the one whose Eq. 3 gain
//     ((D_v + x)'(D_v + x) / (n_v + 1) + (D_u - x)'(D_u - x) / (n_u - 1)) - S_v / n_v - S_u / n_u
// is largest, if that gain is positive.  Each move changes two clusters and one
// label before the next visit reads them, so the visits run in order.
//
// Arithmetic, fixed so that every decision is reproducible: FP64; D_r starts
// as its members' rows summed in ascending sample id; a squared norm squares
// the elements (each rounded once) of the vector zero-padded to a power of two
// and sums them by halving folds (w[j] += w[j + P/2], then P/4, ...); the gain
// is evaluated term by term, left to right, every operation rounded once (no
// fused multiply-add).  A sample alone in its cluster does not move (Eq. 3
// divides by n_u - 1); equal gains go to the smaller label.
//
// Layout: D is k x d row-major FP64; S, counts and labels are k / k / n
// arrays.  One thread-block cluster (up to 16 CTAs, one per SM) walks the
// visits: one warp per candidate (and one for the own cluster) computes the
// squared norm of D_v + x (D_u - x) with lane l holding elements l + 32 m,
// and CTA 0 takes the arg-max and applies the move.  GB300 runs FP64 at a
// small fraction of its FP32 rate, so a visit's FP64 work is spread over the
// cluster's SMs.  After a move, S_u and S_v are the two norms already computed
// for the decision: the new rows are exactly the rounded sums that were
// squared.
#include <map>
#include <mutex>

#include "common.cuh"

namespace gkm {

namespace {

constexpr int BO_MAX_D = 1024;

// Squared norm of a lane-major vector (lane l holds w[l + 32 m], m < PL) by
// halving folds; the total lands in lane 0.  Folds with a stride of 32 or more
// stay inside a lane; the last five are shuffles.
template <int PL>
__device__ __forceinline__ double fold_lanes(double (&w)[PL])
{
#pragma unroll
    for (int h = PL / 2; h >= 1; h /= 2)
#pragma unroll
        for (int m = 0; m < h; m++)
            w[m] = __dadd_rn(w[m], w[m + h]);
    double a = w[0];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
        a = __dadd_rn(a, __shfl_down_sync(FULL_MASK, a, o));
    return a;
}

template <typename XT>
__device__ __forceinline__ double ldx64(const XT *p)
{
    return (double)ldx(p);
}

// ---------------------------------------------------------------------------
// Eq. 2 state from a CSR grouping (members ascending within a cluster).
// ---------------------------------------------------------------------------
constexpr int BS_THREADS = 128;

// D[r][t]: one thread per (cluster, coordinate), members summed in CSR order.
template <typename XT>
__global__ void __launch_bounds__(BS_THREADS) k_boost_sum(const XT *__restrict__ X, int d, int64_t ld,
                                                         const int32_t *__restrict__ offsets,
                                                         const int32_t *__restrict__ members, double *__restrict__ D)
{
    const int r = blockIdx.x;
    const int t = blockIdx.y * BS_THREADS + threadIdx.x;
    if (t >= d)
        return;
    const int b = offsets[r], e = offsets[r + 1];
    double acc = 0.0;
    int p = b;
    for (; p + 4 <= e; p += 4) {  // loads issued ahead of the ordered additions
        const double a0 = ldx64(X + (int64_t)members[p] * ld + t), a1 = ldx64(X + (int64_t)members[p + 1] * ld + t);
        const double a2 = ldx64(X + (int64_t)members[p + 2] * ld + t), a3 = ldx64(X + (int64_t)members[p + 3] * ld + t);
        acc = __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(acc, a0), a1), a2), a3);
    }
    for (; p < e; p++)
        acc = __dadd_rn(acc, ldx64(X + (int64_t)members[p] * ld + t));
    D[(int64_t)r * d + t] = acc;
}

// S[r] = D_r'D_r (the fold) and counts[r], one warp per cluster.
template <int PL>
__global__ void __launch_bounds__(256) k_boost_norms(const double *__restrict__ D, int d, int32_t k,
                                                     const int32_t *__restrict__ offsets, double *__restrict__ S,
                                                     int32_t *__restrict__ counts)
{
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= k)
        return;
    const int lane = lane_id();
    double w[PL];
#pragma unroll
    for (int m = 0; m < PL; m++) {
        const int j = lane + 32 * m;
        const double a = j < d ? D[(int64_t)r * d + j] : 0.0;
        w[m] = __dmul_rn(a, a);
    }
    const double s = fold_lanes<PL>(w);
    if (lane == 0) {
        S[r] = s;
        counts[r] = offsets[r + 1] - offsets[r];
    }
}

// ---------------------------------------------------------------------------
// One epoch of the move step over order[0..m), on one cluster of R CTAs.
//
// Per visit: every CTA stages the sample and gathers the candidate set Q (the
// same labels, so the same Q); the squared norms (task 0: D_u - x, task c:
// D_v + x for the c-th candidate) are spread over the cluster's warps, and
// each task's result (with S_v and n_v) is stored into CTA 0's shared memory;
// a cluster barrier; CTA 0 evaluates the gains (its warps split the
// divisions), takes the arg-max and applies the move; a second cluster barrier
// publishes the move before the next visit reads labels or rows.  Both
// barriers are unconditional, so the barrier sequence never depends on data.
// The FP64 work of a visit thus runs on R SMs; mutable state (labels, D, S,
// counts) is read through L2 (ld.global.cg), which the barriers order.
// ---------------------------------------------------------------------------
constexpr int BE_THREADS = 256;
constexpr int BE_WARPS = BE_THREADS / 32;
constexpr int BE_MAX_CLUSTER = 16;

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t in_rank(const void *p, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_rank(const void *p, int rank, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(in_rank(p, rank)), "d"(v) : "memory");
}

__device__ __forceinline__ void st_rank(const void *p, int rank, int v)
{
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(in_rank(p, rank)), "r"(v) : "memory");
}

template <typename XT, int PL>
__global__ void __launch_bounds__(BE_THREADS, 1)
    k_boost_epoch(const XT *__restrict__ X, int32_t n, int d, int64_t ld, const int32_t *__restrict__ G, int kappa,
                  const int32_t *__restrict__ order, int64_t m, int32_t *L, int32_t k, double *D, int32_t *cnt,
                  double *S, int64_t *n_moved, DevStatus *st)
{
    constexpr int P = 32 * PL;
    constexpr int XR = (P + BE_THREADS - 1) / BE_THREADS;  // sample elements staged per thread
    constexpr int GR = MAX_KAPPA / 32;                      // graph ids per lane of warp 0
    __shared__ double xs[2][P];          // the visited sample in FP64 (zero beyond d), by visit parity
    __shared__ int32_t s_q[MAX_KAPPA];   // candidate clusters (every CTA)
    __shared__ double s_a[MAX_KAPPA];    // CTA 0: (D_v + x)'(D_v + x), stored by the task owners
    __shared__ double s_sv[MAX_KAPPA];   // CTA 0: S_v
    __shared__ int32_t s_nv[MAX_KAPPA];  // CTA 0: n_v
    __shared__ double s_t1[MAX_KAPPA];   // CTA 0: A_v / (n_v + 1)
    __shared__ double s_t3[MAX_KAPPA];   // CTA 0: S_v / n_v
    __shared__ double s_b, s_tu1, s_tu2; // CTA 0: B, B / (n_u - 1), S_u / n_u
    __shared__ int s_nq, s_u, s_nu;
    __shared__ double s_gb[MAX_KAPPA / 32];                      // CTA 0: each group's best gain,
    __shared__ int s_gv[MAX_KAPPA / 32], s_gq[MAX_KAPPA / 32];  // its label and candidate index
    __shared__ int s_mv[3];  // the last visit's move (sample, from, to; to = -1: none), stored by CTA 0

    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int rank = (int)cluster_rank(), R = (int)cluster_size();
    int64_t moves = 0;
    auto visit_id = [&](int64_t s) { return s < m ? __ldg(order + s) : -1; };
    auto valid = [&](int i) { return i >= 0 && i < n; };
    // Pipeline: the sample row of the next visit (all threads), the labels of the next visit's neighbours and
    // the graph row of the one after (warp 0).  Labels read one visit ahead miss only the move of the visit in
    // between, which every CTA patches in from s_mv.
    float xr[XR];
    int gcur[GR], lcur[GR], gnx[GR], lnx[GR];
    int ucur = -1, unx = -1;
    auto load_x = [&](int i) {
#pragma unroll
        for (int c = 0; c < XR; c++) {
            const int j = threadIdx.x + c * BE_THREADS;
            xr[c] = valid(i) && j < d ? ldx(X + (int64_t)i * ld + j) : 0.f;
        }
    };
    auto load_g = [&](int i, int (&g)[GR]) {
#pragma unroll
        for (int c = 0; c < GR; c++) {
            const int j = lane + 32 * c;
            g[c] = valid(i) && j < kappa ? __ldg(G + (int64_t)i * kappa + j) : -1;
        }
    };
    auto load_l = [&](int i, const int (&g)[GR], int (&l)[GR], int &u) {
        u = valid(i) ? __ldcg(L + i) : -1;
#pragma unroll
        for (int c = 0; c < GR; c++)
            l[c] = valid(g[c]) ? __ldcg(L + g[c]) : -2;
    };
    int i_cur = visit_id(0), i_nx = visit_id(1), i_nx2 = visit_id(2);
    load_x(i_cur);
    if (w == 0) {
        load_g(i_cur, gcur);
        load_l(i_cur, gcur, lcur, ucur);
        load_g(i_nx, gnx);
    }
    if (threadIdx.x == 0)
        s_mv[0] = s_mv[1] = s_mv[2] = -1;
    cluster_barrier();  // every CTA of the cluster runs before any stores into another's shared memory

    for (int64_t s = 0; s < m; s++) {
        const int i = i_cur;
        const int buf = (int)(s & 1);
        const int pi = s_mv[0], pu = s_mv[1], pv = s_mv[2];  // the previous visit's move, pending in D
        // ---- stage the sample; gather its candidates (warp 0 of every CTA, from the same labels)
#pragma unroll
        for (int c = 0; c < XR; c++) {
            const int j = threadIdx.x + c * BE_THREADS;
            if (j < P)
                xs[buf][j] = (double)xr[c];
        }
        if (w == 0) {
            int u = ucur;
            if (pv >= 0 && i == pi)
                u = pv;
            if (!valid(i)) {
                if (lane == 0 && rank == 0)
                    flag_error(st, GK_ERR_INVALID, (unsigned)s);
                u = -1;
            } else if (u < 0 || u >= k) {
                if (lane == 0 && rank == 0)
                    flag_error(st, GK_ERR_INVALID, (unsigned)i);
                u = -1;
            }
            int nq = 0;
#pragma unroll
            for (int c = 0; c < GR; c++) {
                if (u < 0 || 32 * c >= kappa)
                    break;
                int v = lcur[c];
                if (pv >= 0 && gcur[c] == pi)
                    v = pv;
                const bool in_row = lane + 32 * c < kappa;
                if (in_row && (v < 0 || v >= k) && rank == 0)
                    flag_error(st, GK_ERR_INVALID, (unsigned)(v == -2 ? i : gcur[c]));
                if (!in_row || v < 0 || v >= k || v == u)
                    v = -1;
                bool keep = v >= 0;
#pragma unroll 8
                for (int q = 0; q < nq; q++)  // broadcast reads, independent of one another
                    keep &= s_q[q] != v;
                const unsigned same = __match_any_sync(FULL_MASK, v);
                keep = keep && (__ffs(same) - 1 == lane);
                const unsigned km = __ballot_sync(FULL_MASK, keep);
                if (keep)
                    s_q[nq + __popc(km & lanemask_lt())] = v;
                nq += __popc(km);
                __syncwarp();
            }
            if (lane == 0) {
                s_nq = nq;
                s_u = u;
            }
            // one visit ahead: the next visit's labels (this visit's move is patched in later), the graph row
            // of the visit after it
            load_l(i_nx, gnx, lnx, unx);
#pragma unroll
            for (int c = 0; c < GR; c++)
                gcur[c] = gnx[c];
            load_g(i_nx2, gnx);
        }
        load_x(i_nx);
        __syncthreads();

        // ---- squared norms: task c = 0 the own cluster (D_u - x), c >= 1 candidate c - 1 (D_v + x); task c runs
        //      on CTA c mod R, warp (c / R) mod BE_WARPS.  Rows pu and pv still lack the previous move.
        const int nq = s_nq, u = s_u;
        if (rank == 0 && w == BE_WARPS - 1 && nq > 0 && lane == 0) {  // S_u / n_u, beside task 0's fold
            const int nu = __ldcg(cnt + u);
            s_nu = nu;
            s_tu2 = __ddiv_rn(__ldcg(S + u), (double)nu);
        }
        for (int c = rank + R * w; nq > 0 && c <= nq; c += R * BE_WARPS) {
            const int r = c == 0 ? u : s_q[c - 1];
            const double *Dr = D + (int64_t)r * d;
            double a[PL];
#pragma unroll
            for (int q = 0; q < PL; q++) {
                const int j = lane + 32 * q;
                a[q] = j < d ? __ldcg(Dr + j) : 0.0;
            }
            double sr = 0.0;
            int nr = 0;
            if (lane == 0) {
                sr = __ldcg(S + r);
                nr = __ldcg(cnt + r);
            }
            const int pend = pv < 0 ? 0 : (r == pu ? -1 : (r == pv ? 1 : 0));
#pragma unroll
            for (int q = 0; q < PL; q++) {
                const int j = lane + 32 * q;
                double y = 0.0;
                if (j < d) {
                    double dr = a[q];
                    if (pend < 0)
                        dr = __dsub_rn(dr, xs[buf ^ 1][j]);
                    else if (pend > 0)
                        dr = __dadd_rn(dr, xs[buf ^ 1][j]);
                    y = c == 0 ? __dsub_rn(dr, xs[buf][j]) : __dadd_rn(dr, xs[buf][j]);
                }
                a[q] = __dmul_rn(y, y);
            }
            const double tot = fold_lanes<PL>(a);
            if (lane == 0) {
                if (c == 0) {  // on CTA 0: the own cluster's term B / (n_u - 1)
                    s_b = tot;
                    s_tu1 = __ddiv_rn(tot, (double)(nr - 1));
                } else {
                    st_rank(&s_a[c - 1], 0, tot);
                    st_rank(&s_sv[c - 1], 0, sr);
                    st_rank(&s_nv[c - 1], 0, nr);
                }
            }
        }
        cluster_barrier();

        // ---- CTA 0: the previous move's rows (warps 4-7, overlapping the rest); the Eq. 3 gains, the arg-max,
        //      this move's sizes, norms and label
        if (rank == 0) {
            const int nu = nq > 0 ? s_nu : 0;
            if (w >= 4) {
                if (pv >= 0) {
                    double *Du = D + (int64_t)pu * d, *Dv = D + (int64_t)pv * d;
                    for (int j = threadIdx.x - 128; j < d; j += BE_THREADS - 128) {
                        Du[j] = __dsub_rn(__ldcg(Du + j), xs[buf ^ 1][j]);
                        Dv[j] = __dadd_rn(__ldcg(Dv + j), xs[buf ^ 1][j]);
                    }
                }
            } else if (nq > 0 && nu >= 2) {
                // division job t: group t / 2 (32 candidates); t even: (D_v + x)'(D_v + x) / (n_v + 1), odd: S_v / n_v
                for (int t = w; t < 2 * ((nq + 31) / 32); t += 4) {
                    const int q = (t >> 1) * 32 + lane;
                    if (q < nq) {
                        if (t & 1)
                            s_t3[q] = __ddiv_rn(s_sv[q], (double)s_nv[q]);
                        else
                            s_t1[q] = __ddiv_rn(s_a[q], (double)(s_nv[q] + 1));
                    }
                }
            }
            __syncthreads();
            // warp g: the gains of group g and their arg-max (the larger gain, then the smaller label)
            if (w < (nq + 31) / 32 && nu >= 2) {
                const int q = w * 32 + lane;
                int bv = -1, bq = -1;
                double best = 0.0;
                if (q < nq) {
                    bv = s_q[q];
                    bq = q;
                    best = __dsub_rn(__dsub_rn(__dadd_rn(s_t1[q], s_tu1), s_t3[q]), s_tu2);
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const double ob = __shfl_xor_sync(FULL_MASK, best, o);
                    const int ov = __shfl_xor_sync(FULL_MASK, bv, o), oq = __shfl_xor_sync(FULL_MASK, bq, o);
                    if (ov >= 0 && (bv < 0 || ob > best || (ob == best && ov < bv))) {
                        best = ob;
                        bv = ov;
                        bq = oq;
                    }
                }
                if (lane == 0) {
                    s_gb[w] = best;
                    s_gv[w] = bv;
                    s_gq[w] = bq;
                }
            }
            __syncthreads();
            if (w == 0) {
                const int groups = nq > 0 && nu >= 2 ? (nq + 31) / 32 : 0;
                int bv = -1, bq = -1;
                double best = 0.0;
                for (int g = 0; g < groups; g++) {
                    const int ov = s_gv[g];
                    const double ob = s_gb[g];
                    if (ov >= 0 && (bv < 0 || ob > best || (ob == best && ov < bv))) {
                        best = ob;
                        bv = ov;
                        bq = s_gq[g];
                    }
                }
                const int v = best > 0.0 ? bv : -1;
                if (lane < R) {  // every CTA learns the move (its rows stay pending in D until the next visit)
                    st_rank(&s_mv[0], lane, i);
                    st_rank(&s_mv[1], lane, u);
                    st_rank(&s_mv[2], lane, v);
                }
                if (lane == 0 && v >= 0) {
                    cnt[u] = nu - 1;
                    cnt[v] = s_nv[bq] + 1;
                    S[u] = s_b;
                    S[v] = s_a[bq];
                    L[i] = v;
                    moves++;
                }
            }
        }
        cluster_barrier();  // the move's label, sizes and norms, and the previous move's rows, before the next visit
        i_cur = i_nx;
        i_nx = i_nx2;
        i_nx2 = visit_id(s + 3);
        if (w == 0) {
            ucur = unx;
#pragma unroll
            for (int c = 0; c < GR; c++)
                lcur[c] = lnx[c];
        }
    }
    // the last move's rows
    if (rank == 0 && m > 0 && s_mv[2] >= 0) {
        const int pu = s_mv[1], pv = s_mv[2], pb = (int)((m - 1) & 1);
        double *Du = D + (int64_t)pu * d, *Dv = D + (int64_t)pv * d;
        for (int j = threadIdx.x; j < d; j += BE_THREADS) {
            Du[j] = __dsub_rn(__ldcg(Du + j), xs[pb][j]);
            Dv[j] = __dadd_rn(__ldcg(Dv + j), xs[pb][j]);
        }
    }
    if (rank == 0 && threadIdx.x == 0 && n_moved)
        *n_moved = moves;
}

// Largest cluster (at most BE_MAX_CLUSTER CTAs) the device can run for this kernel, once per device and kernel.
template <typename KernelT>
int epoch_cluster_size(KernelT kern)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> known;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(dev, reinterpret_cast<const void *>(kern));
    auto it = known.find(key);
    if (it != known.end())
        return it->second;
    int r = 8;  // portable size
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(BE_MAX_CLUSTER);
        cfg.blockDim = dim3(BE_THREADS);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = BE_MAX_CLUSTER;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int most = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&most, kern, &cfg) == cudaSuccess && most > 0)
            r = most < BE_MAX_CLUSTER ? most : BE_MAX_CLUSTER;
    }
    cudaGetLastError();
    known[key] = r;
    return r;
}

template <typename XT, int PL>
cudaError_t boost_epoch_t(const XT *X, int64_t n, int64_t d, int64_t ld, const int32_t *G, int32_t kappa,
                          const int32_t *order, int64_t m, int32_t *L, int32_t k, double *D, int32_t *cnt, double *S,
                          int64_t *n_moved, DevStatus *st, cudaStream_t s)
{
    auto kern = k_boost_epoch<XT, PL>;
    const int R = epoch_cluster_size(kern);
    if (R < 1)
        return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)R);
    cfg.blockDim = dim3(BE_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)R;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, X, (int32_t)n, (int)d, ld, G, (int)kappa, order, m, L, k, D, cnt, S,
                              n_moved, st);
}

template <int PL>
cudaError_t boost_epoch_pl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *G, int32_t kappa,
                           const int32_t *order, int64_t m, int32_t *L, int32_t k, double *D, int32_t *cnt, double *S,
                           int64_t *n_moved, DevStatus *st, cudaStream_t s)
{
    if (bf16)
        return boost_epoch_t<__nv_bfloat16, PL>(static_cast<const __nv_bfloat16 *>(X), n, d, ld, G, kappa, order, m, L,
                                                k, D, cnt, S, n_moved, st, s);
    return boost_epoch_t<float, PL>(static_cast<const float *>(X), n, d, ld, G, kappa, order, m, L, k, D, cnt, S,
                                    n_moved, st, s);
}

template <int PL>
cudaError_t boost_norms_pl(const double *D, int64_t d, int32_t k, const int32_t *offsets, double *S, int32_t *counts,
                           cudaStream_t s)
{
    k_boost_norms<PL><<<(k + 7) / 8, 256, 0, s>>>(D, (int)d, k, offsets, S, counts);
    return cudaGetLastError();
}

int lanes_per_row(int64_t d)
{
    int pl = 1;
    while (32 * pl < d)
        pl <<= 1;
    return pl;
}

}  // namespace

int64_t boost_max_d() { return BO_MAX_D; }

cudaError_t launch_boost_init(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *labels,
                              int32_t k, double *D, int32_t *counts, double *S, int32_t *offsets, int32_t *members,
                              int32_t *grp_counts, void *grp_scratch, DevStatus *st, cudaStream_t s)
{
    cudaError_t e = launch_group(labels, n, k, offsets, members, grp_counts, grp_scratch, st, s);
    if (e != cudaSuccess)
        return e;
    const dim3 grid((unsigned)k, (unsigned)((d + BS_THREADS - 1) / BS_THREADS));
    if (bf16)
        k_boost_sum<__nv_bfloat16><<<grid, BS_THREADS, 0, s>>>(static_cast<const __nv_bfloat16 *>(X), (int)d, ld,
                                                               offsets, members, D);
    else
        k_boost_sum<float><<<grid, BS_THREADS, 0, s>>>(static_cast<const float *>(X), (int)d, ld, offsets, members, D);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    switch (lanes_per_row(d)) {
    case 1: return boost_norms_pl<1>(D, d, k, offsets, S, counts, s);
    case 2: return boost_norms_pl<2>(D, d, k, offsets, S, counts, s);
    case 4: return boost_norms_pl<4>(D, d, k, offsets, S, counts, s);
    case 8: return boost_norms_pl<8>(D, d, k, offsets, S, counts, s);
    case 16: return boost_norms_pl<16>(D, d, k, offsets, S, counts, s);
    default: return boost_norms_pl<32>(D, d, k, offsets, S, counts, s);
    }
}

cudaError_t launch_boost_epoch(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *G,
                               int32_t kappa, const int32_t *order, int64_t m, int32_t *labels, int32_t k, double *D,
                               int32_t *counts, double *S, int64_t *n_moved, DevStatus *st, cudaStream_t s)
{
    switch (lanes_per_row(d)) {
    case 1: return boost_epoch_pl<1>(X, bf16, n, d, ld, G, kappa, order, m, labels, k, D, counts, S, n_moved, st, s);
    case 2: return boost_epoch_pl<2>(X, bf16, n, d, ld, G, kappa, order, m, labels, k, D, counts, S, n_moved, st, s);
    case 4: return boost_epoch_pl<4>(X, bf16, n, d, ld, G, kappa, order, m, labels, k, D, counts, S, n_moved, st, s);
    case 8: return boost_epoch_pl<8>(X, bf16, n, d, ld, G, kappa, order, m, labels, k, D, counts, S, n_moved, st, s);
    case 16: return boost_epoch_pl<16>(X, bf16, n, d, ld, G, kappa, order, m, labels, k, D, counts, S, n_moved, st, s);
    default: return boost_epoch_pl<32>(X, bf16, n, d, ld, G, kappa, order, m, labels, k, D, counts, S, n_moved, st, s);
    }
}

}  // namespace gkm
