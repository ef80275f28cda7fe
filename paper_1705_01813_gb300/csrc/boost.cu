// Boost form of GK-means (Sec. 3.1 Eq. 2 and Eq. 3; the move step of Alg. 2,
// Sec. 4.2).  State per cluster r: the composite vector D_r (FP64, the sum of
// its members, Eq. 2), its size n_r and S_r = D_r'D_r.  Alg. 2 visits samples
// one at a time; sample i in cluster u looks at the clusters of its kappa
// neighbours and moves to the one whose Eq. 3 gain
//     ((D_v + x)'(D_v + x) / (n_v + 1) + (D_u - x)'(D_u - x) / (n_u - 1)) - S_v / n_v - S_u / n_u
// is largest, if that gain is positive.  Each move changes two clusters and one
// label before the next visit reads them, so the result is that of visiting in
// order; the kernel below evaluates windows of visits at once and commits them
// in order only as far as that result allows.
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
// arrays.  One thread-block cluster (up to 16 CTAs, one per SM) runs the
// epoch: one warp per (visit, cluster) task computes the squared norm of
// D_v + x (D_u - x) with lane l holding elements l + 32 m, the owning CTA
// divides its tasks' terms, and CTA 0 takes the arg-max of each visit, finds
// how far the window may commit and applies the moves.  GB300 runs FP64 at a
// small fraction of its FP32 rate, so the FP64 work is spread over the
// cluster's SMs.  After a move, S_u and S_v are the two norms already computed
// for the decision: the new rows are exactly the rounded sums that were
// squared.
#include <climits>
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
    return widen(ldx(p));
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
// One epoch of the move step over order[0..m), on one cluster of R CTAs, in
// windows of up to W visits.
//
// A window's visits are evaluated together against the state at its start:
// every CTA stages the window's samples and gathers the candidate sets; the
// squared norms of all the window's (visit, cluster) tasks are spread over the
// cluster's warps, and each CTA divides its own tasks' terms (lanes over
// tasks) and stores them into CTA 0.  CTA 0 takes each visit's arg-max (a
// shared atomicMax of the gain keys, then an atomicMin of (label, candidate)
// among the tasks at the maximum), then commits the visits in order up to the
// first one whose inputs an earlier committed move of the window changed (its
// sample or one of its neighbours moved; its own cluster or a candidate was
// the source or target of a move), found by looking every visit's items up in
// two small hash tables of the moving visits' samples and clusters.
// A committed visit therefore saw exactly the state the sequential walk gives
// it, and the committed moves touch disjoint clusters, so CTA 0 applies them
// together; the next window starts at the first visit not committed (the
// first visit of a window always commits).  The window grows while windows
// commit whole and shrinks to twice what the last one committed, so that few
// evaluations are thrown away where moves collide often.  Both cluster
// barriers of a window are unconditional.  Mutable state (labels, D, S,
// counts) is read through L2 (ld.global.cg), which the barriers order.
// ---------------------------------------------------------------------------
constexpr int BE_THREADS = 256;
constexpr int BE_WARPS = BE_THREADS / 32;
constexpr int BE_MAX_CLUSTER = 16;
constexpr int BE_MAX_WINDOW = 32;
constexpr int BE_HASH = 128;  // entries of each commit hash table (at most 32 samples, 64 clusters)
constexpr size_t BE_SMEM_BUDGET = 200 * 1024;

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

// Dynamic shared memory of one CTA for windows of W visits (the same layout in every CTA of the cluster).
struct WinLayout {
    int W, kp, TM, TL;
    size_t xs, ra, r1, r3, gk, vbest, vwin, la, ls, rn, ln, lo, tv, sq, sg, svis, su, snq, sbase, dq, ml, tl, mvj,
        hkey, hval, bytes;
    __host__ __device__ WinLayout(int W_, int P, int kappa, int R)
    {
        W = W_;
        kp = (kappa + 31) / 32 * 32;
        TM = W * (kappa + 1);
        TL = (TM + R - 1) / R;
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o += (bytes + 15) / 16 * 16;
            return at;
        };
        xs = take((size_t)W * P * 8);
        ra = take((size_t)TM * 8);
        r1 = take((size_t)TM * 8);
        r3 = take((size_t)TM * 8);
        gk = take((size_t)TM * 8);
        vbest = take((size_t)W * 8);
        vwin = take((size_t)W * 8);
        la = take((size_t)TL * 8);
        ls = take((size_t)TL * 8);
        rn = take((size_t)TM * 4);
        ln = take((size_t)TL * 4);
        lo = take((size_t)TL * 4);
        tv = take((size_t)TM * 4);
        sq = take((size_t)W * kp * 4);
        sg = take((size_t)W * kp * 4);
        svis = take((size_t)W * 4);
        su = take((size_t)W * 4);
        snq = take((size_t)W * 4);
        sbase = take((size_t)(W + 1) * 4);
        dq = take((size_t)W * 4);
        ml = take((size_t)W * 4);
        tl = take((size_t)2 * W * 4);
        mvj = take((size_t)W * 4);
        hkey = take((size_t)2 * BE_HASH * 4);
        hval = take((size_t)2 * BE_HASH * 4);
        bytes = o;
    }
};

template <typename XT, int PL>
__global__ void __launch_bounds__(BE_THREADS, 1)
    k_boost_epoch(const XT *__restrict__ X, int32_t n, int d, int64_t ld, const int32_t *__restrict__ G, int kappa,
                  const int32_t *__restrict__ order, int64_t m, int32_t *L, int32_t k, double *D, int32_t *cnt,
                  double *S, int64_t *n_moved, DevStatus *st, int W)
{
    constexpr int P = 32 * PL;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_win, s_nm, s_T, s_first;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int rank = (int)cluster_rank(), R = (int)cluster_size();
    const WinLayout Y(W, P, kappa, R);
    const int kp = Y.kp;
    double *xs = reinterpret_cast<double *>(smem + Y.xs);
    double *ra = reinterpret_cast<double *>(smem + Y.ra), *r1 = reinterpret_cast<double *>(smem + Y.r1);
    double *r3 = reinterpret_cast<double *>(smem + Y.r3);
    long long *gk = reinterpret_cast<long long *>(smem + Y.gk);
    long long *vbest = reinterpret_cast<long long *>(smem + Y.vbest);
    unsigned long long *vwin = reinterpret_cast<unsigned long long *>(smem + Y.vwin);
    int *hkey = reinterpret_cast<int *>(smem + Y.hkey), *hval = reinterpret_cast<int *>(smem + Y.hval);
    int *tv = reinterpret_cast<int *>(smem + Y.tv);
    double *la = reinterpret_cast<double *>(smem + Y.la), *ls = reinterpret_cast<double *>(smem + Y.ls);
    int *rn = reinterpret_cast<int *>(smem + Y.rn), *ln = reinterpret_cast<int *>(smem + Y.ln);
    int *lo = reinterpret_cast<int *>(smem + Y.lo);
    int *sq = reinterpret_cast<int *>(smem + Y.sq), *sg = reinterpret_cast<int *>(smem + Y.sg);
    int *svis = reinterpret_cast<int *>(smem + Y.svis), *su = reinterpret_cast<int *>(smem + Y.su);
    int *snq = reinterpret_cast<int *>(smem + Y.snq), *sbase = reinterpret_cast<int *>(smem + Y.sbase);
    int *dq = reinterpret_cast<int *>(smem + Y.dq), *ml = reinterpret_cast<int *>(smem + Y.ml);
    int *tl = reinterpret_cast<int *>(smem + Y.tl), *mvj = reinterpret_cast<int *>(smem + Y.mvj);
    auto valid = [&](int i) { return i >= 0 && i < n; };
    int64_t moves = 0;
    int We = W;  // this window's size: doubled after a window that commits whole, else twice what committed
    cluster_barrier();  // every CTA of the cluster runs before any stores into another's shared memory

    for (int64_t s = 0; s < m;) {
        const int Wn = (int)(m - s < (int64_t)We ? m - s : (int64_t)We);
        // ---- the window's visits: ids, then samples, graph rows and own labels, then the neighbours' labels
        if (threadIdx.x < Wn) {
            svis[threadIdx.x] = __ldg(order + s + threadIdx.x);
            vbest[threadIdx.x] = LLONG_MIN;
            vwin[threadIdx.x] = ~0ull;
        }
        __syncthreads();
        if (threadIdx.x < Wn) {
            const int i = svis[threadIdx.x];
            int u = -1;
            if (!valid(i)) {
                if (rank == 0)
                    flag_error(st, GK_ERR_INVALID, (unsigned)(s + threadIdx.x));
            } else {
                u = __ldcg(L + i);
                if (u < 0 || u >= k) {
                    if (rank == 0)
                        flag_error(st, GK_ERR_INVALID, (unsigned)i);
                    u = -1;
                }
            }
            su[threadIdx.x] = u;
        }
        // loads issued eight at a time per thread, then stored: one round trip per batch
        for (int e0 = threadIdx.x; e0 < Wn * P; e0 += 8 * BE_THREADS) {
            float v[8];
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const int e = e0 + b * BE_THREADS, j = e / P, t = e - j * P;
                v[b] = e < Wn * P && valid(svis[j]) && t < d ? ldx(X + (int64_t)svis[j] * ld + t) : 0.f;
            }
#pragma unroll
            for (int b = 0; b < 8; b++)
                if (e0 + b * BE_THREADS < Wn * P)
                    xs[e0 + b * BE_THREADS] = widen(v[b]);  // on the integer pipe: the FP64 one is narrow
        }
        for (int e0 = threadIdx.x; e0 < Wn * kp; e0 += 8 * BE_THREADS) {
            int v[8];
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const int e = e0 + b * BE_THREADS, j = e / kp, t = e - j * kp;
                v[b] = e < Wn * kp && valid(svis[j]) && t < kappa ? __ldg(G + (int64_t)svis[j] * kappa + t) : -1;
            }
#pragma unroll
            for (int b = 0; b < 8; b++)
                if (e0 + b * BE_THREADS < Wn * kp)
                    sg[e0 + b * BE_THREADS] = v[b];
        }
        __syncthreads();
        for (int e0 = threadIdx.x; e0 < Wn * kp; e0 += 8 * BE_THREADS) {
            int v[8];
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const int e = e0 + b * BE_THREADS;
                v[b] = -3;  // -3: no label wanted
                if (e < Wn * kp && e % kp < kappa && su[e / kp] >= 0)
                    v[b] = valid(sg[e]) ? __ldcg(L + sg[e]) : -2;
            }
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const int e = e0 + b * BE_THREADS;
                if (e >= Wn * kp)
                    continue;
                if (v[b] == -2 || (v[b] != -3 && (v[b] < 0 || v[b] >= k))) {
                    if (rank == 0)
                        flag_error(st, GK_ERR_INVALID, (unsigned)(v[b] == -2 ? svis[e / kp] : sg[e]));
                    v[b] = -1;
                }
                sq[e] = v[b] == -3 ? -1 : v[b];
            }
        }
        __syncthreads();
        // candidate set of visit j (warp w takes j = w, w + 8, ...): distinct labels other than its own, in place
        for (int j = w; j < Wn; j += BE_WARPS) {
            const int u = su[j];
            int lab[MAX_KAPPA / 32];
#pragma unroll
            for (int c = 0; c < MAX_KAPPA / 32; c++)
                lab[c] = 32 * c < kp ? sq[j * kp + 32 * c + lane] : -1;
            __syncwarp();
            int nq = 0;
#pragma unroll
            for (int c = 0; c < MAX_KAPPA / 32; c++) {
                if (32 * c >= kp)
                    break;
                int v = lab[c] == u ? -1 : lab[c];
                bool keep = v >= 0;
#pragma unroll 8
                for (int q = 0; q < nq; q++)
                    keep &= sq[j * kp + q] != v;
                const unsigned same = __match_any_sync(FULL_MASK, v);
                keep = keep && (__ffs(same) - 1 == lane);
                const unsigned km = __ballot_sync(FULL_MASK, keep);
                if (keep)
                    sq[j * kp + nq + __popc(km & lanemask_lt())] = v;
                nq += __popc(km);
                __syncwarp();
            }
            if (lane == 0)
                snq[j] = u >= 0 ? nq : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {  // tasks of visit j: [sbase[j], sbase[j + 1]), the first its own cluster
            int T = 0;
            for (int j = 0; j < Wn; j++) {
                sbase[j] = T;
                T += snq[j] > 0 ? snq[j] + 1 : 0;
            }
            sbase[Wn] = T;
            s_T = T;
        }
        __syncthreads();
        for (int j = w; j < Wn; j += BE_WARPS)
            for (int t = sbase[j] + lane; t < sbase[j + 1]; t += 32)
                tv[t] = j;
        __syncthreads();

        // ---- squared norms of the tasks: task t on CTA t mod R; c = 0 the own cluster (D_u - x), else a
        //      candidate (D_v + x)
        const int T = s_T;
        for (int t = rank + R * w; t < T; t += R * BE_WARPS) {
            const int j = tv[t];
            const int c = t - sbase[j];
            const int r = c == 0 ? su[j] : sq[j * kp + c - 1];
            const double *Dr = D + (int64_t)r * d;
            const double *xj = xs + (size_t)j * P;
            double a[PL];
#pragma unroll
            for (int q = 0; q < PL; q++) {
                const int e = lane + 32 * q;
                a[q] = e < d ? __ldcg(Dr + e) : 0.0;
            }
            double sr = 0.0;
            int nr = 0;
            if (lane == 0) {
                sr = __ldcg(S + r);
                nr = __ldcg(cnt + r);
            }
#pragma unroll
            for (int q = 0; q < PL; q++) {
                const int e = lane + 32 * q;
                const double y = e < d ? (c == 0 ? __dsub_rn(a[q], xj[e]) : __dadd_rn(a[q], xj[e])) : 0.0;
                a[q] = __dmul_rn(y, y);
            }
            const double tot = fold_lanes<PL>(a);
            if (lane == 0) {
                const int l = t / R;
                la[l] = tot;
                ls[l] = sr;
                ln[l] = nr;
                lo[l] = c == 0;
            }
        }
        __syncthreads();
        // this CTA's tasks' quotients, lanes over tasks; job even: A / (n_v + 1) (own: B / (n_u - 1)), odd: S / n
        const int TLc = T > rank ? (T - rank + R - 1) / R : 0;
        for (int jb = w; jb < 2 * ((TLc + 31) / 32); jb += BE_WARPS) {
            const int l = (jb >> 1) * 32 + lane;
            if (l < TLc) {
                const int t = l * R + rank;
                if (jb & 1) {
                    st_rank(&r3[t], 0, __ddiv_rn(ls[l], (double)ln[l]));
                } else {
                    st_rank(&r1[t], 0, __ddiv_rn(la[l], (double)(lo[l] ? ln[l] - 1 : ln[l] + 1)));
                    st_rank(&ra[t], 0, la[l]);
                    st_rank(&rn[t], 0, ln[l]);
                }
            }
        }
        cluster_barrier();

        // ---- CTA 0: each visit's arg-max, the in-order commit and the committed moves
        if (rank == 0) {
            // the gain of every candidate task as an integer key in the order of the FP64 values (the gains are sums
            // and differences of non-negative terms, never -0, so the keys order them exactly); each visit's largest
            // key, then the smallest (label, candidate) among the tasks that reach it
            for (int t = threadIdx.x; t < T; t += BE_THREADS) {
                const int j = tv[t], o = sbase[j];
                if (t != o) {
                    const double g = __dsub_rn(__dsub_rn(__dadd_rn(r1[t], r1[o]), r3[t]), r3[o]);
                    const long long b = __double_as_longlong(g);
                    const long long key = b ^ ((b >> 63) & 0x7fffffffffffffffll);
                    gk[t] = key;
                    atomicMax(&vbest[j], key);
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < T; t += BE_THREADS) {
                const int j = tv[t], o = sbase[j];
                if (t != o && gk[t] == vbest[j]) {
                    const unsigned long long label = (unsigned)sq[j * kp + t - o - 1];
                    atomicMin(&vwin[j], (label << 16) | (unsigned)(t - o));
                }
            }
            for (int e = threadIdx.x; e < 2 * BE_HASH; e += BE_THREADS) {  // empty hash tables
                hkey[e] = -1;
                hval[e] = 0x7fffffff;
            }
            __syncthreads();
            // the visits that would move (key > 0: gain > +0; the own cluster keeps two members or more), in order:
            // sample ml, clusters tl[2 q] (from) and tl[2 q + 1] (to)
            if (w == 0) {
                int t = -1;
                if (lane < Wn && snq[lane] > 0 && rn[sbase[lane]] >= 2 && vbest[lane] > 0)
                    t = sbase[lane] + (int)(vwin[lane] & 0xffff);
                if (lane < Wn)
                    dq[lane] = t;
                const unsigned mm = __ballot_sync(FULL_MASK, t >= 0);
                if (t >= 0) {
                    const int q = __popc(mm & lanemask_lt());
                    ml[q] = svis[lane];
                    mvj[q] = lane;
                    tl[2 * q] = su[lane];
                    tl[2 * q + 1] = (int)(vwin[lane] >> 16);
                }
                if (lane == 0) {
                    s_nm = __popc(mm);
                    s_first = Wn;
                }
            }
            __syncthreads();
            // hash tables keyed by sample and by cluster: the earliest moving visit that moves that sample, or leaves
            // or joins that cluster
            const int nmv = s_nm;
            if (threadIdx.x < 3 * nmv) {
                const int q = threadIdx.x / 3, part = threadIdx.x - 3 * q;
                const int x = part == 0 ? ml[q] : tl[2 * q + part - 1];
                int *keys = hkey + (part == 0 ? 0 : BE_HASH), *vals = hval + (part == 0 ? 0 : BE_HASH);
                for (int h = (int)(((unsigned)x * 2654435761u) >> 25), probe = 0; probe < BE_HASH;
                     h = (h + 1) & (BE_HASH - 1), probe++) {
                    const int prev = atomicCAS(&keys[h], -1, x);
                    if (prev == -1 || prev == x) {
                        atomicMin(&vals[h], mvj[q]);
                        break;
                    }
                }
            }
            __syncthreads();
            // the window commits up to the first visit that depends on an earlier moving visit: its sample or a
            // neighbour is that visit's sample, or its own cluster or a candidate is one that visit leaves or joins
            auto earliest = [&](int x, int table) {  // the earliest moving visit recorded for x, or Wn
                const int *keys = hkey + table * BE_HASH, *vals = hval + table * BE_HASH;
                for (int h = (int)(((unsigned)x * 2654435761u) >> 25), probe = 0; probe < BE_HASH;
                     h = (h + 1) & (BE_HASH - 1), probe++) {
                    const int kx = keys[h];
                    if (kx == x)
                        return vals[h];
                    if (kx == -1)
                        break;
                }
                return 0x7fffffff;
            };
            if (nmv > 0) {
                for (int j = mvj[0] + 1 + w; j < Wn; j += BE_WARPS) {
                    bool hit = false;
                    for (int c = lane; c <= kappa; c += 32) {  // the sample (c = 0) and its neighbours
                        const int x = c == 0 ? svis[j] : sg[j * kp + c - 1];
                        hit |= x >= 0 && earliest(x, 0) < j;
                    }
                    if (su[j] >= 0)
                        for (int c = lane; c <= snq[j]; c += 32) {  // the own cluster (c = 0) and the candidates
                            const int x = c == 0 ? su[j] : sq[j * kp + c - 1];
                            hit |= earliest(x, 1) < j;
                        }
                    if (__any_sync(FULL_MASK, hit) && lane == 0)
                        atomicMin(&s_first, j);
                }
            }
            __syncthreads();
            const int done = s_first;
            if (w == 0) {
                if (lane < R)
                    st_rank(&s_win, lane, done);
            }
            int nm = 0;  // the committed moves: the moving visits before `done`
            while (nm < nmv && mvj[nm] < done)
                nm++;
            // the committed moves touch disjoint clusters: x leaves S_u for S_v in each
            for (int e = threadIdx.x; e < nm * d; e += BE_THREADS) {
                const int q = e / d, t = e - q * d, j = mvj[q];
                const int u = su[j], v = tl[2 * q + 1];
                const double x = xs[(size_t)j * P + t];
                D[(int64_t)u * d + t] = __dsub_rn(__ldcg(D + (int64_t)u * d + t), x);
                D[(int64_t)v * d + t] = __dadd_rn(__ldcg(D + (int64_t)v * d + t), x);
            }
            if (threadIdx.x < nm) {
                const int j = mvj[threadIdx.x], o = sbase[j], t = dq[j];
                const int u = su[j], v = tl[2 * threadIdx.x + 1];
                cnt[u] = rn[o] - 1;
                cnt[v] = rn[t] + 1;
                S[u] = ra[o];
                S[v] = ra[t];
                L[svis[j]] = v;
            }
            moves += nm;
        }
        cluster_barrier();  // the window's moves before the next window reads labels and rows
        const int got = s_win;  // the same in every CTA
        We = got == Wn ? (2 * We < W ? 2 * We : W) : (2 * got < W ? (2 * got > 2 ? 2 * got : 2) : W);
        s += got;
    }
    if (rank == 0 && threadIdx.x == 0 && n_moved)
        *n_moved = moves;
}

// Largest cluster (at most BE_MAX_CLUSTER CTAs) the device can run for this kernel with `smem` bytes of dynamic
// shared memory per CTA, once per device and kernel.
template <typename KernelT>
int epoch_cluster_size(KernelT kern, size_t smem)
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
    int r = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) {
        r = 8;  // portable size
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(BE_MAX_CLUSTER);
            cfg.blockDim = dim3(BE_THREADS);
            cfg.dynamicSmemBytes = smem;
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
    const int R = epoch_cluster_size(kern, BE_SMEM_BUDGET);
    if (R < 1)
        return cudaErrorInvalidConfiguration;
    int W = BE_MAX_WINDOW;  // the largest window whose layout fits the budget
    while (W > 1 && WinLayout(W, 32 * PL, kappa, R).bytes > BE_SMEM_BUDGET)
        W--;
    const size_t smem = WinLayout(W, 32 * PL, kappa, R).bytes;
    if (smem > BE_SMEM_BUDGET)
        return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)R);
    cfg.blockDim = dim3(BE_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)R;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, X, (int32_t)n, (int)d, ld, G, (int)kappa, order, m, L, k, D, cnt, S,
                              n_moved, st, W);
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
