/*
 * GK-means oracle: a plain, slow, FP64 CPU restatement of the graph-guided
 * k-means of Deng & Zhao, "Fast k-means based on KNN Graph" (arXiv 1705.01813).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker for the CUDA
 * library.  It shares no code, header, table or helper with the CUDA path, and
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  The product path never calls it.
 *
 * Every function follows the paper in its own order and notation:
 *   - k-means objective and the two Lloyd steps: Eq. 1 and the paragraph after it (Sec. 1)
 *   - composite vectors D_r and the objective I: Eq. 2 (Sec. 3.1)
 *   - candidate clusters from the kappa neighbours: Alg. 2 (Sec. 4.2), in the
 *     form given at the end of Sec. 4.2, where a sample takes the nearest
 *     centroid among the collected clusters
 *   - KNN-graph construction by repeated fast k-means: Alg. 3 (Sec. 4.3)
 *   - cluster count k0 = floor(n / xi): Alg. 3 and Sec. 4.3
 *   - one k-means iteration per graph round: Sec. 4.5
 *   - average distortion: Eq. 4 (Sec. 5.1)
 *   - two-means tree, the initial partition of Alg. 2: Alg. 1 (Sec. 3.2),
 *     with its own readings T1-T6 stated where it is defined
 *
 * Readings where the paper is silent (all stated again where they are used):
 *   R1 the sample's own cluster is a candidate as well as its neighbours';
 *   R2 the assignment is synchronous (every sample against the previous centroids);
 *   R3 ties go to the smaller (distance, label) / (distance, index) key;
 *   R4 an empty cluster keeps its previous centroid and has no members;
 *   R5 labels and centroids carry over from one graph round to the next;
 *   R6 a cluster larger than max_cluster is cut into ceil(m / max_cluster)
 *      runs of consecutive members (ascending sample id) whose sizes differ by
 *      at most one;
 *   R7 graph distances are squared Euclidean; graph rows hold no self and no
 *      repeated neighbour and are sorted by (distance, index);
 *   R8 random numbers come from the SplitMix64 generator (Steele, Lea & Flood,
 *      OOPSLA 2014) used as a counter-based function, see or_draw().
 *
 * Inputs X are read as stored (FP32) and widened to FP64 element by element.
 *
 * Threads: with OpenMP the loops over samples, runs and clusters are shared
 * out over the host cores; every result is written by one thread and every sum
 * keeps its order (a cluster's members in ascending id, the distortion over
 * samples in index order), so the results do not depend on the thread count
 * (or_set_threads; tests check it).
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------- */
/* R8: SplitMix64.  The published generator keeps a 64-bit state s, adds the   */
/* constant gamma = 0x9E3779B97F4A7C15 and returns a mixed copy of the state.  */
/* The j-th output (j >= 1) of the generator seeded with `key` is therefore    */
/* mix(key + j * gamma); or_draw(key, c) returns output c + 1.                 */
/* ------------------------------------------------------------------------- */
static const uint64_t OR_GAMMA = 0x9E3779B97F4A7C15ULL;
static const uint64_t OR_TAG_LABELS = 0x4C41424C00000000ULL; /* "LABL" */
static const uint64_t OR_TAG_GRAPH = 0x4752415000000000ULL;  /* "GRAP" */

static uint64_t or_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The generator as published: advance the state, return the mixed state. */
uint64_t or_splitmix64_next(uint64_t *state)
{
    *state += OR_GAMMA;
    return or_mix(*state);
}

uint64_t or_draw(uint64_t key, uint64_t counter)
{
    return or_mix(key + (counter + 1) * OR_GAMMA);
}

/* Threads of the parallel loops (1: single-threaded); returns the count in effect. */
int or_set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0)
        omp_set_num_threads(threads);
    return omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* squared Euclidean distance in FP64, inputs widened exactly */
static double or_d2_ff(const float *a, const float *b, int64_t d)
{
    double s = 0.0;
    for (int64_t t = 0; t < d; t++) {
        double diff = (double)a[t] - (double)b[t];
        s += diff * diff;
    }
    return s;
}

static double or_d2_fd(const float *a, const double *c, int64_t d)
{
    double s = 0.0;
    for (int64_t t = 0; t < d; t++) {
        double diff = (double)a[t] - c[t];
        s += diff * diff;
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* Seeded initial state                                                      */
/* ------------------------------------------------------------------------- */

/* Seeded random initial labelling: label of sample i = draw(seed^LABL, i) mod k. */
void or_init_labels(int64_t n, int32_t k, uint64_t seed, int32_t *labels)
{
    uint64_t key = seed ^ OR_TAG_LABELS;
    for (int64_t i = 0; i < n; i++)
        labels[i] = (int32_t)(or_draw(key, (uint64_t)i) % (uint64_t)k);
}

/* Key order of R3/R7: smaller distance first, then smaller index. */
static int or_key_less(double da, int32_t ia, double db, int32_t ib)
{
    return da < db || (da == db && ia < ib);
}

/* insertion sort of one graph row by (distance, index) */
static void or_sort_row(int32_t *idx, double *dist, int32_t len)
{
    for (int32_t a = 1; a < len; a++) {
        int32_t ii = idx[a];
        double dd = dist[a];
        int32_t b = a - 1;
        while (b >= 0 && or_key_less(dd, ii, dist[b], idx[b])) {
            idx[b + 1] = idx[b];
            dist[b + 1] = dist[b];
            b--;
        }
        idx[b + 1] = ii;
        dist[b + 1] = dd;
    }
}

/*
 * Random initial KNN graph (Alg. 3 begins from random neighbour lists).
 * Row i draws j = draw(seed^GRAP, i * 2^32 + a) mod n for a = 0, 1, ...,
 * rejects j == i and indices it already holds, and stops at kappa accepted.
 * The row is then sorted by (distance, index) (R7).
 */
void or_init_graph(const float *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed,
                   int32_t *g_idx, double *g_dist)
{
    uint64_t key = seed ^ OR_TAG_GRAPH;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        int32_t *row = g_idx + i * kappa;
        double *rd = g_dist + i * kappa;
        int32_t got = 0;
        for (uint64_t a = 0; got < kappa; a++) {
            int64_t j = (int64_t)(or_draw(key, ((uint64_t)i << 32) | a) % (uint64_t)n);
            if (j == i)
                continue;
            int dup = 0;
            for (int32_t q = 0; q < got; q++)
                if (row[q] == j) {
                    dup = 1;
                    break;
                }
            if (dup)
                continue;
            row[got] = (int32_t)j;
            rd[got] = or_d2_ff(X + i * ld, X + j * ld, d);
            got++;
        }
        or_sort_row(row, rd, kappa);
    }
}

/*
 * The same initial rows for a few listed samples only (for spot checks at
 * sizes where the full construction is too slow): row q of g_idx / g_dist
 * receives sample rows[q]'s list, drawn and sorted exactly as above.
 */
void or_init_graph_rows(const float *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed,
                        const int64_t *rows, int64_t nrows, int32_t *g_idx, double *g_dist)
{
    uint64_t key = seed ^ OR_TAG_GRAPH;
    for (int64_t q = 0; q < nrows; q++) {
        const int64_t i = rows[q];
        int32_t *row = g_idx + q * kappa;
        double *rd = g_dist + q * kappa;
        int32_t got = 0;
        for (uint64_t a = 0; got < kappa; a++) {
            int64_t j = (int64_t)(or_draw(key, ((uint64_t)i << 32) | a) % (uint64_t)n);
            if (j == i)
                continue;
            int dup = 0;
            for (int32_t t = 0; t < got; t++)
                if (row[t] == j) {
                    dup = 1;
                    break;
                }
            if (dup)
                continue;
            row[got] = (int32_t)j;
            rd[got] = or_d2_ff(X + i * ld, X + j * ld, d);
            got++;
        }
        or_sort_row(row, rd, kappa);
    }
}

/* ------------------------------------------------------------------------- */
/* Assignment: Alg. 2 with the closest-centroid rule (GK-means^-)            */
/* ------------------------------------------------------------------------- */

/*
 * For each listed sample i (all samples when rows == NULL):
 *   Q = { L[i] } (R1)  union  { L[G[i][j]] : j < kappa }   (Alg. 2, candidate loop)
 *   L'[i] = the r in Q with the smallest (||x_i - C_r||^2, r)  (R2, R3)
 * best[i] receives that distance and uniq[i] (optional) the size of Q.
 * When kappa == 0 and all_clusters != 0 every cluster is a candidate
 * (exhaustive Lloyd assignment, the textbook rule after Eq. 1).
 */
static void or_assign_impl(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *G, int32_t kappa,
                           const double *C, int32_t k, const int32_t *L_in, int32_t *L_out, double *best,
                           int32_t *uniq, const int64_t *rows, int64_t nrows, int all_clusters)
{
    int64_t cnt = rows ? nrows : n;
#pragma omp parallel
    {
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kappa + 1));
#pragma omp for schedule(dynamic, 256)
    for (int64_t r = 0; r < cnt; r++) {
        int64_t i = rows ? rows[r] : r;
        const float *x = X + i * ld;
        int32_t bestr = -1;
        double bestd = 0.0;
        int32_t u = 0;
        if (all_clusters) {
            for (int32_t c = 0; c < k; c++) {
                double dd = or_d2_fd(x, C + (int64_t)c * d, d);
                if (bestr < 0 || or_key_less(dd, c, bestd, bestr)) {
                    bestd = dd;
                    bestr = c;
                }
            }
            u = k;
        } else {
            Q[u++] = L_in[i];
            for (int32_t j = 0; j < kappa; j++) {
                int32_t lab = L_in[G[i * kappa + j]];
                int seen = 0;
                for (int32_t q = 0; q < u; q++)
                    if (Q[q] == lab) {
                        seen = 1;
                        break;
                    }
                if (!seen)
                    Q[u++] = lab;
            }
            for (int32_t q = 0; q < u; q++) {
                double dd = or_d2_fd(x, C + (int64_t)Q[q] * d, d);
                if (bestr < 0 || or_key_less(dd, Q[q], bestd, bestr)) {
                    bestd = dd;
                    bestr = Q[q];
                }
            }
        }
        if (L_out)
            L_out[rows ? r : i] = bestr;
        if (best)
            best[rows ? r : i] = bestd;
        if (uniq)
            uniq[rows ? r : i] = u;
    }
    free(Q);
    }
}

void or_assign(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *G, int32_t kappa,
               const double *C, int32_t k, const int32_t *L_in, int32_t *L_out, double *best, int32_t *uniq,
               const int64_t *rows, int64_t nrows)
{
    or_assign_impl(X, n, d, ld, G, kappa, C, k, L_in, L_out, best, uniq, rows, nrows, 0);
}

/*
 * Near-tie report of the assignment (for the checks of this oracle against
 * arithmetic of another precision; not a step of the paper).  For each sample
 * i: Q as the assignment forms it (own label, then the kappa neighbours'
 * labels, each cluster once), the two smallest squared distances
 * d1 <= d2 to distinct clusters of Q, and margin[i] = (d2 - d1) / d1:
 * 0 for an exact tie, +inf when Q holds one cluster or d1 = 0 < d2.  A
 * sample whose margin is below a tolerance may go to either of its two best
 * clusters under arithmetic that rounds differently.
 */
void or_assign_margin(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *G, int32_t kappa,
                      const double *C, const int32_t *L_in, double *margin)
{
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kappa + 1));
    for (int64_t i = 0; i < n; i++) {
        int32_t u = 0;
        Q[u++] = L_in[i];
        for (int32_t j = 0; j < kappa; j++) {
            int32_t lab = L_in[G[i * kappa + j]];
            int seen = 0;
            for (int32_t q = 0; q < u; q++)
                if (Q[q] == lab) {
                    seen = 1;
                    break;
                }
            if (!seen)
                Q[u++] = lab;
        }
        double d1 = INFINITY, d2 = INFINITY;
        for (int32_t q = 0; q < u; q++) {
            double dd = or_d2_fd(X + i * ld, C + (int64_t)Q[q] * d, d);
            if (dd < d1) {
                d2 = d1;
                d1 = dd;
            } else if (dd < d2) {
                d2 = dd;
            }
        }
        if (u < 2)
            margin[i] = INFINITY;
        else if (d1 > 0.0)
            margin[i] = (d2 - d1) / d1;
        else
            margin[i] = d2 > 0.0 ? INFINITY : 0.0;
    }
    free(Q);
}

/* Exhaustive Lloyd assignment: every one of the k centroids is a candidate. */
void or_assign_exhaustive(const float *X, int64_t n, int64_t d, int64_t ld, const double *C, int32_t k,
                          int32_t *L_out, double *best)
{
    or_assign_impl(X, n, d, ld, NULL, 0, C, k, NULL, L_out, best, NULL, NULL, 0, 1);
}

static void or_group(const int32_t *L, int64_t n, int32_t k, int64_t *offsets, int32_t *members);

/* ------------------------------------------------------------------------- */
/* Update: centroid = mean of members (Sec. 1), D_r of Eq. 2, E of Eq. 4     */
/* ------------------------------------------------------------------------- */

/*
 * counts[r] = n_r, D_r = sum of the members of S_r (ascending sample order),
 * C_r = D_r / n_r, and an empty cluster keeps its previous C_r (R4).
 * On return *E = (1/n) sum_i ||x_i - C_{L[i]}||^2 (Eq. 4, computed directly)
 * and, if I_out is given, *I_out = sum_r D_r'D_r / n_r (Eq. 2).
 */
void or_update(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *L, int32_t k, double *C,
               int64_t *counts, double *E, double *I_out)
{
    double *D = (double *)calloc((size_t)k * (size_t)d, sizeof(double));
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)k + 1));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    or_group(L, n, k, off, mem); /* S_r: the members of cluster r in ascending sample order */
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t r = 0; r < k; r++) {
        counts[r] = off[r + 1] - off[r];
        for (int64_t p = off[r]; p < off[r + 1]; p++) {
            const int64_t i = mem[p];
            for (int64_t t = 0; t < d; t++)
                D[(int64_t)r * d + t] += (double)X[i * ld + t];
        }
    }
    double I = 0.0;
    for (int32_t r = 0; r < k; r++) {
        if (counts[r] == 0)
            continue;
        double dd = 0.0;
        for (int64_t t = 0; t < d; t++) {
            C[(int64_t)r * d + t] = D[(int64_t)r * d + t] / (double)counts[r];
            dd += D[(int64_t)r * d + t] * D[(int64_t)r * d + t];
        }
        I += dd / (double)counts[r];
    }
    if (E) {
        /* the terms in parallel, their sum in index order */
        double *term = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            term[i] = or_d2_fd(X + i * ld, C + (int64_t)L[i] * d, d);
        double s = 0.0;
        for (int64_t i = 0; i < n; i++)
            s += term[i];
        *E = s / (double)n;
        free(term);
    }
    if (I_out)
        *I_out = I;
    free(D);
    free(off);
    free(mem);
}

/* ------------------------------------------------------------------------- */
/* Fit: C^0 = update(L^0); then T times { assign; update }                    */
/* ------------------------------------------------------------------------- */

/*
 * E_log (2*iters + 1 entries): E after the initial update, then for each
 * iteration E after the assignment (mean best distance against the previous
 * centroids) and E after the update.  C starts at zero so that a cluster
 * empty from the start has a defined (unused) centroid.
 */
void or_fit(const float *X, int64_t n, int64_t d, int64_t ld, int32_t k, const int32_t *G, int32_t kappa,
            int32_t iters, const int32_t *L0, int32_t *L, double *C, int64_t *counts, double *E_log)
{
    int32_t *L2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *best = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(L, L0, sizeof(int32_t) * (size_t)n);
    memset(C, 0, sizeof(double) * (size_t)k * (size_t)d);
    or_update(X, n, d, ld, L, k, C, counts, &E_log[0], NULL);
    for (int32_t t = 0; t < iters; t++) {
        or_assign(X, n, d, ld, G, kappa, C, k, L, L2, best, NULL, NULL, 0);
        double s = 0.0;
        for (int64_t i = 0; i < n; i++)
            s += best[i];
        E_log[1 + 2 * t] = s / (double)n;
        memcpy(L, L2, sizeof(int32_t) * (size_t)n);
        or_update(X, n, d, ld, L, k, C, counts, &E_log[2 + 2 * t], NULL);
    }
    free(L2);
    free(best);
}

/* ------------------------------------------------------------------------- */
/* Graph refinement: Alg. 3, exhaustive pairs inside each cluster            */
/* ------------------------------------------------------------------------- */

/* Cluster set S as lists of members in ascending sample id (counting sort). */
static void or_group(const int32_t *L, int64_t n, int32_t k, int64_t *offsets, int32_t *members)
{
    int64_t *fill = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    for (int32_t r = 0; r <= k; r++)
        offsets[r] = 0;
    for (int64_t i = 0; i < n; i++)
        offsets[L[i] + 1]++;
    for (int32_t r = 0; r < k; r++)
        offsets[r + 1] += offsets[r];
    for (int64_t i = 0; i < n; i++) {
        int32_t r = L[i];
        members[offsets[r] + fill[r]] = (int32_t)i;
        fill[r]++;
    }
    free(fill);
}

/*
 * Merge the pair (dist, j) into row i (Alg. 3: a compared pair updates both rows):
 * the row keeps its kappa smallest keys (R3/R7), never holds j twice and never
 * holds i.  The row is sorted, so the new key is placed by insertion.
 */
static void or_merge(int32_t *row, double *rd, int32_t kappa, int32_t i, double dist, int32_t j)
{
    if (j == i)
        return;
    for (int32_t q = 0; q < kappa; q++)
        if (row[q] == j)
            return;
    if (!or_key_less(dist, j, rd[kappa - 1], row[kappa - 1]))
        return;
    int32_t b = kappa - 1;
    while (b > 0 && or_key_less(dist, j, rd[b - 1], row[b - 1])) {
        row[b] = row[b - 1];
        rd[b] = rd[b - 1];
        b--;
    }
    row[b] = j;
    rd[b] = dist;
}

/* R6: sizes and starts of the runs a cluster of m members is cut into. */
static int64_t or_nchunks(int64_t m, int32_t cap)
{
    return (m + cap - 1) / cap;
}

static void or_chunk(int64_t m, int64_t nc, int64_t c, int64_t *start, int64_t *size)
{
    int64_t base = m / nc, rem = m % nc;
    *start = c * base + (c < rem ? c : rem);
    *size = base + (c < rem ? 1 : 0);
}

/* bit set of the pairs compared so far (Alg. 3 skips a pair seen before); n*n bits */
typedef struct {
    uint8_t *bits;
    int64_t n;
} or_visited;

static int or_test_and_set(or_visited *v, int64_t i, int64_t j)
{
    int64_t a = i < j ? i : j, b = i < j ? j : i;
    int64_t bit = a * v->n + b;
    int was = (v->bits[bit >> 3] >> (bit & 7)) & 1;
    v->bits[bit >> 3] |= (uint8_t)(1u << (bit & 7));
    return was;
}

/*
 * One refinement of G given labels L in [0, k): for every run of every
 * cluster (R6) and every pair i < j in it, merge d(x_i, x_j) into rows i and j.
 * With `visited`, a pair seen in an earlier call is skipped.
 */
static void or_refine_impl(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *L, int32_t k,
                           int32_t kappa, int32_t cap, int32_t *g_idx, double *g_dist, or_visited *visited)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)k + 1));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_group(L, n, k, off, mem);
    /* a row belongs to one run of one cluster, so clusters may run in parallel (the shared visited set may not) */
#pragma omp parallel for schedule(dynamic, 4) if (visited == NULL)
    for (int32_t r = 0; r < k; r++) {
        int64_t m = off[r + 1] - off[r];
        if (m < 2)
            continue;
        int64_t nc = or_nchunks(m, cap);
        for (int64_t c = 0; c < nc; c++) {
            int64_t s0, sz;
            or_chunk(m, nc, c, &s0, &sz);
            const int32_t *S = mem + off[r] + s0;
            for (int64_t a = 0; a < sz; a++) {
                for (int64_t b = a + 1; b < sz; b++) {
                    int32_t i = S[a], j = S[b];
                    if (visited && or_test_and_set(visited, i, j))
                        continue;
                    double dist = or_d2_ff(X + (int64_t)i * ld, X + (int64_t)j * ld, d);
                    or_merge(g_idx + (int64_t)i * kappa, g_dist + (int64_t)i * kappa, kappa, i, dist, j);
                    or_merge(g_idx + (int64_t)j * kappa, g_dist + (int64_t)j * kappa, kappa, j, dist, i);
                }
            }
        }
    }
    free(off);
    free(mem);
}

void or_graph_refine(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *L, int32_t k,
                     int32_t kappa, int32_t max_cluster, int32_t *g_idx, double *g_dist)
{
    or_refine_impl(X, n, d, ld, L, k, kappa, max_cluster, g_idx, g_dist, NULL);
}

/*
 * The same refinement for a few listed rows only (for spot checks at sizes
 * where the full refinement is too slow): rows_idx/rows_dist hold the listed
 * rows' lists on entry (nrows x kappa) and their refined lists on return.
 * Row i meets exactly the members of its own run, so this equals the full
 * refinement restricted to those rows.
 */
void or_graph_refine_rows(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *L, int32_t k,
                          int32_t kappa, int32_t max_cluster, const int64_t *rows, int64_t nrows,
                          int32_t *rows_idx, double *rows_dist)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)k + 1));
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_group(L, n, k, off, mem);
    for (int64_t q = 0; q < nrows; q++) {
        int64_t i = rows[q];
        int32_t r = L[i];
        int64_t m = off[r + 1] - off[r];
        int64_t pos = -1;
        for (int64_t a = 0; a < m; a++)
            if (mem[off[r] + a] == i) {
                pos = a;
                break;
            }
        int64_t nc = or_nchunks(m, max_cluster);
        for (int64_t c = 0; c < nc; c++) {
            int64_t s0, sz;
            or_chunk(m, nc, c, &s0, &sz);
            if (pos < s0 || pos >= s0 + sz)
                continue;
            for (int64_t b = 0; b < sz; b++) {
                int32_t j = mem[off[r] + s0 + b];
                if (j == i)
                    continue;
                double dist = or_d2_ff(X + i * ld, X + (int64_t)j * ld, d);
                or_merge(rows_idx + q * kappa, rows_dist + q * kappa, kappa, (int32_t)i, dist, j);
            }
        }
    }
    free(off);
    free(mem);
}

/* CSR of the cluster set, exposed for checks of the grouping step. */
void or_group_csr(const int32_t *L, int64_t n, int32_t k, int64_t *offsets, int32_t *members)
{
    or_group(L, n, k, offsets, members);
}

/* ------------------------------------------------------------------------- */
/* Alg. 3: KNN graph by repeated fast k-means                                */
/* ------------------------------------------------------------------------- */

/*
 * G^0 random (or_init_graph), k0 = floor(n / xi) (at least 1), L^0 seeded
 * random labels in [0, k0), C = update(L^0); then tau rounds of
 *   one GK-means iteration at k0 on G^t (Sec. 4.5: t = 1): L = assign(L, C, G^t), C = update(L)
 *   exhaustive pairs inside each cluster merged into G (R6, R7).
 * use_visited != 0 keeps the visited-pair set of Alg. 3 (needs n*n bits).
 * L_out (optional) receives the final labels, E_log (optional, 2*tau+1
 * entries) the distortion after the initial update and after each assign and
 * update.
 */
int or_build_graph(const float *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, int32_t xi, int32_t tau,
                   int32_t max_cluster, uint64_t seed, int use_visited, int32_t *g_idx, double *g_dist,
                   int32_t *L_out, double *E_log)
{
    int32_t k0 = (int32_t)(n / xi);
    if (k0 < 1)
        k0 = 1;
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *L2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *best = (double *)malloc(sizeof(double) * (size_t)n);
    double *C = (double *)calloc((size_t)k0 * (size_t)d, sizeof(double));
    int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * (size_t)k0);
    or_visited vis = {NULL, n};
    if (use_visited) {
        vis.bits = (uint8_t *)calloc((size_t)((n * n + 7) / 8), 1);
        if (!vis.bits)
            return 1;
    }
    or_init_graph(X, n, d, ld, kappa, seed, g_idx, g_dist);
    or_init_labels(n, k0, seed, L);
    double e0;
    or_update(X, n, d, ld, L, k0, C, counts, &e0, NULL);
    if (E_log)
        E_log[0] = e0;
    for (int32_t t = 0; t < tau; t++) {
        or_assign(X, n, d, ld, g_idx, kappa, C, k0, L, L2, best, NULL, NULL, 0);
        double s = 0.0;
        for (int64_t i = 0; i < n; i++)
            s += best[i];
        memcpy(L, L2, sizeof(int32_t) * (size_t)n);
        double e;
        or_update(X, n, d, ld, L, k0, C, counts, &e, NULL);
        if (E_log) {
            E_log[1 + 2 * t] = s / (double)n;
            E_log[2 + 2 * t] = e;
        }
        or_refine_impl(X, n, d, ld, L, k0, kappa, max_cluster, g_idx, g_dist, use_visited ? &vis : NULL);
    }
    if (L_out)
        memcpy(L_out, L, sizeof(int32_t) * (size_t)n);
    free(L);
    free(L2);
    free(best);
    free(C);
    free(counts);
    free(vis.bits);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Brute force (textbook) checkers                                           */
/* ------------------------------------------------------------------------- */

/* Exact KNN graph: all pairs, rows sorted by (distance, index), no self. */
void or_brute_knn(const float *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, int32_t *g_idx, double *g_dist)
{
    for (int64_t i = 0; i < n; i++) {
        int32_t *row = g_idx + i * kappa;
        double *rd = g_dist + i * kappa;
        int32_t got = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double dist = or_d2_ff(X + i * ld, X + j * ld, d);
            if (got < kappa) {
                row[got] = (int32_t)j;
                rd[got] = dist;
                got++;
                if (got == kappa)
                    or_sort_row(row, rd, kappa);
            } else {
                or_merge(row, rd, kappa, (int32_t)i, dist, (int32_t)j);
            }
        }
        if (got < kappa)
            or_sort_row(row, rd, got);
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. 1: two-means tree (Sec. 3.2)                                          */
/* ------------------------------------------------------------------------- */

/*
 * Starting from one cluster holding every sample, the largest cluster is
 * taken out, bisected, the two halves are made equal in size, and both go
 * back, until there are k clusters.  Readings where the paper is silent:
 *   T1 a bisection is Lloyd's 2-means (the closest-centroid form used by the
 *      rest of this path; the paper bisects with its boost form) for `iters`
 *      iterations from two seed samples;
 *   T2 the seeds are the two members with the smallest keys
 *      (draw(seed ^ TREE, depth * 2^32 + id), id), depth = the cluster's
 *      depth in the tree (the root has depth 0);
 *   T3 each decision is taken in FP32, the precision of the CUDA path: the
 *      squared distance sums fma(x_t - c_t, x_t - c_t, acc) over ascending t
 *      in one FP32 accumulator; a member joins half u when d(x, c_u) <= d(x, c_v);
 *      a centre is the FP32 rounding of the FP64 mean of its half (members in
 *      ascending id); an empty half keeps its centre;
 *   T4 equal sizes: the members are ordered by (d(x, c_u) - d(x, c_v) in FP32,
 *      id) with the final centres; the first ceil(m / 2) form u, the rest v;
 *   T5 among clusters of the largest size the shallowest is taken first, then
 *      the one that comes first in the order of T6;
 *   T6 the clusters are numbered left to right in the tree, u before v.
 */
static const uint64_t OR_TAG_TREE = 0x5452454500000000ULL; /* "TREE" */

/* T3: FP32 squared distance, ascending coordinates, one fused multiply-add per step */
static float or_d2_f32(const float *x, const float *c, int64_t d)
{
    float acc = 0.0f;
    for (int64_t t = 0; t < d; t++) {
        float e = x[t] - c[t];
        acc = fmaf(e, e, acc);
    }
    return acc;
}

typedef struct {
    float key;
    int32_t id;
} or_tree_key;

static int or_tree_key_cmp(const void *a, const void *b)
{
    const or_tree_key *p = (const or_tree_key *)a, *q = (const or_tree_key *)b;
    if (p->key != q->key)
        return p->key < q->key ? -1 : 1;
    return (p->id > q->id) - (p->id < q->id);
}

static int or_id_cmp(const void *a, const void *b)
{
    int32_t p = *(const int32_t *)a, q = *(const int32_t *)b;
    return (p > q) - (p < q);
}

/* One bisection (T1-T4) of the members mem[0..m), m >= 2, in ascending id.
 * On return mem[0..ceil(m/2)) is half u and the rest half v, each in ascending id. */
static void or_bisect(const float *X, int64_t d, int64_t ld, int32_t *mem, int64_t m, int32_t depth,
                      int32_t iters, uint64_t seed, float *cu, float *cv, double *su, double *sv, or_tree_key *keys)
{
    uint64_t key = seed ^ OR_TAG_TREE;
    int64_t a = -1, b = -1;
    uint64_t ha = 0, hb = 0;
    for (int64_t p = 0; p < m; p++) { /* T2: ascending id, so an equal draw keeps the smaller id first */
        uint64_t h = or_draw(key, ((uint64_t)(uint32_t)depth << 32) | (uint64_t)(uint32_t)mem[p]);
        if (a < 0 || h < ha) {
            b = a;
            hb = ha;
            a = p;
            ha = h;
        } else if (b < 0 || h < hb) {
            b = p;
            hb = h;
        }
    }
    memcpy(cu, X + (int64_t)mem[a] * ld, sizeof(float) * (size_t)d);
    memcpy(cv, X + (int64_t)mem[b] * ld, sizeof(float) * (size_t)d);
    for (int32_t it = 0; it < iters; it++) { /* T1, T3 */
        int64_t nu = 0, nv = 0;
        memset(su, 0, sizeof(double) * (size_t)d);
        memset(sv, 0, sizeof(double) * (size_t)d);
        for (int64_t p = 0; p < m; p++) {
            const float *x = X + (int64_t)mem[p] * ld;
            double *s = or_d2_f32(x, cu, d) <= or_d2_f32(x, cv, d) ? su : sv;
            for (int64_t t = 0; t < d; t++)
                s[t] += (double)x[t];
            if (s == su)
                nu++;
            else
                nv++;
        }
        for (int64_t t = 0; t < d; t++) {
            if (nu)
                cu[t] = (float)(su[t] / (double)nu);
            if (nv)
                cv[t] = (float)(sv[t] / (double)nv);
        }
    }
    for (int64_t p = 0; p < m; p++) { /* T4 */
        const float *x = X + (int64_t)mem[p] * ld;
        keys[p].key = or_d2_f32(x, cu, d) - or_d2_f32(x, cv, d);
        keys[p].id = mem[p];
    }
    qsort(keys, (size_t)m, sizeof(or_tree_key), or_tree_key_cmp);
    int64_t h = (m + 1) / 2;
    for (int64_t p = 0; p < m; p++)
        mem[p] = keys[p].id;
    qsort(mem, (size_t)h, sizeof(int32_t), or_id_cmp);
    qsort(mem + h, (size_t)(m - h), sizeof(int32_t), or_id_cmp);
}

/*
 * Alg. 1: labels[i] in [0, k) for every sample, 1 <= k <= n.  A cluster is a
 * range [off, off + m) of one permutation of the samples, so that "left to
 * right" (T6) is the order of off.  Returns 0, or 1 for bad arguments or no memory.
 */
int or_two_means_tree(const float *X, int64_t n, int64_t d, int64_t ld, int32_t k, int32_t iters, uint64_t seed,
                      int32_t *labels)
{
    if (k < 1 || (int64_t)k > n || iters < 0)
        return 1;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int64_t *size = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    float *cu = (float *)malloc(sizeof(float) * (size_t)d);
    float *cv = (float *)malloc(sizeof(float) * (size_t)d);
    double *su = (double *)malloc(sizeof(double) * (size_t)d);
    double *sv = (double *)malloc(sizeof(double) * (size_t)d);
    or_tree_key *keys = (or_tree_key *)malloc(sizeof(or_tree_key) * (size_t)n);
    int rc = 1;
    if (!perm || !off || !size || !depth || !cu || !cv || !su || !sv || !keys)
        goto done;
    for (int64_t i = 0; i < n; i++)
        perm[i] = (int32_t)i;
    off[0] = 0;
    size[0] = n;
    depth[0] = 0;
    for (int32_t t = 1; t < k; t++) {
        int32_t s = 0; /* pop: largest size, then smallest depth, then leftmost (T5) */
        for (int32_t r = 1; r < t; r++)
            if (size[r] > size[s] || (size[r] == size[s] && (depth[r] < depth[s] ||
                                                            (depth[r] == depth[s] && off[r] < off[s]))))
                s = r;
        int64_t m = size[s], h = (m + 1) / 2;
        or_bisect(X, d, ld, perm + off[s], m, depth[s], iters, seed, cu, cv, su, sv, keys);
        off[t] = off[s] + h; /* v */
        size[t] = m - h;
        depth[t] = depth[s] + 1;
        size[s] = h; /* u keeps the left range */
        depth[s] += 1;
    }
    for (int32_t s = 0; s < k; s++) { /* T6: rank of off */
        int32_t rank = 0;
        for (int32_t r = 0; r < k; r++)
            rank += off[r] < off[s];
        for (int64_t p = off[s]; p < off[s] + size[s]; p++)
            labels[perm[p]] = rank;
    }
    rc = 0;
done:
    free(perm);
    free(off);
    free(size);
    free(depth);
    free(cu);
    free(cv);
    free(su);
    free(sv);
    free(keys);
    return rc;
}

/* ======================================================================
 * Boost form of GK-means (Sec. 3.1 Eq. 2 and Eq. 3; the move step of Alg. 2,
 * Sec. 4.2).  State per cluster r: the composite vector D_r = sum of its
 * members (Eq. 2), its size n_r and S_r = D_r'D_r.  Readings:
 *   B1 a visit sequence `order` (sample ids, drawn by the caller) replaces
 *      "one sample is randomly selected"; an epoch is one pass over it.
 *   B2 the candidates of sample i are the distinct labels of its kappa
 *      neighbours other than its own label u = L[i] (Alg. 2 collects Q).
 *   B3 a sample alone in its cluster is not moved (Eq. 3 divides by n_u - 1).
 *   B4 FP64 throughout; D_r starts as its members' rows summed in ascending
 *      sample id; every squared norm is or_fold_sq below; Eq. 3 is evaluated
 *      term by term, left to right, each operation rounded once.
 *   B5 the candidate of largest gain wins, the smaller label on equal gains;
 *      the sample moves iff that gain is > 0 (Alg. 2).
 * ====================================================================== */

/* Squared norm of v[0..d): the squares (each rounded once) of the vector
 * zero-padded to the smallest power of two P >= d, then halving folds:
 * while P > 1, P /= 2 and w[j] = w[j] + w[j + P] for j < P.  w: scratch of at
 * least P doubles. */
static double or_fold_sq_impl(const double *v, int64_t d, double *w)
{
    int64_t P = 1;
    while (P < d)
        P <<= 1;
    for (int64_t j = 0; j < P; j++)
        w[j] = j < d ? v[j] * v[j] : 0.0;
    for (int64_t h = P / 2; h >= 1; h /= 2)
        for (int64_t j = 0; j < h; j++)
            w[j] = w[j] + w[j + h];
    return w[0];
}

double or_fold_sq(const double *v, int64_t d)
{
    int64_t P = 1;
    while (P < d)
        P <<= 1;
    double *w = (double *)malloc(sizeof(double) * (size_t)P);
    if (!w)
        return -1.0;
    double r = or_fold_sq_impl(v, d, w);
    free(w);
    return r;
}

/* Eq. 2 state from labels: D (k x d, row-major), counts, S.  B4: each D_r is
 * the running FP64 sum of its members' rows in ascending sample id. */
int or_boost_init(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *L, int32_t k, double *D,
                  int32_t *counts, double *S)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)(2 * d + 2));
    if (!w)
        return 1;
    for (int64_t e = 0; e < (int64_t)k * d; e++)
        D[e] = 0.0;
    for (int32_t r = 0; r < k; r++)
        counts[r] = 0;
    for (int64_t i = 0; i < n; i++) { /* ascending id: each D_r gets its members in that order */
        int32_t r = L[i];
        for (int64_t t = 0; t < d; t++)
            D[(int64_t)r * d + t] = D[(int64_t)r * d + t] + (double)X[i * ld + t];
        counts[r] += 1;
    }
    for (int32_t r = 0; r < k; r++)
        S[r] = or_fold_sq_impl(D + (int64_t)r * d, d, w);
    free(w);
    return 0;
}

/* Eq. 3: gain of moving x from S_u (size nu, vector Du, S_u = Su) to S_v.
 * Dv_plus_x_sq = (D_v + x)'(D_v + x), Du_minus_x_sq = (D_u - x)'(D_u - x). */
static double or_boost_gain(double Dv_plus_x_sq, int32_t nv, double Sv, double Du_minus_x_sq, int32_t nu, double Su)
{
    return ((Dv_plus_x_sq / (double)(nv + 1) + Du_minus_x_sq / (double)(nu - 1)) - Sv / (double)nv) -
           Su / (double)nu;
}

/* One epoch of Alg. 2's move step over the visits order[0..m): labels L, D,
 * counts and S are updated in place, each move before the next visit is
 * examined.  gains (m doubles, or NULL) receives the gain of the move made at
 * each visit and 0 where the sample stayed.  Returns the number of moves, or
 * -1 if out of memory. */
int64_t or_boost_epoch(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *G, int32_t kappa,
                       const int32_t *order, int64_t m, int32_t *L, int32_t k, double *D, int32_t *counts, double *S,
                       double *gains)
{
    (void)n;
    (void)k;
    double *x = (double *)malloc(sizeof(double) * (size_t)d);
    double *y = (double *)malloc(sizeof(double) * (size_t)d);
    int64_t P = 1;
    while (P < d)
        P <<= 1;
    double *w = (double *)malloc(sizeof(double) * (size_t)P);
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kappa > 0 ? kappa : 1));
    if (!x || !y || !w || !Q) {
        free(x);
        free(y);
        free(w);
        free(Q);
        return -1;
    }
    int64_t moves = 0;
    for (int64_t s = 0; s < m; s++) {
        const int64_t i = order[s];
        const int32_t u = L[i];
        if (gains)
            gains[s] = 0.0;
        if (counts[u] < 2) /* B3 */
            continue;
        for (int64_t t = 0; t < d; t++)
            x[t] = (double)X[i * ld + t];
        /* Q: distinct labels of the neighbours, own label excluded (B2) */
        int32_t nq = 0;
        for (int32_t j = 0; j < kappa; j++) {
            int32_t v = L[G[i * kappa + j]];
            int seen = v == u;
            for (int32_t q = 0; q < nq && !seen; q++)
                seen = Q[q] == v;
            if (!seen)
                Q[nq++] = v;
        }
        if (nq == 0)
            continue;
        const double *Du = D + (int64_t)u * d;
        for (int64_t t = 0; t < d; t++)
            y[t] = Du[t] - x[t];
        const double Bu = or_fold_sq_impl(y, d, w);
        double best = 0.0;
        int32_t bv = -1;
        for (int32_t q = 0; q < nq; q++) {
            const int32_t v = Q[q];
            const double *Dv = D + (int64_t)v * d;
            for (int64_t t = 0; t < d; t++)
                y[t] = Dv[t] + x[t];
            const double g = or_boost_gain(or_fold_sq_impl(y, d, w), counts[v], S[v], Bu, counts[u], S[u]);
            if (bv < 0 || g > best || (g == best && v < bv)) /* B5 */
                best = g, bv = v;
        }
        if (!(best > 0.0))
            continue;
        /* the move (Alg. 2): x leaves S_u and joins S_bv; sizes and S follow their definitions */
        double *Dm = D + (int64_t)u * d, *Dp = D + (int64_t)bv * d;
        for (int64_t t = 0; t < d; t++) {
            Dm[t] = Dm[t] - x[t];
            Dp[t] = Dp[t] + x[t];
        }
        counts[u] -= 1;
        counts[bv] += 1;
        S[u] = or_fold_sq_impl(Dm, d, w);
        S[bv] = or_fold_sq_impl(Dp, d, w);
        L[i] = bv;
        if (gains)
            gains[s] = best;
        moves++;
    }
    free(x);
    free(y);
    free(w);
    free(Q);
    return moves;
}
