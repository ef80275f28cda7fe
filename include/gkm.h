/*
 * gkm.h - C ABI of libgkm, a CUDA (sm_103a) implementation of graph-guided
 * k-means ("GK-means", Deng & Zhao, "Fast k-means based on KNN Graph",
 * arXiv 1705.01813).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument is DEVICE memory owned by the caller unless it is
 *    marked "host".  The library never allocates, frees or keeps a pointer
 *    after the call returns (scratch comes from the caller's workspace `ws`).
 *  - The sample matrix X is row-major: sample i, coordinate t at
 *    X[i * ld + t], n rows (n < 2^31), d coordinates (1 <= d <= 4096),
 *    ld >= d.  Element type: FP32.
 *    X must be 4-byte aligned; with X 16-byte aligned and d, ld multiples
 *    of 4 the kernels use 16-byte vector loads.
 *  - Labels are int32 in [0, k).  A KNN graph is two n x kappa row-major
 *    arrays: g_idx (int32 neighbour ids) and g_dist (FP32 squared Euclidean
 *    distances); each row is sorted by (distance, id), holds no self and no
 *    repeated id.
 *  - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and is asynchronous unless the entry point says it synchronises.
 *  - Arguments are checked on the host before anything is enqueued; a bad
 *    argument returns GK_ERR_INVALID and gk_last_error() says why.  Errors the
 *    kernels find (a label or neighbour id out of range: GK_ERR_INVALID; a
 *    non-finite sample, seen by the update or the two-means tree:
 *    GK_ERR_NUMERIC; a bounded wait that ran out: GK_ERR_TIMEOUT) are recorded
 *    in a status word inside `ws` and read back by gk_read_status().
 *  - ws/ws_bytes: caller-provided device scratch of at least
 *    gk_workspace_size(op, ...) bytes, 256-byte aligned.  A call that needs
 *    more returns GK_ERR_INVALID with the required size in the message.
 *    Concurrent calls must use distinct workspaces.
 *  - The library is reentrant across streams.  Its global state: the
 *    thread-local message returned by gk_last_error(), each kernel's shared
 *    memory limit (set once per device), and, with gk_set_replay on, the
 *    cache of captured request graphs.
 */
#ifndef GKM_H
#define GKM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GK_API __attribute__((visibility("default")))
#else
#define GK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GK_OK = 0,
    GK_ERR_INVALID = 1, /* bad argument, or a kernel found an out-of-range label / id */
    GK_ERR_CUDA = 2,    /* a CUDA runtime call failed */
    GK_ERR_NOMEM = 3,   /* workspace too small for a data-dependent size */
    GK_ERR_TIMEOUT = 4, /* a bounded device-side wait gave up */
    GK_ERR_NUMERIC = 5  /* non-finite value met */
} gk_status;

/* Operation ids for gk_workspace_size(). */
enum {
    GK_OP_ASSIGN = 0,
    GK_OP_UPDATE = 1,
    GK_OP_REFINE = 2,
    GK_OP_FIT = 3,
    GK_OP_BUILD = 4,
    GK_OP_RECALL = 5,
    GK_OP_TREE = 6,
    GK_OP_BOOST = 7
};

/* Parameters of the graph construction (Alg. 3 and Sec. 4.4 of the paper). */
typedef struct {
    int32_t kappa;       /* neighbours per sample, 1 <= kappa <= 128 and kappa < n      */
    int32_t xi;          /* target cluster size; k0 = max(1, floor(n / xi))  (Alg. 3)   */
    int32_t tau;         /* refinement rounds (Alg. 3), >= 0                            */
    int32_t max_cluster; /* a cluster larger than this is cut into runs of consecutive
                            members (ascending id) whose sizes differ by at most one    */
    uint64_t seed;       /* seed of the random initial graph and labels (SplitMix64)    */
    int32_t precision;   /* bits 0-7: 0: FP32 throughout; 1: refinement pair distances from
                            a BF16 Gram on the tensor cores with an exact FP32 recompute
                            of the pairs inside its error bound (64 <= d <= 128; other
                            widths use the FP32 kernels); 2, 3 and 4: 1 and the
                            assignment's screening as in gk_assign_step.  Bits 8-15:
                            the assignment's candidates per group, as there.  All give
                            the same graph.                                             */
    int32_t reserved;    /* must be 0                                                   */
} gk_graph_params;

/* Library version string (static storage). */
GK_API const char *gk_version(void);

/* Message of the last failed call on this host thread (static storage, never NULL). */
GK_API const char *gk_last_error(void);

/*
 * Bytes of workspace the operation `op` (GK_OP_ASSIGN, _UPDATE, _REFINE, _FIT,
 * _RECALL, _TREE, _BOOST) needs for these sizes; 0 for an unknown op.  k is the number of
 * clusters (for GK_OP_RECALL: the number of queries m).  The graph
 * construction has its own query, gk_workspace_size_build().
 */
GK_API size_t gk_workspace_size(int32_t op, int64_t n, int64_t d, int32_t k, int32_t kappa);

/* Workspace bytes of gk_build_knn_graph() for these sizes and parameters. */
GK_API size_t gk_workspace_size_build(int64_t n, int64_t d, const gk_graph_params *p);

/*
 * Seeded random initial labelling (the paper starts from a partition; the
 * random start replaces its two-means tree).  labels[i] = SplitMix64 output
 * (i + 1) of the generator seeded with seed ^ 0x4C41424C00000000, modulo k.
 * labels: device int32[n], written.
 */
GK_API int gk_init_labels(int64_t n, int32_t k, uint64_t seed, int32_t *labels, void *stream);

/*
 * Random initial KNN graph (Alg. 3 begins from random neighbour lists).
 * Row i takes draws j = output(i * 2^32 + a + 1) mod n, a = 0, 1, ..., of the
 * SplitMix64 generator seeded with seed ^ 0x4752415000000000, rejecting j == i
 * and ids it already holds, until kappa are accepted; their squared distances
 * are computed in FP32 and the row sorted by (distance, id).
 * g_idx: device int32[n * kappa], g_dist: device float[n * kappa], written.
 */
GK_API int gk_init_graph(const float *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed, int32_t *g_idx,
                  float *g_dist, void *ws, size_t ws_bytes, void *stream);

/*
 * Graph-guided assignment step (Alg. 2, candidate loop, with the
 * closest-centroid rule given at the end of Sec. 4.2).  For each sample i the
 * candidate clusters are its own label and the labels of its kappa graph
 * neighbours; labels_out[i] is the candidate r with the smallest
 * (||x_i - C_r||^2, r).  All samples use the same input centroids.
 *   g_idx     device int32[n * kappa], neighbour ids in [0, n)
 *   C         device float[k * d], centroids, row-major with stride d
 *   labels_in device int32[n];  labels_out device int32[n] (may not alias labels_in)
 *   best_d2   device float[n] or NULL: the winning squared distance
 *   sum_d2    device double[1] or NULL: sum of best_d2 (n times the distortion
 *             after the assignment, Eq. 4), computed in FP64
 *   n_changed device int64[1] or NULL: samples whose label changed
 *   precision bits 0-7, the level: 0 or 1: candidate distances read the FP32
 *             centroid rows; 2, 3 and 4: they are first screened against a
 *             copy of the centroids (2: BF16, on the SIMT cores, one sample per
 *             warp; 3: BF16, for d <= 128 on the tensor cores, 128 samples of
 *             adjacent clusters at a time; 4: int8 with a per-row scale, on the
 *             SIMT cores, a quarter of the FP32 row's bytes) and every
 *             candidate within a rigorous error bound of the minimum is
 *             recomputed against the FP32 rows in the same order as with 0, so
 *             labels_out, best_d2, sum_d2 and n_changed are identical.
 *             Bits 8-15: candidates per group of the row kernels, 0 (default:
 *             8, or 4 for rows of more than 512 values), 4 or 8 (rows of more
 *             than 512 values always take 4); a tile shape, the results are the
 *             same.  Other bits must be 0.
 *   members   device int32[n] or NULL: the samples grouped by labels_in, as
 *             gk_group_by_label returns them; used by precision 3 to form the
 *             tiles (NULL: the call groups them itself)
 */
GK_API int gk_assign_step(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                          const float *C, int32_t k, const int32_t *labels_in, int32_t *labels_out, float *best_d2,
                          double *sum_d2, int64_t *n_changed, int32_t precision, const int32_t *members, void *ws,
                          size_t ws_bytes, void *stream);

/*
 * Centroid update (Sec. 1: each centroid becomes the mean of its members).
 * Members are grouped by label (CSR, members in ascending id); per cluster the
 * composite vector D_r (Eq. 2) is summed with compensated FP32 arithmetic and
 * widened to FP64, and C_r = D_r / n_r.  An empty cluster keeps its centroid.
 *   C        device float[k * d], in: previous centroids, out: new centroids
 *   counts   device int32[k] or NULL: cluster sizes n_r
 *   sum_d2   device double[1] or NULL: n times the distortion after the update
 *            (Eq. 4), from the Eq. 2 identity sum ||x||^2 - sum_r D_r'D_r / n_r
 *   offsets, members  device int32[k + 1] / int32[n] or NULL: the CSR grouping
 *            (cluster r owns members[offsets[r] .. offsets[r+1]) )
 * A NaN or infinite sample makes its cluster's distortion term non-finite:
 * the update records GK_ERR_NUMERIC (detail: the cluster) in the status word.
 * A label outside [0, k) is recorded as GK_ERR_INVALID; its sample belongs to
 * no cluster (it is listed after every cluster's members, beyond
 * offsets[k]), so the other clusters' results are those of their members.
 * The same holds for every update inside gk_kmeans_fit and gk_build_knn_graph.
 */
GK_API int gk_update_step(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k, float *C,
                   int32_t *counts, double *sum_d2, int32_t *offsets, int32_t *members, void *ws, size_t ws_bytes,
                   void *stream);

/*
 * One graph refinement (Alg. 3, the exhaustive pairs inside each cluster):
 * samples are grouped by label; a cluster of m > max_cluster members is cut
 * into ceil(m / max_cluster) runs of consecutive members whose sizes differ by
 * at most one; every pair (i, j) inside a run is merged into rows i and j, a
 * row keeping its kappa smallest (distance, id) keys with no self and no
 * repeated id.  Pair distances are squared Euclidean in FP32, summed over
 * coordinates in ascending order, so a pair has the same bits in every round.
 *   precision  0: distances on the SIMT cores; 1 to 3: a BF16 Gram matrix per run
 *              on the tensor cores gives d2 = |x|^2 + |y|^2 - 2 x.y, exact when
 *              the run's centred coordinates are integers of magnitude <= 255
 *              (and 2 d 255^2 < 2^24), otherwise every pair within a rigorous
 *              error bound of entering a row is recomputed in FP32 as with 0;
 *              the tensor-core path serves 64 <= d <= 128 (BF16 samples are
 *              staged uncentred, so their Gram carries no BF16 rounding);
 *              other widths use the SIMT kernels of 0; all settings give the
 *              same graph.
 *   g_idx / g_dist  device, n x kappa, in: current graph, out: refined graph
 */
GK_API int gk_graph_refine(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                           int32_t kappa, int32_t max_cluster, int32_t precision, int32_t *g_idx, float *g_dist,
                           void *ws, size_t ws_bytes, void *stream);

/*
 * The three steps the update and the refinement are made of, for callers that
 * sequence the path themselves (they run the same kernels as the calls above).
 *
 * gk_group_by_label: the cluster set S (Alg. 1 and 3 map labels to it) as a
 *   CSR: offsets int32[k + 1], members int32[n] (ascending id within a
 *   cluster), counts int32[k] or NULL.  Workspace: gk_workspace_size(GK_OP_UPDATE, ...).
 * gk_update_from_groups: the centroid update of gk_update_step given that CSR.
 * gk_graph_refine_groups: the refinement of gk_graph_refine given that CSR.
 *   Workspace: gk_workspace_size(GK_OP_REFINE, ...).
 * Labels out of range are reported through the status word, as above.
 */
GK_API int gk_group_by_label(const int32_t *labels, int64_t n, int32_t k, int32_t *offsets, int32_t *members,
                             int32_t *counts, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_update_from_groups(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                                 const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2,
                                 void *ws, size_t ws_bytes, void *stream);
GK_API int gk_graph_refine_groups(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                                  const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster,
                                  int32_t precision, int32_t *g_idx, float *g_dist, void *ws, size_t ws_bytes,
                                  void *stream);

/*
 * KNN-graph construction by repeated fast k-means (Alg. 3): random graph and
 * labels at k0 = max(1, floor(n / xi)), centroids from those labels, then tau
 * rounds of { one graph-guided assignment, one update, one refinement }
 * (one k-means iteration per round, Sec. 4.5; labels and centroids carry over
 * from round to round).
 *   labels_out device int32[n] or NULL: the final labels at k0
 *   e_log      HOST double[2 * tau + 1] or NULL: distortion after the first
 *              update, then after each assignment and update.  A non-NULL
 *              e_log makes the call synchronise the stream.
 */
GK_API int gk_build_knn_graph(const float *X, int64_t n, int64_t d, int64_t ld, const gk_graph_params *p, int32_t *g_idx,
                       float *g_dist, int32_t *labels_out, double *e_log, void *ws, size_t ws_bytes, void *stream);

/*
 * Graph-guided k-means (Alg. 2 with the closest-centroid rule): centroids
 * from the initial labels, then `iters` x { assignment, update }.
 *   init_labels device int32[n] or NULL (NULL: gk_init_labels(seed))
 *   precision   of the assignment steps, as in gk_assign_step (same results)
 *   labels_out  device int32[n]; C_out device float[k * d]; counts_out device int32[k] or NULL
 *   e_log       HOST double[2 * iters + 1] or NULL, as in gk_build_knn_graph
 *               (non-NULL synchronises the stream)
 */
GK_API int gk_kmeans_fit(const float *X, int64_t n, int64_t d, int64_t ld, int32_t k, const int32_t *g_idx,
                         int32_t kappa, int32_t iters, const int32_t *init_labels, uint64_t seed, int32_t precision,
                         int32_t *labels_out, float *C_out, int32_t *counts_out, double *e_log, void *ws,
                         size_t ws_bytes, void *stream);

/*
 * Batches of independent clustering jobs (batching; the paper clusters one
 * data set): several jobs with the same row width d and kappa run as one
 * problem, so every kernel launch of the path serves all of them.  Job j owns
 * the samples first_j .. first_j + n_j - 1 of X (the jobs' samples
 * concatenated in job order; first_0 = 0, first_{j+1} = first_j + n_j) and
 * runs what gk_build_knn_graph and gk_kmeans_fit run for it alone: the graph
 * construction (Alg. 3) at k0_j = max(1, floor(n_j / xi)) from graph_seed,
 * then `iters` iterations of Alg. 2 at k_j clusters from the labels
 * gk_init_labels(n_j, k_j, fit_seed) draws.  Each job's graph rows, labels,
 * centroids and final distortion equal its solo results bit for bit: its rows,
 * labels and clusters are numbered after the jobs before it, so no cluster and
 * no graph row spans two jobs and every tie order is the solo one.
 *   jobs        HOST gk_job[njobs], 1 <= njobs <= GK_MAX_BATCH_JOBS; for every
 *               job n_j >= 2, kappa < n_j, k_j >= 1, reserved 0
 *   p           kappa, xi, tau, max_cluster, precision as for
 *               gk_build_knn_graph (p->seed is not used: seeds are per job)
 *   g_idx, g_dist  device [N x kappa], N = sum n_j: the constructed graph, ids
 *               in batch numbering (job j's ids are first_j + its solo ids)
 *   labels_out  device int32[N]: job j's final labels in [0, k_j)
 *   C_out       device float[(sum k_j) x d]: job j's centroids in rows
 *               sum_{i<j} k_i .. + k_j - 1
 *   distortion  device double[njobs]: each job's final distortion (Eq. 4)
 *   ws          gk_workspace_size_batch(d, njobs, jobs, p) bytes
 * With gk_set_replay on, a call whose arguments and job table equal an
 * earlier call's replays its captured CUDA graph.
 */
#define GK_MAX_BATCH_JOBS 64

typedef struct {
    int64_t n;           /* samples of the job                                           */
    int32_t k;           /* clusters of its fit                                          */
    int32_t reserved;    /* must be 0                                                    */
    uint64_t graph_seed; /* seed of its random initial graph and labels at k0            */
    uint64_t fit_seed;   /* seed of its initial labels at k                              */
} gk_job;

GK_API size_t gk_workspace_size_batch(int64_t d, int32_t njobs, const gk_job *jobs, const gk_graph_params *p);
GK_API int gk_batch_fit(const float *X, int64_t d, int64_t ld, int32_t njobs, const gk_job *jobs,
                        const gk_graph_params *p, int32_t iters, int32_t *g_idx, float *g_dist, int32_t *labels_out,
                        float *C_out, double *distortion, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_batch_fit_bf16(const uint16_t *X, int64_t d, int64_t ld, int32_t njobs, const gk_job *jobs,
                             const gk_graph_params *p, int32_t iters, int32_t *g_idx, float *g_dist,
                             int32_t *labels_out, float *C_out, double *distortion, void *ws, size_t ws_bytes,
                             void *stream);

/*
 * gk_update_step without a workspace, for callers that cannot allocate device
 * memory: for instance an application whose framework owns all device memory
 * through its own pool and forbids raw cudaMalloc, or a latency-bound serving
 * loop where cudaMalloc / cudaFree may synchronise the device.  (The paper has
 * no counterpart: this is an interface choice of the library.)
 *
 * Same arguments and results as gk_update_step (no offsets / members
 * outputs).  Scratch comes from one fixed array compiled into the library's
 * device image: 24 MiB on every GPU that loads the library, held until the
 * process exits.  Limits: n <= 1,048,576 and k <= 32,768; larger sizes return
 * GK_ERR_INVALID with a message.  Nothing is allocated by the call.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call on a device shares the one array: calls whose work overlaps on
 *    the GPU (different streams, or different host threads) race and corrupt
 *    each other's results.  Serialise them, e.g. on one stream.
 *  - The array keeps the previous call's contents; the call clears what must
 *    start at zero.  Labels out of range are not reported through a status
 *    word here (there is no workspace to read it from).  A sample whose label
 *    is outside [0, k) belongs to no cluster: the centroids, counts and
 *    distortion terms of the clusters are those of the other samples alone
 *    (as for gk_update_step, which also records the bad label in its status
 *    word), so sum(counts) < n reveals such samples.
 */
GK_API int gk_update_step_noalloc(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                                  float *C, int32_t *counts, double *sum_d2, void *stream);

/*
 * BF16 samples.  Each call below is the call of the same name without _bf16,
 * with X holding the samples as BF16 values (their 16-bit patterns, row-major,
 * leading dimension ld in elements, 2-byte aligned) instead of FP32.  Every
 * element is widened exactly to FP32 when read and all arithmetic is the FP32
 * path's, so the results are those of the FP32 call on the widened samples,
 * bit for bit; the samples take half the device memory and half the read
 * traffic.  (Deep-feature vectors at the paper's largest scale, 10^7 x 512,
 * Sec. 5, take 10 GB this way.)  At precision 2 the assignment screens its
 * candidates against BF16 centroids with the samples unrounded, as for FP32
 * samples.  The tensor-core screening (precision 3) reads FP32 samples only:
 * with BF16 samples the assignment takes precision 0, 1 or 2
 * (gk_assign_step_bf16, gk_kmeans_fit_bf16, and p->precision of
 * gk_build_knn_graph_bf16), else GK_ERR_INVALID.
 */
GK_API int gk_init_graph_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed,
                              int32_t *g_idx, float *g_dist, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_assign_step_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                               int32_t kappa, const float *C, int32_t k, const int32_t *labels_in,
                               int32_t *labels_out, float *best_d2, double *sum_d2, int64_t *n_changed,
                               int32_t precision, const int32_t *members, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_update_step_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                               float *C, int32_t *counts, double *sum_d2, int32_t *offsets, int32_t *members,
                               void *ws, size_t ws_bytes, void *stream);
GK_API int gk_graph_refine_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                                int32_t kappa, int32_t max_cluster, int32_t precision, int32_t *g_idx, float *g_dist,
                                void *ws, size_t ws_bytes, void *stream);
GK_API int gk_update_from_groups_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                                      const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2,
                                      void *ws, size_t ws_bytes, void *stream);
GK_API int gk_graph_refine_groups_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                                       const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster,
                                       int32_t precision, int32_t *g_idx, float *g_dist, void *ws, size_t ws_bytes,
                                       void *stream);
GK_API int gk_build_knn_graph_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const gk_graph_params *p,
                                   int32_t *g_idx, float *g_dist, int32_t *labels_out, double *e_log, void *ws,
                                   size_t ws_bytes, void *stream);
GK_API int gk_kmeans_fit_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, int32_t k, const int32_t *g_idx,
                              int32_t kappa, int32_t iters, const int32_t *init_labels, uint64_t seed,
                              int32_t precision, int32_t *labels_out, float *C_out, int32_t *counts_out,
                              double *e_log, void *ws, size_t ws_bytes, void *stream);

/*
 * Top-1 recall of a KNN graph on sampled queries (Sec. 5: the recall of the
 * top-1 neighbour, estimated on randomly chosen samples where the full ground
 * truth is too costly).  For each query q = queries[t] the exact nearest
 * neighbour among the other n - 1 samples is found by brute force (squared
 * Euclidean distance in FP32 in the canonical order of the graph's distances,
 * ties to the smaller id: the graph's key order); q is a hit when it is
 * g_idx[q][0].  Graph rows hold exact distances sorted by key, so a row holds
 * its sample's nearest neighbour exactly when that is its first entry.
 *   X, n, d, ld    samples as in gk_assign_step (n >= 2)
 *   g_idx, kappa   device int32[n x kappa]: the graph
 *   queries        device int32[m]: sample ids (drawn by the caller); an id
 *                  outside [0, n) is reported in the status word, never a hit
 *   nn_idx, nn_dist  device int32[m] / float[m] or NULL: each query's exact
 *                  nearest neighbour and its distance (-1 / +inf if none)
 *   hits           device int64[1]: number of hits (overwritten)
 *   ws             gk_workspace_size(GK_OP_RECALL, n, d, m, kappa) bytes
 * Cost: m n d pair terms, on the SIMT cores (FP32 tiles of 64 queries x 64
 * samples).
 */
GK_API int gk_graph_recall(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                           const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist, int64_t *hits,
                           void *ws, size_t ws_bytes, void *stream);
GK_API int gk_graph_recall_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                                int32_t kappa, const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist,
                                int64_t *hits, void *ws, size_t ws_bytes, void *stream);

/*
 * Two-means tree (Alg. 1, Sec. 3.2): the initial partition of the paper's
 * GK-means.  Starting from one cluster of all samples, the largest cluster is
 * bisected and the halves are made equal in size until there are k clusters.
 * One bisection of a cluster of m members: the two members with the smallest
 * (SplitMix64 draw of (seed, depth, id), id) are the starting centres; `iters`
 * Lloyd 2-means iterations follow (a member joins half u when its squared
 * distance to c_u is at most that to c_v; a centre becomes the FP32 rounding of
 * the FP64 mean of its half; an empty half keeps its centre); then the members
 * are ordered by (d(x, c_u) - d(x, c_v), id) and the first ceil(m/2) form u,
 * the rest v.  Distances and their difference are FP32, summed over ascending
 * coordinates with one fused multiply-add per step.  Among clusters of the
 * largest size the shallowest splits first, then the leftmost.  The sizes
 * depend on n and k only: at depth L a cluster has floor(n / 2^L) or one more
 * members.
 *   X, n, d, ld    samples as in gk_assign_step (n >= 1)
 *   k              clusters, 1 <= k <= n
 *   iters          Lloyd iterations per bisection, 0 <= iters <= 64
 *   seed           seed of the starting centres
 *   labels         device int32[n] (out): each sample's cluster; clusters are
 *                  numbered left to right in the tree (u before v)
 *   ws             gk_workspace_size(GK_OP_TREE, n, d, k, 0) bytes
 * Bad arguments return GK_ERR_INVALID; a non-finite distance sets
 * GK_ERR_NUMERIC in the status word (the partition is still complete).
 * Cost per depth: (iters + 1) reads of X plus 8 reads of one 64-bit key per
 * sample; depths = floor(log2 k) + (1 if k is not a power of two).
 */
GK_API int gk_two_means_tree(const float *X, int64_t n, int64_t d, int64_t ld, int32_t k, int32_t iters,
                             uint64_t seed, int32_t *labels, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_two_means_tree_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, int32_t k, int32_t iters,
                                  uint64_t seed, int32_t *labels, void *ws, size_t ws_bytes, void *stream);

/*
 * Boost form of GK-means (Sec. 3.1 Eq. 2 and Eq. 3; the move step of Alg. 2,
 * Sec. 4.2): the paper's standard configuration, in which one visited sample
 * at a time moves to the neighbouring cluster of largest objective gain.
 *
 * State of a partition (Eq. 2), all device memory owned by the caller:
 *   D       FP64 k x d, row-major (row r at D + r * d): D_r, the sum of the
 *           members of cluster r
 *   counts  int32[k]: n_r
 *   S       FP64[k]: S_r = D_r'D_r
 * The objective of Eq. 2 is I = sum over non-empty r of S_r / n_r, and the
 * k-means distortion (Eq. 4) is (sum_i ||x_i||^2 - I) / n.
 *
 * Arithmetic (fixed, so that every move decision is reproducible): FP64.
 * gk_boost_init sums each D_r over its members in ascending sample id.  A
 * squared norm squares each element of the vector zero-padded to the smallest
 * power of two P >= d (each product rounded once) and adds them by halving
 * folds: while P > 1, P /= 2 and w[j] = w[j] + w[j + P] for j < P.  Samples
 * are widened exactly to FP64 (BF16 through FP32).
 *
 * gk_boost_init: the state of the partition `labels` (int32[n] in [0, k)).
 *   ws  gk_workspace_size(GK_OP_BOOST, n, d, k, 0) bytes
 *
 * gk_boost_epoch: one epoch of the move step.  For s = 0 .. m - 1 in order,
 * sample i = order[s] with label u: if n_u >= 2, the candidates are the
 * distinct labels of its kappa neighbours (g_idx row i) other than u, and the
 * gain of moving to candidate v is
 *   ((A_v / (n_v + 1) + B / (n_u - 1)) - S_v / n_v) - S_u / n_u,
 *   A_v = (D_v + x)'(D_v + x),  B = (D_u - x)'(D_u - x)   (squared norms as above),
 * each operation rounded once, left to right.  The candidate of largest gain
 * (the smaller label on equal gains) is taken if its gain is > 0: then
 * labels[i] = v, D_u -= x and D_v += x element by element, n_u -= 1,
 * n_v += 1, S_u = B and S_v = A_v.  The next visit sees these changes.
 *   X, n, d, ld    samples as in gk_assign_step, 1 <= d <= 1024
 *   g_idx, kappa   KNN graph rows (only g_idx is read), 1 <= kappa <= 128
 *   order          device int32[m]: the visited sample ids (the paper draws
 *                  them at random; a permutation of [0, n) is one pass), m >= 0
 *   labels, D, counts, S   the state, updated in place; it must be the state
 *                  of `labels` (as gk_boost_init makes it) for the epoch to
 *                  follow Eq. 3
 *   n_moved        device int64[1] (out) or NULL: moves made
 *   ws             gk_workspace_size(GK_OP_BOOST, n, d, k, kappa) bytes
 * A visit id, label or neighbour id out of range sets GK_ERR_INVALID in the
 * status word and that visit makes no move.
 * The result is that of the visits made one after another.  One thread-block
 * cluster (up to 16 CTAs) runs the epoch: it evaluates windows of up to 32
 * visits against the state at the window's start and commits them in order
 * up to the first visit that depends on an earlier move of the window (its
 * sample or a neighbour moved, or its own cluster or a candidate was left or
 * joined); the rest is evaluated again in the next window.  A visit costs
 * (candidates + 1) FP64 rows of d elements read, and 2 rows written when it
 * moves.
 */
GK_API int gk_boost_init(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                         double *D, int32_t *counts, double *S, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_boost_init_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                              double *D, int32_t *counts, double *S, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_boost_epoch(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                          const int32_t *order, int64_t m, int32_t *labels, int32_t k, double *D, int32_t *counts,
                          double *S, int64_t *n_moved, void *ws, size_t ws_bytes, void *stream);
GK_API int gk_boost_epoch_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                               int32_t kappa, const int32_t *order, int64_t m, int32_t *labels, int32_t k, double *D,
                               int32_t *counts, double *S, int64_t *n_moved, void *ws, size_t ws_bytes, void *stream);

/*
 * Replay of repeated requests (off by default).  With replay on, a call of
 * gk_build_knn_graph(_bf16) or gk_kmeans_fit(_bf16) whose arguments (every
 * pointer, size and parameter; the device) equal an earlier call's is
 * launched as one CUDA graph, captured on that earlier call, instead of its
 * few hundred kernel launches one by one.  The graph reads and writes the
 * same addresses as a direct call, so the results are the same; the host
 * distortion log (e_log) is filled after it as before.  The first call with
 * new arguments pays the capture.  A call on a stream that is being captured
 * already, or on the legacy default stream (NULL), runs directly.  At most 32
 * graphs are kept (the oldest dropped, after a device synchronisation).
 * gk_set_replay(0) drops them all, after synchronising their devices.
 * Meant for a loop that repeats one request on the same buffers; a stream of
 * differently shaped requests would pay a capture per request.
 */
GK_API int gk_set_replay(int enable);

/*
 * Synchronise `stream`, return the status word the kernels of calls that used
 * `ws` recorded (GK_OK if none), and clear it.  Also returns GK_ERR_CUDA if the
 * stream itself reports an error.
 */
GK_API int gk_read_status(void *ws, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GKM_H */
