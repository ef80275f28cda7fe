// C entry points of libgkm (declared in include/gkm.h): argument checks,
// workspace layout and the step sequences of the fit (Alg. 2 with the
// closest-centroid rule) and of the graph construction (Alg. 3).
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "batch.cuh"
#include "common.cuh"

using namespace gkm;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define GK_CUDA(call)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(GK_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                    \
    } while (0)

constexpr int64_t MAX_ROWS = (int64_t)1 << 31;
constexpr int MAX_LOG = 4096;  // e_log entries kept on the device

int check_x(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int64_t min_n)
{
    if (!X)
        return fail(GK_ERR_INVALID, "X is NULL");
    if (n < min_n || n >= MAX_ROWS)
        return fail(GK_ERR_INVALID, "n = %lld out of range [%lld, 2^31)", (long long)n, (long long)min_n);
    if (d < 1 || d > MAX_D)
        return fail(GK_ERR_INVALID, "d = %lld out of range [1, %d]", (long long)d, MAX_D);
    if (ld < d)
        return fail(GK_ERR_INVALID, "ld = %lld < d = %lld", (long long)ld, (long long)d);
    if ((reinterpret_cast<uintptr_t>(X) & (bf16 ? 1 : 3)) != 0)
        return fail(GK_ERR_INVALID, "X is not %d-byte aligned", bf16 ? 2 : 4);
    return GK_OK;
}

int check_kappa(int32_t kappa, int64_t n)
{
    if (kappa < 1 || kappa > MAX_KAPPA || (int64_t)kappa >= n)
        return fail(GK_ERR_INVALID, "kappa = %d out of range [1, min(%d, n - 1)]", kappa, MAX_KAPPA);
    return GK_OK;
}

// The precision argument: bits 0-7 the level (0-4), bits 8-15 the assignment's candidates per group (0: the
// kernels' default, else 4 or 8; a tile shape with the same results), no other bits.
int check_precision(int32_t precision, bool bf16)
{
    const int level = precision & 0xff, gw = (precision >> 8) & 0xff;
    if (precision < 0 || (precision >> 16) != 0 || level > 4 || (gw != 0 && gw != 4 && gw != 8))
        return fail(GK_ERR_INVALID,
                    "precision = %d (bits 0-7: level 0, 1: FP32 rows; 2, 3: BF16 screening (3: on the tensor cores), "
                    "4: int8 screening, each + exact recompute; bits 8-15: 0, 4 or 8 candidates per group)",
                    precision);
    if (bf16 && level == 3)
        return fail(GK_ERR_INVALID, "BF16 samples: precision must be 0, 1 or 2 (3 screens on FP32 samples)");
    return GK_OK;
}

int check_ws(void *ws, size_t ws_bytes, size_t need)
{
    if (!ws)
        return fail(GK_ERR_INVALID, "workspace is NULL (needs %zu bytes)", need);
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0)
        return fail(GK_ERR_INVALID, "workspace is not 256-byte aligned");
    if (ws_bytes < need)
        return fail(GK_ERR_INVALID, "workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
    return GK_OK;
}

// Workspace layouts.  Every layout starts with the device status word.
struct GroupBufs {
    int32_t *offsets, *members, *counts;
    void *scratch;
};

struct Layout {
    DevStatus *st;
    // grouping
    GroupBufs grp;
    void *upd_scratch;
    void *asg_scratch;
    void *ref_scratch;
    void *rec_scratch;
    void *tree_scratch;
    int32_t *labels_a;
    int32_t *labels_b;
    float *cent;
    double *elog;
    size_t bytes;
};

Layout carve(void *ws, int op, int64_t n, int64_t d, int32_t k)
{
    Carver cv{static_cast<char *>(ws), 0, 0};
    Layout L{};
    L.st = cv.take<DevStatus>(1);
    bool need_group = op == GK_OP_ASSIGN || op == GK_OP_UPDATE || op == GK_OP_REFINE || op == GK_OP_FIT ||
                      op == GK_OP_BUILD || op == GK_OP_BOOST;
    bool need_update = op == GK_OP_UPDATE || op == GK_OP_FIT || op == GK_OP_BUILD;
    bool need_assign = op == GK_OP_ASSIGN || op == GK_OP_FIT || op == GK_OP_BUILD;
    if (need_group) {
        L.grp.offsets = cv.take<int32_t>((size_t)k + 1);
        L.grp.members = cv.take<int32_t>((size_t)n);
        L.grp.counts = cv.take<int32_t>((size_t)k);
        L.grp.scratch = cv.take<char>(group_scratch_bytes(n, k));
    }
    if (need_update)
        L.upd_scratch = cv.take<char>(update_scratch_bytes(n, k));
    if (need_assign)
        L.asg_scratch = cv.take<char>(assign_scratch_bytes(n, k, d));
    if (op == GK_OP_REFINE || op == GK_OP_BUILD)
        L.ref_scratch = cv.take<char>(refine_scratch_bytes(n, k, d));
    if (op == GK_OP_FIT || op == GK_OP_BUILD) {
        L.labels_b = cv.take<int32_t>((size_t)n);
        L.elog = cv.take<double>(MAX_LOG);
    }
    if (op == GK_OP_BUILD) {
        L.labels_a = cv.take<int32_t>((size_t)n);
        L.cent = cv.take<float>((size_t)k * (size_t)d);
    }
    if (op == GK_OP_RECALL)  // k: the number of queries
        L.rec_scratch = cv.take<char>(recall_scratch_bytes(n, k));
    if (op == GK_OP_TREE)
        L.tree_scratch = cv.take<char>(tree_scratch_bytes(n, d, k));
    L.bytes = cv.off;
    return L;
}

int32_t build_k0(int64_t n, int32_t xi) { return (int32_t)(n / xi > 0 ? n / xi : 1); }

// ---------------------------------------------------------------------------
// Replay of repeated one-call requests (opt-in, gk_set_replay).  A graph
// construction or fit whose arguments (pointers, sizes, parameters, device)
// equal an earlier call's is launched as the CUDA graph captured on that
// call, instead of its few hundred kernel launches one by one; the graph
// reads and writes the same addresses, so the results are those of a direct
// call.  A call on a stream that is already being captured, or on the legacy
// default stream, enqueues its launches directly.
// ---------------------------------------------------------------------------
constexpr size_t REPLAY_MAX = 32;  // cached graphs; the oldest is dropped beyond

struct Replay {
    std::mutex mu;
    bool on = false;
    std::map<std::vector<uint64_t>, cudaGraphExec_t> execs;
    std::vector<std::vector<uint64_t>> order;  // insertion order, for dropping the oldest

    // Drops every cached graph after the work of the devices they belong to has finished (a graph may still be
    // running from a replay).
    void clear()
    {
        int cur = 0;
        cudaGetDevice(&cur);
        std::set<int> devs;
        for (auto &kv : execs)
            devs.insert((int)kv.first.back());
        for (int dv : devs) {
            cudaSetDevice(dv);
            cudaDeviceSynchronize();
        }
        cudaSetDevice(cur);
        for (auto &kv : execs)
            cudaGraphExecDestroy(kv.second);
        execs.clear();
        order.clear();
    }
};

Replay &replay()
{
    static Replay r;
    return r;
}

// Runs enqueue() (which returns a GK_ code) directly, or through the replay cache under `key`.
template <typename F>
int enqueue_or_replay(std::vector<uint64_t> key, cudaStream_t s, F enqueue)
{
    Replay &R = replay();
    {
        std::lock_guard<std::mutex> lock(R.mu);
        if (!R.on)
            return enqueue();
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s == nullptr || cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return enqueue();
    int dev = 0;
    GK_CUDA(cudaGetDevice(&dev));
    key.push_back((uint64_t)dev);
    {
        std::lock_guard<std::mutex> lock(R.mu);
        auto it = R.execs.find(key);
        if (it != R.execs.end()) {
            GK_CUDA(cudaGraphLaunch(it->second, s));
            return GK_OK;
        }
    }
    GK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    const int rc = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc != GK_OK || e != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        return rc != GK_OK ? rc : fail(GK_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess)
        return fail(GK_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    {
        std::lock_guard<std::mutex> lock(R.mu);
        auto it = R.execs.find(key);
        if (it == R.execs.end()) {
            if (R.order.size() >= REPLAY_MAX) {
                auto old = R.execs.find(R.order.front());
                if (old != R.execs.end()) {
                    cudaDeviceSynchronize();  // the oldest graph may still be running from a replay
                    cudaGraphExecDestroy(old->second);
                    R.execs.erase(old);
                }
                R.order.erase(R.order.begin());
            }
            R.execs[key] = exec;
            R.order.push_back(key);
        } else {  // another thread captured the same call meanwhile
            cudaGraphExecDestroy(exec);
            exec = it->second;
        }
        GK_CUDA(cudaGraphLaunch(exec, s));
    }
    return GK_OK;
}

uint64_t u64(const void *p) { return (uint64_t)reinterpret_cast<uintptr_t>(p); }

}  // namespace

namespace gkm {
// Lets other translation units of the library report through gk_last_error().
void set_last_error(const char *msg)
{
    snprintf(g_err, sizeof(g_err), "%s", msg);
}

cudaError_t set_max_smem(const void *kernel, int bytes)
{
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, kernel}))
        return cudaSuccess;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) == cudaSuccess)
        done.insert({dev, kernel});
    return e;
}

cudaError_t resident_grid(const void *kernel, int threads, size_t smem, int *grid)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> known;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = known.find({dev, kernel});
    if (it != known.end()) {
        *grid = it->second;
        return cudaSuccess;
    }
    int sms = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem)) != cudaSuccess)
        return e;
    *grid = sms * (per > 0 ? per : 1);
    known[{dev, kernel}] = *grid;
    return cudaSuccess;
}
}  // namespace gkm

extern "C" {

const char *gk_version(void) { return "libgkm 0.1 (sm_103a)"; }

const char *gk_last_error(void) { return g_err; }

size_t gk_workspace_size(int32_t op, int64_t n, int64_t d, int32_t k, int32_t kappa)
{
    (void)kappa;
    if (op < GK_OP_ASSIGN || op > GK_OP_BOOST || op == GK_OP_BUILD || n < 0 || d < 0 || k < 0)
        return 0;
    return carve(nullptr, op, n, d, k).bytes;
}

size_t gk_workspace_size_build(int64_t n, int64_t d, const gk_graph_params *p)
{
    if (!p || p->xi < 1 || n < 0 || d < 0)
        return 0;
    return carve(nullptr, GK_OP_BUILD, n, d, build_k0(n, p->xi)).bytes;
}

int gk_init_labels(int64_t n, int32_t k, uint64_t seed, int32_t *labels, void *stream)
{
    if (n < 1 || n >= MAX_ROWS)
        return fail(GK_ERR_INVALID, "n = %lld out of range", (long long)n);
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (!labels)
        return fail(GK_ERR_INVALID, "labels is NULL");
    GK_CUDA(launch_init_labels(n, k, seed, labels, (cudaStream_t)stream));
    return GK_OK;
}

static int init_graph_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed,
                           int32_t *g_idx, float *g_dist, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 2)) || (rc = check_kappa(kappa, n)))
        return rc;
    if (!g_idx || !g_dist)
        return fail(GK_ERR_INVALID, "graph arrays are NULL");
    if ((rc = check_ws(ws, ws_bytes, sizeof(DevStatus))))
        return rc;
    GK_CUDA(launch_init_graph(X, bf16, n, d, ld, kappa, seed, g_idx, g_dist, static_cast<DevStatus *>(ws),
                              (cudaStream_t)stream));
    return GK_OK;
}

int gk_init_graph(const float *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed, int32_t *g_idx,
                  float *g_dist, void *ws, size_t ws_bytes, void *stream)
{
    return init_graph_impl(X, false, n, d, ld, kappa, seed, g_idx, g_dist, ws, ws_bytes, stream);
}

int gk_init_graph_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, int32_t kappa, uint64_t seed,
                       int32_t *g_idx, float *g_dist, void *ws, size_t ws_bytes, void *stream)
{
    return init_graph_impl(X, true, n, d, ld, kappa, seed, g_idx, g_dist, ws, ws_bytes, stream);
}


static int assign_step_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                            int32_t kappa, const float *C, int32_t k, const int32_t *labels_in, int32_t *labels_out,
                            float *best_d2, double *sum_d2, int64_t *n_changed, int32_t precision,
                            const int32_t *members, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 2)) || (rc = check_kappa(kappa, n)))
        return rc;
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (!g_idx || !C || !labels_in || !labels_out)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    if (labels_in == labels_out)
        return fail(GK_ERR_INVALID, "labels_out must not alias labels_in");
    if ((rc = check_precision(precision, bf16)))
        return rc;
    Layout L = carve(nullptr, GK_OP_ASSIGN, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_ASSIGN, n, d, k);
    if ((precision & 0xff) == 3 && !members) {  // group the samples by their input label for the tile screening
        GK_CUDA(launch_group(labels_in, n, k, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st,
                             (cudaStream_t)stream));
        members = L.grp.members;
    }
    GK_CUDA(launch_assign(X, bf16, n, d, ld, g_idx, kappa, C, k, labels_in, labels_out, best_d2, sum_d2, n_changed,
                          L.asg_scratch, L.st, (cudaStream_t)stream, precision, members));
    return GK_OK;
}

int gk_assign_step(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                   const float *C, int32_t k, const int32_t *labels_in, int32_t *labels_out, float *best_d2,
                   double *sum_d2, int64_t *n_changed, int32_t precision, const int32_t *members, void *ws,
                   size_t ws_bytes, void *stream)
{
    return assign_step_impl(X, false, n, d, ld, g_idx, kappa, C, k, labels_in, labels_out, best_d2, sum_d2,
                            n_changed, precision, members, ws, ws_bytes, stream);
}

int gk_assign_step_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                        const float *C, int32_t k, const int32_t *labels_in, int32_t *labels_out, float *best_d2,
                        double *sum_d2, int64_t *n_changed, int32_t precision, const int32_t *members, void *ws,
                        size_t ws_bytes, void *stream)
{
    return assign_step_impl(X, true, n, d, ld, g_idx, kappa, C, k, labels_in, labels_out, best_d2, sum_d2, n_changed,
                            precision, members, ws, ws_bytes, stream);
}


static int update_step_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *labels,
                            int32_t k, float *C, int32_t *counts, double *sum_d2, int32_t *offsets, int32_t *members,
                            void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 1)))
        return rc;
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (!labels || !C)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    Layout L = carve(nullptr, GK_OP_UPDATE, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_UPDATE, n, d, k);
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *off = offsets ? offsets : L.grp.offsets;
    int32_t *mem = members ? members : L.grp.members;
    int32_t *cnt = counts ? counts : L.grp.counts;
    GK_CUDA(launch_group(labels, n, k, off, mem, cnt, L.grp.scratch, L.st, s));
    GK_CUDA(launch_update(X, bf16, n, d, ld, off, mem, k, C, cnt, sum_d2, L.upd_scratch, L.st, s));
    return GK_OK;
}

int gk_update_step(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k, float *C,
                   int32_t *counts, double *sum_d2, int32_t *offsets, int32_t *members, void *ws, size_t ws_bytes,
                   void *stream)
{
    return update_step_impl(X, false, n, d, ld, labels, k, C, counts, sum_d2, offsets, members, ws, ws_bytes, stream);
}

int gk_update_step_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                        float *C, int32_t *counts, double *sum_d2, int32_t *offsets, int32_t *members, void *ws,
                        size_t ws_bytes, void *stream)
{
    return update_step_impl(X, true, n, d, ld, labels, k, C, counts, sum_d2, offsets, members, ws, ws_bytes, stream);
}


static int graph_refine_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *labels,
                             int32_t k, int32_t kappa, int32_t max_cluster, int32_t precision, int32_t *g_idx,
                             float *g_dist, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 2)) || (rc = check_kappa(kappa, n)))
        return rc;
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (max_cluster < 2)
        return fail(GK_ERR_INVALID, "max_cluster = %d < 2", max_cluster);
    if ((rc = check_precision(precision, false)))
        return rc;
    precision &= 0xff;  // the refinement's path: 0 FP32 tiles, >= 1 the tensor-core Gram where d allows
    if (!labels || !g_idx || !g_dist)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    Layout L = carve(nullptr, GK_OP_REFINE, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_REFINE, n, d, k);
    cudaStream_t s = (cudaStream_t)stream;
    GK_CUDA(launch_group(labels, n, k, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st, s));
    GK_CUDA(launch_refine(X, bf16, n, d, ld, L.grp.offsets, L.grp.members, k, kappa, max_cluster, g_idx, g_dist,
                          L.ref_scratch, L.st, s, precision));
    return GK_OK;
}

int gk_graph_refine(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                    int32_t kappa, int32_t max_cluster, int32_t precision, int32_t *g_idx, float *g_dist, void *ws,
                    size_t ws_bytes, void *stream)
{
    return graph_refine_impl(X, false, n, d, ld, labels, k, kappa, max_cluster, precision, g_idx, g_dist, ws,
                             ws_bytes, stream);
}

int gk_graph_refine_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                         int32_t kappa, int32_t max_cluster, int32_t precision, int32_t *g_idx, float *g_dist,
                         void *ws, size_t ws_bytes, void *stream)
{
    return graph_refine_impl(X, true, n, d, ld, labels, k, kappa, max_cluster, precision, g_idx, g_dist, ws,
                             ws_bytes, stream);
}


int gk_group_by_label(const int32_t *labels, int64_t n, int32_t k, int32_t *offsets, int32_t *members,
                      int32_t *counts, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if (n < 1 || n >= MAX_ROWS)
        return fail(GK_ERR_INVALID, "n = %lld out of range", (long long)n);
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (!labels || !offsets || !members)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    Layout L = carve(nullptr, GK_OP_UPDATE, n, 1, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_UPDATE, n, 1, k);
    GK_CUDA(launch_group(labels, n, k, offsets, members, counts ? counts : L.grp.counts, L.grp.scratch, L.st,
                         (cudaStream_t)stream));
    return GK_OK;
}

static int update_from_groups_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                                   const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2,
                                   void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 1)))
        return rc;
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (!offsets || !members || !C)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    Layout L = carve(nullptr, GK_OP_UPDATE, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_UPDATE, n, d, k);
    GK_CUDA(launch_update(X, bf16, n, d, ld, offsets, members, k, C, counts, sum_d2, L.upd_scratch, L.st,
                          (cudaStream_t)stream));
    return GK_OK;
}

int gk_update_from_groups(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2, void *ws,
                          size_t ws_bytes, void *stream)
{
    return update_from_groups_impl(X, false, n, d, ld, offsets, members, k, C, counts, sum_d2, ws, ws_bytes, stream);
}

int gk_update_from_groups_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                               const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2, void *ws,
                               size_t ws_bytes, void *stream)
{
    return update_from_groups_impl(X, true, n, d, ld, offsets, members, k, C, counts, sum_d2, ws, ws_bytes, stream);
}


static int graph_refine_groups_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld,
                                    const int32_t *offsets, const int32_t *members, int32_t k, int32_t kappa,
                                    int32_t max_cluster, int32_t precision, int32_t *g_idx, float *g_dist, void *ws,
                                    size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 2)) || (rc = check_kappa(kappa, n)))
        return rc;
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (max_cluster < 2)
        return fail(GK_ERR_INVALID, "max_cluster = %d < 2", max_cluster);
    if ((rc = check_precision(precision, false)))
        return rc;
    precision &= 0xff;
    if (!offsets || !members || !g_idx || !g_dist)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    Layout L = carve(nullptr, GK_OP_REFINE, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_REFINE, n, d, k);
    GK_CUDA(launch_refine(X, bf16, n, d, ld, offsets, members, k, kappa, max_cluster, g_idx, g_dist, L.ref_scratch,
                          L.st, (cudaStream_t)stream, precision));
    return GK_OK;
}

int gk_graph_refine_groups(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                           const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster, int32_t precision,
                           int32_t *g_idx, float *g_dist, void *ws, size_t ws_bytes, void *stream)
{
    return graph_refine_groups_impl(X, false, n, d, ld, offsets, members, k, kappa, max_cluster, precision, g_idx,
                                    g_dist, ws, ws_bytes, stream);
}

int gk_graph_refine_groups_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                                const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster,
                                int32_t precision, int32_t *g_idx, float *g_dist, void *ws, size_t ws_bytes,
                                void *stream)
{
    return graph_refine_groups_impl(X, true, n, d, ld, offsets, members, k, kappa, max_cluster, precision, g_idx,
                                    g_dist, ws, ws_bytes, stream);
}


static int kmeans_fit_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t k,
                           const int32_t *g_idx, int32_t kappa, int32_t iters, const int32_t *init_labels,
                           uint64_t seed, int32_t precision, int32_t *labels_out, float *C_out, int32_t *counts_out,
                           double *e_log, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 2)) || (rc = check_kappa(kappa, n)))
        return rc;
    if (k < 1)
        return fail(GK_ERR_INVALID, "k = %d < 1", k);
    if (iters < 0 || 2 * iters + 1 > MAX_LOG)
        return fail(GK_ERR_INVALID, "iters = %d out of range [0, %d]", iters, (MAX_LOG - 1) / 2);
    if ((rc = check_precision(precision, bf16)))
        return rc;
    if (!g_idx || !labels_out || !C_out)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    Layout L = carve(nullptr, GK_OP_FIT, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_FIT, n, d, k);
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *cnt = counts_out ? counts_out : L.grp.counts;

    auto enqueue = [&]() -> int {
        // ping-pong the labels so that the final ones land in labels_out
        int32_t *cur = (iters % 2 == 0) ? labels_out : L.labels_b;
        int32_t *nxt = (iters % 2 == 0) ? L.labels_b : labels_out;
        if (init_labels)
            GK_CUDA(cudaMemcpyAsync(cur, init_labels, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        else
            GK_CUDA(launch_init_labels(n, k, seed, cur, s));
        GK_CUDA(cudaMemsetAsync(C_out, 0, sizeof(float) * (size_t)k * (size_t)d, s));
        GK_CUDA(launch_group(cur, n, k, L.grp.offsets, L.grp.members, cnt, L.grp.scratch, L.st, s));
        GK_CUDA(launch_update(X, bf16, n, d, ld, L.grp.offsets, L.grp.members, k, C_out, cnt, L.elog + 0,
                              L.upd_scratch, L.st, s));
        for (int t = 0; t < iters; t++) {
            GK_CUDA(launch_assign(X, bf16, n, d, ld, g_idx, kappa, C_out, k, cur, nxt, nullptr, L.elog + 1 + 2 * t,
                                  nullptr, L.asg_scratch, L.st, s, precision, L.grp.members));
            GK_CUDA(launch_group(nxt, n, k, L.grp.offsets, L.grp.members, cnt, L.grp.scratch, L.st, s));
            GK_CUDA(launch_update(X, bf16, n, d, ld, L.grp.offsets, L.grp.members, k, C_out, cnt, L.elog + 2 + 2 * t,
                                  L.upd_scratch, L.st, s));
            int32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        return GK_OK;
    };
    const std::vector<uint64_t> key = {1, u64(X), (uint64_t)bf16, (uint64_t)n, (uint64_t)d, (uint64_t)ld, (uint64_t)k,
                                       u64(g_idx), (uint64_t)kappa, (uint64_t)iters, u64(init_labels), seed,
                                       (uint64_t)precision, u64(labels_out), u64(C_out), u64(counts_out), u64(ws),
                                       (uint64_t)ws_bytes};
    if ((rc = enqueue_or_replay(key, s, enqueue)) != GK_OK)
        return rc;
    if (e_log) {
        GK_CUDA(cudaMemcpyAsync(e_log, L.elog, sizeof(double) * (size_t)(2 * iters + 1), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < 2 * iters + 1; q++)
            e_log[q] /= (double)n;
    }
    return GK_OK;
}

int gk_kmeans_fit(const float *X, int64_t n, int64_t d, int64_t ld, int32_t k, const int32_t *g_idx, int32_t kappa,
                  int32_t iters, const int32_t *init_labels, uint64_t seed, int32_t precision, int32_t *labels_out,
                  float *C_out, int32_t *counts_out, double *e_log, void *ws, size_t ws_bytes, void *stream)
{
    return kmeans_fit_impl(X, false, n, d, ld, k, g_idx, kappa, iters, init_labels, seed, precision, labels_out,
                           C_out, counts_out, e_log, ws, ws_bytes, stream);
}

int gk_kmeans_fit_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, int32_t k, const int32_t *g_idx,
                       int32_t kappa, int32_t iters, const int32_t *init_labels, uint64_t seed, int32_t precision,
                       int32_t *labels_out, float *C_out, int32_t *counts_out, double *e_log, void *ws,
                       size_t ws_bytes, void *stream)
{
    return kmeans_fit_impl(X, true, n, d, ld, k, g_idx, kappa, iters, init_labels, seed, precision, labels_out,
                           C_out, counts_out, e_log, ws, ws_bytes, stream);
}


static int build_knn_graph_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const gk_graph_params *p,
                                int32_t *g_idx, float *g_dist, int32_t *labels_out, double *e_log, void *ws,
                                size_t ws_bytes, void *stream)
{
    int rc;
    if (!p)
        return fail(GK_ERR_INVALID, "params is NULL");
    if ((rc = check_x(X, bf16, n, d, ld, 2)) || (rc = check_kappa(p->kappa, n)))
        return rc;
    if (p->xi < 1 || p->tau < 0 || 2 * p->tau + 1 > MAX_LOG || p->max_cluster < 2 || p->reserved != 0)
        return fail(GK_ERR_INVALID, "bad params (xi=%d tau=%d max_cluster=%d)", p->xi, p->tau, p->max_cluster);
    if ((rc = check_precision(p->precision, bf16)))
        return rc;
    if (!g_idx || !g_dist)
        return fail(GK_ERR_INVALID, "graph arrays are NULL");
    const int32_t k0 = build_k0(n, p->xi);
    Layout L = carve(nullptr, GK_OP_BUILD, n, d, k0);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_BUILD, n, d, k0);
    cudaStream_t s = (cudaStream_t)stream;
    const int tau = p->tau;
    auto enqueue = [&]() -> int {
        int32_t *cur = L.labels_a, *nxt = L.labels_b;
        GK_CUDA(launch_init_graph(X, bf16, n, d, ld, p->kappa, p->seed, g_idx, g_dist, L.st, s));
        GK_CUDA(launch_init_labels(n, k0, p->seed, cur, s));
        GK_CUDA(cudaMemsetAsync(L.cent, 0, sizeof(float) * (size_t)k0 * (size_t)d, s));
        GK_CUDA(launch_group(cur, n, k0, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st, s));
        GK_CUDA(launch_update(X, bf16, n, d, ld, L.grp.offsets, L.grp.members, k0, L.cent, L.grp.counts, L.elog + 0,
                              L.upd_scratch, L.st, s));
        for (int t = 0; t < tau; t++) {
            // one k-means iteration at k0 on the current graph (Sec. 4.5: t = 1 per round)
            GK_CUDA(launch_assign(X, bf16, n, d, ld, g_idx, p->kappa, L.cent, k0, cur, nxt, nullptr, L.elog + 1 + 2 * t,
                                  nullptr, L.asg_scratch, L.st, s, p->precision, L.grp.members));
            GK_CUDA(launch_group(nxt, n, k0, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st, s));
            GK_CUDA(launch_update(X, bf16, n, d, ld, L.grp.offsets, L.grp.members, k0, L.cent, L.grp.counts,
                                  L.elog + 2 + 2 * t, L.upd_scratch, L.st, s));
            // exhaustive pairs inside the clusters of the new partition
            GK_CUDA(launch_refine(X, bf16, n, d, ld, L.grp.offsets, L.grp.members, k0, p->kappa, p->max_cluster, g_idx,
                                  g_dist, L.ref_scratch, L.st, s, p->precision & 0xff));
            int32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        if (labels_out)
            GK_CUDA(cudaMemcpyAsync(labels_out, cur, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        return GK_OK;
    };
    const std::vector<uint64_t> key = {2, u64(X), (uint64_t)bf16, (uint64_t)n, (uint64_t)d, (uint64_t)ld,
                                       (uint64_t)p->kappa, (uint64_t)p->xi, (uint64_t)p->tau,
                                       (uint64_t)p->max_cluster, p->seed, (uint64_t)p->precision, u64(g_idx),
                                       u64(g_dist), u64(labels_out), u64(ws), (uint64_t)ws_bytes};
    if ((rc = enqueue_or_replay(key, s, enqueue)) != GK_OK)
        return rc;
    if (e_log) {
        GK_CUDA(cudaMemcpyAsync(e_log, L.elog, sizeof(double) * (size_t)(2 * tau + 1), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < 2 * tau + 1; q++)
            e_log[q] /= (double)n;
    }
    return GK_OK;
}

int gk_build_knn_graph(const float *X, int64_t n, int64_t d, int64_t ld, const gk_graph_params *p, int32_t *g_idx,
                       float *g_dist, int32_t *labels_out, double *e_log, void *ws, size_t ws_bytes, void *stream)
{
    return build_knn_graph_impl(X, false, n, d, ld, p, g_idx, g_dist, labels_out, e_log, ws, ws_bytes, stream);
}

int gk_build_knn_graph_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const gk_graph_params *p,
                            int32_t *g_idx, float *g_dist, int32_t *labels_out, double *e_log, void *ws,
                            size_t ws_bytes, void *stream)
{
    return build_knn_graph_impl(X, true, n, d, ld, p, g_idx, g_dist, labels_out, e_log, ws, ws_bytes, stream);
}


// ---------------------------------------------------------------------------
// Batches (gk_batch_fit): the jobs' samples are concatenated; job j's graph
// rows, labels and clusters are shifted by its first sample, first cluster at
// k0 and first cluster at k, so no cluster and no graph row spans two jobs and
// every tie order ((distance, id), (distance, label)) is that of the job alone.
// ---------------------------------------------------------------------------
struct BatchDims {
    BatchTable t{};      // samples and clusters at k (the fit)
    int32_t k0first[MAX_BATCH_JOBS + 1];
    int64_t N = 0;
    int32_t K0 = 0, K = 0;
};

static int batch_dims(int32_t njobs, const gk_job *jobs, const gk_graph_params *p, BatchDims *bd)
{
    if (njobs < 1 || njobs > MAX_BATCH_JOBS)
        return fail(GK_ERR_INVALID, "njobs = %d out of range [1, %d]", njobs, MAX_BATCH_JOBS);
    if (!jobs || !p)
        return fail(GK_ERR_INVALID, "jobs or params is NULL");
    if (p->xi < 1)
        return fail(GK_ERR_INVALID, "xi = %d < 1", p->xi);
    int64_t N = 0, K0 = 0, K = 0;
    bd->t.njobs = njobs;
    for (int j = 0; j < njobs; j++) {
        const gk_job &J = jobs[j];
        if (J.n < 2 || J.k < 1 || J.reserved != 0 || (int64_t)p->kappa >= J.n)
            return fail(GK_ERR_INVALID, "job %d: n = %lld, k = %d (need n >= 2, kappa < n, k >= 1, reserved 0)", j,
                        (long long)J.n, J.k);
        bd->t.first[j] = N;
        bd->t.kfirst[j] = (int32_t)K;
        bd->k0first[j] = (int32_t)K0;
        N += J.n;
        K0 += build_k0(J.n, p->xi);
        K += J.k;
        if (N >= MAX_ROWS || K0 >= INT32_MAX || K >= INT32_MAX)
            return fail(GK_ERR_INVALID, "batch too large: %lld samples, %lld clusters", (long long)N, (long long)K);
    }
    bd->t.first[njobs] = N;
    bd->t.kfirst[njobs] = (int32_t)K;
    bd->k0first[njobs] = (int32_t)K0;
    bd->N = N;
    bd->K0 = (int32_t)K0;
    bd->K = (int32_t)K;
    return GK_OK;
}

static int batch_fit_impl(const void *X, bool bf16, int64_t d, int64_t ld, int32_t njobs, const gk_job *jobs,
                          const gk_graph_params *p, int32_t iters, int32_t *g_idx, float *g_dist, int32_t *labels_out,
                          float *C_out, double *distortion, void *ws, size_t ws_bytes, void *stream)
{
    BatchDims bd;
    int rc;
    if ((rc = batch_dims(njobs, jobs, p, &bd)))
        return rc;
    const int64_t N = bd.N;
    if ((rc = check_x(X, bf16, N, d, ld, 2)) || (rc = check_kappa(p->kappa, N)))
        return rc;
    if (p->tau < 0 || p->max_cluster < 2 || p->reserved != 0)
        return fail(GK_ERR_INVALID, "bad params (tau=%d max_cluster=%d)", p->tau, p->max_cluster);
    if ((rc = check_precision(p->precision, bf16)))
        return rc;
    if (iters < 0)
        return fail(GK_ERR_INVALID, "iters = %d < 0", iters);
    if (!g_idx || !g_dist || !labels_out || !C_out || !distortion)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    const int32_t Km = bd.K0 > bd.K ? bd.K0 : bd.K;
    Layout L = carve(nullptr, GK_OP_BUILD, N, d, Km);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_BUILD, N, d, Km);
    cudaStream_t s = (cudaStream_t)stream;
    const int es = bf16 ? 2 : 4;
    const char *Xc = static_cast<const char *>(X);
    auto enqueue = [&]() -> int {
        int32_t *cur = L.labels_a, *nxt = L.labels_b;
        // each job's random graph and labels at its k0, drawn on its own rows as alone, then shifted
        for (int j = 0; j < njobs; j++) {
            const int64_t f = bd.t.first[j], nj = jobs[j].n;
            GK_CUDA(launch_init_graph(Xc + (size_t)f * (size_t)ld * es, bf16, nj, d, ld, p->kappa, jobs[j].graph_seed,
                                      g_idx + f * p->kappa, g_dist + f * p->kappa, L.st, s, (int32_t)f));
            GK_CUDA(launch_init_labels(nj, build_k0(nj, p->xi), jobs[j].graph_seed, cur + f, s, bd.k0first[j]));
        }
        // Alg. 3 over the whole batch at k0 = sum of the jobs' k0
        GK_CUDA(cudaMemsetAsync(L.cent, 0, sizeof(float) * (size_t)bd.K0 * (size_t)d, s));
        GK_CUDA(launch_group(cur, N, bd.K0, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st, s));
        GK_CUDA(launch_update(X, bf16, N, d, ld, L.grp.offsets, L.grp.members, bd.K0, L.cent, L.grp.counts, nullptr,
                              L.upd_scratch, L.st, s));
        for (int t = 0; t < p->tau; t++) {
            GK_CUDA(launch_assign(X, bf16, N, d, ld, g_idx, p->kappa, L.cent, bd.K0, cur, nxt, nullptr, nullptr,
                                  nullptr, L.asg_scratch, L.st, s, p->precision, L.grp.members));
            GK_CUDA(launch_group(nxt, N, bd.K0, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st, s));
            GK_CUDA(launch_update(X, bf16, N, d, ld, L.grp.offsets, L.grp.members, bd.K0, L.cent, L.grp.counts,
                                  nullptr, L.upd_scratch, L.st, s));
            GK_CUDA(launch_refine(X, bf16, N, d, ld, L.grp.offsets, L.grp.members, bd.K0, p->kappa, p->max_cluster,
                                  g_idx, g_dist, L.ref_scratch, L.st, s, p->precision & 0xff));
            int32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        // Alg. 2 at each job's k from its own seeded labels
        for (int j = 0; j < njobs; j++) {
            const int64_t f = bd.t.first[j];
            GK_CUDA(launch_init_labels(jobs[j].n, jobs[j].k, jobs[j].fit_seed, cur + f, s, bd.t.kfirst[j]));
        }
        GK_CUDA(cudaMemsetAsync(C_out, 0, sizeof(float) * (size_t)bd.K * (size_t)d, s));
        GK_CUDA(launch_group(cur, N, bd.K, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st, s));
        GK_CUDA(launch_update(X, bf16, N, d, ld, L.grp.offsets, L.grp.members, bd.K, C_out, L.grp.counts, nullptr,
                              L.upd_scratch, L.st, s));
        for (int t = 0; t < iters; t++) {
            GK_CUDA(launch_assign(X, bf16, N, d, ld, g_idx, p->kappa, C_out, bd.K, cur, nxt, nullptr, nullptr, nullptr,
                                  L.asg_scratch, L.st, s, p->precision, L.grp.members));
            GK_CUDA(launch_group(nxt, N, bd.K, L.grp.offsets, L.grp.members, L.grp.counts, L.grp.scratch, L.st, s));
            GK_CUDA(launch_update(X, bf16, N, d, ld, L.grp.offsets, L.grp.members, bd.K, C_out, L.grp.counts,
                                  nullptr, L.upd_scratch, L.st, s));
            int32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        // each job's distortion from the last update's per-cluster terms, and labels in each job's numbering
        GK_CUDA(launch_batch_distortion(update_contrib(L.upd_scratch), bd.t, distortion, s));
        GK_CUDA(launch_batch_labels(cur, N, bd.t, labels_out, s));
        return GK_OK;
    };
    std::vector<uint64_t> key = {3, u64(X), (uint64_t)bf16, (uint64_t)d, (uint64_t)ld, (uint64_t)njobs,
                                 (uint64_t)p->kappa, (uint64_t)p->xi, (uint64_t)p->tau, (uint64_t)p->max_cluster,
                                 (uint64_t)p->precision, (uint64_t)iters, u64(g_idx), u64(g_dist), u64(labels_out),
                                 u64(C_out), u64(distortion), u64(ws), (uint64_t)ws_bytes};
    for (int j = 0; j < njobs; j++) {
        key.push_back((uint64_t)jobs[j].n);
        key.push_back((uint64_t)jobs[j].k);
        key.push_back(jobs[j].graph_seed);
        key.push_back(jobs[j].fit_seed);
    }
    return enqueue_or_replay(key, s, enqueue);
}

size_t gk_workspace_size_batch(int64_t d, int32_t njobs, const gk_job *jobs, const gk_graph_params *p)
{
    BatchDims bd;
    if (d < 1 || batch_dims(njobs, jobs, p, &bd) != GK_OK)
        return 0;
    return carve(nullptr, GK_OP_BUILD, bd.N, d, bd.K0 > bd.K ? bd.K0 : bd.K).bytes;
}

int gk_batch_fit(const float *X, int64_t d, int64_t ld, int32_t njobs, const gk_job *jobs,
                 const gk_graph_params *p, int32_t iters, int32_t *g_idx, float *g_dist, int32_t *labels_out,
                 float *C_out, double *distortion, void *ws, size_t ws_bytes, void *stream)
{
    return batch_fit_impl(X, false, d, ld, njobs, jobs, p, iters, g_idx, g_dist, labels_out, C_out, distortion, ws,
                          ws_bytes, stream);
}

int gk_batch_fit_bf16(const uint16_t *X, int64_t d, int64_t ld, int32_t njobs, const gk_job *jobs,
                      const gk_graph_params *p, int32_t iters, int32_t *g_idx, float *g_dist, int32_t *labels_out,
                      float *C_out, double *distortion, void *ws, size_t ws_bytes, void *stream)
{
    return batch_fit_impl(X, true, d, ld, njobs, jobs, p, iters, g_idx, g_dist, labels_out, C_out, distortion, ws,
                          ws_bytes, stream);
}

static int graph_recall_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                             int32_t kappa, const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist,
                             int64_t *hits, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 2)) || (rc = check_kappa(kappa, n)))
        return rc;
    if (m < 1)
        return fail(GK_ERR_INVALID, "m = %d < 1", m);
    if (!g_idx || !queries || !hits)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    Layout L = carve(nullptr, GK_OP_RECALL, n, d, m);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_RECALL, n, d, m);
    GK_CUDA(launch_recall(X, bf16, n, d, ld, g_idx, kappa, queries, m, nn_idx, nn_dist, hits, L.rec_scratch, L.st,
                          (cudaStream_t)stream));
    return GK_OK;
}

int gk_graph_recall(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                    const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist, int64_t *hits, void *ws,
                    size_t ws_bytes, void *stream)
{
    return graph_recall_impl(X, false, n, d, ld, g_idx, kappa, queries, m, nn_idx, nn_dist, hits, ws, ws_bytes,
                             stream);
}

int gk_graph_recall_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                         const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist, int64_t *hits, void *ws,
                         size_t ws_bytes, void *stream)
{
    return graph_recall_impl(X, true, n, d, ld, g_idx, kappa, queries, m, nn_idx, nn_dist, hits, ws, ws_bytes,
                             stream);
}

static int two_means_tree_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t k,
                               int32_t iters, uint64_t seed, int32_t *labels, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 1)))
        return rc;
    if (k < 1 || (int64_t)k > n)
        return fail(GK_ERR_INVALID, "k = %d out of range [1, n = %lld]", k, (long long)n);
    if (iters < 0 || iters > 64)
        return fail(GK_ERR_INVALID, "iters = %d out of range [0, 64]", iters);
    if (!labels)
        return fail(GK_ERR_INVALID, "labels is NULL");
    Layout L = carve(nullptr, GK_OP_TREE, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L.bytes)))
        return rc;
    L = carve(ws, GK_OP_TREE, n, d, k);
    GK_CUDA(launch_tree(X, bf16, n, d, ld, k, iters, seed, labels, L.tree_scratch, L.st, (cudaStream_t)stream));
    return GK_OK;
}

int gk_two_means_tree(const float *X, int64_t n, int64_t d, int64_t ld, int32_t k, int32_t iters, uint64_t seed,
                      int32_t *labels, void *ws, size_t ws_bytes, void *stream)
{
    return two_means_tree_impl(X, false, n, d, ld, k, iters, seed, labels, ws, ws_bytes, stream);
}

int gk_two_means_tree_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, int32_t k, int32_t iters,
                           uint64_t seed, int32_t *labels, void *ws, size_t ws_bytes, void *stream)
{
    return two_means_tree_impl(X, true, n, d, ld, k, iters, seed, labels, ws, ws_bytes, stream);
}

static int boost_check(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t k, const void *D,
                       const void *counts, const void *S, void *ws, size_t ws_bytes, Layout *L)
{
    int rc;
    if ((rc = check_x(X, bf16, n, d, ld, 1)))
        return rc;
    if (d > boost_max_d())
        return fail(GK_ERR_INVALID, "d = %lld > %lld (boost form)", (long long)d, (long long)boost_max_d());
    if (k < 1 || (int64_t)k > n)
        return fail(GK_ERR_INVALID, "k = %d out of range [1, n = %lld]", k, (long long)n);
    if (!D || !counts || !S)
        return fail(GK_ERR_INVALID, "a required array is NULL");
    *L = carve(nullptr, GK_OP_BOOST, n, d, k);
    if ((rc = check_ws(ws, ws_bytes, L->bytes)))
        return rc;
    *L = carve(ws, GK_OP_BOOST, n, d, k);
    return GK_OK;
}

static int boost_init_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *labels,
                           int32_t k, double *D, int32_t *counts, double *S, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    Layout L;
    if ((rc = boost_check(X, bf16, n, d, ld, k, D, counts, S, ws, ws_bytes, &L)))
        return rc;
    if (!labels)
        return fail(GK_ERR_INVALID, "labels is NULL");
    GK_CUDA(launch_boost_init(X, bf16, n, d, ld, labels, k, D, counts, S, L.grp.offsets, L.grp.members,
                              L.grp.counts, L.grp.scratch, L.st, (cudaStream_t)stream));
    return GK_OK;
}

int gk_boost_init(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k, double *D,
                  int32_t *counts, double *S, void *ws, size_t ws_bytes, void *stream)
{
    return boost_init_impl(X, false, n, d, ld, labels, k, D, counts, S, ws, ws_bytes, stream);
}

int gk_boost_init_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *labels, int32_t k,
                       double *D, int32_t *counts, double *S, void *ws, size_t ws_bytes, void *stream)
{
    return boost_init_impl(X, true, n, d, ld, labels, k, D, counts, S, ws, ws_bytes, stream);
}

static int boost_epoch_impl(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                            int32_t kappa, const int32_t *order, int64_t m, int32_t *labels, int32_t k, double *D,
                            int32_t *counts, double *S, int64_t *n_moved, void *ws, size_t ws_bytes, void *stream)
{
    int rc;
    Layout L;
    if ((rc = boost_check(X, bf16, n, d, ld, k, D, counts, S, ws, ws_bytes, &L)))
        return rc;
    if ((rc = check_kappa(kappa, n)))
        return rc;
    if (m < 0)
        return fail(GK_ERR_INVALID, "m = %lld < 0", (long long)m);
    if (!g_idx || !labels || (m > 0 && !order))
        return fail(GK_ERR_INVALID, "a required array is NULL");
    GK_CUDA(launch_boost_epoch(X, bf16, n, d, ld, g_idx, kappa, order, m, labels, k, D, counts, S, n_moved, L.st,
                               (cudaStream_t)stream));
    return GK_OK;
}

int gk_boost_epoch(const float *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                   const int32_t *order, int64_t m, int32_t *labels, int32_t k, double *D, int32_t *counts, double *S,
                   int64_t *n_moved, void *ws, size_t ws_bytes, void *stream)
{
    return boost_epoch_impl(X, false, n, d, ld, g_idx, kappa, order, m, labels, k, D, counts, S, n_moved, ws,
                            ws_bytes, stream);
}

int gk_boost_epoch_bf16(const uint16_t *X, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx, int32_t kappa,
                        const int32_t *order, int64_t m, int32_t *labels, int32_t k, double *D, int32_t *counts,
                        double *S, int64_t *n_moved, void *ws, size_t ws_bytes, void *stream)
{
    return boost_epoch_impl(X, true, n, d, ld, g_idx, kappa, order, m, labels, k, D, counts, S, n_moved, ws, ws_bytes,
                            stream);
}

int gk_set_replay(int enable)
{
    Replay &R = replay();
    std::lock_guard<std::mutex> lock(R.mu);
    R.on = enable != 0;
    if (!R.on)
        R.clear();
    return GK_OK;
}

int gk_read_status(void *ws, void *stream)
{
    if (!ws)
        return fail(GK_ERR_INVALID, "workspace is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    GK_CUDA(cudaStreamSynchronize(s));
    unsigned h[2] = {0, 0};
    GK_CUDA(cudaMemcpy(h, ws, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[0] != 0) {
        GK_CUDA(cudaMemset(ws, 0, sizeof(h)));
        return fail((int)h[0], "device status %u (detail %u)", h[0], h[1]);
    }
    return GK_OK;
}

}  // extern "C"
