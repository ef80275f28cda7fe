// Shared device helpers of libgkm (CUDA, sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gkm.h"

namespace gkm {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int MAX_KAPPA = 128;
constexpr int MAX_D = 4096;  // widest row (the generic assignment stages one sample per warp in shared memory)

// Kernels whose dynamic shared memory depends on kappa or d get the attribute
// cudaFuncAttributeMaxDynamicSharedMemorySize set to their size at the largest
// allowed kappa and d: the attribute is per function, and launches from
// several host threads must not see each other's settings.  It is set once per
// device and kernel (set_max_smem), so that calls after the first issue no
// such API call and can be captured into a CUDA graph.

// Device status word kept at the start of every workspace: the first error a
// kernel meets (code, detail).  Kernels record and skip; they never trap.
struct DevStatus {
    unsigned code;
    unsigned detail;
    unsigned pad[62];  // keeps what follows 256-byte aligned
};

__device__ __forceinline__ void flag_error(DevStatus *st, unsigned code, unsigned detail)
{
    if (st && atomicCAS(&st->code, 0u, code) == 0u)
        st->detail = detail;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the generator advances its
// state by gamma and returns mix(state).  Used as a counter-based function:
// draw(key, c) is output number c + 1 of the generator whose state starts at key.
constexpr uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint64_t TAG_LABELS = 0x4C41424C00000000ull;  // "LABL"
constexpr uint64_t TAG_GRAPH = 0x4752415000000000ull;   // "GRAP"

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sm64_draw(uint64_t key, uint64_t counter)
{
    return sm64_mix(key + (counter + 1ull) * SM64_GAMMA);
}

// Samples are stored as FP32 or BF16; a BF16 element is widened exactly to
// FP32 on load, and all arithmetic is FP32, so BF16 samples give the results
// of their FP32 widening bit for bit.
__device__ __forceinline__ float4 bf16x4_to_float4(uint2 v)
{
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&v.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&v.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

template <typename XT>
__device__ __forceinline__ float ldx(const XT *p);
template <>
__device__ __forceinline__ float ldx<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldx<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

// Four consecutive elements (16-byte aligned for FP32, 8-byte aligned for BF16); STREAM: read once (no L1 reuse).
template <typename XT, bool STREAM = false>
__device__ __forceinline__ float4 ldx4(const XT *p);
template <>
__device__ __forceinline__ float4 ldx4<float, false>(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
template <>
__device__ __forceinline__ float4 ldx4<float, true>(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
template <>
__device__ __forceinline__ float4 ldx4<__nv_bfloat16, false>(const __nv_bfloat16 *p)
{
    return bf16x4_to_float4(__ldg(reinterpret_cast<const uint2 *>(p)));
}
template <>
__device__ __forceinline__ float4 ldx4<__nv_bfloat16, true>(const __nv_bfloat16 *p)
{
    return bf16x4_to_float4(__ldcs(reinterpret_cast<const uint2 *>(p)));
}

// Rows of X can be read four elements at a time.
template <typename XT>
inline bool x_vec4(const XT *X, int64_t d, int64_t ld)
{
    return d % 4 == 0 && ld % 4 == 0 && (reinterpret_cast<uintptr_t>(X) % (4 * sizeof(XT))) == 0;
}

// Squared Euclidean distance between two samples in FP32, one accumulator,
// coordinates in ascending order: acc = fma(x_t - y_t, x_t - y_t, acc).
// Every exact pair distance of the graph (initial graph, refinement, rerank)
// uses this order, so that the distance of a pair is the same bits wherever it
// is computed and d(i, j) == d(j, i).
template <typename XT>
__device__ __forceinline__ float pair_d2_seq(const XT *__restrict__ a, const XT *__restrict__ b, int d)
{
    float acc = 0.f;
    for (int t = 0; t < d; t++) {
        float diff = ldx(a + t) - ldx(b + t);
        acc = fmaf(diff, diff, acc);
    }
    return acc;
}

// FP32 -> FP64 widening on the integer pipe (every binary32 value is a binary64 value: the fields are moved, a
// subnormal is normalised).  GB300's FP64 pipe is narrow, and the kernels that sum or fold in FP64 keep it busy.
__device__ __forceinline__ double widen(float x)
{
    const uint32_t u = __float_as_uint(x);
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    uint64_t bits;
    if (e == 0xFFu) {
        bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
    } else if (e != 0) {
        bits = sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)m << 29);
    } else if (m == 0) {
        bits = sign;
    } else {
        const int p = 31 - __clz(m);  // leading one of the subnormal's m * 2^-149
        bits = sign | ((uint64_t)(p + 874) << 52) | ((uint64_t)(m ^ (1u << p)) << (52 - p));
    }
    return __longlong_as_double((long long)bits);
}

// (distance, index) key order of graph rows: smaller distance first, then smaller id.
__device__ __forceinline__ bool key_less(float da, int ia, float db, int ib)
{
    return da < db || (da == db && ia < ib);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Named barriers (ids 1-15; 0 is __syncthreads): `count` threads, whole warps, complete a phase.  bar_sync
// waits for the phase, bar_arrive counts this warp and goes on.
__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned, L2 only),
// grouping of the copies issued so far, and waits on the groups.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void cp_async_wait_all()
{
    cp_async_commit();
    cp_async_wait<0>();
}

}  // namespace gkm

// ---- host-side launch helpers (internal) ---------------------------------
namespace gkm {

// Workspace carving: bump allocator over the caller's buffer.
struct Carver {
    char *base;
    size_t off;
    size_t cap;
    template <class T>
    T *take(size_t count)
    {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

// cudaFuncSetAttribute(kernel, MaxDynamicSharedMemorySize, bytes) on the current
// device, the first time only (thread-safe); `bytes` must be the same on every call.
cudaError_t set_max_smem(const void *kernel, int bytes);
// SMs x blocks of `kernel` resident on one SM (threads per block, dynamic shared memory smem): a grid that
// runs in one wave.  Computed once per device and kernel.
cudaError_t resident_grid(const void *kernel, int threads, size_t smem, int *grid);

// top-1 recall of a graph on sampled queries (recall.cu)
size_t recall_scratch_bytes(int64_t n, int32_t m);
cudaError_t launch_recall(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                          int32_t kappa, const int32_t *queries, int32_t m, int32_t *nn_idx, float *nn_dist,
                          int64_t *hits, void *scratch, DevStatus *st, cudaStream_t s);

// two-means tree, Alg. 1 (tree.cu): labels[n] in [0, k)
size_t tree_scratch_bytes(int64_t n, int64_t d, int32_t k);
cudaError_t launch_tree(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t k, int32_t iters,
                        uint64_t seed, int32_t *labels, void *scratch, DevStatus *st, cudaStream_t s);

// boost form, Eq. 2 state and the move step of Alg. 2 with Eq. 3 gains (boost.cu); d <= boost_max_d()
int64_t boost_max_d();
cudaError_t launch_boost_init(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *labels,
                              int32_t k, double *D, int32_t *counts, double *S, int32_t *offsets, int32_t *members,
                              int32_t *grp_counts, void *grp_scratch, DevStatus *st, cudaStream_t s);
cudaError_t launch_boost_epoch(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *G,
                               int32_t kappa, const int32_t *order, int64_t m, int32_t *labels, int32_t k, double *D,
                               int32_t *counts, double *S, int64_t *n_moved, DevStatus *st, cudaStream_t s);

// Internal launchers (each returns cudaError_t of the launch).  Those that read the samples take them as
// X (FP32, or BF16 when bf16 is set) with leading dimension ld in elements.
// (label_offset / id_offset are added to every label / neighbour id written: a job's numbering inside a batch)
cudaError_t launch_init_labels(int64_t n, int32_t k, uint64_t seed, int32_t *labels, cudaStream_t s,
                               int32_t label_offset = 0);
cudaError_t launch_init_graph(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, int32_t kappa,
                              uint64_t seed, int32_t *g_idx, float *g_dist, DevStatus *st, cudaStream_t s,
                              int32_t id_offset = 0);

// Grouping of samples by label (CSR).  Scratch sizes via group_scratch_bytes().
size_t group_scratch_bytes(int64_t n, int32_t k);
cudaError_t launch_group(const int32_t *labels, int64_t n, int32_t k, int32_t *offsets, int32_t *members,
                         int32_t *counts_out, void *scratch, DevStatus *st, cudaStream_t s);

// Exclusive scan of int32 counts (count elements) into out (count + 1 elements, out[count] = total).
size_t scan_scratch_bytes(int64_t count);
cudaError_t launch_scan(const int32_t *in, int32_t *out, int64_t count, void *scratch, cudaStream_t s);

size_t update_scratch_bytes(int64_t n, int32_t k);
// the per-cluster distortion terms the last launch_update left in its scratch (k doubles)
const double *update_contrib(const void *scratch);
// distortion of each job of a batch from those terms: the FP64 sum of its clusters' terms in the order of the
// update's own sum (one block per job, the same tree), divided by the job's samples (batch.cu)
struct BatchTable;
cudaError_t launch_batch_distortion(const double *contrib, const BatchTable &t, double *out, cudaStream_t s);
// labels of a batch back to each job's numbering: labels_out[i] = labels[i] - (first cluster of i's job)
cudaError_t launch_batch_labels(const int32_t *labels, int64_t N, const BatchTable &t, int32_t *labels_out,
                                cudaStream_t s);
cudaError_t launch_update(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, float *C, int32_t *counts, double *sum_d2,
                          void *scratch, DevStatus *st, cudaStream_t s);

size_t assign_scratch_bytes(int64_t n, int32_t k, int64_t d);
// precision 0 and 1: FP32 candidate rows; 2: BF16 screening on the SIMT cores; 3: on the tensor cores over
// 128-sample tiles when members, the grouping of labels_in, is given and d <= 128; 4: int8 screening (per-row
// scale) on the SIMT cores; all with the exact FP32 recompute (same results).  3 takes FP32 samples only.
// Bits 8-15 of precision: candidates per group of the row kernels (0: default, 4 or 8).
cudaError_t launch_assign(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *g_idx,
                          int32_t kappa, const float *C, int32_t k, const int32_t *labels_in, int32_t *labels_out,
                          float *best_d2, double *sum_d2, int64_t *n_changed, void *scratch, DevStatus *st,
                          cudaStream_t s, int precision, const int32_t *members);

void set_last_error(const char *msg);

size_t refine_scratch_bytes(int64_t n, int32_t k, int64_t d);
// precision 0: FP32 pair distances on the SIMT cores; 1: tensor-core Gram with exact FP32 rerank
cudaError_t launch_refine(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                          const int32_t *members, int32_t k, int32_t kappa, int32_t max_cluster, int32_t *g_idx,
                          float *g_dist, void *scratch, DevStatus *st, cudaStream_t s, int precision);
size_t refine_tc_scratch_bytes(int64_t n, int32_t k, int64_t d);
cudaError_t launch_refine_tc(const void *X, bool bf16, int64_t n, int64_t d, int64_t ld, const int32_t *offsets,
                             const int32_t *members, const int32_t *run_off, const int32_t *run_cl, int32_t k,
                             int32_t kappa, int32_t max_cluster, int64_t grid, int32_t *g_idx, float *g_dist,
                             void *scratch, DevStatus *st, cudaStream_t s);

}  // namespace gkm
