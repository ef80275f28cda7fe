// gk_update_step_noalloc: the centroid update of gk_update_step for callers
// that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a host application whose framework
// owns every byte of device memory through its own pool (a raw allocation
// would bypass its accounting and fragment it), or a latency-bound serving
// loop where cudaMalloc / cudaFree can synchronise the whole device and stall
// other work.  Such callers cannot hand this library a workspace either, so
// this entry point takes its scratch from one fixed array that lives in the
// library's own device image (a file-scope __device__ array): it exists on
// every GPU that loads the library, from load until process exit, and no call
// allocates anything.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "common.cuh"

using namespace gkm;

namespace {

// Stated limits of the fixed scratch: n <= 2^20 samples, k <= 2^15 clusters.
constexpr int64_t NOALLOC_MAX_N = int64_t(1) << 20;
constexpr int32_t NOALLOC_MAX_K = int32_t(1) << 15;
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(24) << 20;  // 24 MiB, enough for the limits above

constexpr int MAX_DEVICES = 64;

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

struct DeviceScratch {
    std::once_flag once;
    void *ptr = nullptr;
    cudaError_t err = cudaSuccess;
};

DeviceScratch g_dev[MAX_DEVICES];

// Device address of the scratch on the current device, looked up once per
// device (the first call on each device does the look-up).
cudaError_t scratch_ptr(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= MAX_DEVICES)
        return cudaErrorInvalidDevice;
    DeviceScratch &s = g_dev[dev];
    std::call_once(s.once, [&] { s.err = cudaGetSymbolAddress(&s.ptr, g_noalloc_scratch); });
    if (s.err != cudaSuccess)
        return s.err;
    *out = s.ptr;
    return cudaSuccess;
}

}  // namespace

static int report(int code, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

extern "C" GK_API int gk_update_step_noalloc(const float *X, int64_t n, int64_t d, int64_t ld,
                                             const int32_t *labels, int32_t k, float *C, int32_t *counts,
                                             double *sum_d2, void *stream)
{
    // argument checks (same rules as gk_update_step) plus the fixed limits
    if (!X || !labels || !C) {
        return report(GK_ERR_INVALID, "a required array is NULL");
    }
    if (n < 1 || n > NOALLOC_MAX_N || k < 1 || k > NOALLOC_MAX_K) {
        return report(GK_ERR_INVALID,
                      "gk_update_step_noalloc: n = %lld, k = %d beyond its fixed scratch (n <= %lld, k <= %d); "
                      "use gk_update_step with a workspace",
                      (long long)n, k, (long long)NOALLOC_MAX_N, NOALLOC_MAX_K);
    }
    if (d < 1 || d > 4096 || ld < d || (reinterpret_cast<uintptr_t>(X) & 3) != 0) {
        return report(GK_ERR_INVALID, "bad shape: d = %lld, ld = %lld", (long long)d, (long long)ld);
    }
    // layout of the fixed scratch, as gk_update_step lays out its workspace
    Carver probe{nullptr, 0, 0};
    probe.take<DevStatus>(1);
    probe.take<int32_t>((size_t)k + 1);
    probe.take<int32_t>((size_t)n);
    probe.take<int32_t>((size_t)k);
    probe.take<char>(group_scratch_bytes(n, k));
    probe.take<char>(update_scratch_bytes(n, k));
    if (probe.off > NOALLOC_SCRATCH_BYTES) {
        return report(GK_ERR_INVALID, "gk_update_step_noalloc: needs %zu bytes of scratch, has %zu", probe.off,
                      NOALLOC_SCRATCH_BYTES);
    }
    void *base = nullptr;
    cudaError_t e = scratch_ptr(&base);
    if (e != cudaSuccess) {
        return report(GK_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    }
    Carver cv{static_cast<char *>(base), 0, 0};
    DevStatus *st = cv.take<DevStatus>(1);
    int32_t *off = cv.take<int32_t>((size_t)k + 1);
    int32_t *mem = cv.take<int32_t>((size_t)n);
    int32_t *cnt_tmp = cv.take<int32_t>((size_t)k);
    void *gscratch = cv.take<char>(group_scratch_bytes(n, k));
    void *uscratch = cv.take<char>(update_scratch_bytes(n, k));
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *cnt = counts ? counts : cnt_tmp;
    // the status word keeps the previous call's value: clear it (the grouping
    // zeroes its own counters; everything else is overwritten before it is read)
    if ((e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s)) == cudaSuccess &&
        (e = launch_group(labels, n, k, off, mem, cnt, gscratch, st, s)) == cudaSuccess)
        e = launch_update(X, false, n, d, ld, off, mem, k, C, cnt, sum_d2, uscratch, st, s);
    if (e != cudaSuccess) {
        return report(GK_ERR_CUDA, "launch failed: %s", cudaGetErrorString(e));
    }
    return GK_OK;
}
