// Batches of independent clustering jobs (gk_batch_fit): the two kernels that
// turn the batch's results back into each job's own.
//
// k_batch_distortion: job j's distortion from the per-cluster terms of the
// last update, summed over its clusters with the thread mapping and tree of
// the update's own one-block sum (k_sum_f64), so that it equals the job's
// solo distortion bit for bit, then divided by its samples (Eq. 4).
// k_batch_labels: labels back to each job's numbering.
#include "batch.cuh"
#include "common.cuh"

namespace gkm {

__global__ void __launch_bounds__(1024) k_batch_distortion(const double *__restrict__ contrib, const BatchTable t,
                                                           double *__restrict__ out)
{
    __shared__ double s[1024];
    const int j = blockIdx.x;
    const int32_t a = t.kfirst[j], count = t.kfirst[j + 1] - a;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += 1024)
        v += contrib[a + i];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[j] = s[0] / (double)(t.first[j + 1] - t.first[j]);
}

__global__ void __launch_bounds__(256) k_batch_labels(const int32_t *__restrict__ labels, int64_t N, const BatchTable t,
                                                      int32_t *__restrict__ labels_out)
{
    __shared__ int64_t first[MAX_BATCH_JOBS + 1];
    __shared__ int32_t kfirst[MAX_BATCH_JOBS + 1];
    for (int j = threadIdx.x; j <= t.njobs; j += blockDim.x) {
        first[j] = t.first[j];
        kfirst[j] = t.kfirst[j];
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = t.njobs;  // the job j with first[j] <= i < first[j + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (first[mid] <= i)
                lo = mid;
            else
                hi = mid;
        }
        labels_out[i] = labels[i] - kfirst[lo];
    }
}

cudaError_t launch_batch_distortion(const double *contrib, const BatchTable &t, double *out, cudaStream_t s)
{
    k_batch_distortion<<<t.njobs, 1024, 0, s>>>(contrib, t, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_labels(const int32_t *labels, int64_t N, const BatchTable &t, int32_t *labels_out,
                                cudaStream_t s)
{
    int64_t blocks = (N + 255) / 256;
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    k_batch_labels<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(labels, N, t, labels_out);
    return cudaGetLastError();
}

}  // namespace gkm
