// Sample convergence check of Eq. (sample_error): the ensemble-averaged relative L1 error
// between paired samples (the same parameters X_m) at two resolutions, on the common
// restriction grid.  One block per sample forms, in fixed order, the four numerators and
// denominators (components x, y, z with the absolute value, the vector with the Euclidean
// norm); one thread then averages the per-sample ratios over the samples.
#include <string>

#include "internal.h"

namespace mclbm {

namespace {

constexpr int kErrThreads = 256;

__global__ void __launch_bounds__(kErrThreads) k_sample_error(const double* __restrict__ u, const double* __restrict__ ref,
                                                              int G, double* __restrict__ ratio)
{
    __shared__ double sh[8][kErrThreads];
    const int m = blockIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < G; k += kErrThreads) {
        const double* a = u + ((int64_t)m * G + k) * 3;
        const double* b = ref + ((int64_t)m * G + k) * 3;
        double dd = 0, rr = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double d = a[c] - b[c];
            acc[c] += fabs(d);
            acc[4 + c] += fabs(b[c]);
            dd += d * d;
            rr += b[c] * b[c];
        }
        acc[3] += sqrt(dd);
        acc[7] += sqrt(rr);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = kErrThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) ratio[(int64_t)m * 4 + threadIdx.x] = sh[threadIdx.x][0] / sh[4 + threadIdx.x][0];
}

__global__ void k_sample_error_mean(const double* __restrict__ ratio, int M, double* __restrict__ out)
{
    if (threadIdx.x < 4) {
        double s = 0;
        for (int m = 0; m < M; ++m) s += ratio[(int64_t)m * 4 + threadIdx.x];
        out[threadIdx.x] = s / M;
    }
}

}  // namespace

}  // namespace mclbm

using namespace mclbm;

extern "C" {

size_t mclbm_sample_error_work_bytes(int32_t M) { return M < 1 ? 0 : ((size_t)4 * M + 4) * sizeof(double); }

int mclbm_sample_error(const double* d_u, const double* d_ref, int32_t M, int32_t G, void* d_work, size_t work_bytes,
                       void* cuda_stream, double* out)
{
    if (!d_u || !d_ref || !d_work || !out || M < 1 || G < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    if (work_bytes < mclbm_sample_error_work_bytes(M))
        return set_error(MCLBM_ERR_OOM, "work buffer needs " + std::to_string(mclbm_sample_error_work_bytes(M)) + " bytes");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* ratio = (double*)d_work;
    double* res = ratio + 4 * (size_t)M;
    k_sample_error<<<M, kErrThreads, 0, s>>>(d_u, d_ref, G, ratio);
    k_sample_error_mean<<<1, 32, 0, s>>>(ratio, M, res);
    MCLBM_CUDA(cudaGetLastError());
    MCLBM_CUDA(cudaMemcpyAsync(out, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MCLBM_CUDA(cudaStreamSynchronize(s));
    return MCLBM_OK;
}

}  // extern "C"
