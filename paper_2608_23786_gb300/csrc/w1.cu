// One-point 1-Wasserstein distance W_{1,1} of Algorithm "WassersteinDistance1".
//
// For each of the G points and each velocity component, the two empirical laws
// (M_A and M_B equally weighted atoms) are compared by the L1 distance of their
// cumulative distribution functions (Eq. (wassersteinPermutations): for equal
// sizes this is the sorted-rearrangement cost (1/M) sum |a_(m) - b_(m)|).
// One block per (point, component): both samples are loaded into shared memory,
// padded with +inf to a power of two and bitonic-sorted; one thread then merges
// the two sorted lists, accumulating |F_A - F_B| times the gap to the next
// support point, in FP64.  A final fixed-order reduction gives
// W = (1/G) sum_points sum_components W1.
#include <cfloat>
#include <mutex>
#include <string>

#include "internal.h"

namespace mclbm {

namespace {

constexpr int kThreads = 256;

__device__ void bitonic_sort(double* v, int n)  // n a power of two, ascending
{
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const double a = v[i], b = v[ixj];
                    if ((a > b) == up) {
                        v[i] = b;
                        v[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_w1_points(const double* __restrict__ A, int MA, const double* __restrict__ B,
                                                        int MB, int G, int PA, int PB, double* __restrict__ per_point)
{
    extern __shared__ double sm[];
    double* a = sm;       // [PA]
    double* b = sm + PA;  // [PB]
    const int p = blockIdx.x, comp = blockIdx.y;
    for (int m = threadIdx.x; m < PA; m += blockDim.x) a[m] = m < MA ? A[((int64_t)m * G + p) * 3 + comp] : DBL_MAX;
    for (int m = threadIdx.x; m < PB; m += blockDim.x) b[m] = m < MB ? B[((int64_t)m * G + p) * 3 + comp] : DBL_MAX;
    __syncthreads();
    bitonic_sort(a, PA);
    bitonic_sort(b, PB);
    if (threadIdx.x == 0) {
        int i = 0, j = 0;
        double acc = 0.0;
        const double ia = 1.0 / MA, ib = 1.0 / MB;
        // consume the merged support in ascending order; after consuming value z the
        // CDFs are i/MA and j/MB on [z, next)
        while (i < MA || j < MB) {
            double z;
            if (j >= MB || (i < MA && a[i] <= b[j])) z = a[i++];
            else z = b[j++];
            if (i >= MA && j >= MB) break;
            const double next = (j >= MB || (i < MA && a[i] <= b[j])) ? a[i] : b[j];
            acc += fabs(i * ia - j * ib) * (next - z);
        }
        per_point[(int64_t)p * 3 + comp] = acc;
    }
}

__global__ void k_w1_total(const double* __restrict__ per_point, int G, double* __restrict__ out)
{
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < 3 * G; k += blockDim.x) s += per_point[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] / G;
}

int pow2_at_least(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

size_t w1_work_bytes(int MA, int MB, int G)
{
    (void)MA;
    (void)MB;
    return ((size_t)3 * G + 32) * sizeof(double);
}

cudaError_t launch_w1(const double* d_a, int MA, const double* d_b, int MB, int G, char* work, size_t work_bytes,
                      cudaStream_t s, double* h_W, double* h_per_point)
{
    if (work_bytes < w1_work_bytes(MA, MB, G)) return cudaErrorInvalidValue;
    double* per_point = (double*)work;
    double* total = per_point + 3 * G;
    const int PA = pow2_at_least(MA), PB = pow2_at_least(MB);
    const size_t smem = (size_t)(PA + PB) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_w1_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_w1_points<<<dim3(G, 3), kThreads, smem, s>>>(d_a, MA, d_b, MB, G, PA, PB, per_point);
    k_w1_total<<<1, kThreads, 0, s>>>(per_point, G, total);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(h_W, total, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if (h_per_point &&
        (e = cudaMemcpyAsync(h_per_point, per_point, sizeof(double) * 3 * G, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

// ---- W1 on restricted fields without caller-provided scratch ---------------------
// The call below uses, as its only scratch, a fixed array in the library's device
// image: per-point distances [G][3] and the total, for at most kNoAllocMaxPoints points.
// Every GPU that loads the library holds this array (about 96 KiB) until the process
// exits.  Every element the call reads from it is first written by the same call, so
// nothing needs clearing between calls; calls that overlap on the GPU (other streams,
// other host threads) share the array and race.

constexpr int kNoAllocMaxPoints = 4096;

static __device__ __align__(256) double g_w1_scratch[3 * kNoAllocMaxPoints + 32];

namespace {
std::mutex g_scratch_mu;
double* g_scratch_dev[kMaxDevices];  // device address of g_w1_scratch, per device

// Device address of the scratch array on the current device.  Looked up once per device
// (with that device current) on the first call made on it.
cudaError_t scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_w1_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = (double*)p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace mclbm

using namespace mclbm;

extern "C" int mclbm_w1_restricted_noalloc(const double* d_a, int32_t MA, const double* d_b, int32_t MB, int32_t G,
                                           void* cuda_stream, double* W, double* per_point)
{
    if (!d_a || !d_b || !W || G < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    if (G > kNoAllocMaxPoints)
        return set_error(MCLBM_ERR_SHAPE, "mclbm_w1_restricted_noalloc supports at most " +
                                              std::to_string(kNoAllocMaxPoints) + " points (G = " + std::to_string(G) +
                                              "); use mclbm_w1_restricted with a work buffer");
    if (MA < 1 || MB < 1 || MA > kMaxW1Samples || MB > kMaxW1Samples)
        return set_error(MCLBM_ERR_SHAPE, "W1 supports 1..2048 samples per ensemble");
    double* scratch = nullptr;
    MCLBM_CUDA(scratch_address(&scratch));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* pp = scratch;
    double* total = scratch + 3 * G;
    const int PA = pow2_at_least(MA), PB = pow2_at_least(MB);
    const size_t smem = (size_t)(PA + PB) * sizeof(double);  // <= 32 KiB: no opt-in needed
    k_w1_points<<<dim3(G, 3), kThreads, smem, s>>>(d_a, MA, d_b, MB, G, PA, PB, pp);
    k_w1_total<<<1, kThreads, 0, s>>>(pp, G, total);
    MCLBM_CUDA(cudaGetLastError());
    MCLBM_CUDA(cudaMemcpyAsync(W, total, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (per_point) MCLBM_CUDA(cudaMemcpyAsync(per_point, pp, sizeof(double) * 3 * G, cudaMemcpyDeviceToHost, s));
    MCLBM_CUDA(cudaStreamSynchronize(s));
    return MCLBM_OK;
}
