// Arithmetic throughput of the GPU the library runs on: long chains of independent fused
// multiply-adds (FP64, FP32, packed FP32x2, packed half2) or reciprocal approximations (the
// MUFU unit) on every SM, timed with CUDA events.  These are the ceilings that the kernels
// bound by arithmetic rather than by memory (the plain FP64 stepper, the FP64 reductions, the
// FP16-storage collision) are set against.
#include <cuda_fp16.h>

#include "internal.h"

namespace mclbm {
namespace {

constexpr int kChains = 8;         // independent dependency chains per thread
constexpr int kPeakThreads = 256;  // threads per block
constexpr int kPeakBlocksPerSM = 8;

__device__ __forceinline__ double op(double x) { return fma(x, 0.9999999999, 1e-9); }
__device__ __forceinline__ float op(float x)
{
    float d;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(x), "f"(0.9999999f), "f"(1e-7f));
    return d;
}
struct Packed {
    float2 v;
};
__device__ __forceinline__ Packed op(Packed x)
{
    Packed d;
    asm volatile(
        "{\n\t.reg .b64 pa, pb, pc, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %4};\n\t"
        "mov.b64 pc, {%5, %5};\n\tfma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.v.x), "=f"(d.v.y)
        : "f"(x.v.x), "f"(x.v.y), "f"(0.9999999f), "f"(1e-7f));
    return d;
}
__device__ __forceinline__ __half2 op(__half2 x) { return __hfma2(x, __float2half2_rn(0.999f), __float2half2_rn(1e-3f)); }
struct Recip {
    float v;
};
// x <- 1 / (x + 1): an add and a reciprocal per step (consecutive reciprocals alone would
// cancel in pairs); the chain converges to 0.618.., and the reciprocal unit (a quarter of the
// FP32 lanes) bounds its rate.
__device__ __forceinline__ Recip op(Recip x)
{
    Recip d;
    asm volatile("{\n\t.reg .f32 t;\n\tadd.rn.f32 t, %1, 0f3F800000;\n\trcp.approx.ftz.f32 %0, t;\n\t}"
                 : "=f"(d.v)
                 : "f"(x.v));
    return d;
}

template <class T>
__device__ __forceinline__ T seed(int k);
template <>
__device__ __forceinline__ double seed<double>(int k) { return 1.0 + 1e-3 * (threadIdx.x + k); }
template <>
__device__ __forceinline__ float seed<float>(int k) { return 1.f + 1e-3f * (threadIdx.x + k); }
template <>
__device__ __forceinline__ Packed seed<Packed>(int k) { return Packed{make_float2(1.f + 1e-3f * k, 1.f + 1e-3f * threadIdx.x)}; }
template <>
__device__ __forceinline__ __half2 seed<__half2>(int k) { return __float2half2_rn(1.f + 1e-2f * k); }
template <>
__device__ __forceinline__ Recip seed<Recip>(int k) { return Recip{1.f + 1e-3f * (threadIdx.x + k)}; }

__device__ __forceinline__ double value(double x) { return x; }
__device__ __forceinline__ double value(float x) { return x; }
__device__ __forceinline__ double value(Packed x) { return x.v.x + x.v.y; }
__device__ __forceinline__ double value(__half2 x) { return __low2float(x) + __high2float(x); }
__device__ __forceinline__ double value(Recip x) { return x.v; }

template <class T>
__global__ void __launch_bounds__(kPeakThreads) k_alu_rate(double* sink, int iters)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = seed<T>(k);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = op(x[k]);
        }
    }
    double acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += value(x[k]);
    if (acc == -1.0) sink[0] = acc;  // never true for these chains; keeps them live
}

template <class T>
cudaError_t time_rate(double* sink, int iters, cudaStream_t s, int grid, float* ms)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    k_alu_rate<T><<<grid, kPeakThreads, 0, s>>>(sink, iters);  // warm-up
    cudaEventRecord(a, s);
    k_alu_rate<T><<<grid, kPeakThreads, 0, s>>>(sink, iters);
    cudaEventRecord(b, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

}  // namespace
}  // namespace mclbm

using namespace mclbm;

extern "C" int mclbm_alu_rate(int32_t kind, int32_t iters, double* d_sink, void* cuda_stream, double* results_per_s,
                              double* ms_out)
{
    if (!d_sink || !results_per_s || iters < 1 || kind < 0 || kind > 4)
        return set_error(MCLBM_ERR_INVALID_ARG, "mclbm_alu_rate: kind 0..4, iters >= 1, d_sink and results_per_s");
    int dev = 0, sms = 0;
    MCLBM_CUDA(cudaGetDevice(&dev));
    MCLBM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * kPeakBlocksPerSM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float ms = 0;
    cudaError_t e;
    switch (kind) {
        case 0: e = time_rate<double>(d_sink, iters, s, grid, &ms); break;
        case 1: e = time_rate<float>(d_sink, iters, s, grid, &ms); break;
        case 2: e = time_rate<Packed>(d_sink, iters, s, grid, &ms); break;
        case 3: e = time_rate<__half2>(d_sink, iters, s, grid, &ms); break;
        default: e = time_rate<Recip>(d_sink, iters, s, grid, &ms); break;
    }
    MCLBM_CUDA(e);
    const double lanes = (kind == 2 || kind == 3) ? 2.0 : 1.0;  // results per thread and operation
    const double results = (double)grid * kPeakThreads * kChains * 16.0 * iters * lanes;
    *results_per_s = results / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return MCLBM_OK;
}
