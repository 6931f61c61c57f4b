// Population storage and addressing.
//
// Layout of one lattice in HBM: [sample][i][z][y][x] (structure of arrays, x
// fastest), i in the library order of lattice.cuh.  Three element types:
//   double - raw f_i                      (MCLBM_FP64, FP64 arithmetic)
//   float  - h_i = f_i / w_i - 1          (MCLBM_FP32, FP32 arithmetic)
//   __half - h_i rounded to nearest       (MCLBM_FP16, FP32 arithmetic)
//
// Where the pre-collision population f_i(x, t) lives ("pre-collision location"):
//   pull pattern:           slot i of node x - c_i of the current lattice
//                           (the lattice holds the post-collision state of t-1);
//   AA pattern, t even:     slot i of node x;
//   AA pattern, t odd:      slot opp(i) of node x - c_i.
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "lattice.cuh"

namespace mclbm {

template <class E>
struct Storage;

template <>
struct Storage<double> {
    using compute = double;
    static constexpr bool shifted = false;
    __device__ __forceinline__ static double load(const double* p) { return __ldg(p); }
    __device__ __forceinline__ static void store(double* p, double v) { *p = v; }
};
template <>
struct Storage<float> {
    using compute = float;
    static constexpr bool shifted = true;
    __device__ __forceinline__ static float load(const float* p) { return __ldg(p); }
    __device__ __forceinline__ static void store(float* p, float v) { *p = v; }
};
template <>
struct Storage<__half> {
    using compute = float;
    static constexpr bool shifted = true;
    __device__ __forceinline__ static float load(const __half* p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static void store(__half* p, float v) { *p = __float2half_rn(v); }
};

// Lattice geometry of one level (N a power of two).
struct Geom {
    int N, logN;
    int64_t n;  // N^3
    __host__ __device__ __forceinline__ int wrap(int a) const { return a & (N - 1); }
    __host__ __device__ __forceinline__ int64_t node(int x, int y, int z) const
    {
        return ((int64_t)z << (2 * logN)) | ((int64_t)y << logN) | (int64_t)x;
    }
};

enum Pattern { kPull = 0, kAA = 1 };

// Element offset (within one sample) of the pre-collision f_i(x, y, z).
__device__ __forceinline__ int64_t pre_loc(const Geom& g, int pattern, int parity, int i, int x, int y, int z)
{
    if (pattern == kAA && parity == 0) return (int64_t)i * g.n + g.node(x, y, z);
    const int slot = (pattern == kAA) ? opp(i) : i;
    return (int64_t)slot * g.n + g.node(g.wrap(x - cx(i)), g.wrap(y - cy(i)), g.wrap(z - cz(i)));
}

// Convert a stored value to the raw population f_i (FP64).
template <class E>
__device__ __forceinline__ double to_raw(int i, E v);
template <>
__device__ __forceinline__ double to_raw<double>(int, double v) { return v; }
template <>
__device__ __forceinline__ double to_raw<float>(int i, float v) { return weight<double>(i) * (1.0 + (double)v); }
template <>
__device__ __forceinline__ double to_raw<__half>(int i, __half v)
{
    return weight<double>(i) * (1.0 + (double)__half2float(v));
}

// Store a raw population f_i (FP64) in the element type.
template <class E>
__device__ __forceinline__ void store_raw(E* p, int i, double f);
template <>
__device__ __forceinline__ void store_raw<double>(double* p, int, double f) { *p = f; }
template <>
__device__ __forceinline__ void store_raw<float>(float* p, int i, double f)
{
    *p = (float)(f / weight<double>(i) - 1.0);
}
template <>
__device__ __forceinline__ void store_raw<__half>(__half* p, int i, double f)
{
    *p = __double2half(f / weight<double>(i) - 1.0);
}

}  // namespace mclbm
