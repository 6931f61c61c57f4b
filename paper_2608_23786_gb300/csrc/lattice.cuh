// D3Q19 velocity set of the library (Sec. "Entropic multi-relaxation lattice
// Boltzmann scheme": q = 19, c_s^2 = 1/3, weights 1/3, 1/18, 1/36).
//
// Storage order: rest, then opposite pairs (2k-1, 2k): faces +-x, +-y, +-z,
// then edges xy (++,--), (+-,-+), xz (++,--), (+-,-+), yz (++,--), (+-,-+).
// opp(i) = i + 1 for odd i, i - 1 for even i > 0.
#pragma once
#include <cstdint>

namespace mclbm {

constexpr int Q = 19;

__host__ __device__ constexpr int cx(int i)
{
    constexpr int v[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
}
__host__ __device__ constexpr int cy(int i)
{
    constexpr int v[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
}
__host__ __device__ constexpr int cz(int i)
{
    constexpr int v[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr int norm2(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }

template <class T>
__host__ __device__ constexpr T weight(int i)
{
    return norm2(i) == 0 ? T(1) / T(3) : (norm2(i) == 1 ? T(1) / T(18) : T(1) / T(36));
}

}  // namespace mclbm
