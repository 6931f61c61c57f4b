// Velocity set of the library.  Default: D3Q19 (Sec. "Entropic multi-relaxation lattice
// Boltzmann scheme": q = 19, c_s^2 = 1/3, weights 1/3, 1/18, 1/36).  Built with
// -DMCLBM_D3Q27: D3Q27 (all 27 vectors of {-1,0,1}^3, weights 8/27, 2/27, 1/54, 1/216).
//
// Storage order: rest, then opposite pairs (2k-1, 2k): faces +-x, +-y, +-z,
// then edges xy (++,--), (+-,-+), xz (++,--), (+-,-+), yz (++,--), (+-,-+),
// then (D3Q27) corners (+++,---), (++-,--+), (+-+,-+-), (+--,-++).
// opp(i) = i + 1 for odd i, i - 1 for even i > 0; the first non-zero component of an
// odd-numbered velocity is +1.
#pragma once
#include <cstdint>

namespace mclbm {

#ifdef MCLBM_D3Q27
constexpr int Q = 27;
#define MCLBM_LATTICE_NAME "D3Q27"
#else
constexpr int Q = 19;
#define MCLBM_LATTICE_NAME "D3Q19"
#endif

__host__ __device__ constexpr int cx(int i)
{
    constexpr int v[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return v[i];
}
__host__ __device__ constexpr int cy(int i)
{
    constexpr int v[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1, -1, 1};
    return v[i];
}
__host__ __device__ constexpr int cz(int i)
{
    constexpr int v[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr int norm2(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }

template <class T>
__host__ __device__ constexpr T weight(int i)
{
#ifdef MCLBM_D3Q27
    return norm2(i) == 0 ? T(8) / T(27)
                         : (norm2(i) == 1 ? T(2) / T(27) : (norm2(i) == 2 ? T(1) / T(54) : T(1) / T(216)));
#else
    return norm2(i) == 0 ? T(1) / T(3) : (norm2(i) == 1 ? T(1) / T(18) : T(1) / T(36));
#endif
}

// 1 / w_i (exact in binary floating point for both sets)
template <class T>
__host__ __device__ constexpr T inv_weight(int i)
{
#ifdef MCLBM_D3Q27
    return norm2(i) == 0 ? T(27) / T(8) : (norm2(i) == 1 ? T(13.5) : (norm2(i) == 2 ? T(54) : T(216)));
#else
    return norm2(i) == 0 ? T(3) : (norm2(i) == 1 ? T(18) : T(36));
#endif
}

}  // namespace mclbm
