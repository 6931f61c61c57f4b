// Macroscopic fields and ensemble reductions read from the population lattice:
// moments, kinetic energy / enstrophy, ensemble mean and variance (with the energies in
// the same pass when asked), restriction to the common Q^3 grid, and the finiteness scan.
//
// All sums use a fixed assignment of nodes to threads and a fixed reduction tree,
// so results are bitwise reproducible from run to run (no floating-point atomics).
#include <cuda_fp16.h>

#include "internal.h"
#include "storage.cuh"

namespace mclbm {

namespace {

constexpr int kBlock = 256;
constexpr int kEnergyChunks = 64;  // blocks per sample in the energy reduction

// rho and u (lattice units) of the pre-collision state at one node, in type C.
// Shifted storage: rho = 1 + sum w h, rho u = sum w c h.
template <class E, class C>
__device__ __forceinline__ void node_moments(const E* base, const Geom& g, int pattern, int parity, int x, int y, int z,
                                             C& rho, C& ux, C& uy, C& uz)
{
    C r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        C v;
        if constexpr (Storage<E>::shifted)
            v = weight<C>(i) * (C)Storage<E>::load(base + pre_loc(g, pattern, parity, i, x, y, z));
        else
            v = (C)Storage<E>::load(base + pre_loc(g, pattern, parity, i, x, y, z));
        r += v;
        if (cx(i) > 0) jx += v; else if (cx(i) < 0) jx -= v;
        if (cy(i) > 0) jy += v; else if (cy(i) < 0) jy -= v;
        if (cz(i) > 0) jz += v; else if (cz(i) < 0) jz -= v;
    }
    if constexpr (Storage<E>::shifted) r += C(1);
    rho = r;
    ux = jx / r;
    uy = jy / r;
    uz = jz / r;
}

__device__ __forceinline__ void xyz_of(const Geom& g, int64_t node, int& x, int& y, int& z)
{
    x = (int)(node & (g.N - 1));
    y = (int)((node >> g.logN) & (g.N - 1));
    z = (int)(node >> (2 * g.logN));
}

// block-wide sum of a double; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

template <class E>
__global__ void __launch_bounds__(kBlock) k_moments(const E* __restrict__ lat, Geom g, int pattern, int parity, int sample,
                                                    double uscale, double* __restrict__ rho_out, double* __restrict__ u_out)
{
    const E* base = lat + (int64_t)sample * Q * g.n;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n; node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        xyz_of(g, node, x, y, z);
        typename Storage<E>::compute r, ux, uy, uz;  // FP32 arithmetic for FP32/FP16 storage, as the stepper's
        node_moments<E, typename Storage<E>::compute>(base, g, pattern, parity, x, y, z, r, ux, uy, uz);
        if (rho_out) rho_out[node] = (double)r;
        u_out[node] = (double)ux * uscale;
        u_out[g.n + node] = (double)uy * uscale;
        u_out[2 * g.n + node] = (double)uz * uscale;
    }
}

// Per-sample partial sums of |u_phys|^2 / 2; grid (kEnergyChunks, M).
template <class E>
__global__ void __launch_bounds__(kBlock) k_energy_partial(const E* __restrict__ lat, Geom g, int pattern, int parity,
                                                           double uscale, double* __restrict__ partial)
{
    using C = typename Storage<E>::compute;
    __shared__ double sh[32];
    const int m = blockIdx.y;
    const E* base = lat + (int64_t)m * Q * g.n;
    double acc = 0.0;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n; node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        xyz_of(g, node, x, y, z);
        C r, ux, uy, uz;
        node_moments<E, C>(base, g, pattern, parity, x, y, z, r, ux, uy, uz);
        const double vx = (double)ux * uscale, vy = (double)uy * uscale, vz = (double)uz * uscale;
        acc += 0.5 * (vx * vx + vy * vy + vz * vz);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(int64_t)m * gridDim.x + blockIdx.x] = acc;
}

// Kinetic energy and enstrophy partials of one sample from its velocity field.
__global__ void __launch_bounds__(kBlock) k_energy_enstrophy_field(const double* __restrict__ u, Geom g, double inv2dx,
                                                                   double* __restrict__ partial)
{
    __shared__ double sh[32];
    const double* ux = u;
    const double* uy = u + g.n;
    const double* uz = u + 2 * g.n;
    double e = 0.0, zz = 0.0;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n; node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        xyz_of(g, node, x, y, z);
        const double vx = ux[node], vy = uy[node], vz = uz[node];
        e += 0.5 * (vx * vx + vy * vy + vz * vz);
        const int64_t xp = g.node(g.wrap(x + 1), y, z), xm = g.node(g.wrap(x - 1), y, z);
        const int64_t yp = g.node(x, g.wrap(y + 1), z), ym = g.node(x, g.wrap(y - 1), z);
        const int64_t zp = g.node(x, y, g.wrap(z + 1)), zm = g.node(x, y, g.wrap(z - 1));
        const double wx = (uz[yp] - uz[ym]) * inv2dx - (uy[zp] - uy[zm]) * inv2dx;
        const double wy = (ux[zp] - ux[zm]) * inv2dx - (uz[xp] - uz[xm]) * inv2dx;
        const double wz = (uy[xp] - uy[xm]) * inv2dx - (ux[yp] - ux[ym]) * inv2dx;
        zz += 0.5 * (wx * wx + wy * wy + wz * wz);
    }
    e = block_sum(e, sh);
    if (threadIdx.x == 0) partial[2 * blockIdx.x] = e;
    zz = block_sum(zz, sh);
    if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = zz;
}

// out[k] = scale * sum_j partial[k * count * stride + j * stride + offset], fixed order.
__global__ void k_reduce_rows(const double* __restrict__ partial, int rows, int count, int stride, int offset, double scale,
                              double* __restrict__ out)
{
    __shared__ double sh[32];
    const int k = blockIdx.x;
    if (k >= rows) return;
    double acc = 0.0;
    for (int j = threadIdx.x; j < count; j += blockDim.x) acc += partial[((int64_t)k * count + j) * stride + offset];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[k] = acc * scale;
}

// ---- one pass over the ensemble: mean and unbiased variance fields, optionally E_m(t) ----
// Thread t takes the run of kRunVec nodes x0 = kRunVec t .. of one row and walks the samples.
// Its pre-collision populations are gathered with six row offsets per run (rows y - 1..y + 1,
// planes z - 1..z + 1); MODE 0 pull (slot i of x - c_i), 1 AA even (slot i of x), 2 AA odd
// (slot opp(i) of x - c_i).  The moments are formed in the storage's compute type, as the
// stepper's.  Per node the sums of d_m = u_m - u_0 and d_m^2 (m >= 1) are accumulated in FP64
// (one-pass variance about the first sample: mean = u_0 + S1 / M, var = (S2 - S1^2 / M) / (M - 1),
// free of the cancellation of raw sums because d is of the size of the spread), from partial sums
// over chunks of kSampleChunk samples in the compute type.  WANT_E: each sample's sum of |u|^2
// over the run is reduced across the warp in the compute type and accumulated per warp in FP64 in
// shared memory, then per block in a fixed order: partial[m][block].  For FP32 and FP16 storage,
// whose velocity carries FP32 rounding at best, the FP32 partial sums (at most 8 samples, or a
// warp's 64 squares: within 5e-7 relative for the positive terms) leave about one FP64
// operation per node and sample, and the pass runs at memory speed rather than at the rate of
// GB300's FP64 units.
constexpr int kRunVec = 2;
constexpr int kSampleChunk = 8;

template <class E, int MODE>
__device__ __forceinline__ void gather_run(const E* base, const Geom& g, int x0, int y, int z,
                                           typename Storage<E>::compute (&f)[Q][kRunVec])
{
    using C = typename Storage<E>::compute;
    uint32_t yo[3], zo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        yo[k] = (uint32_t)g.wrap(y + k - 1) << g.logN;
        zo[k] = (uint32_t)g.wrap(z + k - 1) << (2 * g.logN);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int slot = MODE == 2 ? opp(i) : i;
        const int dx = MODE == 1 ? 0 : -cx(i), dy = MODE == 1 ? 0 : -cy(i), dz = MODE == 1 ? 0 : -cz(i);
        const E* row = base + ((uint64_t)(uint32_t)slot * (uint32_t)g.n + (uint64_t)(zo[1 + dz] + yo[1 + dy]));
#pragma unroll
        for (int k = 0; k < kRunVec; ++k) f[i][k] = (C)Storage<E>::load(row + ((x0 + k + dx) & (g.N - 1)));
    }
}

template <class E, int MODE, bool WANT_E>
__global__ void __launch_bounds__(kBlock) k_stats_pass(const E* __restrict__ lat, Geom g, int M, double uscale,
                                                       double* __restrict__ mean, double* __restrict__ var,
                                                       double* __restrict__ epart)
{
    using C = typename Storage<E>::compute;
    extern __shared__ double ered[];  // WANT_E: [M][warps of the block]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if constexpr (WANT_E) {
        for (int k = threadIdx.x; k < M * nw; k += blockDim.x) ered[k] = 0.0;
        __syncthreads();
    }
    const int64_t runs = g.n / kRunVec;
    const double invM = 1.0 / M;
    const double vscale = M > 1 ? uscale * uscale / (M - 1) : 0.0;  // var = (S2 - S1^2 / M) uscale^2 / (M - 1)
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < runs; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = t * kRunVec;
        int x0, y, z;
        xyz_of(g, node, x0, y, z);
        C u0[3][kRunVec], p1[3][kRunVec], p2[3][kRunVec];
        double s1[3][kRunVec], s2[3][kRunVec];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < kRunVec; ++k) {
                s1[a][k] = s2[a][k] = 0.0;
                p1[a][k] = p2[a][k] = C(0);
            }
        for (int m = 0; m < M; ++m) {
            C f[Q][kRunVec];
            gather_run<E, MODE>(lat + (int64_t)m * Q * g.n, g, x0, y, z, f);
            C e = C(0);
#pragma unroll
            for (int k = 0; k < kRunVec; ++k) {
                C r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const C v = Storage<E>::shifted ? weight<C>(i) * f[i][k] : f[i][k];
                    r += v;
                    if (cx(i) > 0) jx += v; else if (cx(i) < 0) jx -= v;
                    if (cy(i) > 0) jy += v; else if (cy(i) < 0) jy -= v;
                    if (cz(i) > 0) jz += v; else if (cz(i) < 0) jz -= v;
                }
                if (Storage<E>::shifted) r += C(1);
                const C ri = C(1) / r;
                const C u[3] = {jx * ri, jy * ri, jz * ri};
                if constexpr (WANT_E) e += u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (m == 0) {
                        u0[a][k] = u[a];
                    } else if constexpr (std::is_same<C, double>::value) {  // FP64 storage: directly
                        const double d = u[a] - u0[a][k];
                        s1[a][k] += d;
                        s2[a][k] = fma(d, d, s2[a][k]);
                    } else {
                        const C d = u[a] - u0[a][k];
                        p1[a][k] += d;
                        p2[a][k] = fma(d, d, p2[a][k]);
                    }
                }
            }
            // the chunk's partial sums into the FP64 ones (after samples 8, 16, ... and the last)
            if (!std::is_same<C, double>::value && m > 0 && (m % kSampleChunk == 0 || m == M - 1)) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int k = 0; k < kRunVec; ++k) {
                        s1[a][k] += (double)p1[a][k];
                        s2[a][k] += (double)p2[a][k];
                        p1[a][k] = p2[a][k] = C(0);
                    }
            }
            if constexpr (WANT_E) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
                if (lane == 0) ered[m * nw + warp] += (double)e;
            }
        }
#pragma unroll
        for (int k = 0; k < kRunVec; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                mean[a * g.n + node + k] = fma(s1[a][k], invM, (double)u0[a][k]) * uscale;
                var[a * g.n + node + k] = fma(-s1[a][k] * invM, s1[a][k], s2[a][k]) * vscale;
            }
    }
    if constexpr (WANT_E) {
        __syncthreads();
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < nw; ++w) acc += ered[m * nw + w];
            epart[(int64_t)m * gridDim.x + blockIdx.x] = 0.5 * uscale * uscale * acc;
        }
    }
}

// Restriction of the physical velocity to the Q^3 nodes n = j N / Q: out [M][Q^3][3].
template <class E>
__global__ void k_restrict(const E* __restrict__ lat, Geom g, int M, int Qd, int pattern, int parity, double uscale,
                           double* __restrict__ out)
{
    const int G = Qd * Qd * Qd;
    const int s = g.N / Qd;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)M * G; t += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(t / G), p = (int)(t % G);
        const int jx = p % Qd, jy = (p / Qd) % Qd, jz = p / (Qd * Qd);
        double r, ux, uy, uz;
        node_moments<E, double>(lat + (int64_t)m * Q * g.n, g, pattern, parity, jx * s, jy * s, jz * s, r, ux, uy, uz);
        out[t * 3 + 0] = ux * uscale;
        out[t * 3 + 1] = uy * uscale;
        out[t * 3 + 2] = uz * uscale;
    }
}

template <class E>
__global__ void k_check_finite(const E* __restrict__ lat, int64_t count, int* __restrict__ flag)
{
    int bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if constexpr (sizeof(E) == 2)
            v = (double)__half2float(lat[k]);
        else
            v = (double)lat[k];
        if (!isfinite(v)) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

int grid_for(int64_t total, int cap = 152 * 16)
{
    int64_t b = (total + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    return (int)(b > cap ? cap : b);
}

Geom geom_of(const mclbm_ctx* c) { return Geom{c->N, c->logN, c->n}; }
double uscale_of(const mclbm_ctx* c) { return c->cfg.U_c / c->units.U_lat; }
int parity_of(const mclbm_ctx* c) { return c->cfg.pattern == MCLBM_AA ? (int)(c->steps & 1) : 0; }

template <class E>
cudaError_t moments_t(const mclbm_ctx* c, int sample, double* d_rho, double* d_u)
{
    k_moments<E><<<grid_for(c->n), kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur), geom_of(c), c->cfg.pattern,
                                                           parity_of(c), sample, uscale_of(c), d_rho, d_u);
    return cudaGetLastError();
}

template <class E>
cudaError_t energy_t(mclbm_ctx* c, bool with_z, double* h_E, double* h_Z)
{
    double* partial = (double*)(c->work + c->wl.partial);
    double* res = (double*)(c->work + c->wl.bins);  // [2][M]
    const double invn = 1.0 / (double)c->n;
    if (!with_z) {
        dim3 grid(kEnergyChunks, c->M);
        k_energy_partial<E><<<grid, kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur), geom_of(c), c->cfg.pattern,
                                                            parity_of(c), uscale_of(c), partial);
        k_reduce_rows<<<c->M, kBlock, 0, c->stream>>>(partial, c->M, kEnergyChunks, 1, 0, invn, res);
    } else {
        double* field = (double*)(c->work + c->wl.field);
        const double inv2dx = 1.0 / (2.0 * c->units.dx);
        const int nb = grid_for(c->n, 1024);
        for (int m = 0; m < c->M; ++m) {
            k_moments<E><<<grid_for(c->n), kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur), geom_of(c),
                                                                   c->cfg.pattern, parity_of(c), m, uscale_of(c), nullptr,
                                                                   field);
            k_energy_enstrophy_field<<<nb, kBlock, 0, c->stream>>>(field, geom_of(c), inv2dx, partial + (int64_t)m * 2 * nb);
        }
        k_reduce_rows<<<c->M, kBlock, 0, c->stream>>>(partial, c->M, nb, 2, 0, invn, res);
        k_reduce_rows<<<c->M, kBlock, 0, c->stream>>>(partial, c->M, nb, 2, 1, invn, res + c->M);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(h_E, res, sizeof(double) * c->M, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    if (with_z) {
        e = cudaMemcpyAsync(h_Z, res + c->M, sizeof(double) * c->M, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(c->stream);
}

constexpr int kStatsBlocks = 152 * 6;  // persistent grid of the statistics pass (fixed: deterministic sums)

template <class E>
cudaError_t stats_pass_t(const mclbm_ctx* c, double* d_mean, double* d_var, double* h_E)
{
    const Geom g = geom_of(c);
    const E* lat = (const E*)lattice_ptr(c, c->cur);
    const int mode = c->cfg.pattern == MCLBM_PULL ? 0 : (parity_of(c) == 0 ? 1 : 2);
    int64_t blocks = (g.n / kRunVec + kBlock - 1) / kBlock;
    if (blocks > kStatsBlocks) blocks = kStatsBlocks;
    const double us = uscale_of(c);
    if (!h_E) {
        if (mode == 0) k_stats_pass<E, 0, false><<<(int)blocks, kBlock, 0, c->stream>>>(lat, g, c->M, us, d_mean, d_var, nullptr);
        else if (mode == 1) k_stats_pass<E, 1, false><<<(int)blocks, kBlock, 0, c->stream>>>(lat, g, c->M, us, d_mean, d_var, nullptr);
        else k_stats_pass<E, 2, false><<<(int)blocks, kBlock, 0, c->stream>>>(lat, g, c->M, us, d_mean, d_var, nullptr);
        return cudaGetLastError();
    }
    double* partial = (double*)(c->work + c->wl.partial);
    double* res = (double*)(c->work + c->wl.bins);
    const size_t smem = (size_t)c->M * (kBlock / 32) * sizeof(double);
    cudaError_t e;
    if (mode == 0) {
        if ((e = cudaFuncSetAttribute(k_stats_pass<E, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_stats_pass<E, 0, true><<<(int)blocks, kBlock, smem, c->stream>>>(lat, g, c->M, us, d_mean, d_var, partial);
    } else if (mode == 1) {
        if ((e = cudaFuncSetAttribute(k_stats_pass<E, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_stats_pass<E, 1, true><<<(int)blocks, kBlock, smem, c->stream>>>(lat, g, c->M, us, d_mean, d_var, partial);
    } else {
        if ((e = cudaFuncSetAttribute(k_stats_pass<E, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_stats_pass<E, 2, true><<<(int)blocks, kBlock, smem, c->stream>>>(lat, g, c->M, us, d_mean, d_var, partial);
    }
    k_reduce_rows<<<c->M, kBlock, 0, c->stream>>>(partial, c->M, (int)blocks, 1, 0, 1.0 / (double)c->n, res);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(h_E, res, sizeof(double) * c->M, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

template <class E>
cudaError_t mean_var_t(const mclbm_ctx* c, double* d_mean, double* d_var)
{
    return stats_pass_t<E>(c, d_mean, d_var, nullptr);
}

template <class E>
cudaError_t restrict_t(const mclbm_ctx* c, int Qd, double* d_out)
{
    k_restrict<E><<<grid_for((int64_t)c->M * Qd * Qd * Qd), kBlock, 0, c->stream>>>(
        (const E*)lattice_ptr(c, c->cur), geom_of(c), c->M, Qd, c->cfg.pattern, parity_of(c), uscale_of(c), d_out);
    return cudaGetLastError();
}

template <class E>
cudaError_t finite_t(mclbm_ctx* c, int* h_bad)
{
    int* flag = (int*)(c->work + c->wl.flag);
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    const int64_t count = (int64_t)c->M * Q * c->n;
    k_check_finite<E><<<grid_for(count), kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur), count, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(h_bad, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

}  // namespace

#define MCLBM_DISPATCH(c, fn, ...)                       \
    switch ((c)->cfg.precision) {                        \
        case MCLBM_FP64: return fn<double>(__VA_ARGS__); \
        case MCLBM_FP32: return fn<float>(__VA_ARGS__);  \
        default: return fn<__half>(__VA_ARGS__);         \
    }

cudaError_t launch_moments(const mclbm_ctx* c, int sample, double* d_rho, double* d_u)
{
    MCLBM_DISPATCH(c, moments_t, c, sample, d_rho, d_u);
}
cudaError_t launch_energy(mclbm_ctx* c, bool with_z, double* h_E, double* h_Z)
{
    MCLBM_DISPATCH(c, energy_t, c, with_z, h_E, h_Z);
}
cudaError_t launch_energy_mean_var(const mclbm_ctx* c, double* h_E, double* d_mean, double* d_var)
{
    MCLBM_DISPATCH(c, stats_pass_t, c, d_mean, d_var, h_E);
}

cudaError_t launch_mean_var(const mclbm_ctx* c, double* d_mean, double* d_var)
{
    MCLBM_DISPATCH(c, mean_var_t, c, d_mean, d_var);
}
cudaError_t launch_restrict(const mclbm_ctx* c, int Qd, double* d_out) { MCLBM_DISPATCH(c, restrict_t, c, Qd, d_out); }
cudaError_t launch_check_finite(mclbm_ctx* c, int* h_bad) { MCLBM_DISPATCH(c, finite_t, c, h_bad); }

// Velocity field of one sample into the work buffer (used by the spectral statistics).
cudaError_t launch_field(const mclbm_ctx* c, int sample, double* d_u) { return launch_moments(c, sample, nullptr, d_u); }

}  // namespace mclbm
