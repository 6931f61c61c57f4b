// Macroscopic fields and ensemble reductions read from the population lattice:
// moments, kinetic energy / enstrophy, ensemble mean and variance, restriction to
// the common Q^3 grid, and the finiteness scan.
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

// Ensemble mean and unbiased variance of the physical velocity (Welford, fixed sample order).
template <class E>
__global__ void __launch_bounds__(kBlock) k_mean_var(const E* __restrict__ lat, Geom g, int M, int pattern, int parity,
                                                     double uscale, double* __restrict__ mean, double* __restrict__ var)
{
    using C = typename Storage<E>::compute;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n; node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        xyz_of(g, node, x, y, z);
        double mu[3] = {0, 0, 0}, m2[3] = {0, 0, 0};
        for (int m = 0; m < M; ++m) {
            C r, ux, uy, uz;
            node_moments<E, C>(lat + (int64_t)m * Q * g.n, g, pattern, parity, x, y, z, r, ux, uy, uz);
            const double v[3] = {(double)ux * uscale, (double)uy * uscale, (double)uz * uscale};
            const double inv = 1.0 / (m + 1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double d = v[a] - mu[a];
                mu[a] += d * inv;
                m2[a] += d * (v[a] - mu[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mean[a * g.n + node] = mu[a];
            var[a * g.n + node] = m2[a] / (M - 1);
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

template <class E>
cudaError_t mean_var_t(const mclbm_ctx* c, double* d_mean, double* d_var)
{
    k_mean_var<E><<<grid_for(c->n, 1 << 30), kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur), geom_of(c), c->M,
                                                                    c->cfg.pattern, parity_of(c), uscale_of(c), d_mean,
                                                                    d_var);
    return cudaGetLastError();
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
cudaError_t launch_mean_var(const mclbm_ctx* c, double* d_mean, double* d_var)
{
    MCLBM_DISPATCH(c, mean_var_t, c, d_mean, d_var);
}
cudaError_t launch_restrict(const mclbm_ctx* c, int Qd, double* d_out) { MCLBM_DISPATCH(c, restrict_t, c, Qd, d_out); }
cudaError_t launch_check_finite(mclbm_ctx* c, int* h_bad) { MCLBM_DISPATCH(c, finite_t, c, h_bad); }

// Velocity field of one sample into the work buffer (used by the spectral statistics).
cudaError_t launch_field(const mclbm_ctx* c, int sample, double* d_u) { return launch_moments(c, sample, nullptr, d_u); }

}  // namespace mclbm
