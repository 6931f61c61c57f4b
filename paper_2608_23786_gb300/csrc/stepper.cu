// Ensemble initialisation and the fused stream + KBC collide kernels.
//
// One thread updates one lattice node of one sample per step.  The grid spans
// every node of every sample of the ensemble (the sample index is the slowest
// part of the linear node index), so a whole ensemble advances in one launch.
//
// Streaming (Eq. (lbIteration), f_i(x + c_i, t + 1) = f*_i(x, t)) is fused with
// the collision in two patterns:
//   pull: read f_i(x, t) = S_i(x - c_i) from lattice A, write f*_i(x, t) to
//         slot i of node x in lattice B (A and B swap every step);
//   AA:   one lattice, in place.  Even t: read slot i of x, write f*_i to slot
//         opp(i) of x.  Odd t: read slot opp(i) of x - c_i, write f*_i to slot i
//         of x + c_i.  Each node reads and writes the same 19 slots, so no two
//         threads touch the same element within a step.
#include <cuda_fp16.h>

#include "collide.cuh"
#include "internal.h"
#include "storage.cuh"

namespace mclbm {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ void decode(const Geom& g, int64_t idx, int& m, int& x, int& y, int& z)
{
    m = (int)(idx >> (3 * g.logN));
    const int64_t node = idx & (g.n - 1);
    x = (int)(node & (g.N - 1));
    y = (int)((node >> g.logN) & (g.N - 1));
    z = (int)(node >> (2 * g.logN));
}

template <class E>
__device__ __forceinline__ void collide_node(typename Storage<E>::compute (&v)[Q], typename Storage<E>::compute omega)
{
    if constexpr (Storage<E>::shifted)
        kbc_shifted(v, omega);
    else
        kbc_raw(v, omega);
}

// ---------------------------------------------------------------- init ----
// u_0 = (U_lat / U_c) (u_det + s(X_m)) at node x_n = 2 pi n / N, f_0 = f^eq(rho_0, u_0),
// Eqs. (tgv_init_velo), (alpha_perturbation), (initialRTGV), (initialPopulations).
template <class E>
__global__ void __launch_bounds__(kBlock) k_init(E* __restrict__ lat, Geom g, int64_t total, const double* __restrict__ X,
                                                 double uc, double ulat, int density_mode, int pattern)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int m, x, y, z;
        decode(g, idx, m, x, y, z);
        const double invN = 1.0 / g.N;
        double sx, cxx, sy, cyy, sz, czz, s2x, c2x, s2y, c2y, s2z, c2z;
        sincospi(2.0 * x * invN, &sx, &cxx);
        sincospi(2.0 * y * invN, &sy, &cyy);
        sincospi(2.0 * z * invN, &sz, &czz);
        sincospi(4.0 * x * invN, &s2x, &c2x);
        sincospi(4.0 * y * invN, &s2y, &c2y);
        sincospi(4.0 * z * invN, &s2z, &c2z);
        double u[3] = {uc * sx * cyy * czz, -uc * cxx * sy * czz, 0.0};
        if (X) {
            const double* Xm = X + 24 * (int64_t)m;
            const double ax[2] = {s2x, c2x}, ay[2] = {s2y, c2y}, az[2] = {s2z, c2z};
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int k = 0; k < 2; ++k) s += Xm[8 * al + 4 * i + 2 * j + k] * (ax[i] * ay[j] * az[k]);
                u[al] += s * 0.125;
            }
        }
        const double sc = ulat / uc;
        u[0] *= sc;
        u[1] *= sc;
        u[2] *= sc;
        double drho = 0.0;
        if (density_mode == 1) drho = 3.0 * (ulat * ulat / 16.0) * (c2x + c2y) * (c2z + 2.0);
        const double rho = 1.0 + drho;
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        E* base = lat + (int64_t)m * Q * g.n;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
            const double heq = drho + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);  // f^eq / w - 1
            E* p = base + pre_loc(g, pattern, 0, i, x, y, z);
            if constexpr (Storage<E>::shifted) {
                if constexpr (sizeof(E) == 4)
                    *p = (float)heq;
                else
                    *p = __double2half(heq);
            } else {
                *p = rho * weight<double>(i) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            }
        }
    }
}

// ------------------------------------------------------ fused step: pull ----
template <class E>
__global__ void __launch_bounds__(kBlock) k_step_pull(const E* __restrict__ src, E* __restrict__ dst, Geom g,
                                                      int64_t total, typename Storage<E>::compute omega)
{
    using C = typename Storage<E>::compute;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int m, x, y, z;
        decode(g, idx, m, x, y, z);
        const int64_t base = (int64_t)m * Q * g.n;
        C v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            v[i] = Storage<E>::load(src + base + (int64_t)i * g.n +
                                    g.node(g.wrap(x - cx(i)), g.wrap(y - cy(i)), g.wrap(z - cz(i))));
        collide_node<E>(v, omega);
        const int64_t node = g.node(x, y, z);
#pragma unroll
        for (int i = 0; i < Q; ++i) Storage<E>::store(dst + base + (int64_t)i * g.n + node, v[i]);
    }
}

// -------------------------------------------------------- fused step: AA ----
template <class E, int Parity>
__global__ void __launch_bounds__(kBlock) k_step_aa(E* lat, Geom g, int64_t total, typename Storage<E>::compute omega)
{
    using C = typename Storage<E>::compute;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int m, x, y, z;
        decode(g, idx, m, x, y, z);
        E* base = lat + (int64_t)m * Q * g.n;
        C v[Q];
        if (Parity == 0) {
            const int64_t node = g.node(x, y, z);
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = Storage<E>::load(base + (int64_t)i * g.n + node);
            collide_node<E>(v, omega);
#pragma unroll
            for (int i = 0; i < Q; ++i) Storage<E>::store(base + (int64_t)opp(i) * g.n + node, v[i]);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                v[i] = Storage<E>::load(base + (int64_t)opp(i) * g.n +
                                        g.node(g.wrap(x - cx(i)), g.wrap(y - cy(i)), g.wrap(z - cz(i))));
            collide_node<E>(v, omega);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                Storage<E>::store(base + (int64_t)i * g.n + g.node(g.wrap(x + cx(i)), g.wrap(y + cy(i)), g.wrap(z + cz(i))),
                                  v[i]);
        }
    }
}

// ------------------------------------------------ population gather/scatter ----
template <class E>
__global__ void k_get_pops(const E* __restrict__ lat, Geom g, int pattern, int parity, int sample, double* __restrict__ out)
{
    const E* base = lat + (int64_t)sample * Q * g.n;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n;
         node += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(node & (g.N - 1)), y = (int)((node >> g.logN) & (g.N - 1)), z = (int)(node >> (2 * g.logN));
#pragma unroll
        for (int i = 0; i < Q; ++i) out[(int64_t)i * g.n + node] = to_raw<E>(i, base[pre_loc(g, pattern, parity, i, x, y, z)]);
    }
}

template <class E>
__global__ void k_set_pops(E* __restrict__ lat, Geom g, int pattern, int parity, int sample, const double* __restrict__ in)
{
    E* base = lat + (int64_t)sample * Q * g.n;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n;
         node += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(node & (g.N - 1)), y = (int)((node >> g.logN) & (g.N - 1)), z = (int)(node >> (2 * g.logN));
#pragma unroll
        for (int i = 0; i < Q; ++i) store_raw<E>(base + pre_loc(g, pattern, parity, i, x, y, z), i, in[(int64_t)i * g.n + node]);
    }
}

int grid_for(int64_t total)
{
    int64_t b = (total + kBlock - 1) / kBlock;
    return (int)(b > (int64_t)1 << 30 ? (int64_t)1 << 30 : b);
}

Geom geom_of(const mclbm_ctx* c) { return Geom{c->N, c->logN, c->n}; }

template <class E>
cudaError_t init_t(const mclbm_ctx* c, const double* d_params)
{
    const int64_t total = (int64_t)c->M * c->n;
    k_init<E><<<grid_for(total), kBlock, 0, c->stream>>>((E*)lattice_ptr(c, c->cur), geom_of(c), total, d_params,
                                                         c->cfg.U_c, c->units.U_lat, c->cfg.init_density,
                                                         c->cfg.pattern);
    return cudaGetLastError();
}

template <class E>
cudaError_t step_t(mclbm_ctx* c)
{
    using C = typename Storage<E>::compute;
    const int64_t total = (int64_t)c->M * c->n;
    const C omega = (C)c->units.omega;
    if (c->cfg.pattern == MCLBM_PULL) {
        k_step_pull<E><<<grid_for(total), kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur),
                                                                  (E*)lattice_ptr(c, 1 - c->cur), geom_of(c), total,
                                                                  omega);
        c->cur ^= 1;
    } else if ((c->steps & 1) == 0) {
        k_step_aa<E, 0><<<grid_for(total), kBlock, 0, c->stream>>>((E*)lattice_ptr(c, 0), geom_of(c), total, omega);
    } else {
        k_step_aa<E, 1><<<grid_for(total), kBlock, 0, c->stream>>>((E*)lattice_ptr(c, 0), geom_of(c), total, omega);
    }
    return cudaGetLastError();
}

template <class E>
cudaError_t get_t(const mclbm_ctx* c, int sample, double* d_out)
{
    k_get_pops<E><<<grid_for(c->n), kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur), geom_of(c),
                                                            c->cfg.pattern, (int)(c->steps & 1), sample, d_out);
    return cudaGetLastError();
}

template <class E>
cudaError_t set_t(mclbm_ctx* c, int sample, const double* d_in)
{
    k_set_pops<E><<<grid_for(c->n), kBlock, 0, c->stream>>>((E*)lattice_ptr(c, c->cur), geom_of(c), c->cfg.pattern,
                                                            (int)(c->steps & 1), sample, d_in);
    return cudaGetLastError();
}

}  // namespace

#define MCLBM_DISPATCH(c, fn, ...)                                  \
    switch ((c)->cfg.precision) {                                   \
        case MCLBM_FP64: return fn<double>(__VA_ARGS__);            \
        case MCLBM_FP32: return fn<float>(__VA_ARGS__);             \
        default: return fn<__half>(__VA_ARGS__);                    \
    }

cudaError_t launch_init(const mclbm_ctx* c, const double* d_params) { MCLBM_DISPATCH(c, init_t, c, d_params); }
cudaError_t launch_step(mclbm_ctx* c) { MCLBM_DISPATCH(c, step_t, c); }
cudaError_t launch_get_populations(const mclbm_ctx* c, int sample, double* d_out)
{
    MCLBM_DISPATCH(c, get_t, c, sample, d_out);
}
cudaError_t launch_set_populations(mclbm_ctx* c, int sample, const double* d_in)
{
    MCLBM_DISPATCH(c, set_t, c, sample, d_in);
}

}  // namespace mclbm
