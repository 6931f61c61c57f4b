// Ensemble initialisation: the RTGV velocity of every sample and its equilibrium populations
// (the initial state of the stepper, in the storage's layout and pattern).
#include <cuda_fp16.h>

#include "internal.h"
#include "stepper_impl.cuh"

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

// Per-axis trigonometric tables of the initial condition: for n < N,
// t[4n + 0..3] = sin(x_n), cos(x_n), sin(2 x_n), cos(2 x_n), x_n = 2 pi n / N, and the same
// values rounded to FP32 in tf.
__global__ void k_trig_tables(double* t, float* tf, int N)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double s, c, s2, c2;
        sincospi(2.0 * k / N, &s, &c);
        sincospi(4.0 * k / N, &s2, &c2);
        t[4 * k + 0] = s;
        t[4 * k + 1] = c;
        t[4 * k + 2] = s2;
        t[4 * k + 3] = c2;
        tf[4 * k + 0] = (float)s;
        tf[4 * k + 1] = (float)c;
        tf[4 * k + 2] = (float)s2;
        tf[4 * k + 3] = (float)c2;
    }
}

// u_0 = (U_lat / U_c)(u_det + s(X_m)) at node x_n = 2 pi n / N, f_0 = f^eq(rho_0, u_0):
// Eqs. (tgv_init_velo), (alpha_perturbation), (initialRTGV), (initialPopulations).
// The row factors below in FP64; per node u_0, rho_0 and the equilibrium in the storage's
// arithmetic (FP64 for raw storage; FP32 for the shifted deviations h = f^eq / w - 1, whose
// stored values carry FP32 rounding at best, so the node's FP64 work is only that of its row,
// and the kernel writes at memory speed instead of waiting on GB300's FP64 units).  A block takes kInitChunk
// consecutive nodes of the ensemble (whole rows, or part of one row when N > kInitChunk): one
// thread per row first forms the row's factors in shared memory, the y, z factors of u_det and
// of the perturbation of Eq. (alpha_perturbation),
//   s_a = (1/8) sum_{ijk} X_{a,ijk} A_i(2x) A_j(2y) A_k(2z) = (1/8) sum_i A_i(2x) B_{a,i},
//   B_{a,i} = sum_{jk} X_{a,ijk} A_j(2y) A_k(2z);
// then consecutive threads take consecutive nodes, so every population's stores are coalesced.
constexpr int kInitChunk = 2048;

// Row factors, with U_lat / U_c and the 1/8 of the perturbation folded in: along the row,
// u_x = ux_yz sin x + B[0][0] sin 2x + B[0][1] cos 2x, u_y = uy_yz cos x + B[1][0] sin 2x +
// B[1][1] cos 2x, u_z = B[2][0] sin 2x + B[2][1] cos 2x.
template <class T>
struct InitRow {
    T B[3][2];
    T ux_yz, uy_yz, dr_yz, c2y;
};

// trig: the FP64 table; trig_c: the table in the compute type (the same table for FP64 storage)
template <class E>
__global__ void __launch_bounds__(kBlock) k_init(E* __restrict__ lat, Geom g, int64_t total, const double* __restrict__ X,
                                                 const double* __restrict__ trig,
                                                 const typename Storage<E>::compute* __restrict__ trig_c, double uc,
                                                 double ulat, int density_mode, int pattern)
{
    using C = typename Storage<E>::compute;
    __shared__ InitRow<C> rows[kInitChunk / 8];  // N >= 8
    const int rows_per_chunk = kInitChunk >> g.logN > 0 ? kInitChunk >> g.logN : 1;
    const double sc = ulat / uc;
    for (int64_t c0 = blockIdx.x * (int64_t)kInitChunk; c0 < total; c0 += (int64_t)gridDim.x * kInitChunk) {
        __syncthreads();  // the previous chunk's rows are no longer read
        const int span = kInitChunk < (int)(total - c0) ? kInitChunk : (int)(total - c0);
        const int nrows = ((span + g.N - 1) >> g.logN) < rows_per_chunk ? ((span + g.N - 1) >> g.logN) : rows_per_chunk;
        for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
            int m, x, y, z;
            decode(g, c0 + ((int64_t)r << g.logN), m, x, y, z);
            const double sy = trig[4 * y], cyy = trig[4 * y + 1], s2y = trig[4 * y + 2], c2y = trig[4 * y + 3];
            const double czz = trig[4 * z + 1], s2z = trig[4 * z + 2], c2z = trig[4 * z + 3];
            const double* Xm = X + 24 * (int64_t)m;
            const double ay[2] = {s2y, c2y}, az[2] = {s2z, c2z};
            double P[2][2];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int k = 0; k < 2; ++k) P[j][k] = ay[j] * az[k];
            InitRow<C> ir;
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    double bsum = 0.0;
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int k = 0; k < 2; ++k) bsum = fma(Xm[8 * al + 4 * i + 2 * j + k], P[j][k], bsum);
                    ir.B[al][i] = (C)(0.125 * sc * bsum);
                }
            ir.ux_yz = (C)(sc * (uc * cyy * czz));  // u_det = (ux_yz sin x, uy_yz cos x, 0)
            ir.uy_yz = (C)(sc * (-uc * sy * czz));
            ir.dr_yz = (C)(3.0 * (ulat * ulat / 16.0) * (c2z + 2.0));
            ir.c2y = (C)c2y;
            rows[r] = ir;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < span; q += blockDim.x) {
            int m, x, y, z;
            decode(g, c0 + q, m, x, y, z);
            const InitRow<C>& ir = rows[q >> g.logN < rows_per_chunk ? q >> g.logN : 0];
            const C sx = trig_c[4 * x], cxx = trig_c[4 * x + 1], s2x = trig_c[4 * x + 2], c2x = trig_c[4 * x + 3];
            // three operations per component (the row factors carry U_lat / U_c and 1/8)
            const C u[3] = {fma(sx, ir.ux_yz, fma(s2x, ir.B[0][0], c2x * ir.B[0][1])),
                            fma(cxx, ir.uy_yz, fma(s2x, ir.B[1][0], c2x * ir.B[1][1])),
                            fma(s2x, ir.B[2][0], c2x * ir.B[2][1])};
            const C drho = density_mode == 1 ? ir.dr_yz * (c2x + ir.c2y) : C(0);
            E* base = lat + (int64_t)m * Q * g.n;
            if constexpr (Storage<E>::shifted) {
                const C ux = u[0], uy = u[1], uz = u[2], dr = drho, rho = C(1) + dr;
                const C uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    C cu = 0;
                    MCLBM_SIGNED_ADD(cu, cx(i), ux);
                    MCLBM_SIGNED_ADD(cu, cy(i), uy);
                    MCLBM_SIGNED_ADD(cu, cz(i), uz);
                    const C heq = dr + rho * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
                    base[pre_loc(g, pattern, 0, i, x, y, z)] = from_c<E>(heq);
                }
            } else {
                const double rho = 1.0 + drho;
                const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
                    base[pre_loc(g, pattern, 0, i, x, y, z)] =
                        rho * weight<double>(i) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
                }
            }
        }
    }
}

Geom geom_of(const mclbm_ctx* c) { return Geom{c->N, c->logN, c->n}; }

template <class E>
cudaError_t init_t(const mclbm_ctx* c, const double* d_params, double* d_trig)
{
    float* d_trig_f = reinterpret_cast<float*>(d_trig + 4 * (size_t)c->N);
    k_trig_tables<<<(c->N + 127) / 128, 128, 0, c->stream>>>(d_trig, d_trig_f, c->N);
    using C = typename Storage<E>::compute;
    const C* trig_c;
    if constexpr (std::is_same<C, double>::value)
        trig_c = d_trig;
    else
        trig_c = d_trig_f;
    const int64_t total = (int64_t)c->M * c->n;  // a multiple of kInitChunk when n >= kInitChunk
    int64_t chunks = (total + kInitChunk - 1) / kInitChunk;
    if (chunks > (int64_t)c->num_sms * 8) chunks = (int64_t)c->num_sms * 8;
    k_init<E><<<(int)chunks, kBlock, 0, c->stream>>>((E*)lattice_ptr(c, c->cur), geom_of(c), total, d_params, d_trig,
                                                      trig_c, c->cfg.U_c, c->units.U_lat, c->cfg.init_density,
                                                      c->cfg.pattern);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init(const mclbm_ctx* c, const double* d_params)
{
    double* trig = (double*)(c->work + c->wl.trig);
    switch (c->cfg.precision) {
        case MCLBM_FP64: return init_t<double>(c, d_params, trig);
        case MCLBM_FP32: return init_t<float>(c, d_params, trig);
        default: return init_t<__half>(c, d_params, trig);
    }
}
}  // namespace mclbm
