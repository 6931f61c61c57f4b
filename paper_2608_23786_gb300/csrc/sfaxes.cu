// Longitudinal structure functions along the lattice axes, p = 2..pmax
// (Eq. (structuresLocal) with n in {e_x, e_y, e_z}; the modulus as in Eq.
// (structures)):  S_p(r) = 1/(3 N^3) sum_x sum_a |u_a(x + r e_a) - u_a(x)|^p.
//
// A line is the component u_a along axis a for fixed other coordinates (3 N^2
// lines).  Each block stages L lines in shared memory; thread t owns the lag
// r = t % (N/2) + 1 of line t / (N/2) and accumulates the p-th powers in FP64
// over the whole line, keeping its sums in registers across all batches of lines
// the block handles.  Threads with the same lag are then summed in a fixed
// order, and a second kernel sums the blocks in a fixed order: deterministic.
#include "internal.h"
#include "storage.cuh"

namespace mclbm {

cudaError_t launch_field(const mclbm_ctx* c, int sample, double* d_u);

namespace {

constexpr int kThreads = 256;
constexpr int kMaxP = 8;
constexpr int kSfBlocks = 152 * 2;

__global__ void __launch_bounds__(kThreads) k_sf_axes(const double* __restrict__ u, int N, int logN, int pmax,
                                                      double* __restrict__ partial)
{
    extern __shared__ double sm[];
    const int halfN = N / 2;
    const int L = kThreads / halfN > 0 ? kThreads / halfN : 1;  // lines per batch
    double* line = sm;                                          // [L][N]
    const int t = threadIdx.x;
    const int r = t % halfN + 1;
    const int lsub = t / halfN;
    const bool active = lsub < L && t < L * halfN;
    double acc[kMaxP - 1];
#pragma unroll
    for (int k = 0; k < kMaxP - 1; ++k) acc[k] = 0.0;
    const int64_t n = (int64_t)N * N * N;
    const int nlines = 3 * N * N;
    const int nbatches = (nlines + L - 1) / L;
    for (int b = blockIdx.x; b < nbatches; b += gridDim.x) {
        __syncthreads();
        for (int k = t; k < L * N; k += blockDim.x) {
            const int ls = k / N, j = k % N;
            const int lid = b * L + ls;
            double v = 0.0;
            if (lid < nlines) {
                const int a = lid / (N * N), rest = lid % (N * N);
                const int p = rest / N, q = rest % N;  // the two fixed coordinates
                int64_t idx;
                if (a == 0) idx = ((int64_t)p * N + q) * N + j;       // (z=p, y=q, x=j)
                else if (a == 1) idx = ((int64_t)p * N + j) * N + q;  // (z=p, y=j, x=q)
                else idx = ((int64_t)j * N + p) * N + q;              // (z=j, y=p, x=q)
                v = u[(int64_t)a * n + idx];
            }
            line[ls * N + j] = v;
        }
        __syncthreads();
        if (active && b * L + lsub < nlines) {
            const double* Lp = line + lsub * N;
            for (int x = 0; x < N; ++x) {
                const double d = fabs(Lp[(x + r) & (N - 1)] - Lp[x]);
                double pw = d * d;
                acc[0] += pw;
#pragma unroll
                for (int k = 1; k < kMaxP - 1; ++k) {
                    if (k + 2 > pmax) break;
                    pw *= d;
                    acc[k] += pw;
                }
            }
        }
    }
    // combine threads of equal lag in a fixed order: stage in shared memory
    __syncthreads();
    double* red = sm;  // [L][halfN][kMaxP-1] fits: L * halfN <= kThreads
    if (active) {
#pragma unroll
        for (int k = 0; k < kMaxP - 1; ++k) red[((int64_t)lsub * halfN + (r - 1)) * (kMaxP - 1) + k] = acc[k];
    }
    __syncthreads();
    for (int o = t; o < halfN * (kMaxP - 1); o += blockDim.x) {
        double s = 0.0;
        for (int ls = 0; ls < L; ++ls) s += red[(int64_t)ls * halfN * (kMaxP - 1) + o];
        partial[(int64_t)blockIdx.x * halfN * (kMaxP - 1) + o] = s;
    }
}

__global__ void k_sf_reduce(const double* __restrict__ partial, int nblocks, int halfN, int pmax, double scale,
                            double* __restrict__ out)
{
    // out [pmax-1][halfN]
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < halfN * (pmax - 1); o += gridDim.x * blockDim.x) {
        const int k = o / halfN, r = o % halfN;
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[((int64_t)b * halfN + r) * (kMaxP - 1) + k];
        out[o] = s * scale;
    }
}

}  // namespace

size_t sf_axes_smem(int N)
{
    const int halfN = N / 2;
    const int L = kThreads / halfN > 0 ? kThreads / halfN : 1;
    size_t a = (size_t)L * N * sizeof(double);
    size_t b = (size_t)L * halfN * (kMaxP - 1) * sizeof(double);
    return a > b ? a : b;
}

size_t sf_axes_partial_bytes(int N) { return (size_t)kSfBlocks * (N / 2) * (kMaxP - 1) * sizeof(double); }

cudaError_t launch_sf_axes(mclbm_ctx* c, int pmax, double* h_S)
{
    const int N = c->N, halfN = N / 2;
    double* field = (double*)(c->work + c->wl.field);
    double* partial = (double*)(c->work + c->wl.real);  // reuses the spectrum buffer
    double* out = (double*)(c->work + c->wl.bins);      // [M][pmax-1][N/2]
    const size_t smem = sf_axes_smem(N);
    cudaError_t e = cudaFuncSetAttribute(k_sf_axes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const double scale = 1.0 / (3.0 * (double)c->n);
    for (int m = 0; m < c->M; ++m) {
        if ((e = launch_field(c, m, field)) != cudaSuccess) return e;
        k_sf_axes<<<kSfBlocks, kThreads, smem, c->stream>>>(field, N, c->logN, pmax, partial);
        k_sf_reduce<<<8, 256, 0, c->stream>>>(partial, kSfBlocks, halfN, pmax, scale,
                                               out + (int64_t)m * (pmax - 1) * halfN);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(h_S, out, sizeof(double) * c->M * (pmax - 1) * halfN, cudaMemcpyDeviceToHost, c->stream)) !=
        cudaSuccess)
        return e;
    return cudaStreamSynchronize(c->stream);
}

}  // namespace mclbm
