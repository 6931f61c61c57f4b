// Longitudinal structure functions along the lattice axes, p = 2..pmax
// (Eq. (structuresLocal) with n in {e_x, e_y, e_z}; the modulus as in Eq.
// (structures)):  S_p(r) = 1/(3 N^3) sum_x sum_a |u_a(x + r e_a) - u_a(x)|^p.
//
// A line is the component u_a along axis a for fixed other coordinates (3 N^2
// lines).  Each block stages L lines in shared memory; thread t owns the lag
// r = t % (N/2) + 1 of line t / (N/2) and accumulates the p-th powers in FP64
// over the whole line (contexts with FP32 or FP16 storage: FP32 differences and powers, FP32
// sums of 32 points added up in FP32 over the line, and the line's sums accumulated in FP64),
// keeping its sums in registers across all batches of
// lines the block handles.  Threads with the same lag are then summed in a fixed
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
            if (pmax <= 6) {
                // |d|^p for p = 2..6 from d^2 and d^4, three of them fused into the accumulation:
                // 8 FP64 operations per difference instead of 11
                for (int x = 0; x < N; ++x) {
                    const double d = Lp[(x + r) & (N - 1)] - Lp[x];
                    const double ad = fabs(d);
                    const double d2 = d * d;
                    acc[0] += d2;
                    acc[1] = fma(d2, ad, acc[1]);
                    const double d4 = d2 * d2;
                    acc[2] += d4;
                    acc[3] = fma(d4, ad, acc[3]);
                    acc[4] = fma(d4, d2, acc[4]);
                }
            } else {
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

// The same sums for contexts with FP32 or FP16 storage, whose velocity field carries FP32
// precision at most: the lines are staged in FP32, each difference and its powers (p = 2..6) are
// formed in FP32 and summed in FP32 over 32 consecutive points, the chunk sums of a line are
// added in FP32 (at most N / 32 = 16 of them), and each line's sums are accumulated in FP64.  All
// terms are positive, so a line's FP32 sum is within (32 + 16) 2^-24 < 3e-6 relative, and the
// FP64 units (GB300 runs FP32 at many times their rate) see 10 operations per line instead of 10
// per 32 points.
__global__ void __launch_bounds__(kThreads) k_sf_axes_f32(const double* __restrict__ u, int N, int logN,
                                                          double* __restrict__ partial)
{
    extern __shared__ double sm[];
    const int halfN = N / 2;
    const int L = kThreads / halfN > 0 ? kThreads / halfN : 1;
    float* line = reinterpret_cast<float*>(sm);  // [L][N]
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
    const int chunk = N < 32 ? N : 32;
    for (int b = blockIdx.x; b < nbatches; b += gridDim.x) {
        __syncthreads();
        for (int k = t; k < L * N; k += blockDim.x) {
            const int ls = k / N, j = k % N;
            const int lid = b * L + ls;
            float v = 0.f;
            if (lid < nlines) {
                const int a = lid / (N * N), rest = lid % (N * N);
                const int p = rest / N, q = rest % N;
                int64_t idx;
                if (a == 0) idx = ((int64_t)p * N + q) * N + j;
                else if (a == 1) idx = ((int64_t)p * N + j) * N + q;
                else idx = ((int64_t)j * N + p) * N + q;
                v = (float)u[(int64_t)a * n + idx];
            }
            line[ls * N + j] = v;
        }
        __syncthreads();
        if (active && b * L + lsub < nlines) {
            const float* Lp = line + lsub * N;
            float l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f, l4 = 0.f;  // the line's sums
            for (int x0 = 0; x0 < N; x0 += chunk) {
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
                for (int x = x0; x < x0 + chunk; ++x) {
                    const float d = Lp[(x + r) & (N - 1)] - Lp[x];
                    const float ad = fabsf(d);
                    const float d2 = d * d;
                    s0 += d2;
                    s1 = fmaf(d2, ad, s1);
                    const float d4 = d2 * d2;
                    s2 += d4;
                    s3 = fmaf(d4, ad, s3);
                    s4 = fmaf(d4, d2, s4);
                }
                l0 += s0;
                l1 += s1;
                l2 += s2;
                l3 += s3;
                l4 += s4;
            }
            acc[0] += (double)l0;
            acc[1] += (double)l1;
            acc[2] += (double)l2;
            acc[3] += (double)l3;
            acc[4] += (double)l4;
        }
    }
    __syncthreads();
    double* red = sm;
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
    // FP32/FP16 storage and p <= 6: FP32 differences with FP64 accumulation; otherwise FP64
    const bool f32 = c->cfg.precision != MCLBM_FP64 && pmax <= 6;
    cudaError_t e = f32 ? cudaFuncSetAttribute(k_sf_axes_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                        : cudaFuncSetAttribute(k_sf_axes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const double scale = 1.0 / (3.0 * (double)c->n);
    for (int m = 0; m < c->M; ++m) {
        if ((e = launch_field(c, m, field)) != cudaSuccess) return e;
        if (f32)
            k_sf_axes_f32<<<kSfBlocks, kThreads, smem, c->stream>>>(field, N, c->logN, partial);
        else
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
