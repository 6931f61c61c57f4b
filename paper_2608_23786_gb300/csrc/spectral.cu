// Spectral statistics: FP64 3-D FFT, shell energy spectrum and the trace
// second-order structure function of Algorithm "SF_spectral".
//
// FFT: complex-to-complex, N a power of two.  A 3-D transform is three passes of
// batched 1-D transforms, one per axis.  Each block stages a tile of T lines in
// shared memory (T consecutive x for the y and z passes, so every global access is
// a coalesced run of T complex values), applies the bit-reversal permutation on
// load, the butterfly stages in place (radix-2^2: stages in pairs), and writes the
// tile back.  Twiddles exp(-2 pi i k / N) come from a table made
// once per context.  Real fields share complex transforms two at a time: samples
// are taken in pairs (a, b), u_x + i u_y of each sample is one transform (only the
// sum of the two powers is needed), and u_z of a with u_z of b is a third, whose two
// powers are separated through Z_k and Z_-k: 1.5 forward transforms per sample.  The
// autocorrelations of a pair come from one inverse transform of psi_a + i psi_b
// (each psi is real and even, so each inverse is real).  An odd last sample takes
// two forward and one inverse transform of its own.
//
// Shell sums: the blocks of shell kappa (or lag radius r) enumerate its integer
// points {k in K_N : round(|k|) = kappa}, K_N = {-N/2+1..N/2}^3, with an exact
// integer test 4|k|^2 in [(2 kappa - 1)^2, (2 kappa + 1)^2), each thread over a
// fixed subset of (k_z, k_y) rows, then fixed reduction trees: deterministic.
#include "internal.h"
#include "storage.cuh"

namespace mclbm {

cudaError_t launch_field(const mclbm_ctx* c, int sample, double* d_u);

namespace {

constexpr int kFftThreads = 256;

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a conj(b)
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b)
{
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Batched 1-D FFT of length N along one axis; `stride` is the element distance
// along the line (1, N or N^2).  Block b handles T lines.
__global__ void __launch_bounds__(kFftThreads) k_fft_pass(double2* __restrict__ data, const double2* __restrict__ tw,
                                                          int N, int logN, int T, int64_t stride, int inverse)
{
    extern __shared__ double2 buf[];  // [T][N]
    const int64_t n = (int64_t)N * N * N;
    (void)n;
    // line t of this block starts at base(t)
    const int lines_per_plane = N * N;  // lines of one axis
    const int first = blockIdx.x * T;   // first line id
    auto base_of = [&](int line) -> int64_t {
        if (stride == 1) return (int64_t)line * N;        // line = z*N + y
        const int a = line / N, b = line % N;             // b = x (fastest across the tile)
        if (stride == N) return (int64_t)a * N * N + b;   // a = z: elements (z, j, x)
        return (int64_t)a * N + b;                        // stride N^2: a = y: elements (j, y, x)
    };
    (void)lines_per_plane;
    const int total = T * N;
    if (stride == 1) {
        for (int k = threadIdx.x; k < total; k += blockDim.x) {
            const int t = k / N, j = k % N;
            buf[t * N + bitrev(j, logN)] = data[base_of(first + t) + j];
        }
    } else {
        for (int k = threadIdx.x; k < total; k += blockDim.x) {
            const int t = k % T, j = k / T;
            buf[t * N + bitrev(j, logN)] = data[base_of(first + t) + (int64_t)j * stride];
        }
    }
    __syncthreads();
    // Decimation in time on the bit-reversed tile, the stages in pairs as radix-2^2 butterflies
    // (three twiddle products per four points where the two radix-2 stages take four; the first
    // pair's twiddles are all 1): with w = W_{4h}^p for position p of a group of 4h points,
    // t1 = w^2 x1, t2 = w x2, t3 = w^3 x3, the stages h and 2h give (x0 + t1) +- (t2 + t3) and
    // (x0 - t1) -+ i (t2 - t3) (forward; the inverse conjugates w and i).  An odd log2 N ends with
    // one radix-2 stage.  tw holds W_N^j for j < N.
    const int quarterN = N >> 2;
    int s = 0;
    for (; s + 1 < logN; s += 2) {
        const int half = 1 << s;
        const int tstep = N >> (s + 2);  // W_{4h}^k = W_N^{k tstep}
        for (int b = threadIdx.x; b < T * quarterN; b += blockDim.x) {
            const int t = b / quarterN, q = b % quarterN;
            const int pos = q & (half - 1);
            double2* L = buf + t * N + ((q >> s) << (s + 2)) + pos;
            const double2 x0 = L[0];
            double2 t1 = L[half], t2 = L[2 * half], t3 = L[3 * half];
            if (half > 1) {  // uniform: the first pair has p = 0
                const int j1 = pos * tstep;
                if (inverse) {
                    t1 = cmul_conj(t1, tw[2 * j1]);
                    t2 = cmul_conj(t2, tw[j1]);
                    t3 = cmul_conj(t3, tw[3 * j1]);
                } else {
                    t1 = cmul(t1, tw[2 * j1]);
                    t2 = cmul(t2, tw[j1]);
                    t3 = cmul(t3, tw[3 * j1]);
                }
            }
            const double2 a = make_double2(x0.x + t1.x, x0.y + t1.y), c = make_double2(x0.x - t1.x, x0.y - t1.y);
            const double2 e = make_double2(t2.x + t3.x, t2.y + t3.y), d = make_double2(t2.x - t3.x, t2.y - t3.y);
            L[0] = make_double2(a.x + e.x, a.y + e.y);
            L[2 * half] = make_double2(a.x - e.x, a.y - e.y);
            if (inverse) {  // c +- i d
                L[half] = make_double2(c.x - d.y, c.y + d.x);
                L[3 * half] = make_double2(c.x + d.y, c.y - d.x);
            } else {  // c -+ i d
                L[half] = make_double2(c.x + d.y, c.y - d.x);
                L[3 * half] = make_double2(c.x - d.y, c.y + d.x);
            }
        }
        __syncthreads();
    }
    if (s < logN) {  // the last stage, h = N/2: W_N^p
        const int halfN = N >> 1;
        for (int b = threadIdx.x; b < T * halfN; b += blockDim.x) {
            const int t = b / halfN, pos = b % halfN;
            double2* L = buf + t * N + pos;
            const double2 u = L[0];
            const double2 v = inverse ? cmul_conj(L[halfN], tw[pos]) : cmul(L[halfN], tw[pos]);
            L[0] = make_double2(u.x + v.x, u.y + v.y);
            L[halfN] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    if (stride == 1) {
        for (int k = threadIdx.x; k < total; k += blockDim.x) {
            const int t = k / N, j = k % N;
            data[base_of(first + t) + j] = buf[t * N + j];
        }
    } else {
        for (int k = threadIdx.x; k < total; k += blockDim.x) {
            const int t = k % T, j = k / T;
            data[base_of(first + t) + (int64_t)j * stride] = buf[t * N + j];
        }
    }
}

__global__ void k_twiddles(double2* tw, int N)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * k / N, &s, &c);
        tw[k] = make_double2(c, s);
    }
}

__global__ void k_real_to_complex(const double* __restrict__ in, double2* __restrict__ out, int64_t n)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = make_double2(in[k], 0.0);
}

// Two real fields in one complex transform: out = a + i b.
__global__ void k_pack_complex(const double* __restrict__ a, const double* __restrict__ b, double2* __restrict__ out,
                               int64_t n)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = make_double2(a[k], b[k]);
}

// Power of the two real fields packed as Z = a + i b: with A, B their transforms,
// A_k = (Z_k + conj(Z_-k)) / 2 and B_k = (Z_k - conj(Z_-k)) / (2i), so
// |A_k|^2 + |B_k|^2 = (|Z_k|^2 + |Z_-k|^2) / 2 (index -k taken mod N per axis).
__global__ void k_accum_power_pair(const double2* __restrict__ in, double* __restrict__ psi, int N, int logN, int first)
{
    const int64_t n = (int64_t)N << (2 * logN);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(k & (N - 1)), iy = (int)((k >> logN) & (N - 1)), iz = (int)(k >> (2 * logN));
        const int64_t km = ((int64_t)((N - iz) & (N - 1)) << (2 * logN)) | ((int64_t)((N - iy) & (N - 1)) << logN) |
                           (int64_t)((N - ix) & (N - 1));
        const double2 v = in[k], w = in[km];
        const double p = 0.5 * ((v.x * v.x + v.y * v.y) + (w.x * w.x + w.y * w.y));
        psi[k] = first ? p : psi[k] + p;
    }
}

// Powers of the two real fields packed as Z = a + i b, each on its own: 2 A_k = Z_k + conj(Z_-k)
// and 2 i B_k = Z_k - conj(Z_-k), so |A_k|^2 and |B_k|^2 are a quarter of the squared moduli;
// added to psi_a and psi_b.
__global__ void k_accum_power_split(const double2* __restrict__ in, double* __restrict__ psi_a,
                                    double* __restrict__ psi_b, int N, int logN)
{
    const int64_t n = (int64_t)N << (2 * logN);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(k & (N - 1)), iy = (int)((k >> logN) & (N - 1)), iz = (int)(k >> (2 * logN));
        const int64_t km = ((int64_t)((N - iz) & (N - 1)) << (2 * logN)) | ((int64_t)((N - iy) & (N - 1)) << logN) |
                           (int64_t)((N - ix) & (N - 1));
        const double2 v = in[k], w = in[km];
        const double ar = v.x + w.x, ai = v.y - w.y;  // 2 A_k
        const double br = v.x - w.x, bi = v.y + w.y;  // 2 i B_k
        psi_a[k] += 0.25 * (ar * ar + ai * ai);
        psi_b[k] += 0.25 * (br * br + bi * bi);
    }
}

__global__ void k_accum_power(const double2* __restrict__ in, double* __restrict__ psi, int64_t n, int first)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = in[k];
        const double p = v.x * v.x + v.y * v.y;
        psi[k] = first ? p : psi[k] + p;
    }
}

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

// Shell sums.  mode 0 (spectrum): out[kappa] = 4 pi / |S| sum |k|^2 psi / 2 * scale.
// mode 1 (structure function): out[r] = 1/|C| sum 2 (R_0 - R_h), R_h = cbuf[h] * scale, taking
// the real (comp 0) or imaginary (comp 1) part of the complex buffer.
// Block (kappa, s) takes every kShellSplit-th thread stride of the rows (k_z, k_y) with
// |k_z|, |k_y| <= kappa (no other row meets the shell) and, per row, the k_x >= 0 with
// 4|k|^2 in [(2 kappa - 1)^2, (2 kappa + 1)^2), found in integers; partial[kappa][s] = (sum,
// count), summed over s in order by k_shell_finish.  One FP64 fma per point (the factors 1/2
// and 2 are applied once per shell) and an integer count keep the work off the FP64 pipe.
constexpr int kShellSplit = 16;

// Largest x >= 0 with 4 x^2 < v (v > 0): a single-precision guess (v < 2^24 here), corrected
// in integers.
__device__ __forceinline__ int isqrt_below(int64_t v)
{
    int x = (int)sqrtf(0.25f * (float)v);
    while (x >= 0 && 4 * (int64_t)x * x >= v) --x;
    while (4 * (int64_t)(x + 1) * (x + 1) < v) ++x;
    return x;
}

__global__ void k_shells(const double* __restrict__ psi, const double2* __restrict__ cbuf, int comp, int N, int mode,
                         double scale, double* __restrict__ partial)
{
    __shared__ double sh[32];
    const int kap = blockIdx.x, s = blockIdx.y;
    const int64_t lo4 = kap == 0 ? 0 : (int64_t)(2 * kap - 1) * (2 * kap - 1);  // 4|k|^2 >= lo4
    const int64_t hi4 = (int64_t)(2 * kap + 1) * (2 * kap + 1);                   // 4|k|^2 <  hi4
    const int half = N / 2;
    const int R = kap < half ? kap : half;
    const int lo = -R > -half + 1 ? -R : -half + 1;  // K_N: -N/2+1..N/2
    const int side = R - lo + 1;
    const int64_t rows = (int64_t)side * side;
    const double* cpart = reinterpret_cast<const double*>(cbuf) + comp;  // element h at cpart[2 h]
    const double R0 = mode == 1 ? cpart[0] * scale : 0.0;
    double acc = 0.0;
    int cnt = 0;
    for (int64_t p = (int64_t)s * blockDim.x + threadIdx.x; p < rows; p += (int64_t)gridDim.y * blockDim.x) {
        const int kz = lo + (int)(p / side), ky = lo + (int)(p % side);
        const int64_t kzy = (int64_t)kz * kz + (int64_t)ky * ky;
        const int64_t need = lo4 - 4 * kzy, below = hi4 - 4 * kzy;  // 4 kx^2 >= need, 4 kx^2 < below
        if (below <= 0) continue;
        const int kx0 = need <= 0 ? 0 : isqrt_below(need) + 1;
        int kx1 = isqrt_below(below);
        if (kx1 > half) kx1 = half;
        const int iz = kz < 0 ? kz + N : kz, iy = ky < 0 ? ky + N : ky;
        const int64_t row = ((int64_t)iz * N + iy) * N;
        for (int kx = kx0; kx <= kx1; ++kx) {
            const double k2 = (double)(kzy + (int64_t)kx * kx);
            for (int sgn = 0; sgn < 2; ++sgn) {
                int sx;
                if (sgn == 0) sx = kx;
                else {
                    if (kx == 0 || kx == half) continue;  // -0 is +0; -N/2 is not in K_N
                    sx = -kx;
                }
                const int64_t idx = row + (sx < 0 ? sx + N : sx);
                if (mode == 0)
                    acc = fma(k2, psi[idx], acc);
                else
                    acc += fma(-cpart[2 * idx], scale, R0);
                ++cnt;
            }
        }
    }
    acc = block_sum(acc, sh);
    const double count = block_sum((double)cnt, sh);
    if (threadIdx.x == 0) {
        partial[((int64_t)kap * gridDim.y + s) * 2] = acc;
        partial[((int64_t)kap * gridDim.y + s) * 2 + 1] = count;
    }
}

__global__ void k_shell_finish(const double* __restrict__ partial, int nb, int split, int mode, double scale,
                               double* __restrict__ out)
{
    for (int kap = blockIdx.x * blockDim.x + threadIdx.x; kap < nb; kap += gridDim.x * blockDim.x) {
        double acc = 0.0, cnt = 0.0;
        for (int s = 0; s < split; ++s) {
            acc += partial[((int64_t)kap * split + s) * 2];
            cnt += partial[((int64_t)kap * split + s) * 2 + 1];
        }
        if (mode == 0)
            out[kap] = cnt > 0 ? 4.0 * 3.14159265358979323846 / cnt * (0.5 * acc) * scale : 0.0;
        else
            out[kap] = cnt > 0 ? 2.0 * acc / cnt : 0.0;
    }
}

cudaError_t shells(const mclbm_ctx* c, const double* psi, const double2* cbuf, int comp, int mode, double scale,
                   double* out)
{
    const int nb = c->N / 2 + 1;
    double* partial = (double*)(c->work + c->wl.partial);
    k_shells<<<dim3(nb, kShellSplit), 256, 0, c->stream>>>(psi, cbuf, comp, c->N, mode, scale, partial);
    k_shell_finish<<<(nb + 255) / 256, 256, 0, c->stream>>>(partial, nb, kShellSplit, mode, mode == 0 ? scale : 1.0, out);
    return cudaGetLastError();
}

int grid_for(int64_t total)
{
    int64_t b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

int fft_tile(int N) { return N >= 8 ? 8 : N; }

cudaError_t fft3d(const mclbm_ctx* c, double2* data, const double2* tw, int inverse)
{
    const int N = c->N, logN = c->logN, T = fft_tile(N);
    const size_t smem = (size_t)T * N * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_fft_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = N * N / T;
    const int64_t strides[3] = {1, N, (int64_t)N * N};
    for (int a = 0; a < 3; ++a) {
        k_fft_pass<<<blocks, kFftThreads, smem, c->stream>>>(data, tw, N, logN, T, strides[a], inverse);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_twiddles(const mclbm_ctx* c)
{
    k_twiddles<<<grid_for(c->N), 256, 0, c->stream>>>((double2*)(c->work + c->wl.twiddle), c->N);
    return cudaGetLastError();
}

// Spectrum E [M][N/2+1] and/or S2 [M][N/2+1] (host, may be NULL).
cudaError_t launch_spectral(mclbm_ctx* c, double* h_E, double* h_S2)
{
    const int64_t n = c->n;
    const int nb = c->N / 2 + 1;
    double* field = (double*)(c->work + c->wl.field);  // [4][n]
    double2* cb = (double2*)(c->work + c->wl.cplx);
    double* psi_a = (double*)(c->work + c->wl.real);
    double* psi_b = (double*)(c->work + c->wl.real2);
    const double2* tw = (const double2*)(c->work + c->wl.twiddle);
    double* bins = (double*)(c->work + c->wl.bins);  // [2][M][nb]
    const double N3 = (double)n;
    const double s6 = 1.0 / (N3 * N3);  // Phi = |u~|^2 with u~ = F(u) / N^3, so Phi = psi / N^6
    const int gn = grid_for(n);
    cudaStream_t st = c->stream;
    cudaError_t e;
    int m = 0;
    for (; m + 1 < c->M; m += 2) {
        // sample m at field + n (its u_z at field + 3n), then sample m + 1 at field (u_z at field + 2n)
        if ((e = launch_field(c, m, field + n)) != cudaSuccess) return e;
        k_pack_complex<<<gn, 256, 0, st>>>(field + n, field + 2 * n, cb, n);
        if ((e = fft3d(c, cb, tw, 0)) != cudaSuccess) return e;
        k_accum_power_pair<<<gn, 256, 0, st>>>(cb, psi_a, c->N, c->logN, 1);
        if ((e = launch_field(c, m + 1, field)) != cudaSuccess) return e;
        k_pack_complex<<<gn, 256, 0, st>>>(field, field + n, cb, n);
        if ((e = fft3d(c, cb, tw, 0)) != cudaSuccess) return e;
        k_accum_power_pair<<<gn, 256, 0, st>>>(cb, psi_b, c->N, c->logN, 1);
        k_pack_complex<<<gn, 256, 0, st>>>(field + 3 * n, field + 2 * n, cb, n);
        if ((e = fft3d(c, cb, tw, 0)) != cudaSuccess) return e;
        k_accum_power_split<<<gn, 256, 0, st>>>(cb, psi_a, psi_b, c->N, c->logN);
        if (h_E) {
            if ((e = shells(c, psi_a, nullptr, 0, 0, s6, bins + (int64_t)m * nb)) != cudaSuccess) return e;
            if ((e = shells(c, psi_b, nullptr, 0, 0, s6, bins + (int64_t)(m + 1) * nb)) != cudaSuccess) return e;
        }
        if (h_S2) {
            // R = N^-3 F^-1(psi), F^-1 with the factor N^-3: R_h = re(sum_k psi_k e^{+2 pi i k.h/N}) / N^6;
            // the pair's two autocorrelations are the real and imaginary parts of one inverse
            k_pack_complex<<<gn, 256, 0, st>>>(psi_a, psi_b, cb, n);
            if ((e = fft3d(c, cb, tw, 1)) != cudaSuccess) return e;
            if ((e = shells(c, nullptr, cb, 0, 1, s6, bins + (int64_t)(c->M + m) * nb)) != cudaSuccess) return e;
            if ((e = shells(c, nullptr, cb, 1, 1, s6, bins + (int64_t)(c->M + m + 1) * nb)) != cudaSuccess) return e;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (m < c->M) {  // the odd last sample: u_x + i u_y, then u_z alone
        if ((e = launch_field(c, m, field)) != cudaSuccess) return e;
        k_pack_complex<<<gn, 256, 0, st>>>(field, field + n, cb, n);
        if ((e = fft3d(c, cb, tw, 0)) != cudaSuccess) return e;
        k_accum_power_pair<<<gn, 256, 0, st>>>(cb, psi_a, c->N, c->logN, 1);
        k_real_to_complex<<<gn, 256, 0, st>>>(field + 2 * n, cb, n);
        if ((e = fft3d(c, cb, tw, 0)) != cudaSuccess) return e;
        k_accum_power<<<gn, 256, 0, st>>>(cb, psi_a, n, 0);
        if (h_E && (e = shells(c, psi_a, nullptr, 0, 0, s6, bins + (int64_t)m * nb)) != cudaSuccess) return e;
        if (h_S2) {
            k_real_to_complex<<<gn, 256, 0, st>>>(psi_a, cb, n);
            if ((e = fft3d(c, cb, tw, 1)) != cudaSuccess) return e;
            if ((e = shells(c, nullptr, cb, 0, 1, s6, bins + (int64_t)(c->M + m) * nb)) != cudaSuccess) return e;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (h_E && (e = cudaMemcpyAsync(h_E, bins, sizeof(double) * c->M * nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    if (h_S2 && (e = cudaMemcpyAsync(h_S2, bins + (int64_t)c->M * nb, sizeof(double) * c->M * nb, cudaMemcpyDeviceToHost,
                                     st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

}  // namespace mclbm
