// Two-point 1-Wasserstein distances between the laws of two ensembles on the restriction
// grid: W_{1,2}^v of Eq. (W1_vector) / Algorithm "WassersteinDistance2_vector" (atoms
// (u(x_i), u(x_j)) in R^6) and the component-wise W_{1,2} of Algorithm
// "WassersteinDistance2" (atoms (u_c(x_i), u_c(x_j)) in R^2 for each component c), with
// the Euclidean ground metric, for every point pair i <= j; pairs with i != j count twice
// and the sum is divided by G^2.
//
// Each pair (and component) is one exact optimal-transport problem between two uniform
// empirical measures.  With M_A and M_B atoms and L = lcm(M_A, M_B), repeating every atom
// of A L / M_A times and every atom of B L / M_B times gives uniform weights 1/L on both
// sides without changing the optimum, and an optimal plan is then a permutation: an L x L
// assignment problem.  One warp solves one problem with the shortest-augmenting-path
// (Hungarian) method on integer costs: the Euclidean distance of the FP32 atoms (taken
// relative to the atoms' mean) in fixed point (2^40 units for the largest possible cost), so
// that the potentials and reduced costs are exact and the matching is optimal for those costs.  The distance of the problem is then the mean FP64 cost of the
// matched pairs, recomputed from the FP64 atoms.  Each lane owns columns lane and lane + 32.
#include <cmath>
#include <string>

#include "internal.h"

namespace mclbm {

namespace {

constexpr int kPairMaxL = 64;  // largest assignment size (two columns per lane)
constexpr int kPairWarps = 8;  // warps (problems in flight) per block
constexpr long long kInf = 0x3fffffffffffffffLL;

struct PairProblem {
    int i, j, c;  // point pair (i <= j) and component (vector problems: c = 0)
};

// Pair k of the row-major upper triangle of G x G: row start s(i) = i (2G - i + 1) / 2.
__device__ __forceinline__ void pair_of(int64_t k, int G, int& i, int& j)
{
    const double b = 2.0 * G + 1.0;
    int r = (int)floor((b - sqrt(b * b - 8.0 * (double)k)) * 0.5);
    auto start = [G](int64_t t) { return t * (2 * (int64_t)G - t + 1) / 2; };
    if (r < 0) r = 0;
    if (r > G - 1) r = G - 1;
    while (r > 0 && start(r) > k) --r;
    while (r < G - 1 && start(r + 1) <= k) ++r;
    i = r;
    j = r + (int)(k - start(r));
}

// Atom of sample m for the problem in FP64: K = 6 (vector) or 2 (component c).
template <int K>
__device__ __forceinline__ void atom64(const double* U, int G, int m, const PairProblem& pb, double (&x)[K])
{
    if constexpr (K == 6) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            x[d] = U[((int64_t)m * G + pb.i) * 3 + d];
            x[3 + d] = U[((int64_t)m * G + pb.j) * 3 + d];
        }
    } else {
        x[0] = U[((int64_t)m * G + pb.i) * 3 + pb.c];
        x[1] = U[((int64_t)m * G + pb.j) * 3 + pb.c];
    }
}

template <int K>
__device__ __forceinline__ double cost64(const double* A, const double* B, int G, int ma, int mb, const PairProblem& pb)
{
    double s = 0.0;
    if constexpr (K == 6) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double e1 = A[((int64_t)ma * G + pb.i) * 3 + d] - B[((int64_t)mb * G + pb.i) * 3 + d];
            const double e2 = A[((int64_t)ma * G + pb.j) * 3 + d] - B[((int64_t)mb * G + pb.j) * 3 + d];
            s += e1 * e1 + e2 * e2;
        }
    } else {
        const double e1 = A[((int64_t)ma * G + pb.i) * 3 + pb.c] - B[((int64_t)mb * G + pb.i) * 3 + pb.c];
        const double e2 = A[((int64_t)ma * G + pb.j) * 3 + pb.c] - B[((int64_t)mb * G + pb.j) * 3 + pb.c];
        s = e1 * e1 + e2 * e2;
    }
    return sqrt(s);
}

template <int K>
__device__ __forceinline__ long long qcost(const float (&x)[K], const float (&y)[K], float scale)
{
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < K; ++d) {
        const float e = x[d] - y[d];
        s = fmaf(e, e, s);
    }
    return __float2ll_rn(sqrtf(s) * scale);
}

// One problem per warp.  Shared memory per warp: row atoms X [L][K] (FP32), row potentials
// u [L], matched row of each column p [L + 1] (slot L: the virtual column of the row being
// inserted) and the predecessor column way [L].
template <int K>
__global__ void __launch_bounds__(32 * kPairWarps) k_w1_pairs(const double* __restrict__ A, int MA,
                                                              const double* __restrict__ B, int MB, int G, int L,
                                                              int ncomp, int64_t nprob, double* __restrict__ per)
{
    __shared__ float sX[kPairWarps][kPairMaxL][K];
    __shared__ long long su[kPairWarps][kPairMaxL];
    __shared__ int sp[kPairWarps][kPairMaxL + 1];
    __shared__ int sway[kPairWarps][kPairMaxL];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float(*X)[K] = sX[w];
    long long* u = su[w];
    int* p = sp[w];
    int* way = sway[w];
    const int ra = L / MA, rb = L / MB;  // repetitions of each atom
    const int VIRT = L;
    for (int64_t prob = (int64_t)blockIdx.x * kPairWarps + w; prob < nprob; prob += (int64_t)gridDim.x * kPairWarps) {
        PairProblem pb;
        pair_of(prob / ncomp, G, pb.i, pb.j);
        pb.c = (int)(prob % ncomp);
        // The costs depend on differences only: atoms are taken relative to the mean of both
        // ensembles' atoms (in FP64), so that their FP32 values resolve the spread of the
        // ensembles rather than the magnitude of the velocity.
        double cen[K];
#pragma unroll
        for (int d = 0; d < K; ++d) cen[d] = 0.0;
        for (int m = lane; m < MA; m += 32) {
            double x[K];
            atom64<K>(A, G, m, pb, x);
#pragma unroll
            for (int d = 0; d < K; ++d) cen[d] += x[d] / MA;
        }
        for (int m = lane; m < MB; m += 32) {
            double x[K];
            atom64<K>(B, G, m, pb, x);
#pragma unroll
            for (int d = 0; d < K; ++d) cen[d] += x[d] / MB;
        }
#pragma unroll
        for (int d = 0; d < K; ++d) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) cen[d] += __shfl_xor_sync(0xffffffffu, cen[d], off);
            cen[d] *= 0.5;
        }
        // rows: atoms of A (row r is sample r / ra); columns: atoms of B (column s is sample s / rb)
        float amax = 0.f;
        for (int r = lane; r < L; r += 32) {
            double x[K];
            atom64<K>(A, G, r / ra, pb, x);
#pragma unroll
            for (int d = 0; d < K; ++d) {
                X[r][d] = (float)(x[d] - cen[d]);
                amax = fmaxf(amax, fabsf(X[r][d]));
            }
            u[r] = 0;
        }
        float y[2][K];
        long long v[2], minv[2];
        bool used[2], mine[2];
        int col[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            col[q] = lane + 32 * q;
            mine[q] = col[q] < L;
            if (mine[q]) {
                double x[K];
                atom64<K>(B, G, col[q] / rb, pb, x);
#pragma unroll
                for (int d = 0; d < K; ++d) {
                    y[q][d] = (float)(x[d] - cen[d]);
                    amax = fmaxf(amax, fabsf(y[q][d]));
                }
            }
            v[q] = 0;
            if (mine[q]) p[col[q]] = -1;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        // fixed-point unit: costs are at most 2 sqrt(K) amax; 2^40 units for that bound leaves
        // room for the potentials (sums of at most L costs) in 64 bits
        const float scale = amax > 0.f ? 1099511627776.0f / (2.0f * sqrtf((float)K) * amax) : 1.0f;
        __syncwarp();
        for (int i = 0; i < L; ++i) {
            if (lane == 0) p[VIRT] = i;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                minv[q] = kInf;
                used[q] = false;
            }
            __syncwarp();
            int j0 = VIRT;
            bool found = false;  // a free column was reached (always within i + 1 scans)
            for (int guard = 0; guard <= L; ++guard) {
                const int i0 = p[j0];
                const long long ui0 = u[i0];
                long long best = kInf;
                int bj = VIRT;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (mine[q] && !used[q]) {
                        float x[K];
#pragma unroll
                        for (int d = 0; d < K; ++d) x[d] = X[i0][d];
                        const long long cur = qcost<K>(x, y[q], scale) - ui0 - v[q];
                        if (cur < minv[q]) {
                            minv[q] = cur;
                            way[col[q]] = j0;
                        }
                        if (minv[q] < best || (minv[q] == best && col[q] < bj)) {
                            best = minv[q];
                            bj = col[q];
                        }
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
                    const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
                    if (ob < best || (ob == best && oj < bj)) {
                        best = ob;
                        bj = oj;
                    }
                }
                const long long delta = best;
                // potentials: used columns (and the virtual column) raise the potential of their
                // row, the others lower their reduced distance
                if (lane == 0) u[i] += delta;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (!mine[q]) continue;
                    if (used[q]) {
                        u[p[col[q]]] += delta;
                        v[q] -= delta;
                    } else {
                        minv[q] -= delta;
                    }
                }
                __syncwarp();
                j0 = bj;
                if (j0 >= VIRT) break;
                if (p[j0] < 0) {
                    found = true;
                    break;
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    if (col[q] == j0) used[q] = true;
            }
            __syncwarp();
            // augment along the predecessor columns back to the virtual column
            if (lane == 0 && found) {
                int jj = j0;
                for (int guard = 0; guard <= L && jj != VIRT; ++guard) {
                    const int j1 = way[jj];
                    p[jj] = p[j1];
                    jj = j1;
                }
            }
            __syncwarp();
        }
        // W1 of the problem: mean FP64 cost of the matched pairs
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (mine[q] && p[col[q]] >= 0) s += cost64<K>(A, B, G, p[col[q]] / ra, col[q] / rb, pb);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) per[prob] = s / L;
        __syncwarp();
    }
}

// Fixed-order total: per-block partial sums of w_k D_k over contiguous chunks, then one thread.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_pair_partials(const double* __restrict__ per, int G, int ncomp,
                                                               int64_t nprob, int64_t chunk, double* __restrict__ partial)
{
    __shared__ double sh[kSumThreads];
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < nprob ? lo + chunk : nprob;
    double acc = 0.0;
    for (int64_t t = lo + threadIdx.x; t < hi; t += kSumThreads) {
        int i, j;
        pair_of(t / ncomp, G, i, j);
        acc += (i == j ? 1.0 : 2.0) * per[t];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kSumThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_pair_total(const double* __restrict__ partial, int nparts, double scale, double* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += partial[b];
        out[0] = s * scale;
    }
}

constexpr int kPairParts = 256;

int gcd_int(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace

size_t w1_pair_work_bytes(int G, int vector)
{
    const int64_t npairs = (int64_t)G * (G + 1) / 2;
    return ((size_t)npairs * (vector ? 1 : 3) + kPairParts + 32) * sizeof(double);
}

}  // namespace mclbm

using namespace mclbm;

extern "C" {

size_t mclbm_w1_2pt_work_bytes(int32_t G, int32_t vector)
{
    return G < 1 ? 0 : w1_pair_work_bytes(G, vector);
}

int mclbm_w1_2pt(const double* d_a, int32_t MA, const double* d_b, int32_t MB, int32_t G, int32_t vector, void* d_work,
                 size_t work_bytes, void* cuda_stream, double* W, double* d_per_pair)
{
    if (!d_a || !d_b || !d_work || !W || MA < 1 || MB < 1 || G < 1 || (vector != 0 && vector != 1))
        return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    const int g = gcd_int(MA, MB);
    const int64_t L = (int64_t)MA / g * MB;
    if (L > kPairMaxL)
        return set_error(MCLBM_ERR_SHAPE, "lcm(MA, MB) = " + std::to_string(L) + " exceeds " +
                                              std::to_string(kPairMaxL) + " atoms per side");
    if (work_bytes < w1_pair_work_bytes(G, vector))
        return set_error(MCLBM_ERR_OOM, "work buffer needs " + std::to_string(w1_pair_work_bytes(G, vector)) + " bytes");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int ncomp = vector ? 1 : 3;
    const int64_t nprob = (int64_t)G * (G + 1) / 2 * ncomp;
    double* per = d_per_pair ? d_per_pair : (double*)d_work;
    double* partial = (double*)d_work + nprob;
    double* total = partial + kPairParts;
    int dev = 0, sms = 0;
    MCLBM_CUDA(cudaGetDevice(&dev));
    MCLBM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (nprob + kPairWarps - 1) / kPairWarps;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (vector)
        k_w1_pairs<6><<<(unsigned)blocks, 32 * kPairWarps, 0, s>>>(d_a, MA, d_b, MB, G, (int)L, ncomp, nprob, per);
    else
        k_w1_pairs<2><<<(unsigned)blocks, 32 * kPairWarps, 0, s>>>(d_a, MA, d_b, MB, G, (int)L, ncomp, nprob, per);
    const int64_t chunk = (nprob + kPairParts - 1) / kPairParts;
    k_pair_partials<<<kPairParts, kSumThreads, 0, s>>>(per, G, ncomp, nprob, chunk, partial);
    k_pair_total<<<1, 32, 0, s>>>(partial, kPairParts, 1.0 / ((double)G * G), total);
    MCLBM_CUDA(cudaGetLastError());
    MCLBM_CUDA(cudaMemcpyAsync(W, total, sizeof(double), cudaMemcpyDeviceToHost, s));
    MCLBM_CUDA(cudaStreamSynchronize(s));
    return MCLBM_OK;
}

}  // extern "C"
