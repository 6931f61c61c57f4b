// Two-point 1-Wasserstein distances between the laws of two ensembles on the restriction
// grid: W_{1,2}^v of Eq. (W1_vector) / Algorithm "WassersteinDistance2_vector" (atoms
// (u(x_i), u(x_j)) in R^6) and the component-wise W_{1,2} of Algorithm
// "WassersteinDistance2" (atoms (u_c(x_i), u_c(x_j)) in R^2 for each component c), with
// the Euclidean ground metric, for every point pair i <= j; pairs with i != j count twice
// and the sum is divided by G^2.
//
// Each pair (and component) is one exact optimal-transport problem between two uniform
// empirical measures of M_A and M_B atoms.  Costs are the Euclidean distances of the FP32 atoms
// (taken relative to the atoms' mean) in fixed point (2^40 units for the largest possible cost),
// so that potentials and reduced costs are exact integers and the plan found is optimal for those
// costs; the distance of the problem is then the FP64 cost of that plan, recomputed from the FP64
// atoms.  Two solvers:
//
//  - L = lcm(M_A, M_B) <= 64: repeating every atom of A L / M_A times and every atom of B L / M_B
//    times gives uniform weights 1/L on both sides without changing the optimum, and an optimal
//    plan is then a permutation: one warp solves the L x L assignment problem with the
//    shortest-augmenting-path (Hungarian) method, each lane owning columns lane and lane + 32.
//  - otherwise (M_A, M_B <= 1024): one block solves the transportation problem directly, with
//    g = gcd(M_A, M_B), integer supply M_B / g at every atom of A and demand M_A / g at every atom
//    of B (the plan pi = x / (M_A M_B / g)), by successive shortest paths: rows (atoms of A) are
//    inserted one at a time, and each insertion ships the row's supply along shortest paths of
//    reduced costs (Dijkstra over the columns, with the rows that ship to a reached column reached
//    through its flow at no reduced cost), updating the potentials after each path.  Equal sample
//    counts are assignment problems again (supply and demand 1): the matching is kept in shared
//    memory.  Otherwise the integer flows x_ij (at most min(supply, demand) <= 1024, 16 bits) are
//    kept in a column-major matrix in the work buffer, one per block in flight.
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

// ---- transportation problems beyond the warp kernel: one block per problem -----------------
constexpr int kTpMaxM = 1024;          // atoms per side
constexpr int kTpThreads = 256;        // threads per block
constexpr int kTpWarps = kTpThreads / 32;
constexpr int kTpGeneralBlocks = 256;  // blocks in flight for unequal sample counts (one flow matrix each)

// Shared-memory layout of one block: 8-byte arrays first, then 4-byte, then bytes.
struct TpLayout {
    int u, v, dcol, drow;           // long long [MA], [MB], [MB], [MA]: potentials, distances
    int X, Y;                       // float [MA][K], [MB][K]: atoms relative to the mean
    int predc, predr, dem, pcol, newr;  // int [MB], [MA], [MB], [MB], [MA]
    int used, reached;              // unsigned char [MB], [MA]
    int red;                        // scratch: long long [kTpWarps] + int [kTpWarps] + scalars
    int total;
};

__host__ __device__ inline int tp_align(int x) { return (x + 15) & ~15; }

__host__ __device__ inline TpLayout tp_layout(int MA, int MB, int K)
{
    TpLayout L;
    int o = 0;
    L.u = o; o = tp_align(o + 8 * MA);
    L.v = o; o = tp_align(o + 8 * MB);
    L.dcol = o; o = tp_align(o + 8 * MB);
    L.drow = o; o = tp_align(o + 8 * MA);
    L.X = o; o = tp_align(o + 4 * MA * K);
    L.Y = o; o = tp_align(o + 4 * MB * K);
    L.predc = o; o = tp_align(o + 4 * MB);
    L.predr = o; o = tp_align(o + 4 * MA);
    L.dem = o; o = tp_align(o + 4 * MB);
    L.pcol = o; o = tp_align(o + 4 * MB);
    L.newr = o; o = tp_align(o + 4 * MA);
    L.used = o; o = tp_align(o + MB);
    L.reached = o; o = tp_align(o + MA);
    L.red = o; o = tp_align(o + 8 * kTpWarps * (6 + 1) + 4 * kTpWarps + 64);
    L.total = o;
    return L;
}

// Block-wide sum of one double per thread (fixed order: warp trees, then warp 0 over the warps).
__device__ __forceinline__ double tp_block_sum(double x, double* scratch)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    __syncthreads();
    if (lane == 0) scratch[w] = x;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < kTpWarps; ++k) t += scratch[k];
    return t;
}

// Block-wide minimum of (value, index) pairs, ties to the smaller index; every thread gets it.
__device__ __forceinline__ void tp_block_argmin(long long& best, int& bj, long long* sv, int* si)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
        if (ob < best || (ob == best && oj < bj)) {
            best = ob;
            bj = oj;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sv[w] = best;
        si[w] = bj;
    }
    __syncthreads();
    best = sv[0];
    bj = si[0];
    for (int k = 1; k < kTpWarps; ++k)
        if (sv[k] < best || (sv[k] == best && si[k] < bj)) {
            best = sv[k];
            bj = si[k];
        }
}

// One transportation problem per block (grid-strided over the problems).  MATCH: equal sample
// counts (supply = demand = 1), matching in shared memory; otherwise the block's flow matrix
// flowT [MB][MA] (column-major: the rows shipping to one column are contiguous).  err: set to 1
// if a shortest-path search ends without reaching a column with open demand (it cannot while the
// total supply equals the total demand; the check keeps every loop bounded).
template <int K, bool MATCH>
__global__ void __launch_bounds__(kTpThreads, 2) k_w1_transport(const double* __restrict__ A, int MA,
                                                             const double* __restrict__ B, int MB, int G, int ncomp,
                                                             int64_t nprob, int supply, int demand,
                                                             unsigned short* __restrict__ flows,
                                                             double* __restrict__ per, int* __restrict__ err)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    const TpLayout Lo = tp_layout(MA, MB, K);
    long long* u = reinterpret_cast<long long*>(tsm + Lo.u);
    long long* v = reinterpret_cast<long long*>(tsm + Lo.v);
    long long* dcol = reinterpret_cast<long long*>(tsm + Lo.dcol);
    long long* drow = reinterpret_cast<long long*>(tsm + Lo.drow);
    float* X = reinterpret_cast<float*>(tsm + Lo.X);
    float* Y = reinterpret_cast<float*>(tsm + Lo.Y);
    int* predc = reinterpret_cast<int*>(tsm + Lo.predc);
    int* predr = reinterpret_cast<int*>(tsm + Lo.predr);
    int* dem = reinterpret_cast<int*>(tsm + Lo.dem);
    int* pcol = reinterpret_cast<int*>(tsm + Lo.pcol);
    int* newr = reinterpret_cast<int*>(tsm + Lo.newr);
    unsigned char* used = tsm + Lo.used;
    unsigned char* reached = tsm + Lo.reached;
    long long* sv = reinterpret_cast<long long*>(tsm + Lo.red);
    double* sd = reinterpret_cast<double*>(sv + kTpWarps);
    int* si = reinterpret_cast<int*>(sd + 6 * kTpWarps);
    int* s_nnew = si + kTpWarps;
    int* s_sup = s_nnew + 1;
    int* s_fail = s_sup + 1;
    const int tid = threadIdx.x;
    // each block's matrix starts on a 16-byte boundary (its zeroing writes whole 16-byte words)
    const size_t fstride = ((size_t)MA * MB + 7) / 8 * 8;
    unsigned short* flowT = MATCH ? nullptr : flows + (size_t)blockIdx.x * fstride;
    const long long total_flow = MATCH ? MA : (long long)MA * supply;

    for (int64_t prob = blockIdx.x; prob < nprob; prob += gridDim.x) {
        PairProblem pb;
        pair_of(prob / ncomp, G, pb.i, pb.j);
        pb.c = (int)(prob % ncomp);
        // atoms relative to the mean of both ensembles' atoms (FP64), as in the warp kernel
        double cen[K];
#pragma unroll
        for (int d = 0; d < K; ++d) cen[d] = 0.0;
        for (int m = tid; m < MA; m += kTpThreads) {
            double x[K];
            atom64<K>(A, G, m, pb, x);
#pragma unroll
            for (int d = 0; d < K; ++d) cen[d] += x[d] / MA;
        }
        for (int m = tid; m < MB; m += kTpThreads) {
            double x[K];
            atom64<K>(B, G, m, pb, x);
#pragma unroll
            for (int d = 0; d < K; ++d) cen[d] += x[d] / MB;
        }
#pragma unroll
        for (int d = 0; d < K; ++d) cen[d] = 0.5 * tp_block_sum(cen[d], sd + d * kTpWarps);
        float amax = 0.f;
        for (int m = tid; m < MA; m += kTpThreads) {
            double x[K];
            atom64<K>(A, G, m, pb, x);
#pragma unroll
            for (int d = 0; d < K; ++d) {
                X[m * K + d] = (float)(x[d] - cen[d]);
                amax = fmaxf(amax, fabsf(X[m * K + d]));
            }
            u[m] = 0;
        }
        for (int m = tid; m < MB; m += kTpThreads) {
            double x[K];
            atom64<K>(B, G, m, pb, x);
#pragma unroll
            for (int d = 0; d < K; ++d) {
                Y[m * K + d] = (float)(x[d] - cen[d]);
                amax = fmaxf(amax, fabsf(Y[m * K + d]));
            }
            v[m] = 0;
            dem[m] = demand;
            pcol[m] = -1;
        }
        if (!MATCH) {
            uint4* f4 = reinterpret_cast<uint4*>(flowT);
            const size_t n4 = fstride / 8;
            for (size_t k = tid; k < n4; k += kTpThreads) f4[k] = make_uint4(0, 0, 0, 0);
        }
        {
            // fixed-point unit: 2^40 for the largest possible cost 2 sqrt(K) amax
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
            __syncthreads();
            if ((tid & 31) == 0) sd[tid >> 5] = amax;
            __syncthreads();
            for (int k = 0; k < kTpWarps; ++k) amax = fmaxf(amax, (float)sd[k]);
        }
        const float scale = amax > 0.f ? 1099511627776.0f / (2.0f * sqrtf((float)K) * amax) : 1.0f;
        if (tid == 0) *s_fail = 0;
        __syncthreads();

        for (int r0 = 0; r0 < MA; ++r0) {
            if (tid == 0) *s_sup = supply;
            __syncthreads();
            // each pass ships at least one unit of the row's supply
            for (int pass = 0; pass < supply && *s_sup > 0; ++pass) {
                for (int j = tid; j < MB; j += kTpThreads) {
                    dcol[j] = kInf;
                    used[j] = 0;
                }
                for (int i = tid; i < MA; i += kTpThreads) reached[i] = 0;
                __syncthreads();
                if (tid == 0) {
                    reached[r0] = 1;
                    drow[r0] = 0;
                    newr[0] = r0;
                    *s_nnew = 1;
                }
                __syncthreads();
                long long dstar = 0;
                int jstar = -1;
                bool found = false;
                for (int it = 0; it <= MB; ++it) {
                    // relax the columns from the rows reached in the last step (ties to the
                    // smaller row, so that the tree does not depend on the order of the list)
                    const int nn = *s_nnew;
                    for (int q = 0; q < nn; ++q) {
                        const int i = newr[q];
                        const long long base = drow[i] - u[i];
                        float xi[K];
#pragma unroll
                        for (int d = 0; d < K; ++d) xi[d] = X[i * K + d];
                        for (int j = tid; j < MB; j += kTpThreads) {
                            if (used[j]) continue;
                            float yj[K];
#pragma unroll
                            for (int d = 0; d < K; ++d) yj[d] = Y[j * K + d];
                            const long long cand = base + qcost<K>(xi, yj, scale) - v[j];
                            if (cand < dcol[j] || (cand == dcol[j] && i < predc[j])) {
                                dcol[j] = cand;
                                predc[j] = i;
                            }
                        }
                    }
                    long long best = kInf;
                    int bj = 0x7fffffff;
                    for (int j = tid; j < MB; j += kTpThreads)
                        if (!used[j] && (dcol[j] < best || (dcol[j] == best && j < bj))) {
                            best = dcol[j];
                            bj = j;
                        }
                    tp_block_argmin(best, bj, sv, si);
                    if (bj >= MB || best >= kInf) break;  // nothing reachable: failure, reported below
                    jstar = bj;
                    dstar = best;
                    if (dem[jstar] > 0) {
                        found = true;
                        break;
                    }
                    __syncthreads();  // every thread has read the search state
                    if (tid == 0) {
                        used[jstar] = 1;
                        *s_nnew = 0;
                    }
                    __syncthreads();
                    // the rows that ship to jstar are reached through their flow at no reduced cost
                    if (MATCH) {
                        if (tid == 0) {
                            const int i = pcol[jstar];
                            if (i >= 0 && !reached[i]) {
                                reached[i] = 1;
                                drow[i] = dstar;
                                predr[i] = jstar;
                                newr[0] = i;
                                *s_nnew = 1;
                            }
                        }
                    } else {
                        const unsigned short* fc = flowT + (size_t)jstar * MA;
                        for (int i = tid; i < MA; i += kTpThreads)
                            if (fc[i] > 0 && !reached[i]) {
                                reached[i] = 1;
                                drow[i] = dstar;
                                predr[i] = jstar;
                                newr[atomicAdd(s_nnew, 1)] = i;
                            }
                    }
                    __syncthreads();
                }
                if (!found) {
                    if (tid == 0) {
                        *s_fail = 1;
                        *s_sup = 0;
                    }
                    __syncthreads();
                    break;
                }
                // potentials: reached rows u += d* - d(row), used columns v -= d* - d(column)
                for (int i = tid; i < MA; i += kTpThreads)
                    if (reached[i]) u[i] += dstar - drow[i];
                for (int j = tid; j < MB; j += kTpThreads)
                    if (used[j]) v[j] -= dstar - dcol[j];
                __syncthreads();
                // augment along the path back to r0 (one thread; at most min(MA, MB) + 1 steps)
                if (tid == 0) {
                    int b = *s_sup < dem[jstar] ? *s_sup : dem[jstar];
                    if (MATCH) {
                        b = 1;
                        int j = jstar;
                        for (int guard = 0; guard <= MB; ++guard) {
                            const int i = predc[j];
                            const int jp = i == r0 ? -1 : predr[i];
                            pcol[j] = i;
                            if (i == r0) break;
                            j = jp;
                        }
                    } else {
                        int j = jstar;
                        for (int guard = 0; guard <= MB; ++guard) {  // bottleneck of the reverse edges
                            const int i = predc[j];
                            if (i == r0) break;
                            const int jp = predr[i];
                            const int f = flowT[(size_t)jp * MA + i];
                            if (f < b) b = f;
                            j = jp;
                        }
                        j = jstar;
                        for (int guard = 0; guard <= MB; ++guard) {
                            const int i = predc[j];
                            flowT[(size_t)j * MA + i] += (unsigned short)b;
                            if (i == r0) break;
                            const int jp = predr[i];
                            flowT[(size_t)jp * MA + i] -= (unsigned short)b;
                            j = jp;
                        }
                    }
                    dem[jstar] -= b;
                    *s_sup -= b;
                }
                __syncthreads();
            }
        }
        // W1 of the problem: the FP64 cost of the plan, sum x_ij c_ij / (total flow)
        double s = 0.0;
        if (MATCH) {
            for (int j = tid; j < MB; j += kTpThreads)
                if (pcol[j] >= 0) s += cost64<K>(A, B, G, pcol[j], j, pb);
        } else {
            const size_t n = (size_t)MA * MB;
            for (size_t k = tid; k < n; k += kTpThreads) {
                const int f = flowT[k];
                if (f > 0) s += f * cost64<K>(A, B, G, (int)(k % MA), (int)(k / MA), pb);
            }
        }
        s = tp_block_sum(s, sd);
        if (tid == 0) {
            per[prob] = s / (double)total_flow;
            if (*s_fail) atomicExch(err, 1);
        }
        __syncthreads();
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

// Work buffer: per-problem values [nprob], partial sums [kPairParts], the total and an error
// word, then (unequal sample counts beyond the warp kernel) one flow matrix per block in flight.
struct PairWork {
    size_t per, partial, total, err, flows, bytes;
};

PairWork pair_work(int MA, int MB, int G, int vector)
{
    const int64_t nprob = (int64_t)G * (G + 1) / 2 * (vector ? 1 : 3);
    PairWork w;
    w.per = 0;
    w.partial = (size_t)nprob * sizeof(double);
    w.total = w.partial + kPairParts * sizeof(double);
    w.err = w.total + 32 * sizeof(double);
    w.flows = (w.err + 16 + 255) / 256 * 256;
    const int g = gcd_int(MA, MB);
    const int64_t L = (int64_t)MA / g * MB;
    const bool general = L > kPairMaxL && MA != MB;
    const size_t fstride = ((size_t)MA * MB + 7) / 8 * 8;  // elements per block, as in the kernel
    w.bytes = w.flows + (general ? (size_t)kTpGeneralBlocks * fstride * sizeof(unsigned short) : 0);
    return w;
}

}  // namespace mclbm

using namespace mclbm;

extern "C" {

size_t mclbm_w1_2pt_work_bytes(int32_t MA, int32_t MB, int32_t G, int32_t vector)
{
    if (G < 1 || MA < 1 || MB < 1 || MA > kTpMaxM || MB > kTpMaxM) return 0;
    return pair_work(MA, MB, G, vector).bytes;
}

int mclbm_w1_2pt(const double* d_a, int32_t MA, const double* d_b, int32_t MB, int32_t G, int32_t vector, void* d_work,
                 size_t work_bytes, void* cuda_stream, double* W, double* d_per_pair)
{
    if (!d_a || !d_b || !d_work || !W || MA < 1 || MB < 1 || G < 1 || (vector != 0 && vector != 1))
        return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    if (MA > kTpMaxM || MB > kTpMaxM)
        return set_error(MCLBM_ERR_SHAPE, "sample counts " + std::to_string(MA) + ", " + std::to_string(MB) +
                                              " exceed " + std::to_string(kTpMaxM) + " per ensemble");
    const int g = gcd_int(MA, MB);
    const int64_t L = (int64_t)MA / g * MB;
    const PairWork pw = pair_work(MA, MB, G, vector);
    if (work_bytes < pw.bytes)
        return set_error(MCLBM_ERR_OOM, "work buffer needs " + std::to_string(pw.bytes) + " bytes");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int ncomp = vector ? 1 : 3;
    const int64_t nprob = (int64_t)G * (G + 1) / 2 * ncomp;
    char* wb = (char*)d_work;
    double* per = d_per_pair ? d_per_pair : (double*)(wb + pw.per);
    double* partial = (double*)(wb + pw.partial);
    double* total = (double*)(wb + pw.total);
    int* err = (int*)(wb + pw.err);
    int dev = 0, sms = 0;
    MCLBM_CUDA(cudaGetDevice(&dev));
    MCLBM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (L <= kPairMaxL) {
        int64_t blocks = (nprob + kPairWarps - 1) / kPairWarps;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        if (vector)
            k_w1_pairs<6><<<(unsigned)blocks, 32 * kPairWarps, 0, s>>>(d_a, MA, d_b, MB, G, (int)L, ncomp, nprob, per);
        else
            k_w1_pairs<2><<<(unsigned)blocks, 32 * kPairWarps, 0, s>>>(d_a, MA, d_b, MB, G, (int)L, ncomp, nprob, per);
        MCLBM_CUDA(cudaGetLastError());
    } else {
        const bool match = MA == MB;
        const int K = vector ? 6 : 2;
        const int smem = tp_layout(MA, MB, K).total;
        const int supply = MB / g, demand = MA / g;
        unsigned short* flows = match ? nullptr : (unsigned short*)(wb + pw.flows);
        MCLBM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        auto launch = [&](auto kernel) -> cudaError_t {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTpThreads, smem);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            int64_t blocks = (int64_t)sms * per_sm;
            if (!match && blocks > kTpGeneralBlocks) blocks = kTpGeneralBlocks;
            if (blocks > nprob) blocks = nprob;
            kernel<<<(unsigned)blocks, kTpThreads, smem, s>>>(d_a, MA, d_b, MB, G, ncomp, nprob, supply, demand, flows,
                                                              per, err);
            return cudaGetLastError();
        };
        cudaError_t e;
        if (vector)
            e = match ? launch(k_w1_transport<6, true>) : launch(k_w1_transport<6, false>);
        else
            e = match ? launch(k_w1_transport<2, true>) : launch(k_w1_transport<2, false>);
        MCLBM_CUDA(e);
    }
    const int64_t chunk = (nprob + kPairParts - 1) / kPairParts;
    k_pair_partials<<<kPairParts, kSumThreads, 0, s>>>(per, G, ncomp, nprob, chunk, partial);
    k_pair_total<<<1, 32, 0, s>>>(partial, kPairParts, 1.0 / ((double)G * G), total);
    MCLBM_CUDA(cudaGetLastError());
    int h_err = 0;
    MCLBM_CUDA(cudaMemcpyAsync(W, total, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (L > kPairMaxL) MCLBM_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MCLBM_CUDA(cudaStreamSynchronize(s));
    if (h_err)
        return set_error(MCLBM_ERR_NONFINITE, "a transport search found no column with open demand (non-finite atoms?)");
    return MCLBM_OK;
}

}  // extern "C"
