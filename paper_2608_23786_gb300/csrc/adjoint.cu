// Discrete adjoint of the ensemble time stepping: gradients of the per-sample kinetic
// energy or enstrophy at step T with respect to the 24 initial-uncertainty parameters
// (Eq. (alpha_perturbation)) of every sample.
//
// Forward:  f^{t+1} = S(C(f^t)), S the streaming permutation (Eq. (lbIteration)),
//           C the per-node KBC collision.
// Reverse:  lambda^T = dJ/df^T;  lambda^t_i(x) = [dC(f^t(x))]^T mu(x),
//           mu_i(x) = lambda^{t+1}_i(x + c_i)   (the transpose of streaming);
// Params:   dJ/dX = sum_x (df^0(x)/du_0)(du_0/dX) . lambda^0(x), with
//           f^0 = f^eq(rho_0, u_0), u_0 = (U_lat/U_c)(u_det + s(X)), s linear in X.
// Storage:  checkpoints of the whole lattice every K steps, and for the segment being
//           reversed the K - 1 intermediate lattices recomputed from its checkpoint
//           (states cannot all be kept).  lambda is kept in natural layout
//           [sample][i][node] in the arithmetic of the stepper (FP32 or FP64).
#include <cuda_fp16.h>

#include <string>
#include <vector>

#include "adjoint.cuh"
#include "internal.h"
#include "stepper_async.cuh"
#include "stepper_impl.cuh"

namespace mclbm {

cudaError_t launch_pull_explicit(mclbm_ctx* c, const void* src, void* dst);  // stepper.cu

namespace {

constexpr int kBlock = 128;
constexpr int kGradChunks = 64;  // blocks per sample in the parameter reduction

__device__ __forceinline__ void xyz(const Geom& g, int64_t node, int& x, int& y, int& z)
{
    x = (int)(node & (g.N - 1));
    y = (int)((node >> g.logN) & (g.N - 1));
    z = (int)(node >> (2 * g.logN));
}

// normalised deviation h_i of the pre-collision population f_i(x) of a pull-layout lattice
template <class E, class C>
__device__ __forceinline__ C load_h(const E* sample, const Geom& g, int i, int x, int y, int z)
{
    const E v = sample[pre_loc(g, kPull, 0, i, x, y, z)];
    if constexpr (Storage<E>::shifted)
        return (C)to_c<E>(v);
    else
        return (C)(v / weight<double>(i) - 1.0);
}

template <class E, class C>
__global__ void __launch_bounds__(kBlock) k_adjoint_step(const E* __restrict__ state, const C* __restrict__ lam_next,
                                                         C* __restrict__ lam_out, Geom g, int M, C omega, C guard)
{
    const int64_t total = (int64_t)M * g.n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(idx >> (3 * g.logN));
        const int64_t node = idx & (g.n - 1);
        int x, y, z;
        xyz(g, node, x, y, z);
        const E* sample = state + (int64_t)m * Q * g.n;
        const C* ln = lam_next + (int64_t)m * Q * g.n;
        C h[Q], mu[Q], lam[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            h[i] = load_h<E, C>(sample, g, i, x, y, z);
            mu[i] = ln[(int64_t)i * g.n + g.node(g.wrap(x + cx(i)), g.wrap(y + cy(i)), g.wrap(z + cz(i)))];
        }
        kbc_vjp<C>(h, mu, omega, guard, lam);
        C* lo = lam_out + (int64_t)m * Q * g.n;
#pragma unroll
        for (int i = 0; i < Q; ++i) lo[(int64_t)i * g.n + node] = lam[i];
    }
}

// Threads per block of the FP32 adjoint kernel.  It works on runs of VEC consecutive x-nodes
// with the thread mapping and x-shift shuffles of the forward stepper; runs = M N^3 / VEC is a
// multiple of 32, so warps stay whole.
constexpr int kRunBlock = 128;

// Shared-memory ring of the adjoint run kernel: per stage, the Q state vectors, the Q lambda^{t+1}
// vectors and the edge words (state and lambda, x-moving populations only) of every thread.
// WRAP: every x-row lies within one warp (N <= 32 VEC), the periodic neighbours of a row's end
// runs are in the same warp, and the ring holds no edge words.
template <class E, int VEC, int STAGES, bool WRAP>
struct AdjRing {
    static constexpr int kVS = VEC * (int)sizeof(E), kVL = VEC * 4;
    static constexpr int kStateBytes = STAGES * Q * kRunBlock * kVS;
    static constexpr int kLamBytes = STAGES * Q * kRunBlock * kVL;
    static constexpr int kBytes = kStateBytes + kLamBytes + (WRAP ? 0 : STAGES * 2 * kEdges * kRunBlock * 4);
    __device__ __forceinline__ static int state_off(int stage, int i, int tid) { return ((stage * Q + i) * kRunBlock + tid) * kVS; }
    __device__ __forceinline__ static int lam_off(int stage, int i, int tid)
    {
        return kStateBytes + ((stage * Q + i) * kRunBlock + tid) * kVL;
    }
    __device__ __forceinline__ static int edge_off(int stage, int which, int i, int tid)
    {
        return kStateBytes + kLamBytes + (((stage * 2 + which) * kEdges + edge_index(i)) * kRunBlock + tid) * 4;
    }
};

struct RunPos {
    int m, x0, y, z;
    int64_t node;
};

__device__ __forceinline__ RunPos run_pos(const Geom& g, int64_t t, int vec)
{
    RunPos r;
    const int64_t first = t * vec;
    r.m = (int)(first >> (3 * g.logN));
    r.node = first & (g.n - 1);
    r.x0 = (int)(r.node & (g.N - 1));
    r.y = (int)((r.node >> g.logN) & (g.N - 1));
    r.z = (int)(r.node >> (2 * g.logN));
    return r;
}

// Issue the copies of one run: state f_i(x) from slot i of x - c_i, lambda^{t+1} from slot i of x + c_i.
template <class E, int VEC, int STAGES, bool WRAP, int I = 0>
__device__ __forceinline__ void adj_issue(const E* sbase, const float* lbase, const Geom& g, const RunPos& p, int lane,
                                          uint32_t smem, int stage)
{
    if constexpr (I < Q) {
        using Ring = AdjRing<E, VEC, STAGES, WRAP>;
        const int tid = threadIdx.x;
        const E* srow = sbase + (int64_t)I * g.n + g.node(0, g.wrap(p.y - Dir<I>::y), g.wrap(p.z - Dir<I>::z));
        const float* lrow = lbase + (int64_t)I * g.n + g.node(0, g.wrap(p.y + Dir<I>::y), g.wrap(p.z + Dir<I>::z));
        // one 16-byte copy per group of lanes: consecutive lanes hold consecutive runs of the same
        // row in consecutive slots, and the group's first run starts on a 16-byte boundary
        constexpr int kLS = 16 / Ring::kVS, kLL = 16 / Ring::kVL;  // lanes per 16-byte copy
        if (lane % kLS == 0) cp_async<16>(smem + Ring::state_off(stage, I, tid), srow + p.x0);
        if (lane % kLL == 0) cp_async<16>(smem + Ring::lam_off(stage, I, tid), lrow + p.x0);
        const bool first = lane == 0 || p.x0 == 0, last = lane == 31 || p.x0 + VEC == g.N;
        const int before = (p.x0 - 1) & (g.N - 1), after = (p.x0 + VEC) & (g.N - 1);
        if constexpr (WRAP) {
        } else if constexpr (Dir<I>::x > 0) {  // state from x - 1, lambda from x + 1
            if (first) cp_async<4>(smem + Ring::edge_off(stage, 0, I, tid), edge_word(srow, before));
            if (last) cp_async<4>(smem + Ring::edge_off(stage, 1, I, tid), lrow + after);
        } else if constexpr (Dir<I>::x < 0) {  // state from x + 1, lambda from x - 1
            if (last) cp_async<4>(smem + Ring::edge_off(stage, 0, I, tid), edge_word(srow, after));
            if (first) cp_async<4>(smem + Ring::edge_off(stage, 1, I, tid), lrow + before);
        }
        adj_issue<E, VEC, STAGES, WRAP, I + 1>(sbase, lbase, g, p, lane, smem, stage);
    }
}

template <class T, int VEC, int CXI, bool WRAP>
__device__ __forceinline__ RawRun<T, VEC> adj_raw(const unsigned char* smem, int vec_off, int edge_off)
{
    using R = typename RawOf<VEC * sizeof(T)>::type;
    RawRun<T, VEC> r;
    const R w = *reinterpret_cast<const R*>(smem + vec_off);
    memcpy(r.w, &w, sizeof(R));
    if constexpr (CXI != 0 && !WRAP) {
        const unsigned int e = *reinterpret_cast<const unsigned int*>(smem + edge_off);
        if constexpr (sizeof(T) == 2) {  // source x - 1 is odd (high half), x + VEC even (low half)
            const unsigned short hv = CXI > 0 ? (unsigned short)(e >> 16) : (unsigned short)(e & 0xffffu);
            memcpy(&r.edge, &hv, 2);
        } else {
            memcpy(&r.edge, &e, 4);
        }
    }
    return r;
}

// The x-shift of a run when every x-row lies within one warp: a row is L = N / VEC consecutive
// lanes (L divides 32, N being a power of two), and the element before (after) the row's first
// (last) run is the row's last (first) element, read with one shuffle inside the row's lanes.
template <class E, int VEC, int CXI>
__device__ __forceinline__ void finish_row_wrap(const RawRun<E, VEC>& r, int L, int lane,
                                                typename Storage<E>::compute (&v)[VEC])
{
    if constexpr (CXI == 0) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[k] = to_c<E>(r.w[k]);
    } else {
        const int row = lane & ~(L - 1);
        if constexpr (CXI > 0) {
            const E prev = __shfl_sync(0xffffffffu, r.w[VEC - 1], row | ((lane - 1) & (L - 1)));
            v[0] = to_c<E>(prev);
#pragma unroll
            for (int k = 1; k < VEC; ++k) v[k] = to_c<E>(r.w[k - 1]);
        } else {
            const E next = __shfl_sync(0xffffffffu, r.w[0], row | ((lane + 1) & (L - 1)));
#pragma unroll
            for (int k = 0; k < VEC - 1; ++k) v[k] = to_c<E>(r.w[k + 1]);
            v[VEC - 1] = to_c<E>(next);
        }
    }
}

template <class E, int VEC, int STAGES, bool WRAP, int I = 0>
__device__ __forceinline__ void adj_finish(const unsigned char* smem, int stage, const Geom& g, const RunPos& p,
                                           int lane, float (&hv)[Q][VEC], float (&mv)[Q][VEC])
{
    if constexpr (I < Q) {
        using Ring = AdjRing<E, VEC, STAGES, WRAP>;
        const int tid = threadIdx.x;
        const int eo0 = WRAP ? 0 : Ring::edge_off(stage, 0, I, tid), eo1 = WRAP ? 0 : Ring::edge_off(stage, 1, I, tid);
        const RawRun<E, VEC> rs = adj_raw<E, VEC, Dir<I>::x, WRAP>(smem, Ring::state_off(stage, I, tid), eo0);
        const RawRun<float, VEC> rl = adj_raw<float, VEC, -Dir<I>::x, WRAP>(smem, Ring::lam_off(stage, I, tid), eo1);
        if constexpr (WRAP) {
            finish_row_wrap<E, VEC, Dir<I>::x>(rs, g.N / VEC, lane, hv[I]);
            finish_row_wrap<float, VEC, -Dir<I>::x>(rl, g.N / VEC, lane, mv[I]);
        } else {
            finish_row<E, VEC, Dir<I>::x>(rs, p.x0, g.N, lane, hv[I]);
            finish_row<float, VEC, -Dir<I>::x>(rl, p.x0, g.N, lane, mv[I]);
        }
        adj_finish<E, VEC, STAGES, WRAP, I + 1>(smem, stage, g, p, lane, hv, mv);
    }
}

// FP32 adjoint step: gather the pre-collision state (pull layout, shifted storage; f_i(x) from
// slot i of x - c_i) and lambda^{t+1}(x + c_i) (the transpose of pull streaming), apply the paired
// lane-form product to node pairs in packed FP32x2, store lambda^t aligned.  The next run's state
// and lambda^{t+1} are copied into shared memory (cp.async, STAGES - 1 runs ahead) during the
// current run's product; each thread reads back only its own slots after its own wait_group (no
// block barrier, no spin).
template <class E, int VEC, int STAGES, bool WRAP>
__global__ void __launch_bounds__(kRunBlock) k_adjoint_async(const E* __restrict__ state,
                                                             const float* __restrict__ lam_next,
                                                             float* __restrict__ lam_out, Geom g, int64_t runs,
                                                             float omega, float a, float b)
{
    static_assert(VEC == 2, "node pairs");
    // the D3Q27 FP32 transposed collision takes the intrinsic arithmetic (the same bits; its
    // schedule measured 89.5% -> 92.6% of the copy bandwidth for the reverse sweep at 64^3 x 16);
    // the D3Q19 one and the FP16-state kernels keep the assembly form (FP16 state: 85.2% against
    // 82.1% for D3Q19, 89.6% against 82.0% for D3Q27)
    using Arith = std::conditional_t<Q == 27 && std::is_same<E, float>::value, lanes::Native, lanes::Asm>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kRunBlock;
    int64_t t = blockIdx.x * (int64_t)kRunBlock + threadIdx.x;
    if (t >= runs) return;  // whole warps: runs and strides are multiples of 32
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        const int64_t ts = t + s * stride;
        if (ts < runs) {
            const RunPos p = run_pos(g, ts, VEC);
            adj_issue<E, VEC, STAGES, WRAP>(state + (int64_t)p.m * Q * g.n, lam_next + (int64_t)p.m * Q * g.n, g, p,
                                            lane, sbase, s);
        }
        cp_async_commit();
    }
    int stage = 0;
    for (;;) {
        const int64_t ta = t + (int64_t)(STAGES - 1) * stride;
        if (ta < runs) {
            const RunPos p = run_pos(g, ta, VEC);
            int sa = stage + STAGES - 1;
            if (sa >= STAGES) sa -= STAGES;
            adj_issue<E, VEC, STAGES, WRAP>(state + (int64_t)p.m * Q * g.n, lam_next + (int64_t)p.m * Q * g.n, g, p,
                                            lane, sbase, sa);
        }
        cp_async_commit();
        cp_async_wait<STAGES - 1>();
        __syncwarp();  // the copies of the lane groups (issued by their first lanes) are complete
        const RunPos p = run_pos(g, t, VEC);
        float hv[Q][VEC], mv[Q][VEC];
        adj_finish<E, VEC, STAGES, WRAP>(smem, stage, g, p, lane, hv, mv);
        __syncwarp();  // every lane has read this stage before a group's next copy overwrites it
        float2 h2[Q], m2[Q], l2[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            h2[i] = make_float2(hv[i][0], hv[i][1]);
            m2[i] = make_float2(mv[i][0], mv[i][1]);
        }
        kbc_vjp_shifted<float2, Arith>(h2, m2, omega, a, b, l2);
        float* lo = lam_out + (int64_t)p.m * Q * g.n + p.node;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float o[2] = {l2[i].x, l2[i].y};
            vstore<float, 2>(lo + (int64_t)i * g.n, o);
        }
        t += stride;
        if (t >= runs) break;
        stage = stage + 1 == STAGES ? 0 : stage + 1;
    }
    cp_async_wait<0>();
}

// rho and u (lattice units) of f(x) in FP64
template <class E>
__device__ __forceinline__ void moments64(const E* sample, const Geom& g, int x, int y, int z, double& rho, double (&u)[3])
{
    double r = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double f = to_raw<E>(i, sample[pre_loc(g, kPull, 0, i, x, y, z)]);
        r += f;
        j[0] += cx(i) * f;
        j[1] += cy(i) * f;
        j[2] += cz(i) * f;
    }
    rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

// Seed lambda^T = dJ/df^T.  dJ/du_phys(x) is given per node by g_u ([3][n] FP64, one sample) or,
// when g_u is null, is the kinetic-energy derivative u_phys / N^3.  With u_phys = s j / rho:
// dJ/df_q = sum_a dJ/du_phys_a s (c_qa - u_a) / rho.
template <class E, class C>
__global__ void k_seed(const E* __restrict__ state, int sample, const double* __restrict__ g_u, Geom g, double s,
                       C* __restrict__ lam)
{
    const E* smp = state + (int64_t)sample * Q * g.n;
    C* lo = lam + (int64_t)sample * Q * g.n;
    const double invn = 1.0 / (double)g.n;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n; node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        xyz(g, node, x, y, z);
        double rho, u[3];
        moments64<E>(smp, g, x, y, z, rho, u);
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = g_u ? g_u[a * g.n + node] : s * u[a] * invn;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const double v = (d[0] * (cx(q) - u[0]) + d[1] * (cy(q) - u[1]) + d[2] * (cz(q) - u[2])) * s / rho;
            lo[(int64_t)q * g.n + node] = (C)v;
        }
    }
}

// omega = curl u (central differences), u physical [3][n]
__global__ void k_curl(const double* __restrict__ u, double* __restrict__ w, Geom g, double inv2dx, double scale)
{
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n; node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        xyz(g, node, x, y, z);
        const double* ux = u;
        const double* uy = u + g.n;
        const double* uz = u + 2 * g.n;
        const int64_t xp = g.node(g.wrap(x + 1), y, z), xm = g.node(g.wrap(x - 1), y, z);
        const int64_t yp = g.node(x, g.wrap(y + 1), z), ym = g.node(x, g.wrap(y - 1), z);
        const int64_t zp = g.node(x, y, g.wrap(z + 1)), zm = g.node(x, y, g.wrap(z - 1));
        w[node] = ((uz[yp] - uz[ym]) - (uy[zp] - uy[zm])) * inv2dx * scale;
        w[g.n + node] = ((ux[zp] - ux[zm]) - (uz[xp] - uz[xm])) * inv2dx * scale;
        w[2 * g.n + node] = ((uy[xp] - uy[xm]) - (ux[yp] - ux[ym])) * inv2dx * scale;
    }
}

// Parameter gradient partials: per sample and block, 24 sums of
// G_a(x) (U_lat / U_c) / 8 a_i(2x) a_j(2y) a_k(2z),  G_a = sum_q lambda_q d f^eq_q / d u_a.
template <class E, class C>
__global__ void __launch_bounds__(kBlock) k_param_grad(const E* __restrict__ state0, const C* __restrict__ lam0,
                                                       const double* __restrict__ trig, Geom g, double coef,
                                                       double* __restrict__ partial)
{
    __shared__ double sh[24][kBlock / 32];
    const int m = blockIdx.y;
    const E* smp = state0 + (int64_t)m * Q * g.n;
    const C* lm = lam0 + (int64_t)m * Q * g.n;
    double acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0.0;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n; node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        xyz(g, node, x, y, z);
        double rho, u[3];
        moments64<E>(smp, g, x, y, z, rho, u);
        double G[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const double l = (double)lm[(int64_t)q * g.n + node];
            const double cu = cx(q) * u[0] + cy(q) * u[1] + cz(q) * u[2];
            const double rw = rho * weight<double>(q) * l;
            G[0] += rw * (3.0 * cx(q) + 9.0 * cu * cx(q) - 3.0 * u[0]);
            G[1] += rw * (3.0 * cy(q) + 9.0 * cu * cy(q) - 3.0 * u[1]);
            G[2] += rw * (3.0 * cz(q) + 9.0 * cu * cz(q) - 3.0 * u[2]);
        }
        const double ax[2] = {trig[4 * x + 2], trig[4 * x + 3]};
        const double ay[2] = {trig[4 * y + 2], trig[4 * y + 3]};
        const double az[2] = {trig[4 * z + 2], trig[4 * z + 3]};
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int k = 0; k < 2; ++k) acc[8 * al + 4 * i + 2 * j + k] += G[al] * (ax[i] * ay[j] * az[k]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 24) {
        double v = 0;
        for (int w = 0; w < kBlock / 32; ++w) v += sh[threadIdx.x][w];
        partial[((int64_t)m * gridDim.x + blockIdx.x) * 24 + threadIdx.x] = v * coef;
    }
}

__global__ void k_param_reduce(const double* __restrict__ partial, int M, int chunks, double* __restrict__ out)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M * 24; t += gridDim.x * blockDim.x) {
        const int m = t / 24, k = t % 24;
        double v = 0;
        for (int b = 0; b < chunks; ++b) v += partial[((int64_t)m * chunks + b) * 24 + k];
        out[t] = v;
    }
}

int grid_for(int64_t total)
{
    int64_t b = (total + kBlock - 1) / kBlock;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

struct GradLayout {
    size_t lattice, lam, ckpt, seg, lam0, lam1, fields, partial, out, total;
    int64_t nckpt, nseg;
};

GradLayout grad_layout(const mclbm_ctx* c, int64_t nsteps, int K)
{
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    GradLayout L;
    L.lattice = al(c->elem_bytes * Q * (size_t)c->n * c->M);
    const size_t csize = c->cfg.precision == MCLBM_FP64 ? sizeof(double) : sizeof(float);
    L.lam = al(csize * Q * (size_t)c->n * c->M);
    L.nckpt = (nsteps + K - 1) / K;
    if (L.nckpt < 1) L.nckpt = 1;
    L.nseg = K - 1;
    size_t off = 0;
    L.ckpt = off;
    off += L.lattice * L.nckpt;
    L.seg = off;
    off += L.lattice * L.nseg;
    L.lam0 = off;
    off += L.lam;
    L.lam1 = off;
    off += L.lam;
    L.fields = off;
    off += al(6 * (size_t)c->n * sizeof(double));
    L.partial = off;
    off += al((size_t)c->M * kGradChunks * 24 * sizeof(double));
    L.out = off;
    off += al((size_t)c->M * 24 * sizeof(double));
    L.total = off;
    return L;
}

// Occupancy-sized launch of the adjoint run kernel (two ring stages; resident blocks per SM
// queried once per instantiation).
template <class E, int VEC, bool WRAP>
cudaError_t launch_adjoint_async(mclbm_ctx* c, const Geom& g, int64_t runs, const void* state, const void* lin,
                                 void* lout, float om, float a, float b)
{
    constexpr int kStages = 2;
    auto kern = k_adjoint_async<E, VEC, kStages, WRAP>;
    constexpr int smem = AdjRing<E, VEC, kStages, WRAP>::kBytes;
    static std::atomic<int> occ_cache[kMaxDevices];
    int occ = 0;
    const cudaError_t e = resident_blocks(kern, kRunBlock, smem, occ_cache, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t blocks = (runs + kRunBlock - 1) / kRunBlock;
    if (blocks > (int64_t)c->num_sms * occ) blocks = (int64_t)c->num_sms * occ;
    kern<<<(unsigned)blocks, kRunBlock, smem, c->stream>>>((const E*)state, (const float*)lin, (float*)lout, g, runs,
                                                           om, a, b);
    return cudaGetLastError();
}

template <class E>
cudaError_t adjoint_step_t(mclbm_ctx* c, const void* state, const void* lin, void* lout)
{
    const Geom g{c->N, c->logN, c->n};
    if constexpr (std::is_same<E, double>::value) {
        k_adjoint_step<double, double><<<grid_for((int64_t)c->M * c->n), kBlock, 0, c->stream>>>(
            (const double*)state, (const double*)lin, (double*)lout, g, c->M, c->units.omega, 0.0);
    } else {
        constexpr int kVec = 2;
        const int64_t runs = (int64_t)c->M * c->n / kVec;
        const float om = (float)c->units.omega;
        const float a = (float)(2.0 / c->units.omega), b = (float)(2.0 - 2.0 / c->units.omega);
        const cudaError_t e = c->N <= 32 * kVec
                                  ? launch_adjoint_async<E, kVec, true>(c, g, runs, state, lin, lout, om, a, b)
                                  : launch_adjoint_async<E, kVec, false>(c, g, runs, state, lin, lout, om, a, b);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t adjoint_step(mclbm_ctx* c, const void* state, const void* lin, void* lout)
{
    switch (c->cfg.precision) {
        case MCLBM_FP64: return adjoint_step_t<double>(c, state, lin, lout);
        case MCLBM_FP32: return adjoint_step_t<float>(c, state, lin, lout);
        default: return adjoint_step_t<__half>(c, state, lin, lout);
    }
}

template <class E>
cudaError_t seed_t(mclbm_ctx* c, int objective, void* lam, double* fields)
{
    using C = typename std::conditional<std::is_same<E, double>::value, double, float>::type;
    const Geom g{c->N, c->logN, c->n};
    const double s = c->cfg.U_c / c->units.U_lat;
    const E* state = (const E*)lattice_ptr(c, c->cur);
    const double inv2dx = 1.0 / (2.0 * c->units.dx);
    for (int m = 0; m < c->M; ++m) {
        const double* gu = nullptr;
        if (objective == 1) {
            // dZ/du_phys = curl(curl u) / N^3 (the central-difference curl is self-adjoint)
            cudaError_t e = launch_field(c, m, fields);
            if (e != cudaSuccess) return e;
            k_curl<<<grid_for(c->n), kBlock, 0, c->stream>>>(fields, fields + 3 * c->n, g, inv2dx, 1.0);
            k_curl<<<grid_for(c->n), kBlock, 0, c->stream>>>(fields + 3 * c->n, fields, g, inv2dx, 1.0 / (double)c->n);
            gu = fields;
        }
        k_seed<E, C><<<grid_for(c->n), kBlock, 0, c->stream>>>(state, m, gu, g, s, (C*)lam);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class E>
cudaError_t param_grad_t(mclbm_ctx* c, const void* state0, const void* lam0, double* partial, double* out)
{
    using C = typename std::conditional<std::is_same<E, double>::value, double, float>::type;
    const Geom g{c->N, c->logN, c->n};
    const double* trig = (const double*)(c->work + c->wl.trig);
    const double coef = c->units.U_lat / c->cfg.U_c * 0.125;
    k_param_grad<E, C><<<dim3(kGradChunks, c->M), kBlock, 0, c->stream>>>((const E*)state0, (const C*)lam0, trig, g, coef,
                                                                          partial);
    k_param_reduce<<<(c->M * 24 + 255) / 256, 256, 0, c->stream>>>(partial, c->M, kGradChunks, out);
    return cudaGetLastError();
}

}  // namespace

size_t grad_required_bytes(const mclbm_ctx* c, int64_t nsteps, int K) { return grad_layout(c, nsteps, K).total; }

// CUDA events bracketing the phases of one gradient computation (for mclbm_grad_timing)
struct PhaseEvents {
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ok = true;
    PhaseEvents()
    {
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) ok = false;
    }
    ~PhaseEvents()
    {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
    void mark(int k, cudaStream_t s)
    {
        if (ok) cudaEventRecord(ev[k], s);
    }
};

int run_grad(mclbm_ctx* c, int objective, int64_t nsteps, int K, char* buf, size_t bytes, double* h_J, double* h_dJdX)
{
    const GradLayout L = grad_layout(c, nsteps, K);
    if (bytes < L.total) return set_error(MCLBM_ERR_OOM, "gradient buffer needs " + std::to_string(L.total) + " bytes");
    PhaseEvents pe;
    double recompute_ms = 0, adjoint_ms = 0;
    pe.mark(0, c->stream);
    // ---- forward with checkpoints every K steps
    for (int64_t t = 0; t < nsteps; ++t) {
        if (t % K == 0)
            MCLBM_CUDA(cudaMemcpyAsync(buf + L.ckpt + (size_t)(t / K) * L.lattice, lattice_ptr(c, c->cur), L.lattice,
                                       cudaMemcpyDeviceToDevice, c->stream));
        MCLBM_CUDA(launch_step(c));
    }
    if (nsteps == 0)
        MCLBM_CUDA(cudaMemcpyAsync(buf + L.ckpt, lattice_ptr(c, c->cur), L.lattice, cudaMemcpyDeviceToDevice, c->stream));
    pe.mark(1, c->stream);
    // ---- objective and its derivative at T
    std::vector<double> E((size_t)c->M), Z((size_t)c->M);
    MCLBM_CUDA(launch_energy(c, objective == 1, E.data(), Z.data()));
    for (int m = 0; m < c->M; ++m) h_J[m] = objective == 1 ? Z[m] : E[m];
    char* lam_a = buf + L.lam0;
    char* lam_b = buf + L.lam1;
    double* fields = (double*)(buf + L.fields);
    cudaError_t e;
    switch (c->cfg.precision) {
        case MCLBM_FP64: e = seed_t<double>(c, objective, lam_a, fields); break;
        case MCLBM_FP32: e = seed_t<float>(c, objective, lam_a, fields); break;
        default: e = seed_t<__half>(c, objective, lam_a, fields); break;
    }
    MCLBM_CUDA(e);
    // ---- reverse sweep, one segment at a time (recompute from the checkpoint)
    for (int64_t j = L.nckpt - 1; j >= 0; --j) {
        const int64_t t0 = j * K, t1 = (t0 + K < nsteps) ? t0 + K : nsteps;
        const char* ck = buf + L.ckpt + (size_t)j * L.lattice;
        auto state_at = [&](int64_t t) -> const char* {
            return t == t0 ? ck : buf + L.seg + (size_t)(t - t0 - 1) * L.lattice;
        };
        pe.mark(2, c->stream);
        for (int64_t t = t0 + 1; t < t1; ++t)
            MCLBM_CUDA(launch_pull_explicit(c, state_at(t - 1), (void*)state_at(t)));
        pe.mark(3, c->stream);
        for (int64_t t = t1 - 1; t >= t0; --t) {
            MCLBM_CUDA(adjoint_step(c, state_at(t), lam_a, lam_b));
            char* tmp = lam_a;
            lam_a = lam_b;
            lam_b = tmp;
        }
        pe.mark(4, c->stream);
        if (pe.ok) {
            float a = 0, b = 0;
            MCLBM_CUDA(cudaEventSynchronize(pe.ev[4]));
            cudaEventElapsedTime(&a, pe.ev[2], pe.ev[3]);
            cudaEventElapsedTime(&b, pe.ev[3], pe.ev[4]);
            recompute_ms += a;
            adjoint_ms += b;
        }
    }
    pe.mark(2, c->stream);
    // ---- dJ/dX from lambda^0 and the initial state
    double* partial = (double*)(buf + L.partial);
    double* out = (double*)(buf + L.out);
    switch (c->cfg.precision) {
        case MCLBM_FP64: e = param_grad_t<double>(c, buf + L.ckpt, lam_a, partial, out); break;
        case MCLBM_FP32: e = param_grad_t<float>(c, buf + L.ckpt, lam_a, partial, out); break;
        default: e = param_grad_t<__half>(c, buf + L.ckpt, lam_a, partial, out); break;
    }
    MCLBM_CUDA(e);
    pe.mark(5, c->stream);
    MCLBM_CUDA(cudaMemcpyAsync(h_dJdX, out, sizeof(double) * 24 * c->M, cudaMemcpyDeviceToHost, c->stream));
    MCLBM_CUDA(cudaStreamSynchronize(c->stream));
    // with the Leray option the kernels differentiate with respect to the evaluated
    // coefficients Y = L X; dJ/dX = L^T dJ/dY
    if (c->cfg.options & MCLBM_OPT_LERAY) leray_map(h_dJdX, c->M, true, h_dJdX);
    if (pe.ok) {
        float f = 0, p = 0;
        cudaEventElapsedTime(&f, pe.ev[0], pe.ev[1]);
        cudaEventElapsedTime(&p, pe.ev[2], pe.ev[5]);
        c->grad_ms[0] = f;
        c->grad_ms[1] = recompute_ms;
        c->grad_ms[2] = adjoint_ms;
        c->grad_ms[3] = p;
    }
    return MCLBM_OK;
}

// One adjoint step on caller data (natural layouts): state f^t [M][19][n] FP64 raw populations,
// lambda^{t+1} and lambda^t [M][19][n] FP64.  For tests of the transposed step.
template <class T>
__global__ void k_adjoint_step_natural(const double* __restrict__ f, const double* __restrict__ lam_next,
                                       double* __restrict__ lam_out, Geom g, int M, T omega, T guard)
{
    const int64_t total = (int64_t)M * g.n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(idx >> (3 * g.logN));
        const int64_t node = idx & (g.n - 1);
        int x, y, z;
        xyz(g, node, x, y, z);
        const double* fm = f + (int64_t)m * Q * g.n;
        const double* ln = lam_next + (int64_t)m * Q * g.n;
        T h[Q], mu[Q], lam[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            h[i] = (T)(fm[(int64_t)i * g.n + node] / weight<double>(i) - 1.0);
            mu[i] = (T)ln[(int64_t)i * g.n + g.node(g.wrap(x + cx(i)), g.wrap(y + cy(i)), g.wrap(z + cz(i)))];
        }
        if constexpr (std::is_same<T, float>::value)  // the FP32 path's product (as in k_adjoint_run)
            kbc_vjp_shifted<float>(h, mu, omega, 2.0f / omega, 2.0f - 2.0f / omega, lam);
        else
            kbc_vjp<T>(h, mu, omega, guard, lam);
        for (int i = 0; i < Q; ++i) lam_out[(int64_t)m * Q * g.n + (int64_t)i * g.n + node] = (double)lam[i];
    }
}

cudaError_t launch_adjoint_natural(const mclbm_ctx* c, const double* f, const double* lin, double* lout)
{
    const Geom g{c->N, c->logN, c->n};
    if (c->cfg.precision == MCLBM_FP64)
        k_adjoint_step_natural<double><<<grid_for((int64_t)c->M * c->n), kBlock, 0, c->stream>>>(f, lin, lout, g, c->M,
                                                                                               c->units.omega, 0.0);
    else
        k_adjoint_step_natural<float><<<grid_for((int64_t)c->M * c->n), kBlock, 0, c->stream>>>(
            f, lin, lout, g, c->M, (float)c->units.omega, kHHGuard);
    return cudaGetLastError();
}

}  // namespace mclbm

using namespace mclbm;

extern "C" {

int mclbm_grad_required_bytes(const mclbm_ctx* ctx, int64_t nsteps, int32_t ckpt_every, size_t* bytes)
{
    if (!ctx || !bytes || nsteps < 0 || ckpt_every < 1) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    *bytes = grad_required_bytes(ctx, nsteps, ckpt_every);
    return MCLBM_OK;
}

int mclbm_grad(mclbm_ctx* ctx, int32_t objective, int64_t nsteps, int32_t ckpt_every, void* d_buf, size_t buf_bytes,
               double* J, double* dJdX)
{
    if (ctx && (ctx->cfg.options & MCLBM_OPT_EXACT_GAMMA))
        return set_error(MCLBM_ERR_INVALID_ARG, "the adjoint covers the closed-form gamma only (not MCLBM_OPT_EXACT_GAMMA)");
    if (!ctx || !d_buf || !J || !dJdX || nsteps < 0 || ckpt_every < 1 || (objective != 0 && objective != 1))
        return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    if (ctx->cfg.pattern != MCLBM_PULL) return set_error(MCLBM_ERR_INVALID_ARG, "the adjoint needs pull streaming");
    if (ctx->steps != 0) return set_error(MCLBM_ERR_INVALID_ARG, "mclbm_grad must directly follow an initialisation");
    if ((uintptr_t)d_buf & 255) return set_error(MCLBM_ERR_INVALID_ARG, "gradient buffer must be 256-byte aligned");
    return run_grad(ctx, objective, nsteps, ckpt_every, (char*)d_buf, buf_bytes, J, dJdX);
}

int mclbm_grad_timing(const mclbm_ctx* ctx, double* ms)
{
    if (!ctx || !ms) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    for (int k = 0; k < 4; ++k) ms[k] = ctx->grad_ms[k];
    return MCLBM_OK;
}

int mclbm_adjoint_step(const mclbm_ctx* ctx, const double* d_f, const double* d_lambda_next, double* d_lambda)
{
    if (!ctx || !d_f || !d_lambda_next || !d_lambda) return set_error(MCLBM_ERR_INVALID_ARG, "bad argument");
    MCLBM_ON_DEVICE(ctx->device);
    MCLBM_CUDA(launch_adjoint_natural(ctx, d_f, d_lambda_next, d_lambda));
    return MCLBM_OK;
}

}  // extern "C"
