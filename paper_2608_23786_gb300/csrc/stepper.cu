// Population gather/scatter and the host side of the batched stream + collide launch (the
// kernels live in stepper_impl.cuh and are compiled per element type and pattern in
// stepper_<type>_<pattern>.cu; the initialisation is in init.cu).
#include <cuda_fp16.h>

#include "internal.h"
#include "launch.h"
#include "stepper_impl.cuh"
#include "stepper_staged.cuh"

namespace mclbm {

namespace {

constexpr int kBlock = 256;

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

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing arrives at,
// gives up after `limit_ns` nanoseconds and records MCLBM_ERR_TIMEOUT in the error word,
// exactly as the staged stepper does when a wait runs out.  No copy is in flight.
__global__ void k_wait_selftest(int* err, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_u32(&bar), 1);
    mbar_fence_init();
    if (!mbar_wait_bounded(smem_u32(&bar), 0u, limit_ns)) atomicExch(err, kTimeoutCode);
}


int grid_for(int64_t total)
{
    int64_t b = (total + kBlock - 1) / kBlock;
    return (int)(b > (int64_t)1 << 30 ? (int64_t)1 << 30 : b);
}

Geom geom_of(const mclbm_ctx* c) { return Geom{c->N, c->logN, c->n}; }
int parity_of(const mclbm_ctx* c) { return c->cfg.pattern == MCLBM_AA ? (int)(c->steps & 1) : 0; }

template <class E>
cudaError_t get_t(const mclbm_ctx* c, int sample, double* d_out)
{
    k_get_pops<E><<<grid_for(c->n), kBlock, 0, c->stream>>>((const E*)lattice_ptr(c, c->cur), geom_of(c), c->cfg.pattern,
                                                            parity_of(c), sample, d_out);
    return cudaGetLastError();
}

template <class E>
cudaError_t set_t(mclbm_ctx* c, int sample, const double* d_in)
{
    k_set_pops<E><<<grid_for(c->n), kBlock, 0, c->stream>>>((E*)lattice_ptr(c, c->cur), geom_of(c), c->cfg.pattern,
                                                            parity_of(c), sample, d_in);
    return cudaGetLastError();
}

template <class E>
void fill_level(LevelArgs<E>& L, const mclbm_ctx* c)
{
    if (c->cfg.pattern == MCLBM_PULL) {
        L.src = (const E*)lattice_ptr(c, c->cur);
        L.dst = (E*)lattice_ptr(c, 1 - c->cur);
    } else {
        L.src = (const E*)lattice_ptr(c, 0);
        L.dst = (E*)lattice_ptr(c, 0);
    }
    L.g = geom_of(c);
    L.M = c->M;
    L.parity = parity_of(c);
    L.omega32 = (float)c->units.omega;
    L.omega64 = c->units.omega;
    L.a32 = (float)(2.0 / c->units.omega);
    L.b32 = (float)(2.0 - 2.0 / c->units.omega);
    if constexpr (std::is_same<E, double>::value) {
        L.a64 = 2.0 / c->units.omega;
        L.b64 = 2.0 - 2.0 / c->units.omega;
    }
}

template <class E>
cudaError_t staged_t(mclbm_ctx* const* lv, int nlev, const LaunchConfig& cfg, int grid_cap, cudaStream_t s)
{
    StagedArgs<E> a;
    memset(&a, 0, sizeof(a));
    a.nlev = nlev;
    a.tile_prefix[0] = 0;
    const int target = kConsumerWarps * 32 * cfg.vec;  // nodes per tile
    int max_nodes = 0;
    for (int k = 0; k < nlev; ++k) {
        const int N = lv[k]->N;
        int ty = target / N;
        ty = ty < 1 ? 1 : (ty > N ? N : ty);
        a.ty[k] = ty;
        if (ty * N > max_nodes) max_nodes = ty * N;
        fill_level<E>(a.lev[k], lv[k]);
        a.tile_prefix[k + 1] = a.tile_prefix[k] + (int64_t)lv[k]->M * N * (N / ty);
    }
    a.stage_elems = Q * max_nodes;
    a.err = (int*)(lv[0]->work + lv[0]->wl.flag) + 1;
    const bool pull = lv[0]->cfg.pattern == MCLBM_PULL;
    if constexpr (std::is_same<E, double>::value)
        return pull ? launch_staged_f64_pull(a, cfg, grid_cap, s) : launch_staged_f64_aa(a, cfg, grid_cap, s);
    else if constexpr (std::is_same<E, float>::value)
        return pull ? launch_staged_f32_pull(a, cfg, grid_cap, s) : launch_staged_f32_aa(a, cfg, grid_cap, s);
    else
        return pull ? launch_staged_f16_pull(a, cfg, grid_cap, s) : launch_staged_f16_aa(a, cfg, grid_cap, s);
}

template <class E>
cudaError_t levels_t(mclbm_ctx* const* lv, int nlev, const LaunchConfig& cfg, int grid_cap, cudaStream_t s, int* occ)
{
    if (cfg.kind == 1) return staged_t<E>(lv, nlev, cfg, grid_cap, s);
    BatchArgs<E> a;
    memset(&a, 0, sizeof(a));
    a.nlev = nlev;
    a.prefix[0] = 0;
    for (int k = 0; k < nlev; ++k) {
        fill_level<E>(a.lev[k], lv[k]);
        a.prefix[k + 1] = a.prefix[k] + (int64_t)lv[k]->M * lv[k]->n / cfg.vec;
    }
    const bool pull = lv[0]->cfg.pattern == MCLBM_PULL;
    if constexpr (std::is_same<E, double>::value)
        return pull ? launch_batch_f64_pull(a, cfg, grid_cap, s, occ) : launch_batch_f64_aa(a, cfg, grid_cap, s, occ);
    else if constexpr (std::is_same<E, float>::value)
        return pull ? launch_batch_f32_pull(a, cfg, grid_cap, s, occ) : launch_batch_f32_aa(a, cfg, grid_cap, s, occ);
    else
        return pull ? launch_batch_f16_pull(a, cfg, grid_cap, s, occ) : launch_batch_f16_aa(a, cfg, grid_cap, s, occ);
}

}  // namespace

#define MCLBM_DISPATCH(prec, fn, ...)                    \
    switch (prec) {                                      \
        case MCLBM_FP64: return fn<double>(__VA_ARGS__); \
        case MCLBM_FP32: return fn<float>(__VA_ARGS__);  \
        default: return fn<__half>(__VA_ARGS__);         \
    }

cudaError_t launch_get_populations(const mclbm_ctx* c, int sample, double* d_out)
{
    MCLBM_DISPATCH(c->cfg.precision, get_t, c, sample, d_out);
}
cudaError_t launch_set_populations(mclbm_ctx* c, int sample, const double* d_in)
{
    MCLBM_DISPATCH(c->cfg.precision, set_t, c, sample, d_in);
}

bool launch_supported(int precision, const LaunchConfig& c)
{
    if (c.kind == 6) return c.block == 128 && c.vec == exact_vec(precision);
    if (c.kind == 1) return c.vec == 1 || c.vec == 2;
    if (c.kind < 0 || c.kind > 5 || c.kind == 1 || (c.block != 128 && c.block != 256)) return false;
    if (c.kind == 3 && (precision == MCLBM_FP64 || c.vec % 2 != 0)) return false;
    if (c.kind >= 4 && (!kAsyncKinds || precision == MCLBM_FP64 || c.block != 128)) return false;
    return vec_supported(precision, c.vec);
}

int exact_vec(int precision)
{
    return precision == MCLBM_FP64 ? kVecF64[0] : (precision == MCLBM_FP32 ? kVecF32[0] : kVecF16[0]);
}

bool vec_supported(int precision, int vec)
{
    auto in = [vec](const int* a, int n) {
        for (int k = 0; k < n; ++k)
            if (a[k] == vec) return true;
        return false;
    };
    if (precision == MCLBM_FP64) return in(kVecF64, sizeof(kVecF64) / sizeof(int));
    if (precision == MCLBM_FP32) return in(kVecF32, sizeof(kVecF32) / sizeof(int));
    return in(kVecF16, sizeof(kVecF16) / sizeof(int));
}

cudaError_t launch_levels(mclbm_ctx* const* lv, int nlev, const LaunchConfig& cfg, const LaunchConfig& cfg_odd,
                          cudaStream_t s, int* occ)
{
    if (nlev < 1 || nlev > kMaxLevels) return cudaErrorInvalidValue;
    const int grid_cap = lv[0]->num_sms;
    auto run = [&](mclbm_ctx* const* group, int n, const LaunchConfig& c) {
        switch (lv[0]->cfg.precision) {
            case MCLBM_FP64: return levels_t<double>(group, n, c, grid_cap, s, occ);
            case MCLBM_FP32: return levels_t<float>(group, n, c, grid_cap, s, occ);
            default: return levels_t<__half>(group, n, c, grid_cap, s, occ);
        }
    };
    cudaError_t e = cudaSuccess;
    if (lv[0]->cfg.pattern == MCLBM_AA && cfg.kind != 1) {
        // AA: one launch per parity, each with the kernel specialised for that parity and the
        // parity's own launch shape (the levels are independent, so the order does not matter)
        mclbm_ctx* even[kMaxLevels];
        mclbm_ctx* odd[kMaxLevels];
        int ne = 0, no = 0;
        for (int k = 0; k < nlev; ++k) (lv[k]->steps & 1 ? odd[no++] : even[ne++]) = lv[k];
        if (ne > 0) e = run(even, ne, cfg);
        if (e == cudaSuccess && no > 0) e = run(odd, no, cfg_odd);
    } else {
        e = run(lv, nlev, cfg);
    }
    if (e != cudaSuccess) return e;
    for (int k = 0; k < nlev; ++k) {
        if (lv[k]->cfg.pattern == MCLBM_PULL) lv[k]->cur ^= 1;
        lv[k]->steps += 1;
    }
    return cudaSuccess;
}

cudaError_t launch_step(mclbm_ctx* c) { return launch_step_with(c, c->launch, c->launch_odd); }

cudaError_t launch_wait_selftest(mclbm_ctx* c)
{
    k_wait_selftest<<<1, 32, 0, c->stream>>>((int*)(c->work + c->wl.flag) + 1, 1000ull * 1000);  // 1 ms
    return cudaGetLastError();
}

// One pull step from an explicit source lattice to an explicit destination lattice (both
// pull layout, same shape as the context's); the context's own state is not touched.
cudaError_t launch_pull_explicit(mclbm_ctx* c, const void* src, void* dst)
{
    const LaunchConfig cfg = c->launch.kind == 1 ? default_launch(c->cfg.precision, MCLBM_PULL, c->cfg.options) : c->launch;
    switch (c->cfg.precision) {
        case MCLBM_FP64: {
            BatchArgs<double> a;
            memset(&a, 0, sizeof(a));
            a.nlev = 1;
            fill_level<double>(a.lev[0], c);
            a.lev[0].src = (const double*)src;
            a.lev[0].dst = (double*)dst;
            a.prefix[1] = (int64_t)c->M * c->n / cfg.vec;
            return launch_batch_f64_pull(a, cfg, c->num_sms, c->stream, nullptr);
        }
        case MCLBM_FP32: {
            BatchArgs<float> a;
            memset(&a, 0, sizeof(a));
            a.nlev = 1;
            fill_level<float>(a.lev[0], c);
            a.lev[0].src = (const float*)src;
            a.lev[0].dst = (float*)dst;
            a.prefix[1] = (int64_t)c->M * c->n / cfg.vec;
            return launch_batch_f32_pull(a, cfg, c->num_sms, c->stream, nullptr);
        }
        default: {
            BatchArgs<__half> a;
            memset(&a, 0, sizeof(a));
            a.nlev = 1;
            fill_level<__half>(a.lev[0], c);
            a.lev[0].src = (const __half*)src;
            a.lev[0].dst = (__half*)dst;
            a.prefix[1] = (int64_t)c->M * c->n / cfg.vec;
            return launch_batch_f16_pull(a, cfg, c->num_sms, c->stream, nullptr);
        }
    }
}

cudaError_t launch_step_with(mclbm_ctx* c, const LaunchConfig& cfg, const LaunchConfig& cfg_odd)
{
    mclbm_ctx* one[1] = {c};
    return launch_levels(one, 1, cfg, cfg_odd, c->stream, nullptr);
}

}  // namespace mclbm
