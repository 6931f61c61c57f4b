// Instantiation and launch of the batched stepper kernel for one element type and
// pattern.  Each stepper_<type>_<pattern>.cu translation unit includes this file
// once, so the variants compile in parallel.
#pragma once
#include <mutex>

#include "launch.h"
#include "stepper_async.cuh"
#include "stepper_impl.cuh"
#include "stepper_staged.cuh"

namespace mclbm {

template <class E, int VEC, int PATTERN, int BLOCK, bool EXACT = false>
cudaError_t launch_variant(const BatchArgs<E>& a, int grid_cap, cudaStream_t s, int* occupancy_out)
{
    auto kern = k_step_batch<E, VEC, PATTERN, BLOCK, EXACT>;
    static std::atomic<int> occ_cache[kMaxDevices];  // resident blocks per SM, per device
    int occ = 0;
    const cudaError_t e = resident_blocks(kern, BLOCK, 0, occ_cache, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (occupancy_out) *occupancy_out = occ;
    const int64_t total = a.prefix[a.nlev];
    int64_t blocks = (total + BLOCK - 1) / BLOCK;
    const int64_t cap = (int64_t)grid_cap * occ;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

template <class E, int VEC, int PATTERN, int BLOCK, int FIX, bool PACK, bool WRAP = false>
cudaError_t launch_prefetch_fixed(const BatchArgs<E>& a, int grid_cap, cudaStream_t s, int* occupancy_out)
{
    auto kern = k_step_prefetch<E, VEC, PATTERN, BLOCK, FIX, PACK, WRAP>;
    static std::atomic<int> occ_cache[kMaxDevices];
    int occ = 0;
    const cudaError_t e = resident_blocks(kern, BLOCK, 0, occ_cache, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (occupancy_out) *occupancy_out = occ;
    const int64_t total = a.prefix[a.nlev];
    int64_t blocks = (total + BLOCK - 1) / BLOCK;
    const int64_t cap = (int64_t)grid_cap * occ;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// Whether every level's x-row lies within one warp (N <= 32 VEC): the launch then takes the
// kernels' row-rotation variant (WRAP) for its shifted rows.
template <class E>
bool rows_in_warp(const BatchArgs<E>& a, int vec)
{
    for (int l = 0; l < a.nlev; ++l)
        if (a.lev[l].g.N > 32 * vec) return false;
    return true;
}

// Parity of an AA launch: the host launches AA levels of different parity separately
// (launch_levels), so every launch here has one parity; -1 if not (not launched).
template <class E>
int launch_parity(const BatchArgs<E>& a)
{
    for (int l = 1; l < a.nlev; ++l)
        if (a.lev[l].parity != a.lev[0].parity) return -1;
    return a.lev[0].parity;
}

// Pull launches take the pull-only kernel, AA launches the kernel of their parity.
template <class E, int VEC, int PATTERN, int BLOCK, bool PACK>
cudaError_t launch_prefetch_variant(const BatchArgs<E>& a, int grid_cap, cudaStream_t s, int* occ)
{
    if constexpr (PATTERN == 0) {
        // pull: FP16 storage takes the row rotation where rows lie within one warp (measured: FP16
        // pull with 4 nodes per thread 75.6% -> 82.3% of the copy bandwidth at 128^3); FP32, at the
        // memory bound, keeps the end elements (no gain measured)
        if constexpr (std::is_same<E, __half>::value)
            if (rows_in_warp(a, VEC)) return launch_prefetch_fixed<E, VEC, 0, BLOCK, 0, PACK, true>(a, grid_cap, s, occ);
        return launch_prefetch_fixed<E, VEC, 0, BLOCK, 0, PACK>(a, grid_cap, s, occ);
    } else {
        const int par = launch_parity(a);
        if (par == 0) return launch_prefetch_fixed<E, VEC, 1, BLOCK, 1, PACK>(a, grid_cap, s, occ);
        if (par == 1) {
            // odd steps shift loads and stores: where every level's x-row lies within one warp the
            // row's lanes rotate (no separate end elements)
            if (rows_in_warp(a, VEC)) return launch_prefetch_fixed<E, VEC, 1, BLOCK, 2, PACK, true>(a, grid_cap, s, occ);
            return launch_prefetch_fixed<E, VEC, 1, BLOCK, 2, PACK>(a, grid_cap, s, occ);
        }
        return cudaErrorInvalidValue;
    }
}

template <class E, int VEC, int PATTERN, int BLOCK, int FIX, int STAGES, bool WRAP, bool ONE>
cudaError_t launch_async_fixed(const BatchArgs<E>& a, int grid_cap, cudaStream_t s, int* occupancy_out)
{
    auto kern = k_step_async<E, VEC, PATTERN, BLOCK, FIX, STAGES, WRAP, ONE>;
    constexpr int smem = AsyncRing<E, VEC, BLOCK, STAGES>::kBytes;
    static std::atomic<int> occ_cache[kMaxDevices];
    int occ = 0;
    const cudaError_t e = resident_blocks(kern, BLOCK, smem, occ_cache, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (occupancy_out) *occupancy_out = occ;
    const int64_t total = a.prefix[a.nlev];
    int64_t blocks = (total + BLOCK - 1) / BLOCK;
    const int64_t cap = (int64_t)grid_cap * occ;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <class E, int VEC, int PATTERN, int BLOCK, int STAGES, bool ONE>
cudaError_t launch_async_levels(const BatchArgs<E>& a, int grid_cap, cudaStream_t s, int* occ)
{
    // steps with shifted rows (pull, AA odd) of FP16 storage take the row rotation where every
    // level's row lies within one warp (measured at 128^3 x 32 with 8 nodes per thread: FP16 pull
    // 81.6% -> 90.6% of the copy bandwidth, AA odd steps 65% -> 81.4%; FP32, already at the memory
    // bound, loses with it: AA odd 100% -> 89%, so FP32 ring launches keep the end elements)
    constexpr bool kWrapKind = std::is_same<E, __half>::value;
    const bool wrap = kWrapKind && rows_in_warp(a, VEC);
    if constexpr (PATTERN == 0) {
        if constexpr (kWrapKind)
            if (wrap) return launch_async_fixed<E, VEC, 0, BLOCK, 0, STAGES, true, ONE>(a, grid_cap, s, occ);
        return launch_async_fixed<E, VEC, 0, BLOCK, 0, STAGES, false, ONE>(a, grid_cap, s, occ);
    } else {
        const int par = launch_parity(a);
        if (par == 0) return launch_async_fixed<E, VEC, 1, BLOCK, 1, STAGES, false, ONE>(a, grid_cap, s, occ);
        if (par == 1) {
            if constexpr (kWrapKind)
                if (wrap) return launch_async_fixed<E, VEC, 1, BLOCK, 2, STAGES, true, ONE>(a, grid_cap, s, occ);
            return launch_async_fixed<E, VEC, 1, BLOCK, 2, STAGES, false, ONE>(a, grid_cap, s, occ);
        }
        return cudaErrorInvalidValue;
    }
}

// A launch of one level (a context's own step) of FP16 storage takes the single-level kernel
// (measured at 128^3 x 32: D3Q19 pull 90.7% -> 94.4% of the copy bandwidth, AA even steps 89.6% ->
// 90.0%, AA odd steps 81.4% -> 83.8%, D3Q27 pull 82.9% -> 85.1%); FP32 ring launches, and the
// prefetching kernels, measured slower with it (FP32 AA odd steps 100.3% -> 92.4%; the prefetching
// kernel's FP32 pull 99.6% -> 86.6%, D3Q27 FP16 AA even steps 87.7% -> 69.8%) and keep the level index.
template <class E, int VEC, int PATTERN, int BLOCK, int STAGES>
cudaError_t launch_async_variant(const BatchArgs<E>& a, int grid_cap, cudaStream_t s, int* occ)
{
    if constexpr (std::is_same<E, __half>::value)
        if (a.nlev == 1) return launch_async_levels<E, VEC, PATTERN, BLOCK, STAGES, true>(a, grid_cap, s, occ);
    return launch_async_levels<E, VEC, PATTERN, BLOCK, STAGES, false>(a, grid_cap, s, occ);
}

template <class E, int PATTERN, int... VECS>
cudaError_t launch_vec_block_rest(const BatchArgs<E>& a, const LaunchConfig& cfg, int grid_cap, cudaStream_t s,
                                  int* occ)
{
    cudaError_t e = cudaErrorInvalidConfiguration;
    bool found = false;
    auto try_one = [&](auto vec_tag) {
        constexpr int V = decltype(vec_tag)::value;
        if (found || cfg.vec != V) return;
        found = true;
        if (cfg.kind == 2) {
            if (cfg.block == 128)
                e = launch_prefetch_variant<E, V, PATTERN, 128, false>(a, grid_cap, s, occ);
            else if (cfg.block == 256)
                e = launch_prefetch_variant<E, V, PATTERN, 256, false>(a, grid_cap, s, occ);
            else
                e = cudaErrorInvalidConfiguration;
        } else if (cfg.kind == 3) {
            if constexpr (Storage<E>::shifted && V % 2 == 0) {
                if (cfg.block == 128)
                    e = launch_prefetch_variant<E, V, PATTERN, 128, true>(a, grid_cap, s, occ);
                else if (cfg.block == 256)
                    e = launch_prefetch_variant<E, V, PATTERN, 256, true>(a, grid_cap, s, occ);
                else
                    e = cudaErrorInvalidConfiguration;
            } else {
                e = cudaErrorInvalidConfiguration;
            }
        } else if (cfg.kind == 4 || cfg.kind == 5) {
            if constexpr (Storage<E>::shifted && kAsyncKinds) {
                if (cfg.block != 128)
                    e = cudaErrorInvalidConfiguration;
                else if (cfg.kind == 4)
                    e = launch_async_variant<E, V, PATTERN, 128, 2>(a, grid_cap, s, occ);
                else
                    e = launch_async_variant<E, V, PATTERN, 128, 3>(a, grid_cap, s, occ);
            } else {
                e = cudaErrorInvalidConfiguration;
            }
        } else if (cfg.block == 128)
            e = launch_variant<E, V, PATTERN, 128>(a, grid_cap, s, occ);
        else if (cfg.block == 256)
            e = launch_variant<E, V, PATTERN, 256>(a, grid_cap, s, occ);
        else
            e = cudaErrorInvalidConfiguration;
    };
    (try_one(std::integral_constant<int, VECS>{}), ...);
    return e;
}

template <class E, int PATTERN, int FIRST_VEC, int... VECS>
cudaError_t launch_vec_block(const BatchArgs<E>& a, const LaunchConfig& cfg, int grid_cap, cudaStream_t s, int* occ)
{
    // kind 6 (exact entropic gamma): the direct kernel, the type's first VEC, 128 threads
    if (cfg.kind == 6) {
        if (cfg.vec != FIRST_VEC || cfg.block != 128) return cudaErrorInvalidConfiguration;
        return launch_variant<E, FIRST_VEC, PATTERN, 128, true>(a, grid_cap, s, occ);
    }
    return launch_vec_block_rest<E, PATTERN, FIRST_VEC, VECS...>(a, cfg, grid_cap, s, occ);
}

// Staged kernel: pick the number of stages so that two blocks fit on an SM, size the
// dynamic shared memory, and launch a persistent grid (SM count x resident blocks).
template <class E, int PATTERN, int VEC>
cudaError_t launch_staged_variant(StagedArgs<E>& a, int grid_cap, cudaStream_t s)
{
    auto kern = k_step_staged<E, PATTERN, VEC>;
    const size_t stage_bytes = (size_t)a.stage_elems * sizeof(E);
    int stages = (int)((size_t)(110 * 1024) / stage_bytes);
    stages = stages < 2 ? 2 : (stages > 4 ? 4 : stages);
    a.stages = stages;
    const size_t smem = 256 + (size_t)stages * stage_bytes;
    // the dynamic shared-memory limit is a per-device attribute: the largest set so far, per device
    static std::mutex mu;
    static size_t configured[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        const bool cached = dev >= 0 && dev < kMaxDevices;
        if (!cached || smem > configured[dev]) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            if (cached) configured[dev] = smem;
        }
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStagedThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t total = a.tile_prefix[a.nlev];
    int64_t blocks = (int64_t)grid_cap * occ;
    if (blocks > total) blocks = total;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kStagedThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <class E, int PATTERN>
cudaError_t launch_staged_vec(StagedArgs<E>& a, const LaunchConfig& cfg, int grid_cap, cudaStream_t s)
{
    if (cfg.vec == 1) return launch_staged_variant<E, PATTERN, 1>(a, grid_cap, s);
    if (cfg.vec == 2) return launch_staged_variant<E, PATTERN, 2>(a, grid_cap, s);
    return cudaErrorInvalidConfiguration;
}

}  // namespace mclbm
