// Launch configuration of the stepper kernel variants (chosen by the autotuner).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <type_traits>

namespace mclbm {

constexpr int kMaxLevels = 8;  // levels of one batched launch

// Launch facts of one kernel per device, filled on its first launch on each device: the kernel's
// dynamic shared-memory limit is set there (a per-device attribute) and its resident blocks per
// SM recorded.  Concurrent first launches may both fill a slot, with the same value.
constexpr int kMaxDevices = 64;
template <class K>
cudaError_t resident_blocks(K kern, int block, int smem, std::atomic<int> (&cache)[kMaxDevices], int* occ)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::atomic<int>* slot = (dev >= 0 && dev < kMaxDevices) ? &cache[dev] : nullptr;
    int o = slot ? slot->load(std::memory_order_acquire) : 0;
    if (o > 0) {
        *occ = o;
        return cudaSuccess;
    }
    if (smem > 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, block, smem);
    if (e != cudaSuccess) return e;
    if (o > 0 && slot) slot->store(o, std::memory_order_release);
    *occ = o;
    return cudaSuccess;
}

struct LaunchConfig {
    int vec;       // nodes per thread along x
    int block;     // threads per block (128 or 256); the staged kernel always uses 288
    int kind = 0;  // 0: direct loads (stepper_impl.cuh), 1: shared-memory staging (stepper_staged.cuh),
                   // 2: direct loads with the next run prefetched, 3: as 2 with the packed FP32
                   // collision of node pairs (shifted storage, even vec), 4 / 5: runs ahead
                   // prefetched by cp.async into shared memory, 1 / 2 runs deep (shifted
                   // storage, block 128; packed collision for even vec)
};

// Variants compiled per element type (nodes per thread; VEC * sizeof(E) <= 16 bytes).  The
// D3Q27 build compiles a reduced set (its collision is heavier to compile): one VEC per
// type.
#ifdef MCLBM_D3Q27
#define MCLBM_VECS_F64 1
#define MCLBM_VECS_F32 2
#define MCLBM_VECS_F16 4
constexpr int kVecF64[] = {1};
constexpr int kVecF32[] = {2};
constexpr int kVecF16[] = {4};
constexpr bool kAsyncKinds = true;  // kinds 4 and 5
#else
#define MCLBM_VECS_F64 1, 2
#define MCLBM_VECS_F32 1, 2, 4
#define MCLBM_VECS_F16 2, 4, 8
constexpr int kVecF64[] = {1, 2};
constexpr int kVecF32[] = {1, 2, 4};
constexpr int kVecF16[] = {2, 4, 8};
constexpr bool kAsyncKinds = true;
#endif
constexpr int kBlocks[] = {128, 256};

template <class E>
struct BatchArgs;
template <class E>
struct StagedArgs;

constexpr int kVecStaged[] = {1, 2};  // nodes per consumer thread of the staged kernel

// Launchers defined in stepper_<type>_<pattern>.cu.  grid_cap: SM count (the grid is
// grid_cap times the variant's resident blocks per SM, or less for small batches).
#define MCLBM_DECLARE_LAUNCH(T, E)                                                                              \
    cudaError_t launch_batch_##T##_pull(const BatchArgs<E>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s, \
                                        int* occ);                                                               \
    cudaError_t launch_batch_##T##_aa(const BatchArgs<E>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s,   \
                                      int* occ);                                                                 \
    cudaError_t launch_staged_##T##_pull(StagedArgs<E>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s);    \
    cudaError_t launch_staged_##T##_aa(StagedArgs<E>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s);
MCLBM_DECLARE_LAUNCH(f64, double)
MCLBM_DECLARE_LAUNCH(f32, float)
MCLBM_DECLARE_LAUNCH(f16, __half)
#undef MCLBM_DECLARE_LAUNCH

}  // namespace mclbm
