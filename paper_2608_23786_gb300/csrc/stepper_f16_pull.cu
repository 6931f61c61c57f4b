// Stepper variants: element type __half, pull streaming.
#include "stepper_launch.cuh"

namespace mclbm {

cudaError_t launch_batch_f16_pull(const BatchArgs<__half>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s, int* occ)
{
    return launch_vec_block<__half, 0, MCLBM_VECS_F16>(a, c, grid_cap, s, occ);
}

cudaError_t launch_staged_f16_pull(StagedArgs<__half>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s)
{
    return launch_staged_vec<__half, 0>(a, c, grid_cap, s);
}

}  // namespace mclbm
