// Stepper variants: element type float, aa streaming.
#include "stepper_launch.cuh"

namespace mclbm {

cudaError_t launch_batch_f32_aa(const BatchArgs<float>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s, int* occ)
{
    return launch_vec_block<float, 1, MCLBM_VECS_F32>(a, c, grid_cap, s, occ);
}

cudaError_t launch_staged_f32_aa(StagedArgs<float>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s)
{
    return launch_staged_vec<float, 1>(a, c, grid_cap, s);
}

}  // namespace mclbm
