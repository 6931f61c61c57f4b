// Stepper variants: element type double, pull streaming.
#include "stepper_launch.cuh"

namespace mclbm {

cudaError_t launch_batch_f64_pull(const BatchArgs<double>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s, int* occ)
{
    return launch_vec_block<double, 0, MCLBM_VECS_F64>(a, c, grid_cap, s, occ);
}

cudaError_t launch_staged_f64_pull(StagedArgs<double>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s)
{
    return launch_staged_vec<double, 0>(a, c, grid_cap, s);
}

}  // namespace mclbm
