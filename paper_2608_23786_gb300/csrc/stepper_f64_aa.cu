// Stepper variants: element type double, aa streaming.
#include "stepper_launch.cuh"

namespace mclbm {

cudaError_t launch_batch_f64_aa(const BatchArgs<double>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s, int* occ)
{
    return launch_vec_block<double, 1, MCLBM_VECS_F64>(a, c, grid_cap, s, occ);
}

cudaError_t launch_staged_f64_aa(StagedArgs<double>& a, const LaunchConfig& c, int grid_cap, cudaStream_t s)
{
    return launch_staged_vec<double, 1>(a, c, grid_cap, s);
}

}  // namespace mclbm
