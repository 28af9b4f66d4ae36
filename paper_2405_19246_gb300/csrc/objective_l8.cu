// Objective kernels for l = 8 marginals (warp tiles, 256 states).
#include "warp.cuh"

namespace mmot {
template <>
cudaError_t launch_objective_warp8<float>(const SweepArgs &a, cudaStream_t s, int kind, int level, int fwd)
{
    return launch_wobj_impl<8, float, WShape<7, float>::K>(a, s, kind, level, fwd);
}
template <>
cudaError_t launch_objective_warp8<double>(const SweepArgs &a, cudaStream_t s, int kind, int level, int fwd)
{
    return launch_wobj_impl<8, double, WShape<7, double>::K>(a, s, kind, level, fwd);
}
}  // namespace mmot
