// Euler sweep kernels, element type float, 2D (all layouts, schemes, tiles),
// and the strip-walk sweeps of the split FORCE step.
#include "euler_force_walk.cuh"
#include "sweep_table.cuh"

namespace ripple {
cudaError_t sweep_launch_f32_2d(int layout, int scheme, int v, const SweepLaunch& L)
{
    return SweepDim<float, 2>::launch(layout, scheme, v, L);
}
int sweep_smem_f32_2d(int layout, int scheme, int v) { return SweepDim<float, 2>::smem(layout, scheme, v); }
int sweep_occ_f32_2d(int layout, int scheme, int v) { return SweepDim<float, 2>::occ(layout, scheme, v); }

cudaError_t force_walk_launch_f32_2d(int layout, int axis, const WalkLaunch& L)
{
    if (axis != 0 && axis != 1) return cudaErrorInvalidValue;
    if (layout == LAYOUT_SOA) return axis == 0 ? walk_launch<2, LAYOUT_SOA, 0>(L) : walk_launch<2, LAYOUT_SOA, 1>(L);
    return axis == 0 ? walk_launch<2, LAYOUT_AOS, 0>(L) : walk_launch<2, LAYOUT_AOS, 1>(L);
}
int force_walk_occ_f32_2d(int layout, int axis)
{
    if (layout == LAYOUT_SOA) return axis == 0 ? walk_occ<2, LAYOUT_SOA, 0>() : walk_occ<2, LAYOUT_SOA, 1>();
    return axis == 0 ? walk_occ<2, LAYOUT_AOS, 0>() : walk_occ<2, LAYOUT_AOS, 1>();
}
}  // namespace ripple
