// Euler sweep kernels, element type float, 3D (all layouts, schemes, tiles),
// and the strip-walk sweeps of the split FORCE step.
#include "euler_force_walk.cuh"
#include "sweep_table.cuh"

namespace ripple {
cudaError_t sweep_launch_f32_3d(int layout, int scheme, int v, const SweepLaunch& L)
{
    return SweepDim<float, 3>::launch(layout, scheme, v, L);
}
int sweep_smem_f32_3d(int layout, int scheme, int v) { return SweepDim<float, 3>::smem(layout, scheme, v); }
int sweep_occ_f32_3d(int layout, int scheme, int v) { return SweepDim<float, 3>::occ(layout, scheme, v); }

cudaError_t force_walk_launch_f32_3d(int layout, int axis, const WalkLaunch& L)
{
    if (layout == LAYOUT_SOA)
        return axis == 0 ? walk_launch<3, LAYOUT_SOA, 0>(L) : axis == 1 ? walk_launch<3, LAYOUT_SOA, 1>(L)
                                                                        : walk_launch<3, LAYOUT_SOA, 2>(L);
    return axis == 0 ? walk_launch<3, LAYOUT_AOS, 0>(L) : axis == 1 ? walk_launch<3, LAYOUT_AOS, 1>(L)
                                                                    : walk_launch<3, LAYOUT_AOS, 2>(L);
}
int force_walk_occ_f32_3d(int layout, int axis)
{
    if (layout == LAYOUT_SOA)
        return axis == 0 ? walk_occ<3, LAYOUT_SOA, 0>() : axis == 1 ? walk_occ<3, LAYOUT_SOA, 1>()
                                                                    : walk_occ<3, LAYOUT_SOA, 2>();
    return axis == 0 ? walk_occ<3, LAYOUT_AOS, 0>() : axis == 1 ? walk_occ<3, LAYOUT_AOS, 1>()
                                                                : walk_occ<3, LAYOUT_AOS, 2>();
}
}  // namespace ripple
