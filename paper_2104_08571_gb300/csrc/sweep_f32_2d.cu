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

template <int LAYOUT, int AXIS>
static cudaError_t walk_configure()
{
    static cudaError_t e = cudaFuncSetAttribute(euler_force_walk2d_kernel<LAYOUT, AXIS, kWalkSlots>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                WalkCfg<kWalkSlots>::SMEM);
    return e;
}
template <int LAYOUT, int AXIS>
static cudaError_t walk_launch(const WalkLaunch& L)
{
    const cudaError_t e = walk_configure<LAYOUT, AXIS>();
    if (e != cudaSuccess) return e;
    euler_force_walk2d_kernel<LAYOUT, AXIS, kWalkSlots>
        <<<L.grid, kWalkWarps * 32, WalkCfg<kWalkSlots>::SMEM, L.stream>>>(
            static_cast<const float*>(L.in), static_cast<float*>(L.out), L.ctl, L.wg, L.prm);
    return cudaGetLastError();
}
template <int LAYOUT, int AXIS>
static int walk_occ()
{
    if (walk_configure<LAYOUT, AXIS>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, euler_force_walk2d_kernel<LAYOUT, AXIS, kWalkSlots>,
                                                      kWalkWarps * 32, WalkCfg<kWalkSlots>::SMEM) != cudaSuccess)
        return 0;
    return n;
}
cudaError_t force_walk_launch_f32_2d(int layout, int axis, const WalkLaunch& L)
{
    if (axis != 0 && axis != 1) return cudaErrorInvalidValue;
    if (layout == LAYOUT_SOA) return axis == 0 ? walk_launch<LAYOUT_SOA, 0>(L) : walk_launch<LAYOUT_SOA, 1>(L);
    return axis == 0 ? walk_launch<LAYOUT_AOS, 0>(L) : walk_launch<LAYOUT_AOS, 1>(L);
}
int force_walk_occ_f32_2d(int layout, int axis)
{
    if (layout == LAYOUT_SOA) return axis == 0 ? walk_occ<LAYOUT_SOA, 0>() : walk_occ<LAYOUT_SOA, 1>();
    return axis == 0 ? walk_occ<LAYOUT_AOS, 0>() : walk_occ<LAYOUT_AOS, 1>();
}
}  // namespace ripple
