// Euler sweep kernels, element type double, 3D (all layouts, schemes, tiles).
#include "sweep_table.cuh"

namespace ripple {
cudaError_t sweep_launch_f64_3d(int layout, int scheme, int v, const SweepLaunch& L)
{
    return SweepDim<double, 3>::launch(layout, scheme, v, L);
}
int sweep_smem_f64_3d(int layout, int scheme, int v) { return SweepDim<double, 3>::smem(layout, scheme, v); }
int sweep_occ_f64_3d(int layout, int scheme, int v) { return SweepDim<double, 3>::occ(layout, scheme, v); }
}  // namespace ripple
