// Euler sweep kernels, element type double, 2D (all layouts, schemes, tiles).
#include "sweep_table.cuh"

namespace ripple {
cudaError_t sweep_launch_f64_2d(int layout, int scheme, int v, const SweepLaunch& L)
{
    return SweepDim<double, 2>::launch(layout, scheme, v, L);
}
int sweep_smem_f64_2d(int layout, int scheme, int v) { return SweepDim<double, 2>::smem(layout, scheme, v); }
int sweep_occ_f64_2d(int layout, int scheme, int v) { return SweepDim<double, 2>::occ(layout, scheme, v); }
}  // namespace ripple
