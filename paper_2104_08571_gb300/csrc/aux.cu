// Launchers of the auxiliary Euler kernels and the layout scatter/gather.
#include "euler_aux.cuh"
#include "runtime.h"

namespace ripple {

cudaError_t launch_prep(int dtype, int dim, void* buf, FieldCtl* ctl, const FieldGeom& g, int bc, double gamma,
                        const double inv_dx[3], int slot, int grid, cudaStream_t s)
{
    if (dtype == RIPPLE_F32) {
        if (dim == 2)
            euler_prep_kernel<float, 2><<<grid, 256, 0, s>>>(static_cast<float*>(buf), ctl, g, bc, gamma, inv_dx[0],
                                                             inv_dx[1], inv_dx[2], slot);
        else
            euler_prep_kernel<float, 3><<<grid, 256, 0, s>>>(static_cast<float*>(buf), ctl, g, bc, gamma, inv_dx[0],
                                                             inv_dx[1], inv_dx[2], slot);
    } else {
        if (dim == 2)
            euler_prep_kernel<double, 2><<<grid, 256, 0, s>>>(static_cast<double*>(buf), ctl, g, bc, gamma,
                                                              inv_dx[0], inv_dx[1], inv_dx[2], slot);
        else
            euler_prep_kernel<double, 3><<<grid, 256, 0, s>>>(static_cast<double*>(buf), ctl, g, bc, gamma,
                                                              inv_dx[0], inv_dx[1], inv_dx[2], slot);
    }
    return cudaGetLastError();
}

cudaError_t launch_pad_nan(int dtype, void* buf, const FieldGeom& g, int grid, cudaStream_t s)
{
    if (dtype == RIPPLE_F32) pad_fill_nan_kernel<float><<<grid, 256, 0, s>>>(static_cast<float*>(buf), g);
    else pad_fill_nan_kernel<double><<<grid, 256, 0, s>>>(static_cast<double*>(buf), g);
    return cudaGetLastError();
}

cudaError_t launch_totals(int dtype, int ncomp, const void* buf, const FieldGeom& g, double* partials, int nblocks,
                          FieldCtl* ctl, cudaStream_t s)
{
#define RIPPLE_TOTALS(T, NCOMP) \
    totals_partial_kernel<T, NCOMP><<<nblocks, 256, 0, s>>>(static_cast<const T*>(buf), g, partials)
    if (dtype == RIPPLE_F32) {
        switch (ncomp) {
            case 1: RIPPLE_TOTALS(float, 1); break;
            case 2: RIPPLE_TOTALS(float, 2); break;
            case 3: RIPPLE_TOTALS(float, 3); break;
            case 4: RIPPLE_TOTALS(float, 4); break;
            default: RIPPLE_TOTALS(float, 5); break;
        }
    } else {
        switch (ncomp) {
            case 1: RIPPLE_TOTALS(double, 1); break;
            case 2: RIPPLE_TOTALS(double, 2); break;
            case 3: RIPPLE_TOTALS(double, 3); break;
            case 4: RIPPLE_TOTALS(double, 4); break;
            default: RIPPLE_TOTALS(double, 5); break;
        }
    }
#undef RIPPLE_TOTALS
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    totals_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, ncomp, ctl);
    return cudaGetLastError();
}

cudaError_t launch_interior_copy(int dtype, void* buf, const FieldGeom& g, void* dense, int dense_layout, int dir,
                                 int grid, cudaStream_t s)
{
    if (dtype == RIPPLE_F32)
        interior_copy_kernel<float><<<grid, 256, 0, s>>>(static_cast<float*>(buf), g, static_cast<float*>(dense),
                                                         dense_layout, dir);
    else
        interior_copy_kernel<double><<<grid, 256, 0, s>>>(static_cast<double*>(buf), g, static_cast<double*>(dense),
                                                          dense_layout, dir);
    return cudaGetLastError();
}

cudaError_t launch_group(int dtype, int op, const GroupItem* items, int n, long long blocks, cudaStream_t s)
{
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)blocks;
    if (dtype == RIPPLE_F32) {
        if (op == GROUP_ADMIT_FILL) group_admit_fill_kernel<float><<<grid, 256, 0, s>>>(items, n);
        else if (op == GROUP_ADMIT_PREP) group_admit_prep_kernel<float><<<grid, 256, 0, s>>>(items, n);
        else group_pack_kernel<float><<<grid, 256, 0, s>>>(items, n);
    } else {
        if (op == GROUP_ADMIT_FILL) group_admit_fill_kernel<double><<<grid, 256, 0, s>>>(items, n);
        else if (op == GROUP_ADMIT_PREP) group_admit_prep_kernel<double><<<grid, 256, 0, s>>>(items, n);
        else group_pack_kernel<double><<<grid, 256, 0, s>>>(items, n);
    }
    return cudaGetLastError();
}

}  // namespace ripple
