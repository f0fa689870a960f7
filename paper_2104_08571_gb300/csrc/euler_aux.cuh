// Auxiliary kernels of the Euler path: the first padding fill + wave-speed
// reduction of a freshly uploaded state, the FP64 compensated conserved
// totals, and the interior scatter/gather used by upload and download.
#pragma once
#include <cstdint>

#include "euler_sweep.cuh"
#include "field.cuh"

namespace ripple {

// Read the conserved state of interior cell (i, j, k).
template <typename T, int DIM>
__device__ __forceinline__ void load_cell(const T* __restrict__ buf, const FieldGeom& g, int i, int j, int k,
                                          T (&q)[DIM + 2])
{
    const long long base = geom_cell(g, i, j, k) * g.cell_stride;
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) q[m] = buf[base + (long long)m * g.comp_stride];
}

__device__ __forceinline__ void cell_coords(const FieldGeom& g, long long lin, int& i, int& j, int& k)
{
    i = (int)(lin % g.n[0]);
    const long long r = lin / g.n[0];
    j = (int)(r % g.n[1]);
    k = (int)(r / g.n[1]);
}

// set_boundary + set_wavespeeds + MaxReducer on the current buffer (used once
// after an upload or a change of boundary condition / gamma / dx; the sweep
// itself keeps both up to date afterwards).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) euler_prep_kernel(T* __restrict__ buf, FieldCtl* __restrict__ ctl,
                                                         const FieldGeom g, int bc, double gamma, double idx0,
                                                         double idx1, double idx2, int slot)
{
    const T gm = (T)gamma, gm1 = (T)(gamma - 1.0);
    const T inv_dx[3] = {(T)idx0, (T)idx1, (T)idx2};
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    T smax = T(0);
    bool bad = false;
    for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
         lin += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(g, lin, i, j, k);
        T q[DIM + 2];
        load_cell<T, DIM>(buf, g, i, j, k, q);
        bool ok;
        smax = fmax(smax, wave_sum<T, DIM>(q, gm, gm1, inv_dx, ok));
        if (!ok) { bad = true; record_bad(ctl, BAD_INPUT, i, j, k); }
        write_ghost_images<T, DIM>(buf, g, bc, i, j, k, q);
    }
    __shared__ double red[8];
    double v = (double)smax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        atomic_max_pos_double(&ctl->smax[slot], m);
        if (any_bad) atomicOr(&ctl->err, DEV_ERR_NUMERIC);
    }
}

// Quiet NaN in every padded cell outside the interior (all components).  The
// sweep rewrites the face ghosts each step; edge and corner ghosts and the
// alignment padding stay NaN, so a stencil item that reaches beyond the
// ghost layers carries NaN, which the admissibility minimum ignores.
template <typename T>
__global__ void __launch_bounds__(256) pad_fill_nan_kernel(T* __restrict__ buf, const FieldGeom g)
{
    const long long cells = g.px * g.py * g.pz;
    const T qnan = (T)__int_as_float(0x7fc00000);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
         c += (long long)gridDim.x * blockDim.x) {
        const long long x = c % g.px, r = c / g.px;
        const long long y = r % g.py, z = r / g.py;
        const bool inside = x >= g.lead + g.h && x < g.lead + g.h + g.n[0] && y >= g.h && y < g.h + g.n[1] &&
                            (g.ndim < 3 || (z >= g.h && z < g.h + g.n[2]));
        if (inside) continue;
        for (int m = 0; m < g.ncomp; ++m) buf[c * g.cell_stride + (long long)m * g.comp_stride] = qnan;
    }
}

// Neumaier (improved Kahan-Babuska) compensated accumulation in FP64.
struct Neumaier {
    double s, c;
    __device__ void add(double x)
    {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ void merge(const Neumaier& o)
    {
        add(o.s);
        c += o.c;
    }
};

// Per-block compensated partial sums of each component over interior cells.
// partials[(block * ncomp + m) * 2 + {0: sum, 1: compensation}]
template <typename T, int NCOMP>
__global__ void __launch_bounds__(256) totals_partial_kernel(const T* __restrict__ buf, const FieldGeom g,
                                                             double* __restrict__ partials)
{
    Neumaier acc[NCOMP];
#pragma unroll
    for (int m = 0; m < NCOMP; ++m) acc[m] = Neumaier{0.0, 0.0};
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
         lin += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(g, lin, i, j, k);
        const long long base = geom_cell(g, i, j, k) * g.cell_stride;
#pragma unroll
        for (int m = 0; m < NCOMP; ++m) acc[m].add((double)buf[base + (long long)m * g.comp_stride]);
    }
    // fixed-order block combination: warp tree, then warps in order
    __shared__ double sh[8][NCOMP][2];
#pragma unroll
    for (int m = 0; m < NCOMP; ++m) {
        for (int o = 16; o > 0; o >>= 1) {
            Neumaier other{__shfl_down_sync(0xffffffffu, acc[m].s, o), __shfl_down_sync(0xffffffffu, acc[m].c, o)};
            acc[m].merge(other);
        }
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int m = 0; m < NCOMP; ++m) {
            sh[w][m][0] = acc[m].s;
            sh[w][m][1] = acc[m].c;
        }
    __syncthreads();
    if (threadIdx.x < NCOMP) {
        const int m = threadIdx.x;
        Neumaier b{0.0, 0.0};
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) b.merge(Neumaier{sh[ww][m][0], sh[ww][m][1]});
        partials[((long long)blockIdx.x * NCOMP + m) * 2 + 0] = b.s;
        partials[((long long)blockIdx.x * NCOMP + m) * 2 + 1] = b.c;
    }
}

// Fixed-order final pass over the block partials (one thread per component).
__global__ void totals_final_kernel(const double* __restrict__ partials, int nblocks, int ncomp,
                                    FieldCtl* __restrict__ ctl)
{
    const int m = threadIdx.x;
    if (m >= ncomp) return;
    Neumaier b{0.0, 0.0};
    for (int blk = 0; blk < nblocks; ++blk)
        b.merge(Neumaier{partials[((long long)blk * ncomp + m) * 2], partials[((long long)blk * ncomp + m) * 2 + 1]});
    ctl->totals[m] = b.s + b.c;
}

// Interior copy between a dense array in the given layout and the padded field.
// dir = 0: dense -> field (upload), dir = 1: field -> dense (download).
template <typename T>
__global__ void __launch_bounds__(256) interior_copy_kernel(T* __restrict__ buf, const FieldGeom g,
                                                            T* __restrict__ dense, int dense_layout, int dir)
{
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
         lin += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(g, lin, i, j, k);
        const long long base = geom_cell(g, i, j, k) * g.cell_stride;
        for (int m = 0; m < g.ncomp; ++m) {
            const long long di = dense_layout == LAYOUT_SOA ? (long long)m * total + lin : lin * g.ncomp + m;
            const long long fi = base + (long long)m * g.comp_stride;
            if (dir == 0) buf[fi] = dense[di];
            else dense[di] = buf[fi];
        }
    }
}

}  // namespace ripple
