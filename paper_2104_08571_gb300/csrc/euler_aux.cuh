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


// ---------------------------------------------------------------------------
// Grouped admission and download of the batch runtime: one launch covers every
// instance of a group, each instance owning a contiguous run of blocks
// (GroupItem::blk[pass] = its first block in launch `pass`; instances with no
// blocks in a launch repeat the next instance's value).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int group_find(const GroupItem* __restrict__ items, int n, int pass, long long b)
{
    // last item whose first block is <= b
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].blk[pass] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool padded_inside(const FieldGeom& g, long long c, int& i, int& j, int& k)
{
    const long long x = c % g.px, r = c / g.px;
    const long long y = r % g.py, z = r / g.py;
    i = (int)(x - g.lead - g.h);
    j = (int)(y - g.h);
    k = g.ndim < 3 ? 0 : (int)(z - g.h);
    return i >= 0 && i < g.n[0] && j >= 0 && j < g.n[1] && (g.ndim < 3 || (k >= 0 && k < g.n[2]));
}

// Admission, launch 0 (padded cells of buffer 0): interior cells from the dense
// component-major input held in buffer 1, every other cell quiet NaN; the
// first block of an instance also clears its slot (control block, status,
// counters).  Eikonal instances own one block, which only clears the slot.
template <typename T>
__global__ void __launch_bounds__(256) group_admit_fill_kernel(const GroupItem* __restrict__ items, int n)
{
    const int it = group_find(items, n, 0, blockIdx.x);
    const GroupItem& d = items[it];
    const long long local = blockIdx.x - d.blk[0];
    if (local == 0) {
        unsigned* w = reinterpret_cast<unsigned*>(d.ctl);
        for (int q = threadIdx.x; q < (int)(sizeof(FieldCtl) / sizeof(unsigned)); q += blockDim.x) w[q] = 0u;
        if (threadIdx.x == 0) *d.status = 0ull;
        if (threadIdx.x < 3) d.counters[threadIdx.x] = 0;
    }
    if (!d.euler) return;
    const FieldGeom& g = d.g;
    T* buf = static_cast<T*>(d.buf);
    const T* dense = static_cast<const T*>(d.other);
    const long long cells = g.px * g.py * g.pz;
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    const T qnan = (T)__int_as_float(0x7fc00000);
    const long long c0 = local * kGroupCellsPerBlock;
    for (long long c = c0 + threadIdx.x; c < c0 + kGroupCellsPerBlock && c < cells; c += blockDim.x) {
        int i, j, k;
        const bool inside = padded_inside(g, c, i, j, k);
        const long long lin = ((long long)k * g.n[1] + j) * g.n[0] + i;
        for (int m = 0; m < g.ncomp; ++m)
            buf[c * g.cell_stride + (long long)m * g.comp_stride] = inside ? dense[(long long)m * total + lin] : qnan;
    }
}

// Admission, launch 1 (padded cells again): on buffer 0 the boundary images
// of each interior cell, the largest wave-speed sum (ring slot 0) and the
// admissibility check of the input; on buffer 1 quiet NaN outside the
// interior.  Runs after launch 0 (buffer 1's dense input has been read).
template <typename T>
__global__ void __launch_bounds__(256) group_admit_prep_kernel(const GroupItem* __restrict__ items, int n)
{
    const int it = group_find(items, n, 1, blockIdx.x);
    const GroupItem& d = items[it];
    const long long local = blockIdx.x - d.blk[1];
    const FieldGeom& g = d.g;
    T* buf = static_cast<T*>(d.buf);
    T* other = static_cast<T*>(d.other);
    const T gm = (T)d.gamma, gm1 = (T)(d.gamma - 1.0);
    const T inv_dx[3] = {(T)d.inv_dx0, (T)d.inv_dx1, (T)0};
    const long long cells = g.px * g.py * g.pz;
    const T qnan = (T)__int_as_float(0x7fc00000);
    T smax = T(0);
    bool bad = false;
    const long long c0 = local * kGroupCellsPerBlock;
    for (long long c = c0 + threadIdx.x; c < c0 + kGroupCellsPerBlock && c < cells; c += blockDim.x) {
        int i, j, k;
        if (!padded_inside(g, c, i, j, k)) {
            for (int m = 0; m < g.ncomp; ++m) other[c * g.cell_stride + (long long)m * g.comp_stride] = qnan;
            continue;
        }
        T q[4];
        load_cell<T, 2>(buf, g, i, j, k, q);
        bool ok;
        smax = fmax(smax, wave_sum<T, 2>(q, gm, gm1, inv_dx, ok));
        if (!ok) { bad = true; record_bad(d.ctl, BAD_INPUT, i, j, k); }
        write_ghost_images<T, 2>(buf, g, d.bc, i, j, k, q);
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
        atomic_max_pos_double(&d.ctl->smax[0], m);
        if (any_bad) atomicOr(&d.ctl->err, DEV_ERR_NUMERIC);
    }
}

// Download: the interior of each instance's result buffer into its dense
// component-major stage (interior cells, blk[0]).
template <typename T>
__global__ void __launch_bounds__(256) group_pack_kernel(const GroupItem* __restrict__ items, int n)
{
    const int it = group_find(items, n, 0, blockIdx.x);
    const GroupItem& d = items[it];
    const long long local = blockIdx.x - d.blk[0];
    const FieldGeom& g = d.g;
    const T* buf = static_cast<const T*>(d.buf);
    T* dense = static_cast<T*>(d.other);
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long l0 = local * kGroupCellsPerBlock;
    for (long long lin = l0 + threadIdx.x; lin < l0 + kGroupCellsPerBlock && lin < total; lin += blockDim.x) {
        int i, j, k;
        cell_coords(g, lin, i, j, k);
        const long long base = geom_cell(g, i, j, k) * g.cell_stride;
        for (int m = 0; m < g.ncomp; ++m) dense[(long long)m * total + lin] = buf[base + (long long)m * g.comp_stride];
    }
}

}  // namespace ripple
