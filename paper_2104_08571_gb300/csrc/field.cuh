// Field geometry and per-field device control block, shared by the kernels and
// the host runtime.
//
// A field is the padded tensor of the paper's Section 4.1 with the layouts of
// Section 4.2.  Every axis carries `h` ghost layers on both sides (2D fields
// have a single z plane).  Along x an extra `lead` column pad precedes the
// ghosts so that the first interior cell starts on a 16-byte boundary: TMA
// tile stores of interior boxes then satisfy the 16-byte start rule.
//   padded x of interior cell i  = lead + h + i
//   padded y of interior cell j  = h + j
//   padded z of interior cell k  = h + k (3D) or 0 (2D)
//   cell index c = (pz * py + pyy) * px + pxx
//   element      = c * cell_stride + m * comp_stride
//     SoA: cell_stride = 1,     comp_stride = px * py * pz
//     AoS: cell_stride = ncomp, comp_stride = 1
#pragma once
#include <cstdint>

namespace ripple {

enum { LAYOUT_AOS = 0, LAYOUT_SOA = 1 };

// Device-side error flags (FieldCtl::err), mapped to ripple_status by the host.
// DEV_ERR_BARRIER: a bounded grid-barrier wait ran out (a CTA was not resident
// or stalled), as distinct from an iteration cap reached (DEV_ERR_TIMEOUT).
enum : unsigned { DEV_ERR_NUMERIC = 1u, DEV_ERR_TIMEOUT = 2u, DEV_ERR_INTERNAL = 4u, DEV_ERR_BARRIER = 8u };

struct FieldGeom {
    int ndim, ncomp, h, lead;
    int n[3];              // interior cells (n[2] = 1 in 2D)
    long long px, py, pz;  // padded extents
    long long cell_stride, comp_stride;
};

__host__ __device__ inline long long geom_cell(const FieldGeom& g, int i, int j, int k)
{
    long long pzz = g.ndim == 3 ? (long long)(k + g.h) : 0;
    return (pzz * g.py + (j + g.h)) * g.px + (g.lead + g.h + i);
}

__host__ __device__ inline long long geom_elem(const FieldGeom& g, int i, int j, int k, int m)
{
    return geom_cell(g, i, j, k) * g.cell_stride + (long long)m * g.comp_stride;
}

// Per-field control block in device memory.
struct FieldCtl {
    unsigned long long smax[3];  // ring of max wave-speed sums (bits of a positive double)
    double t;                    // simulated time advanced by the current call
    double dt_last;              // last dt
    unsigned int err;            // DEV_ERR_* flags
    unsigned int pad0;
    double totals[5];            // FP64 compensated totals (written by the totals kernel)
    long long counters[8];       // solver counters (eikonal iterations, visits, ...)
};


// One instance of a grouped admission or download of the batch runtime (the
// kernels are in euler_aux.cuh): every instance of a group owns a contiguous
// run of blocks of one launch, blk[pass] its first block in launch `pass`
// (an instance with no blocks in a launch repeats the next one's value).
constexpr int kGroupCellsPerBlock = 2048;  // 256 threads x 8 cells

struct GroupItem {
    void* buf;                    // admission: buffer 0; download: the buffer holding the result
    void* other;                  // admission: buffer 1, dense input on entry; download: the dense stage
    FieldCtl* ctl;                // the instance's slot entries
    unsigned long long* status;
    long long* counters;
    FieldGeom g;
    double gamma, inv_dx0, inv_dx1;
    int bc;
    int euler;                    // 1: Euler state (fill and prepare), 0: eikonal (slot reset only)
    long long blk[2];
};

}  // namespace ripple
