// FP32 2D and 3D sweeps of the dimensionally split FORCE step (the paper's
// own Euler solver, Section 7.3, Listing euler_graph) on strip walks, sm_103a.
//
// One sweep of the split step reads the one-cell neighbours along a single
// axis, so it needs no tile and no block barrier.  Each warp walks a strip
// 64 cells wide along the swept axis, one chunk of 64 cells (one row
// segment) at a time; every lane owns a pair of x-adjacent cells held as
// f32x2 values, so the flux and update arithmetic issues once for two cells
// (pair_math.cuh).
//   x sweep (AXIS 0): a walk runs along a row (one y, one z).  Lane l
//     evaluates the right faces of its two cells as one pair; the left faces
//     are lane l - 1's right faces (a shuffle) and, for lane 0, the last face
//     of the previous chunk, carried in registers.  The right neighbour of
//     lane 31 is the first cell after the chunk, staged with it.
//   y or z sweep (AXIS 1, 2): a walk runs along the swept axis through the
//     rows of a 64-column strip (of one z plane for y, one y row for z); the
//     face below a row is the face above the next one.  The two differ only
//     in the stride between rows.
// Either way every face of a walk is evaluated once; the first face of a walk
// is evaluated again by the walk before it (the host makes walks long enough
// that this stays a few per cent of the arithmetic).
//
// Staging: every warp owns a ring of NS shared-memory slots of one chunk
// (1 KB) each, filled by per-thread asynchronous copies (cp.async) NS - 1
// chunks (x) or NS - 2 rows (y) ahead of the arithmetic, so the loads in
// flight cost no registers.  A thread waits for its own copy groups only
// (cp.async.wait_group), so no wait can hang, and no CTA barrier is needed.
// AoS lanes copy exactly the cells they read (two 16-byte cells); SoA chunks
// move as 16-byte copies that span two lanes' pairs (half the copies of
// per-lane 8-byte ones, measured 2 % faster), so there __syncwarp publishes
// the lanes' copies to each other and ends their reads of a slot before it
// is refilled (AoS without the barrier: 1 % faster).  Stores are
// coalesced and direct.  dt, t and the CFL maximum follow the tiled sweep: dt
// from the wave-speed maximum of the step's input state; the last sweep of a
// step advances t and reduces the maximum of the new state.  Cells on the
// boundary write their ghost images for the next sweep, as in every sweep.
#pragma once
#include <cstdint>

#include "euler_sweep.cuh"
#include "pair_math.cuh"

namespace ripple {

template <int DIM, int NS_>
struct WalkCfg {
    static constexpr int NC = DIM + 2;
    static constexpr int NS = NS_;                                // ring slots per warp
    static constexpr int SLOT = ((64 * NC + NC + 3) / 4) * 4;     // floats: a chunk + lane 31's right neighbour
    static constexpr int SMEM = kWalkWarps * NS * SLOT * 4;       // dynamic shared memory per CTA
    static_assert(NS >= 3, "the y and z sweeps keep two rows resident");
};
constexpr int kWalkSlots = 6;

template <int DIM, int LAYOUT, int AXIS, int NS>
__global__ void __launch_bounds__(kWalkWarps * 32, 2)
    euler_force_walk_kernel(const float* __restrict__ in, float* __restrict__ out, FieldCtl* __restrict__ ctl,
                            const WalkGeom wg, const SweepParams prm)
{
    constexpr int NC = DIM + 2, SLOT = WalkCfg<DIM, NS>::SLOT;
    // 2D AoS cells are 16 bytes: a lane stages exactly the two cells it reads.
    // Otherwise a chunk moves as 16-byte pieces that span several lanes' cells,
    // published to the warp by __syncwarp.
    constexpr bool kOwnCells = LAYOUT == LAYOUT_AOS && NC == 4;
    const FieldGeom& g = wg.f;
    const int tid = threadIdx.x, lane = tid & 31;
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    extern __shared__ __align__(128) float wsm[];
    float* ring = wsm + warp * NS * SLOT;
    __shared__ float sdt[4];
    __shared__ double red[kWalkWarps];
    if (tid == 0) {
        // dt from the max wave-speed sum of the step's input state (FP64, as the
        // tiled sweep); its FP32 forms rounded here once
        const double dt = prm.cfl / __longlong_as_double((long long)ctl->smax[prm.slot_in]);
        sdt[0] = (float)dt;
        sdt[1] = (float)(0.5 * dt * prm.inv_dx[AXIS]);
        sdt[2] = (float)(0.5 / (dt * prm.inv_dx[AXIS]));  // (dx/dt)/2
        if (blockIdx.x == 0 && prm.last) {
            ctl->t = prm.first ? dt : ctl->t + dt;
            ctl->dt_last = dt;
            ctl->smax[(prm.slot_in + 2) % 3] = 0ull;
        }
    }
    __syncthreads();
    const f2 gamma = splat<f2>(prm.gamma_f), gm1 = splat<f2>(prm.gm1_f);
    const f2 hdt = splat<f2>(sdt[1]), hidt = splat<f2>(sdt[2]);
    const float dtf = sdt[0];
    const f2 ndt = f2{-dtf, -dtf};
    f2 ivx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ivx[d] = splat<f2>(prm.inv_dx_f[d]);
    const f2 iv = ivx[AXIS];
    const int nx = g.n[0];
    const long long cs = g.comp_stride;
    float smax_local = 0.f;
    bool bad = false;

    // Stage the chunk of 64 cells from x0 of the row whose x = 0 cell is the
    // padded cell rb into slot s.  Slot layout: SoA component m at [64 m, 64 m
    // + 64); AoS cell i at [NC i, NC i + NC).  A whole chunk moves as 16-byte
    // copies coalesced across the warp (SoA: 16 per component row; AoS: the
    // chunk's contiguous bytes, or in 2D the lane's own two cells); the lane's
    // pieces (slot offset, source offset from the chunk's first cell) are
    // formed once here.  A chunk past the last cell copies each lane's two
    // cells with the index clamped to the ghost cell x = nx (never stored).
    constexpr int NPIECE = kOwnCells ? 64 : 16 * NC;  // 16-byte pieces of a full chunk
    constexpr int PPL = (NPIECE + 31) / 32;           // per lane
    int pdst[PPL];
    long long psrc[PPL];
#pragma unroll
    for (int t = 0; t < PPL; ++t) {
        const int i = kOwnCells ? 2 * lane + t : lane + 32 * t;
        if constexpr (kOwnCells) {
            pdst[t] = 4 * i;
            psrc[t] = (long long)i * NC;
        } else if constexpr (LAYOUT == LAYOUT_SOA) {
            const int m = i >> 4, part = i & 15;
            pdst[t] = 64 * m + 4 * part;
            psrc[t] = (long long)m * cs + 4 * part;
        } else {
            pdst[t] = 4 * i;
            psrc[t] = 4LL * i;
        }
        if (i >= NPIECE) pdst[t] = -1;
    }
    auto stage = [&](float* s, long long rb, int x0) {
        if (x0 + 64 <= nx) {
            const float* src = LAYOUT == LAYOUT_SOA ? in + rb + x0 : in + (rb + x0) * NC;
#pragma unroll
            for (int t = 0; t < PPL; ++t)
                if (t * 32 + 31 < NPIECE || pdst[t] >= 0) cp_async16(s + pdst[t], src + psrc[t]);
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = 2 * lane + h;
                const long long src = rb + min(x0 + c, nx);
                if constexpr (LAYOUT == LAYOUT_SOA) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) cp_async4(s + 64 * m + c, in + src + m * cs);
                } else if constexpr (kOwnCells) {
                    cp_async16(s + 4 * c, in + src * NC);
                } else {
#pragma unroll
                    for (int m = 0; m < NC; ++m) cp_async4(s + NC * c + m, in + src * NC + m);
                }
            }
        }
    };
    // lane 31: the cell after the chunk (the next chunk's first, or the ghost
    // x = nx), components at [256, 260) of the slot
    constexpr int NEXT = 64 * NC;  // offset of the cell after the chunk in a slot
    auto stage_next = [&](float* s, long long rb, int x0) {
        if (lane != 31) return;
        const long long src = rb + min(x0 + 64, nx);
        if constexpr (LAYOUT == LAYOUT_SOA) {
#pragma unroll
            for (int m = 0; m < NC; ++m) cp_async4(s + NEXT + m, in + src + m * cs);
        } else if constexpr (kOwnCells) {
            cp_async16(s + NEXT, in + src * NC);
        } else {
#pragma unroll
            for (int m = 0; m < NC; ++m) cp_async4(s + NEXT + m, in + src * NC + m);
        }
    };
    // lanes read cells that other lanes copied (see above)
    auto ring_sync = [&]() {
        if constexpr (!kOwnCells) __syncwarp();
    };
    // the lane's pair of cells (2 lane, 2 lane + 1) of a staged chunk
    auto read_pair = [&](const float* s, f2 (&q)[NC]) {
        if constexpr (LAYOUT == LAYOUT_SOA) {
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                const float2 v = *reinterpret_cast<const float2*>(s + 64 * m + 2 * lane);
                q[m] = f2{v.x, v.y};
            }
        } else if constexpr (kOwnCells) {
            const float4 A = *reinterpret_cast<const float4*>(s + 8 * lane);
            const float4 B = *reinterpret_cast<const float4*>(s + 8 * lane + 4);
            q[0] = f2{A.x, B.x}; q[1] = f2{A.y, B.y}; q[2] = f2{A.z, B.z}; q[3] = f2{A.w, B.w};
        } else {
#pragma unroll
            for (int m = 0; m < NC; ++m) q[m] = f2{s[NC * 2 * lane + m], s[NC * (2 * lane + 1) + m]};
        }
    };
    auto load_cell = [&](long long c, float (&v)[NC]) {
        if constexpr (LAYOUT == LAYOUT_SOA) {
#pragma unroll
            for (int m = 0; m < NC; ++m) v[m] = in[c + m * cs];
        } else if constexpr (kOwnCells) {
            const float4 A = *reinterpret_cast<const float4*>(in + c * NC);
            v[0] = A.x; v[1] = A.y; v[2] = A.z; v[3] = A.w;
        } else {
#pragma unroll
            for (int m = 0; m < NC; ++m) v[m] = in[c * NC + m];
        }
    };
    // updated pair of cells (x, x + 1) of row (y, z): checks, CFL maximum, store, ghost images
    auto finish = [&](const f2 (&qn)[NC], long long c, int x, int y, int z, bool v0, bool v1, bool near) {
        // the wave speeds (and the admissibility of the new state) in the last
        // sweep of a step only: the step's CFL maximum is that of its result,
        // and an intermediate state reaches the next sweep's faces, whose
        // states are checked there
        bool ok0 = true, ok1 = true;
        if (prm.last) {
            const f2 sw = wave_sum2<DIM>(qn, gamma, gm1, ivx, ok0, ok1);
            smax_local = fmaxf(smax_local, fmaxf(v0 ? sw.x : 0.f, v1 ? sw.y : 0.f));
        }
        const bool b0 = v0 && !ok0, b1 = v1 && !ok1;
        // warp-uniform branches around the rare paths (a non-admissible cell, a
        // ragged last chunk), so the common path has no divergent region
        if (__any_sync(0xffffffffu, b0 || b1)) {
            if (b0 || b1) {
                bad = true;
                record_bad(ctl, BAD_CELL, b0 ? x : x + 1, y, z);
            }
        }
        if (__all_sync(0xffffffffu, v0 && v1) || (v0 && v1)) {
            if constexpr (LAYOUT == LAYOUT_SOA) {
#pragma unroll
                for (int m = 0; m < NC; ++m)
                    *reinterpret_cast<float2*>(out + c + m * cs) = make_float2(qn[m].x, qn[m].y);
            } else if constexpr (kOwnCells) {
                *reinterpret_cast<float4*>(out + c * NC) = make_float4(qn[0].x, qn[1].x, qn[2].x, qn[3].x);
                *reinterpret_cast<float4*>(out + c * NC + NC) = make_float4(qn[0].y, qn[1].y, qn[2].y, qn[3].y);
            } else {
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    out[c * NC + m] = qn[m].x;
                    out[(c + 1) * NC + m] = qn[m].y;
                }
            }
        } else if (v0) {
#pragma unroll
            for (int m = 0; m < NC; ++m) out[c * g.cell_stride + m * cs] = qn[m].x;
        }
        if (near) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h == 0 ? v0 : v1)) continue;
                float q1[NC];
#pragma unroll
                for (int m = 0; m < NC; ++m) q1[m] = h == 0 ? qn[m].x : qn[m].y;
                write_ghost_images<float, DIM>(out, g, prm.bc, x + h, y, z, q1);
            }
        }
    };
    // padded cell index of cell (0, y, z)
    auto row_base = [&](int y, int z) -> long long {
        return ((long long)(DIM == 3 ? g.h + z : 0) * g.py + (g.h + y)) * g.px + g.lead + g.h;
    };

    // x sweep: the face xs - 1/2 that starts each walk, for 32 of the warp's
    // walks at a time (lane j: the warp's walk jb + j), in the packed
    // arithmetic of the walk before, which gives the same bits: the two walks
    // agree on their common face exactly.  One evaluation per 32 walks instead
    // of one per walk (a 256-cell row is a walk of only four chunks).
    const int wstride = gridDim.x * kWalkWarps;
    float bface[NC];
    float bchk = 1.f;
    int jw = 0;  // walks of this warp so far
    for (int w = blockIdx.x * kWalkWarps + warp; w < wg.walks; w += wstride, ++jw) {
        float chk = 1.f;
        int wx, wy, wz = 0;  // first cell of the walk (reported with a non-admissible face state)
        ring_sync();  // the previous walk's reads of the ring come before its refill
        if constexpr (AXIS == 0) {
            const int r = w / wg.nseg, xs = (w % wg.nseg) * wg.seg;
            const int y = r % g.n[1], z = r / g.n[1];
            const int xe = min(xs + wg.seg, nx);
            const int nch = (xe - xs + 63) >> 6;
            const long long rb = row_base(y, z);  // padded cell of x = 0
            const bool row_near = y < g.h || y >= g.n[1] - g.h || (DIM == 3 && (z < g.h || z >= g.n[2] - g.h));
            wx = xs;
            wy = y;
            wz = z;
            // chunk k in slot k % NS, staged NS - 1 chunks ahead (one copy group per chunk)
#pragma unroll
            for (int k = 0; k < NS - 1; ++k) {
                if (k < nch) {
                    stage(ring + k * SLOT, rb, xs + 64 * k);
                    stage_next(ring + k * SLOT, rb, xs + 64 * k);
                }
                cp_async_commit();
            }
            // face xs - 1/2, the left face of lane 0's first chunk
            if ((jw & 31) == 0) {
                const int wl = w + lane * wstride;  // this lane's walk of the batch
                const int rl = min(wl, wg.walks - 1) / wg.nseg, xl = (min(wl, wg.walks - 1) % wg.nseg) * wg.seg;
                const long long rbl = row_base(rl % g.n[1], rl / g.n[1]);
                float l[NC], r[NC];
                load_cell(rbl + xl - 1, l);
                load_cell(rbl + xl, r);
                f2 a[NC], b[NC], F[NC];
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    a[m] = splat<f2>(l[m]);
                    b[m] = splat<f2>(r[m]);
                }
                bchk = 1.f;
                force<f2, DIM, 0>(a, b, gm1, hdt, hidt, F, bchk);
#pragma unroll
                for (int m = 0; m < NC; ++m) bface[m] = F[m].x;
            }
            float carry[NC];
#pragma unroll
            for (int m = 0; m < NC; ++m) carry[m] = __shfl_sync(0xffffffffu, bface[m], jw & 31);
            chk = __shfl_sync(0xffffffffu, bchk, jw & 31);
            int slot = 0;  // slot of chunk k
#pragma unroll 1
            for (int k = 0; k < nch; ++k) {
                const int x0 = xs + (k << 6), x = x0 + 2 * lane;
                {
                    // refill the slot read in the previous iteration with chunk k + NS - 1
                    const int kn = k + NS - 1;
                    float* s = ring + (slot == 0 ? NS - 1 : slot - 1) * SLOT;
                    ring_sync();
                    if (kn < nch) {
                        stage(s, rb, xs + 64 * kn);
                        stage_next(s, rb, xs + 64 * kn);
                    }
                    cp_async_commit();
                }
                cp_async_wait<NS - 1>();  // chunk k has landed
                ring_sync();
                const float* s = ring + slot * SLOT;
                f2 q[NC], b[NC], Fr[NC], qn[NC];
                read_pair(s, q);
                // right faces of the lane's cells: (x | x + 1) and (x + 1 | x + 2)
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    float rn = __shfl_down_sync(0xffffffffu, q[m].x, 1);
                    if (lane == 31) rn = s[NEXT + m];
                    b[m] = f2{q[m].y, rn};
                }
                force<f2, DIM, 0>(q, b, gm1, hdt, hidt, Fr, chk);
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    float fl = __shfl_up_sync(0xffffffffu, Fr[m].y, 1);
                    if (lane == 0) fl = carry[m];
                    carry[m] = __shfl_sync(0xffffffffu, Fr[m].y, 31);
                    qn[m] = fma_v(ndt, (Fr[m] - f2{fl, Fr[m].x}) * iv, q[m]);
                }
                finish(qn, rb + x, x, y, z, x < xe, x + 1 < xe, row_near || x0 < g.h || x0 + 64 > nx - g.h);
                slot = slot == NS - 1 ? 0 : slot + 1;
            }
        } else {
            // walk: strip of columns x0 .. x0 + 63, line (z for a y sweep, y for a z
            // sweep), rows ys .. ye - 1 along the swept axis
            const int na = g.n[AXIS];
            const int strip = w % wg.nstrips, rest = w / wg.nstrips;
            const int line = rest % wg.nlines, ys = (rest / wg.nlines) * wg.seg;
            const int ye = min(ys + wg.seg, na);
            const int x0 = strip << 6, x = x0 + 2 * lane;
            const bool v0 = x < nx, v1 = x + 1 < nx;
            const int nl = DIM == 3 ? g.n[AXIS == 1 ? 2 : 1] : 1;
            const bool col_near = x0 < g.h || x0 + 64 > nx - g.h || (DIM == 3 && (line < g.h || line >= nl - g.h));
            const long long stride = AXIS == 1 ? g.px : g.px * g.py;
            const long long base = AXIS == 1 ? row_base(0, line) : row_base(line, 0);  // padded cell of (0, row 0)
            auto coords = [&](int row, int& y, int& z) {
                y = AXIS == 1 ? row : line;
                z = AXIS == 1 ? line : row;
            };
            wx = x0;
            coords(ys, wy, wz);
            // row ys - 1 + i in slot i % NS, i = 0 .. ye - ys + 1 (rows ys - 1 and ye
            // are ghost rows at the field's edges), staged NS - 2 rows ahead
            const int nrows = ye - ys + 2;
#pragma unroll
            for (int i = 0; i < NS - 1; ++i) {
                if (i < nrows) stage(ring + i * SLOT, base + (long long)(ys - 1 + i) * stride, x0);
                cp_async_commit();
            }
            cp_async_wait<NS - 3>();  // rows ys - 1 and ys
            ring_sync();
            f2 Fl[NC];  // face below row r (between rows r - 1 and r)
            {
                f2 up[NC], q0[NC];
                read_pair(ring, up);
                read_pair(ring + SLOT, q0);
                force<f2, DIM, AXIS>(up, q0, gm1, hdt, hidt, Fl, chk);
            }
            int slot = 1;  // slot of row r
            long long rb_next = base + (long long)(ys + NS - 2) * stride;  // row ys - 1 + (i + NS - 2)
            long long c_row = base + (long long)ys * stride + x;            // the lane's first cell of row r
#pragma unroll 1
            for (int r = ys; r < ye; ++r, rb_next += stride, c_row += stride) {
                const int i = r - ys + 1;
                {
                    // refill the slot of row i - 2 (read in the previous iteration) with row i + NS - 2
                    const int ir = i + NS - 2;
                    const int sr = slot >= 2 ? slot - 2 : slot + NS - 2;
                    ring_sync();
                    if (ir < nrows) stage(ring + sr * SLOT, rb_next, x0);
                    cp_async_commit();
                }
                cp_async_wait<NS - 3>();  // rows r and r + 1
                ring_sync();
                const int sn = slot == NS - 1 ? 0 : slot + 1;
                f2 q[NC], qd[NC], Fr[NC], qn[NC];
                read_pair(ring + slot * SLOT, q);
                read_pair(ring + sn * SLOT, qd);
                force<f2, DIM, AXIS>(q, qd, gm1, hdt, hidt, Fr, chk);
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    qn[m] = fma_v(ndt, (Fr[m] - Fl[m]) * iv, q[m]);
                    Fl[m] = Fr[m];
                }
                int y, z;
                coords(r, y, z);
                finish(qn, c_row, x, y, z, v0, v1, col_near || r < g.h || r >= na - g.h);
                slot = sn;
            }
        }
        if (!(chk > 0.f)) {
            bad = true;
            record_bad(ctl, BAD_STATE, wx, wy, wz);
        }
    }
    cp_async_wait<0>();

    double v = (double)smax_local;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int k = 0; k < kWalkWarps; ++k) m = fmax(m, red[k]);
        if (prm.last) atomic_max_pos_double(&ctl->smax[(prm.slot_in + 1) % 3], m);
        if (any_bad) atomicOr(&ctl->err, DEV_ERR_NUMERIC);
    }
}

}  // namespace ripple

#include "runtime.h"

namespace ripple {

// Host launch helpers of the walk sweeps (one instantiation per dim, layout, axis).
template <int DIM, int LAYOUT, int AXIS>
static cudaError_t walk_configure()
{
    static cudaError_t e = cudaFuncSetAttribute(euler_force_walk_kernel<DIM, LAYOUT, AXIS, kWalkSlots>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                WalkCfg<DIM, kWalkSlots>::SMEM);
    return e;
}
template <int DIM, int LAYOUT, int AXIS>
static cudaError_t walk_launch(const WalkLaunch& L)
{
    const cudaError_t e = walk_configure<DIM, LAYOUT, AXIS>();
    if (e != cudaSuccess) return e;
    euler_force_walk_kernel<DIM, LAYOUT, AXIS, kWalkSlots>
        <<<L.grid, kWalkWarps * 32, WalkCfg<DIM, kWalkSlots>::SMEM, L.stream>>>(
            static_cast<const float*>(L.in), static_cast<float*>(L.out), L.ctl, L.wg, L.prm);
    return cudaGetLastError();
}
template <int DIM, int LAYOUT, int AXIS>
static int walk_occ()
{
    if (walk_configure<DIM, LAYOUT, AXIS>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, euler_force_walk_kernel<DIM, LAYOUT, AXIS, kWalkSlots>,
                                                      kWalkWarps * 32, WalkCfg<DIM, kWalkSlots>::SMEM) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace ripple
