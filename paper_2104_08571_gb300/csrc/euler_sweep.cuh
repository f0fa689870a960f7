// Halo-padded, block-tiled finite-volume Euler sweep for sm_103a.
//
// One launch advances the whole field by one explicit step (the flux
// difference of the paper's Section 7.3 applied inside the solver step of
// Section 8, Listing "euler_graph"), out of place (Section 5.4 double
// buffering: in -> out).  The step fuses what the paper runs as separate
// graph nodes:
//   set_dt         dt = cfl / smax(in), read from the ring slot the previous
//                  step (or the prep kernel) reduced into;
//   update         unsplit flux difference with Rusanov faces, first order or
//                  MUSCL-Hancock (minmod slopes, per-direction half-step
//                  predictor);
//   set_boundary   the ghost images of every new interior cell are written
//                  to `out` (periodic wrap or constant extrapolation), so the
//                  next step finds its padding filled;
//   set_wavespeeds + MaxReducer
//                  max_cells sum_d (|u_d| + c)/dx_d of the NEW state, warp
//                  shuffles -> block -> one atomicMax per CTA into the next
//                  ring slot (the max is order-independent, so dt is
//                  deterministic);
//   positivity     any non-positive/NaN density or pressure in a cell,
//                  reconstructed or predicted state sets DEV_ERR_NUMERIC.
//
// Tiling ("in_shared" access of Section 5.4, re-designed for Blackwell):
//   * a CTA owns a TX x TY column of cells and streams along z over a chunk
//     of planes (2.5-D); 2D fields are the one-plane case;
//   * each plane of the tile plus its ghost cells (TX+2R) x (TY+2R), all
//     components, arrives in shared memory by ONE TMA tile load
//     (cp.async.bulk.tensor) into a ring of NS slots with one mbarrier per
//     slot, prefetched NS - R - 1 planes ahead;
//   * in-plane (x, y) work is split into phases over shared-memory arrays so
//     that each face flux is evaluated exactly once and read by both cells
//     (bit-exact telescoping); the z direction is carried in registers
//     (predicted states and the lower face flux of the next plane);
//   * the new plane is written to a shared staging tile and leaves by ONE TMA
//     tile store, clipped by the tensor map at the interior's y/z ends (tiles
//     that cross the x end store with plain stores instead).
// The CTA count is a multiple of the SM count (persistent, work items strided
// over CTAs).
#pragma once
#include <cuda.h>
#include <cstdint>
#include <type_traits>

#include "field.cuh"
#include "tma.cuh"

namespace ripple {

enum { SCHEME_RUSANOV1 = 0, SCHEME_MUSCL = 1, SCHEME_FORCE = 2 };

struct SweepGeom {
    FieldGeom f;
    int tiles_x, tiles_y, zchunk, chunks_z;
    int items;  // tiles_x * tiles_y * chunks_z
};

// Strip walks of a one-axis sweep (euler_force_walk.cuh).  x sweep: walk w
// covers `seg` cells of row w / nseg (rows of all y, then z) from
// x = (w % nseg) * seg.  y or z sweep: walk w covers `seg` rows along the
// swept axis of the 64-column strip w % nstrips, on line (w / nstrips) % nlines
// (the z plane of a y sweep, the y row of a z sweep; 1 line in 2D), from
// ((w / nstrips) / nlines) * seg.
struct WalkGeom {
    FieldGeom f;
    int seg, nseg, nstrips, nlines, walks;
};
constexpr int kWalkWarps = 8;  // walks in flight per CTA (one per warp)

struct SweepParams {
    double gamma, cfl;
    double inv_dx[3];
    int bc;       // 0 periodic, 1 transmissive
    int slot_in;  // ring slot holding smax of the input state
    int first;    // first step of a call: t = dt instead of t += dt
    int axis;     // -1: all axes (the unsplit step); 0/1/2: one sweep of a split step along that axis
    int last;     // this launch completes the step: advance t, reduce the new wave speeds
    // FP32 copies of gamma, gamma - 1 and 1/dx, rounded once on the host: FP32
    // kernels read them as constant operands instead of converting the FP64
    // values on the device (a conversion runs on the narrow FP64 pipe, and the
    // compiler may repeat it wherever it rematerialises the value)
    float gamma_f, gm1_f;
    float inv_dx_f[3];
};

// ---------------------------------------------------------------------------
// Arithmetic helpers (field precision).  FP32 uses the hardware approximate
// reciprocal and square root (relative error of about one unit in the last
// place, far inside the FP32 error budget against the FP64 oracle); FP64 keeps
// IEEE division and square root.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_t(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_t(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T minmod_t(T a, T b)
{
    // 0 if the one-sided differences disagree in sign, else the smaller one
    if (a * b <= T(0)) return T(0);
    return fabs(a) < fabs(b) ? a : b;
}

// Physical flux along axis D from the state and its 1/rho; also returns the
// normal velocity and the pressure.
template <typename T, int DIM, int D>
__device__ __forceinline__ void phys_flux_ir(const T (&q)[DIM + 2], T inv_rho, T gm1, T (&F)[DIM + 2], T& un, T& p)
{
    T mm = q[1] * q[1];
#pragma unroll
    for (int e = 1; e < DIM; ++e) mm = fma(q[1 + e], q[1 + e], mm);
    p = gm1 * (q[DIM + 1] - T(0.5) * mm * inv_rho);
    un = q[1 + D] * inv_rho;
    F[0] = q[1 + D];
#pragma unroll
    for (int e = 0; e < DIM; ++e) F[1 + e] = q[1 + e] * un;
    F[1 + D] += p;
    F[DIM + 1] = (q[DIM + 1] + p) * un;
}

// Physical flux along axis D; also returns 1/rho, the normal velocity and the pressure.
template <typename T, int DIM, int D>
__device__ __forceinline__ void phys_flux(const T (&q)[DIM + 2], T gm1, T (&F)[DIM + 2], T& inv_rho, T& un, T& p)
{
    inv_rho = rcp_t(q[0]);
    T mm = q[1] * q[1];
#pragma unroll
    for (int e = 1; e < DIM; ++e) mm = fma(q[1 + e], q[1 + e], mm);
    p = gm1 * (q[DIM + 1] - T(0.5) * mm * inv_rho);
    un = q[1 + D] * inv_rho;
    F[0] = q[1 + D];
#pragma unroll
    for (int e = 0; e < DIM; ++e) F[1 + e] = q[1 + e] * un;
    F[1 + D] += p;
    F[DIM + 1] = (q[DIM + 1] + p) * un;
}

// Admissibility bookkeeping: `chk` keeps the smallest density or pressure
// seen in the states of in-domain items; a non-positive value flags the plane.
// (A NaN state is skipped by fmin but reaches the updated cells, whose own
// check catches it.)
__device__ __forceinline__ void track_min(double& chk, bool valid, double a, double b, double c, double d)
{
    const double m = fmin(fmin(a, b), fmin(c, d));
    if (valid) chk = fmin(chk, m);
}
__device__ __forceinline__ void track_min(float& chk, bool valid, float a, float b, float c, float d)
{
    float m;  // three-operand minimum: one ALU instruction on sm_100 and later
    asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
    if (valid) asm("min.f32 %0, %1, %2, %3;" : "=f"(chk) : "f"(chk), "f"(m), "f"(d));
}

// Rusanov face flux along D between left state a and right state b.
template <typename T, int DIM, int D>
__device__ __forceinline__ void rusanov(const T (&a)[DIM + 2], const T (&b)[DIM + 2], T gamma, T gm1,
                                        T (&F)[DIM + 2], T& chk, bool valid)
{
    T Fa[DIM + 2], Fb[DIM + 2], ia, ua, pa, ib, ub, pb;
    phys_flux<T, DIM, D>(a, gm1, Fa, ia, ua, pa);
    phys_flux<T, DIM, D>(b, gm1, Fb, ib, ub, pb);
    track_min(chk, valid, a[0], pa, b[0], pb);
    const T ca = sqrt_t(gamma * pa * ia);
    const T cb = sqrt_t(gamma * pb * ib);
    const T s = fmax(fabs(ua) + ca, fabs(ub) + cb);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) F[m] = T(0.5) * (Fa[m] + Fb[m]) - T(0.5) * s * (b[m] - a[m]);
}

// First-order conservative update of one component of a 2D cell from its
// four face fluxes (x: left, right; y: below, above).  The batched step and
// the multi-step solo solver share this arithmetic, so a problem's state does
// not depend on which of them advanced it.
template <typename T>
__device__ __forceinline__ T cell_update2(T q, T fxl, T fxr, T fyd, T fyu, T inv_dx0, T inv_dx1, T dt)
{
    T acc = (fxr - fxl) * inv_dx0;
    acc += (fyu - fyd) * inv_dx1;
    return q - dt * acc;
}

// Rusanov face flux from states whose 1/rho and sound speed were formed once
// per cell beforehand (the FP64 path, where division and square root are
// the costly operations): the same flux as rusanov().
template <typename T, int DIM, int D>
__device__ __forceinline__ void rusanov_pre(const T (&a)[DIM + 2], const T (&b)[DIM + 2], T ia, T ib, T ca, T cb,
                                            T gm1, T (&F)[DIM + 2], T& chk, bool valid)
{
    T Fa[DIM + 2], Fb[DIM + 2], ua, pa, ub, pb;
    phys_flux_ir<T, DIM, D>(a, ia, gm1, Fa, ua, pa);
    phys_flux_ir<T, DIM, D>(b, ib, gm1, Fb, ub, pb);
    track_min(chk, valid, a[0], pa, b[0], pb);
    const T s = fmax(fabs(ua) + ca, fabs(ub) + cb);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) F[m] = T(0.5) * (Fa[m] + Fb[m]) - T(0.5) * s * (b[m] - a[m]);
}

// FORCE face flux along D (Toro's first-order centred scheme, the flux of
// Section 7.3): the mean of the Lax-Friedrichs flux and the Richtmyer flux of
// the intermediate state q = (a + b)/2 - (dt/dx)(F(b) - F(a))/2, for
// dtdx = dt/dx_D and inv_dtdx = dx_D/dt.  The admissibility of a and b goes to
// chk; q is an intermediate of the formula and is not checked.
template <typename T, int DIM, int D>
__device__ __forceinline__ void force_flux(const T (&a)[DIM + 2], const T (&b)[DIM + 2], T gm1, T dtdx, T inv_dtdx,
                                           T (&F)[DIM + 2], T& chk, bool valid)
{
    T Fa[DIM + 2], Fb[DIM + 2], q[DIM + 2], Fq[DIM + 2], ia, ua, pa, ib, ub, pb, iq, uq, pq;
    phys_flux<T, DIM, D>(a, gm1, Fa, ia, ua, pa);
    phys_flux<T, DIM, D>(b, gm1, Fb, ib, ub, pb);
    track_min(chk, valid, a[0], pa, b[0], pb);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) q[m] = T(0.5) * (a[m] + b[m]) - T(0.5) * dtdx * (Fb[m] - Fa[m]);
    phys_flux<T, DIM, D>(q, gm1, Fq, iq, uq, pq);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m)
        F[m] = T(0.5) * (T(0.5) * (Fa[m] + Fb[m]) - T(0.5) * inv_dtdx * (b[m] - a[m]) + Fq[m]);
}

// First-order face flux of a scheme: Rusanov, or FORCE for the split step.
template <int SCHEME, typename T, int DIM, int D>
__device__ __forceinline__ void face_flux1(const T (&a)[DIM + 2], const T (&b)[DIM + 2], T gamma, T gm1, T dtdx,
                                           T inv_dtdx, T (&F)[DIM + 2], T& chk, bool valid)
{
    if constexpr (SCHEME == SCHEME_FORCE) force_flux<T, DIM, D>(a, b, gm1, dtdx, inv_dtdx, F, chk, valid);
    else rusanov<T, DIM, D>(a, b, gamma, gm1, F, chk, valid);
}

// MUSCL-Hancock face states of a cell along D from (left, centre, right):
// slopes by minmod, boundary extrapolation, half-step predictor with the
// direction-D flux difference (admissibility of the extrapolated states goes to chk).
template <typename T, int DIM, int D>
__device__ __forceinline__ void muscl_states(const T (&qm)[DIM + 2], const T (&q)[DIM + 2],
                                             const T (&qp)[DIM + 2], T gm1, T half_dtdx,
                                             T (&L)[DIM + 2], T (&R)[DIM + 2], T& chk, bool valid)
{
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) {
        const T slope = minmod_t(q[m] - qm[m], qp[m] - q[m]);
        L[m] = q[m] - T(0.5) * slope;
        R[m] = q[m] + T(0.5) * slope;
    }
    T FL[DIM + 2], FR[DIM + 2], il, ir, u, pl, pr;
    phys_flux<T, DIM, D>(L, gm1, FL, il, u, pl);
    phys_flux<T, DIM, D>(R, gm1, FR, ir, u, pr);
    track_min(chk, valid, L[0], pl, R[0], pr);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) {
        const T inc = half_dtdx * (FL[m] - FR[m]);
        L[m] += inc;
        R[m] += inc;
    }
}

// Separately rounded product and sum (never contracted into a fused
// multiply-add): the wave-speed sum then does not depend on the order of the
// axes, so a problem and its axis-permuted twin get the same dt.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Wave-speed sum and admissibility of a conserved state.
template <typename T, int DIM>
__device__ __forceinline__ T wave_sum(const T (&q)[DIM + 2], T gamma, T gm1, const T (&inv_dx)[3], bool& ok)
{
    const T inv_rho = rcp_t(q[0]);
    T mm = q[1] * q[1];
#pragma unroll
    for (int e = 1; e < DIM; ++e) mm = fma(q[1 + e], q[1 + e], mm);
    const T p = gm1 * (q[DIM + 1] - T(0.5) * mm * inv_rho);
    ok = (q[0] > T(0)) & (p > T(0));
    const T c = sqrt_t(gamma * p * inv_rho);
    T s = T(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) s = add_rn(s, mul_rn(fabs(q[1 + d] * inv_rho) + c, inv_dx[d]));
    return s;
}

// Write the ghost images of interior cell (i, j, k): along each axis, the
// periodic copy on the far side (cells within h of an edge) or the constant
// extrapolation into all h layers (edge cells).  Only face ghosts are
// written: the cross-shaped stencils never read edge or corner ghosts.
template <typename T, int DIM>
__device__ __forceinline__ void write_ghost_images(T* __restrict__ out, const FieldGeom& g, int bc, int i,
                                                   int j, int k, const T (&q)[DIM + 2])
{
    const int c[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const int n = g.n[d];
        if (bc == 0) {
            int img = c[d] < g.h ? c[d] + n : (c[d] >= n - g.h ? c[d] - n : INT32_MIN);
            int img2 = (c[d] < g.h && c[d] >= n - g.h) ? c[d] - n : INT32_MIN;  // n < 2h
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int v = r == 0 ? img : img2;
                if (v == INT32_MIN) continue;
                int cc[3] = {c[0], c[1], c[2]};
                cc[d] = v;
                const long long base = geom_cell(g, cc[0], cc[1], cc[2]) * g.cell_stride;
#pragma unroll
                for (int m = 0; m < DIM + 2; ++m) out[base + (long long)m * g.comp_stride] = q[m];
            }
        } else {
            int lo = 0, cnt = 0;
            if (c[d] == 0) { lo = -g.h; cnt = g.h; }
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) {
                    if (c[d] == n - 1) { lo = n; cnt = g.h; } else cnt = 0;
                }
                for (int r = 0; r < cnt; ++r) {
                    int cc[3] = {c[0], c[1], c[2]};
                    cc[d] = lo + r;
                    const long long base = geom_cell(g, cc[0], cc[1], cc[2]) * g.cell_stride;
#pragma unroll
                    for (int m = 0; m < DIM + 2; ++m) out[base + (long long)m * g.comp_stride] = q[m];
                }
            }
        }
    }
}

// Where the first non-admissible state was found (FieldCtl::counters[4..7]):
// stage code + 1, then x, y, z of the cell (or of the left cell of a face).
// BAD_STATE: a reconstructed, predicted or face state of the tile whose
// first cell is (x, y) on plane z; BAD_CELL / BAD_INPUT: that cell itself.
enum : int { BAD_STATE = 1, BAD_CELL = 7, BAD_INPUT = 8 };
static __device__ __noinline__ void record_bad(FieldCtl* ctl, int code, int x, int y, int z)
{
    if (atomicCAS(reinterpret_cast<unsigned long long*>(&ctl->counters[4]), 0ull, (unsigned long long)code) == 0ull) {
        ctl->counters[5] = x;
        ctl->counters[6] = y;
        ctl->counters[7] = z;
    }
}

__device__ __forceinline__ void atomic_max_pos_double(unsigned long long* addr, double v)
{
    // positive doubles order like their bit patterns
    if (v > 0.0) atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Geometry of the TMA box that stages one plane of a tile plus its ghost
// cells.  Shared by the kernel (shared-memory slot size, expected bytes) and
// the host (tensor-map box), so the two can never disagree.
//   a   : x alignment in cells of a box start (16 bytes of elements)
//   off : the box starts off cells before x0 - r so that its start is aligned
//   bx  : box width in cells (multiple of a), by: box height
// ---------------------------------------------------------------------------
struct BoxGeom {
    int a, off, bx, by;
};
__host__ __device__ constexpr int pow2_divisor16(int v)
{
    return (v % 16 == 0) ? 16 : (v % 8 == 0) ? 8 : (v % 4 == 0) ? 4 : (v % 2 == 0) ? 2 : 1;
}
__host__ __device__ constexpr BoxGeom plane_box(int elem_bytes, int ncomp, bool aos, int r, int tx, int ty)
{
    const int a = 16 / pow2_divisor16(elem_bytes * (aos ? ncomp : 1));
    const int off = (a - r % a) % a;
    return BoxGeom{a, off, ((off + tx + 2 * r + a - 1) / a) * a, ty + 2 * r};
}

// ---------------------------------------------------------------------------
// Compile-time tile configuration.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int LAYOUT, int SCHEME, int TX, int TY>
struct SweepCfg {
    static constexpr int NC = DIM + 2;
    static constexpr int R = SCHEME == SCHEME_MUSCL ? 2 : 1;
    static constexpr int ES = (int)sizeof(T);
    static constexpr BoxGeom BOX = plane_box(ES, NC, LAYOUT == LAYOUT_AOS, R, TX, TY);
    static constexpr int A = BOX.a;
    static constexpr int OFF = BOX.off;
    static constexpr int BX = BOX.bx;
    static constexpr int BY = BOX.by;
    static constexpr int NT = TX * TY;
    static constexpr int NS = DIM == 3 ? 2 * R + 2 : 3;  // ring slots
    static constexpr int SLOT_ELEMS = BX * BY * NC;
    static constexpr int SLOT_BYTES = ((SLOT_ELEMS * ES + 127) / 128) * 128;
    static constexpr int OUT_ELEMS = TX * TY * NC;
    static constexpr int OUT_BYTES = ((OUT_ELEMS * ES + 127) / 128) * 128;
    static constexpr int NPX = (TX + 2) * TY, NPY = TX * (TY + 2);  // predicted-state cells
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);  // faces
    static constexpr int P_BYTES = SCHEME == SCHEME_MUSCL ? ((2 * NC * (NPX + NPY) * ES + 127) / 128) * 128 : 0;
    static constexpr int F_BYTES = ((NC * (NFX + NFY) * ES + 127) / 128) * 128;
    static constexpr int HDR_BYTES = 384;  // mbarriers, reduction scratch, abort flag, step scalars
    // FP64 first-order 2D: 1/rho and the sound speed of every staged cell are
    // formed once per tile (division and square root are costly in FP64)
    static constexpr bool PRIM = std::is_same<T, double>::value && SCHEME == SCHEME_RUSANOV1 && DIM == 2;
    static constexpr int Q_BYTES = PRIM ? ((2 * BX * BY * ES + 127) / 128) * 128 : 0;
    static constexpr int SMEM = HDR_BYTES + NS * SLOT_BYTES + 2 * OUT_BYTES + P_BYTES + F_BYTES + Q_BYTES;
    static_assert(TX % A == 0, "tile width must keep TMA x coordinates 16-byte aligned");
    static_assert(BX * (LAYOUT == LAYOUT_AOS ? NC : 1) <= 256 && BY <= 256, "TMA box too large");
    static_assert(TX * (LAYOUT == LAYOUT_AOS ? NC : 1) <= 256, "TMA store box too large");
    static_assert(NT % 32 == 0 && NT <= 512, "whole warps, at most 16 (header reduction scratch)");
};

// Shared-memory accessors of a staged plane and of the output staging tile.
template <class C, int LAYOUT>
struct PlaneView {
    __device__ static __forceinline__ int idx(int lx, int ly, int m)
    {
        // lx in [-R, TX+R), ly in [-R, TY+R)
        if (LAYOUT == LAYOUT_SOA) return (m * C::BY + ly + C::R) * C::BX + C::OFF + C::R + lx;
        return ((ly + C::R) * C::BX + C::OFF + C::R + lx) * C::NC + m;
    }
};

// ---------------------------------------------------------------------------
// The sweep kernel.
//
// Per plane z of a work item (3D MUSCL shown; Rusanov has no phase P and
// computes its z face in phase F; 2D has no z work):
//   B2  barrier; thread 0 flushes the previous staging tile and refills freed
//       ring slots; every thread checks the abort flag
//   F   x and y face fluxes from the predicted states -> shared arrays
//   B3  barrier
//   U   conservative update of the thread's cell (x, y faces from shared
//       memory, z faces from registers) -> staging tile, ghost images,
//       wave-speed max, positivity; then, if the item has another plane, wait
//       for its planes and run phase P of plane z+1:
//   P   x and y predicted states -> shared arrays; z predicted state of the
//       thread's own column at z+2 and the z face z+3/2 in registers
// so that each plane costs two CTA barriers.  Each thread's work items in
// phases P and F are fixed for the whole tile; their shared-memory offsets
// are decoded once per tile.
// ---------------------------------------------------------------------------
template <typename T, int DIM, int LAYOUT, int SCHEME, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (TX * TY >= 256 ? 2 : 4))
    euler_sweep_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_out,
                       T* __restrict__ out, FieldCtl* __restrict__ ctl, const SweepGeom sg, const SweepParams prm)
{
    using C = SweepCfg<T, DIM, LAYOUT, SCHEME, TX, TY>;
    using PV = PlaneView<C, LAYOUT>;
    constexpr int NC = C::NC, R = C::R, NS = C::NS, NT = C::NT;
    constexpr bool MUSCL = SCHEME == SCHEME_MUSCL;
    // element strides inside a staged plane
    constexpr int SX = LAYOUT == LAYOUT_SOA ? 1 : NC;          // +1 cell in x
    constexpr int SY = LAYOUT == LAYOUT_SOA ? C::BX : C::BX * NC;  // +1 cell in y
    constexpr int SM = LAYOUT == LAYOUT_SOA ? C::BX * C::BY : 1;   // +1 component
    constexpr int NP = C::NPX + C::NPY;  // predicted-state items (MUSCL)
    constexpr int NPXr = ((C::NPX + 31) / 32) * 32, NPYr = ((C::NPY + 31) / 32) * 32;
    constexpr int NFXr = ((C::NFX + 31) / 32) * 32, NFYr = ((C::NFY + 31) / 32) * 32;
    constexpr int KP = MUSCL ? (NPXr + NPYr + NT - 1) / NT : 0;  // phase-P items per thread
    constexpr int KF = (NFXr + NFYr + NT - 1) / NT;              // phase-F items per thread

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);      // NS mbarriers
    double* red = reinterpret_cast<double*>(smem + 64);      // one double per warp (<= 16)
    int* flags = reinterpret_cast<int*>(smem + 64 + 8 * 16);  // abort flag
    T* ring = reinterpret_cast<T*>(smem + C::HDR_BYTES);
    T* stage = reinterpret_cast<T*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES);
    T* P = reinterpret_cast<T*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES + 2 * C::OUT_BYTES);
    T* Fs = reinterpret_cast<T*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES + 2 * C::OUT_BYTES + C::P_BYTES);
    T* PL = P;            // [NC][NPX + NPY]
    T* PR = P + NC * NP;  // [NC][NPX + NPY]
    T* FX = Fs;           // [NC][NFX]
    T* FY = Fs + NC * C::NFX;  // [NC][NFY]
    T* QI = reinterpret_cast<T*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES + 2 * C::OUT_BYTES + C::P_BYTES +
                                 C::F_BYTES);  // [BX * BY] 1/rho of each staged cell (PRIM only)
    T* QC = QI + C::BX * C::BY;                // [BX * BY] sound speed of each staged cell (PRIM only)

    double* sdt = reinterpret_cast<double*>(smem + 256);  // step scalars formed by thread 0

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const FieldGeom& g = sg.f;

    if (tid == 0) {
        // dt from the max wave-speed sum of the input state, in FP64 once per
        // CTA (FP64 throughput is small on this part); every sweep of a split
        // step reads the same ring slot and so uses the same dt
        const double dt = prm.cfl / __longlong_as_double((long long)ctl->smax[prm.slot_in]);
        sdt[0] = dt;
        for (int d = 0; d < 3; ++d) {
            sdt[1 + d] = 0.5 * dt * prm.inv_dx[d];
            sdt[4 + d] = dt * prm.inv_dx[d];
            sdt[7 + d] = prm.inv_dx[d] > 0.0 ? 1.0 / (dt * prm.inv_dx[d]) : 0.0;
        }
        if (blockIdx.x == 0 && prm.last) {
            ctl->t = prm.first ? dt : ctl->t + dt;
            ctl->dt_last = dt;
            ctl->smax[(prm.slot_in + 2) % 3] = 0ull;  // slot the next step reduces into after this one
        }
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        flags[0] = 0;
        fence_mbar_init();
        prefetch_tensormap(&map_in);
        prefetch_tensormap(&map_out);
    }
    __syncthreads();
    const T gamma = (T)prm.gamma, gm1 = (T)(prm.gamma - 1.0);
    const T dtT = (T)sdt[0];
    T inv_dx[3], half_dtdx[3], dtdx[3], inv_dtdx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        inv_dx[d] = (T)prm.inv_dx[d];
        half_dtdx[d] = (T)sdt[1 + d];
        dtdx[d] = (T)sdt[4 + d];
        inv_dtdx[d] = (T)sdt[7 + d];
    }
    // axes whose faces this launch evaluates (all of them for the unsplit step)
    const bool ax0 = prm.axis < 0 || prm.axis == 0;
    const bool ax1 = prm.axis < 0 || prm.axis == 1;
    const bool ax2 = DIM == 3 && (prm.axis < 0 || prm.axis == 2);

    // ---- plane sequence of this CTA: items strided over CTAs ----
    auto item_planes = [&](int item) -> int {
        if (DIM == 2) return 1;
        const int chunk = item % sg.chunks_z;
        return min(sg.zchunk, g.n[2] - chunk * sg.zchunk) + 2 * R;
    };
    int ld_item = blockIdx.x, ld_j = 0;  // loader cursor (thread 0 only)
    unsigned ld_seq = 0;
    auto issue_until = [&](unsigned limit) {
        while (ld_item < sg.items && ld_seq < limit) {
            const int item = ld_item;
            const int chunk = DIM == 3 ? item % sg.chunks_z : 0;
            const int tile = DIM == 3 ? item / sg.chunks_z : item;
            const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
            const int xs = g.lead + g.h + x0 - R - C::OFF;
            const int ys = g.h + y0 - R;
            const int slot = (int)(ld_seq % NS);
            T* dst = ring + (size_t)slot * (C::SLOT_BYTES / sizeof(T));
            mbar_arrive_expect_tx(&bars[slot], (uint32_t)(C::SLOT_ELEMS * sizeof(T)));
            if (DIM == 3) {
                const int pz = g.h + chunk * sg.zchunk - R + ld_j;
                if (LAYOUT == LAYOUT_SOA) tma_load_4d(dst, &map_in, xs, ys, pz, 0, &bars[slot]);
                else tma_load_3d(dst, &map_in, xs * NC, ys, pz, &bars[slot]);
            } else {
                if (LAYOUT == LAYOUT_SOA) tma_load_3d(dst, &map_in, xs, ys, 0, &bars[slot]);
                else tma_load_2d(dst, &map_in, xs * NC, ys, &bars[slot]);
            }
            ++ld_seq;
            if (++ld_j == item_planes(item)) { ld_j = 0; ld_item += gridDim.x; }
        }
    };

    // plane sequence numbers are 32-bit: a CTA streams far fewer than 2^32 planes
    unsigned ready_upto = 0;  // planes with seq < ready_upto have been waited for
    unsigned seq_base = 0;    // seq of plane j = 0 of the current item
    int out_count = 0;         // TMA-stored planes (staging slot parity)
    bool store_pending = false;
    int st_x = 0, st_y = 0, st_z = 0, st_slot = 0;
    bool bad = false;
    T smax_local = T(0);
    bool aborted = false;

    auto plane_ptr = [&](unsigned seq) -> const T* {
        return ring + (seq % NS) * (unsigned)(C::SLOT_BYTES / sizeof(T));
    };
    // wait (all threads) for planes up to seq `need` inclusive; a wait that
    // runs out raises the abort flag, read by every thread after the next barrier
    auto wait_planes = [&](unsigned need) {
        bool ok = true;
        for (unsigned sq = ready_upto; sq <= need; ++sq)
            ok &= mbar_wait_bounded(&bars[sq % NS], (uint32_t)((sq / NS) & 1));
        ready_upto = need + 1;
        if (!ok) flags[0] = 1;
    };
    auto store_tile = [&]() {
        const T* src = stage + (size_t)st_slot * (C::OUT_BYTES / sizeof(T));
        if (DIM == 3) {
            if (LAYOUT == LAYOUT_SOA) tma_store_4d(&map_out, src, st_x, st_y, st_z, 0);
            else tma_store_3d(&map_out, src, st_x * NC, st_y, st_z);
        } else {
            if (LAYOUT == LAYOUT_SOA) tma_store_3d(&map_out, src, st_x, st_y, 0);
            else tma_store_2d(&map_out, src, st_x * NC, st_y);
        }
        bulk_commit();
    };
    // Thread 0, called only right after a CTA barrier that follows every read
    // of the planes with seq < free_before and every write of the staging tile
    // that is still pending: flush that tile by TMA store, make sure the other
    // staging slot has been read out, refill the freed ring slots.
    auto producer_step = [&](unsigned free_before) {
        if (tid != 0) return;
        if (store_pending) {
            store_tile();
            store_pending = false;
        }
        bulk_wait_read<1>();
        issue_until(free_before + NS);
    };

    // load the NC components of the cell at element offset `o` of plane S
    auto load_q = [&](const T* S, int o, T (&q)[NC]) {
#pragma unroll
        for (int m = 0; m < NC; ++m) q[m] = S[o + m * SM];
    };

    for (int item = blockIdx.x; item < sg.items; item += gridDim.x) {
        const int chunk = DIM == 3 ? item % sg.chunks_z : 0;
        const int tile = DIM == 3 ? item / sg.chunks_z : item;
        const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
        const int z0 = chunk * sg.zchunk;
        const int zn = DIM == 3 ? min(sg.zchunk, g.n[2] - z0) : 1;
        const int gx = x0 + lx, gy = y0 + ly;
        const bool col_valid = (gx < g.n[0]) & (gy < g.n[1]);
        // A TMA store clipped at the interior's x end drops the last partial
        // 16-byte chunk of each row when the row length is not a multiple of
        // 16 bytes, so tiles that cross the x end store with plain stores.
        const bool tma_store_ok = x0 + TX <= g.n[0];
        // only tiles within h cells of a domain face have ghost images to write
        const bool near_xy = (x0 < g.h) || (x0 + TX > g.n[0] - g.h) || (y0 < g.h) || (y0 + TY > g.n[1] - g.h);
        T chk = T(1);  // smallest density/pressure of this thread's in-domain states

        // ---- per-tile decode of this thread's phase-P and phase-F items ----
        // Item k of this thread is it = tid + k * NT.  Kept per item: the element
        // offset of its (left) cell in a staged plane; packed in *_bits: bit 2k
        // = x item, bit 2k+1 = y item, bit 16+k = the item touches the domain
        // (its positivity check counts).  Array indices follow from `it`.
        int p_off[KP > 0 ? KP : 1];
        unsigned p_bits = 0u;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int it = tid + k * NT;
            p_off[k] = 0;
            if (it < C::NPX) {
                const int cx = it % (TX + 2) - 1, cy = it / (TX + 2);
                p_off[k] = PV::idx(cx, cy, 0);
                p_bits |= 1u << (2 * k);
                if ((x0 + cx <= g.n[0]) && (y0 + cy < g.n[1])) p_bits |= 1u << (16 + k);
            } else if (it >= NPXr && it - NPXr < C::NPY) {
                const int kk = it - NPXr;
                const int cx = kk % TX, cy = kk / TX - 1;
                p_off[k] = PV::idx(cx, cy, 0);
                p_bits |= 2u << (2 * k);
                if ((x0 + cx < g.n[0]) && (y0 + cy <= g.n[1])) p_bits |= 1u << (16 + k);
            }
        }
        int f_off[KF], f_il[KF];
        unsigned f_bits = 0u;
#pragma unroll
        for (int k = 0; k < KF; ++k) {
            const int it = tid + k * NT;
            f_off[k] = 0;
            f_il[k] = 0;
            if (it < C::NFX) {
                const int fx = it % (TX + 1), cy = it / (TX + 1);  // face between fx-1 and fx
                f_off[k] = PV::idx(fx - 1, cy, 0);
                f_il[k] = cy * (TX + 2) + fx;
                f_bits |= 1u << (2 * k);
                if ((x0 + fx <= g.n[0]) && (y0 + cy < g.n[1])) f_bits |= 1u << (16 + k);
            } else if (it >= NFXr && it - NFXr < C::NFY) {
                const int kk = it - NFXr;
                const int cx = kk % TX, fy = kk / TX;  // face between fy-1 and fy
                f_off[k] = PV::idx(cx, fy - 1, 0);
                f_il[k] = C::NPX + fy * TX + cx;
                f_bits |= 2u << (2 * k);
                if ((x0 + cx < g.n[0]) && (y0 + fy <= g.n[1])) f_bits |= 1u << (16 + k);
            }
        }
        const int my_off = PV::idx(lx, ly, 0);

        // z registers (3D): lower face flux of the current plane, the high-face
        // predicted state of the next plane, and the column values of the
        // current plane (qa) and the one above (qb)
        T Fzm[NC], Fzp[NC], zR[NC], qa[NC], qb[NC], qz2[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            Fzm[m] = T(0); Fzp[m] = T(0); zR[m] = T(0); qa[m] = T(0); qb[m] = T(0); qz2[m] = T(0);
        }

        // Phase P of the plane with index j (seq_base + j); z = z0 - R + j.
        auto phase_p = [&](unsigned j, int z) {
            const T* S = plane_ptr(seq_base + j);
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const unsigned kind = (p_bits >> (2 * k)) & 3u;
                if (kind == 0u) continue;
                const int it = tid + k * NT;
                const int pidx = kind == 1u ? it : C::NPX + it - NPXr;
                const int o = p_off[k];
                const int st = kind == 1u ? SX : SY;
                T qm[NC], q[NC], qp[NC], L[NC], Rs[NC];
                load_q(S, o - st, qm);
                load_q(S, o, q);
                load_q(S, o + st, qp);
                const bool v = (p_bits >> (16 + k)) & 1u;
                if (kind == 1u) muscl_states<T, DIM, 0>(qm, q, qp, gm1, half_dtdx[0], L, Rs, chk, v);
                else muscl_states<T, DIM, 1>(qm, q, qp, gm1, half_dtdx[1], L, Rs, chk, v);
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    PL[m * NP + pidx] = L[m];
                    PR[m * NP + pidx] = Rs[m];
                }
            }
            if (DIM == 3) {
                // z: predicted states of plane z+1 and the face z + 1/2
                T L[NC], Rn[NC];
                load_q(plane_ptr(seq_base + j + 2), my_off, qz2);
                muscl_states<T, DIM, 2 % DIM>(qa, qb, qz2, gm1, half_dtdx[2], L, Rn, chk, col_valid);
                rusanov<T, DIM, 2 % DIM>(zR, L, gamma, gm1, Fzp, chk, col_valid);
#pragma unroll
                for (int m = 0; m < NC; ++m) zR[m] = Rn[m];  // qa, qb shift after phase U
            }
        };

        // every plane of earlier items is free once all threads pass here
        __syncthreads();  // B0
        producer_step(seq_base);

        if (DIM == 3) {
            // planes j = 0 .. 2R-1 (z0-R .. z0+R-1) give the face z0 - 1/2;
            // phase P of z0 needs up to j = 2R (MUSCL)
            wait_planes(seq_base + (MUSCL ? 2 * R : 2 * R - 1));
            __syncthreads();
            if (flags[0]) { aborted = true; break; }
            if (!MUSCL) {
                load_q(plane_ptr(seq_base + 0), my_off, qa);  // z0 - 1
                load_q(plane_ptr(seq_base + 1), my_off, qb);  // z0
                if (ax2)
                    face_flux1<SCHEME, T, DIM, 2 % DIM>(qa, qb, gamma, gm1, dtdx[2], inv_dtdx[2], Fzm, chk,
                                                        col_valid);
#pragma unroll
                for (int m = 0; m < NC; ++m) qa[m] = qb[m];  // qa = column value of z0
            } else {
                T q0[NC], q1[NC], L1[NC], R1[NC], L2[NC];
                load_q(plane_ptr(seq_base + 0), my_off, q0);  // z0 - 2
                load_q(plane_ptr(seq_base + 1), my_off, q1);  // z0 - 1
                load_q(plane_ptr(seq_base + 2), my_off, qa);  // z0
                load_q(plane_ptr(seq_base + 3), my_off, qb);  // z0 + 1
                muscl_states<T, DIM, 2 % DIM>(q0, q1, qa, gm1, half_dtdx[2], L1, R1, chk, col_valid);
                muscl_states<T, DIM, 2 % DIM>(q1, qa, qb, gm1, half_dtdx[2], L2, zR, chk, col_valid);
                rusanov<T, DIM, 2 % DIM>(R1, L2, gamma, gm1, Fzm, chk, col_valid);
                // qa, qb now hold the column values of z0 and z0 + 1
            }
        } else {
            wait_planes(seq_base);
        }
        if (MUSCL) phase_p(DIM == 3 ? R : 0, z0);

        for (int zl = 0; zl < zn; ++zl) {
            const int z = z0 + zl;
            const unsigned jc = DIM == 3 ? (unsigned)(zl + R) : 0u;  // plane index of z
            __syncthreads();  // B2: phase P of this plane (and U of the previous) done
            if (flags[0]) { aborted = true; break; }
            producer_step(seq_base + jc);
            const T* S = plane_ptr(seq_base + jc);
            if constexpr (C::PRIM) {
                // 1/rho and c of every staged cell (padding and beyond-domain cells
                // give values no face in the domain reads)
                for (int c = tid; c < C::BX * C::BY; c += NT) {
                    T q[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) q[m] = S[(LAYOUT == LAYOUT_SOA ? c : c * NC) + m * SM];
                    const T ir = rcp_t(q[0]);
                    T mm = q[1] * q[1];
#pragma unroll
                    for (int e = 1; e < DIM; ++e) mm = fma(q[1 + e], q[1 + e], mm);
                    const T p = gm1 * (q[DIM + 1] - T(0.5) * mm * ir);
                    QI[c] = ir;
                    QC[c] = sqrt_t(gamma * p * ir);
                }
                __syncthreads();
            }

            // ---------------- phase F: face fluxes ----------------
            if (DIM == 3 && !MUSCL) {
                T qc[NC];
                load_q(plane_ptr(seq_base + jc + 1), my_off, qc);
                if (ax2)
                    face_flux1<SCHEME, T, DIM, 2 % DIM>(qa, qc, gamma, gm1, dtdx[2], inv_dtdx[2], Fzp, chk,
                                                        col_valid);
#pragma unroll
                for (int m = 0; m < NC; ++m) qb[m] = qc[m];
            }
#pragma unroll
            for (int k = 0; k < KF; ++k) {
                const unsigned kind = (f_bits >> (2 * k)) & 3u;
                if (kind == 0u || (kind == 1u && !ax0) || (kind == 2u && !ax1)) continue;
                const int it = tid + k * NT;
                T a[NC], b[NC], F[NC];
                if (MUSCL) {
                    const int il = f_il[k], ir = il + (kind == 1u ? 1 : TX);
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        a[m] = PR[m * NP + il];
                        b[m] = PL[m * NP + ir];
                    }
                } else {
                    load_q(S, f_off[k], a);
                    load_q(S, f_off[k] + (kind == 1u ? SX : SY), b);
                }
                const bool v = (f_bits >> (16 + k)) & 1u;
                if constexpr (C::PRIM) {
                    const int ca = LAYOUT == LAYOUT_SOA ? f_off[k] : f_off[k] / NC;
                    const int cb = ca + (kind == 1u ? 1 : C::BX);
                    if (kind == 1u) rusanov_pre<T, DIM, 0>(a, b, QI[ca], QI[cb], QC[ca], QC[cb], gm1, F, chk, v);
                    else rusanov_pre<T, DIM, 1>(a, b, QI[ca], QI[cb], QC[ca], QC[cb], gm1, F, chk, v);
                } else if (MUSCL) {
                    if (kind == 1u) rusanov<T, DIM, 0>(a, b, gamma, gm1, F, chk, v);
                    else rusanov<T, DIM, 1>(a, b, gamma, gm1, F, chk, v);
                } else if (kind == 1u) {
                    face_flux1<SCHEME, T, DIM, 0>(a, b, gamma, gm1, dtdx[0], inv_dtdx[0], F, chk, v);
                } else {
                    face_flux1<SCHEME, T, DIM, 1>(a, b, gamma, gm1, dtdx[1], inv_dtdx[1], F, chk, v);
                }
                if (kind == 1u) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) FX[m * C::NFX + it] = F[m];
                } else {
#pragma unroll
                    for (int m = 0; m < NC; ++m) FY[m * C::NFY + it - NFXr] = F[m];
                }
            }
            __syncthreads();  // B3

            // ---------------- phase U: conservative update + epilogue ----------------
            {
                T* st = stage + (size_t)(out_count & 1) * (C::OUT_BYTES / sizeof(T));
                T qc[NC];
                if (DIM == 3) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) qc[m] = qa[m];
                } else {
                    load_q(S, my_off, qc);
                }
                T qn[NC];
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const T fxp = FX[m * C::NFX + ly * (TX + 1) + lx + 1];
                    const T fxm = FX[m * C::NFX + ly * (TX + 1) + lx];
                    const T fyp = FY[m * C::NFY + (ly + 1) * TX + lx];
                    const T fym = FY[m * C::NFY + ly * TX + lx];
                    T acc = ax0 ? (fxp - fxm) * inv_dx[0] : T(0);
                    if (ax1) acc += (fyp - fym) * inv_dx[1];
                    if (ax2) acc += (Fzp[m] - Fzm[m]) * inv_dx[2];
                    qn[m] = qc[m] - dtT * acc;
                    if (tma_store_ok) {
                        if (LAYOUT == LAYOUT_SOA) st[(m * TY + ly) * TX + lx] = qn[m];
                        else st[(ly * TX + lx) * NC + m] = qn[m];
                    }
                }
                if (!tma_store_ok && col_valid) {
                    const long long base = geom_cell(g, gx, gy, z) * g.cell_stride;
#pragma unroll
                    for (int m = 0; m < NC; ++m) out[base + (long long)m * g.comp_stride] = qn[m];
                }
                if (DIM == 3) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        Fzm[m] = Fzp[m];
                        qa[m] = qb[m];
                        if (MUSCL) qb[m] = qz2[m];
                    }
                }
                fence_proxy_async_smem();
                if (col_valid) {
                    bool ok;
                    const T s = wave_sum<T, DIM>(qn, gamma, gm1, inv_dx, ok);
                    if (!ok) {
                        bad = true;
                        record_bad(ctl, BAD_CELL, gx, gy, z);
                    }
                    smax_local = fmax(smax_local, s);
                    if (near_xy || (DIM == 3 && (z < g.h || z >= g.n[2] - g.h)))
                        write_ghost_images<T, DIM>(out, g, prm.bc, gx, gy, z, qn);
                }
                if (!(chk > T(0))) {
                    bad = true;
                    record_bad(ctl, BAD_STATE, x0, y0, z);
                    chk = T(1);
                }
                if (tma_store_ok) {
                    store_pending = true;
                    st_x = x0; st_y = y0; st_z = z; st_slot = out_count & 1;
                    ++out_count;
                }
            }
            // ---------------- phase P of the next plane ----------------
            if (DIM == 3 && zl + 1 < zn) {
                wait_planes(seq_base + jc + 1 + R);
                if (MUSCL) phase_p(jc + 1, z + 1);
            }
        }
        if (aborted) break;
        seq_base += DIM == 3 ? (unsigned)(zn + 2 * R) : 1u;
    }

    // ---- drain: last store, wait for completion ----
    __syncthreads();
    if (tid == 0) {
        if (store_pending && !aborted) store_tile();
        bulk_wait<0>();
        if (aborted) {
            // loads still in flight complete into this CTA's shared memory:
            // wait for them (bounded) before the CTA exits
            for (unsigned sq = ready_upto; sq < ld_seq; ++sq)
                mbar_wait_bounded(&bars[sq % NS], (uint32_t)((sq / NS) & 1));
            atomicOr(&ctl->err, DEV_ERR_TIMEOUT);
        }
    }

    // ---- block reductions: max wave speed, positivity ----
    double v = (double)smax_local;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < NT / 32; ++w) m = fmax(m, red[w]);
        if (prm.last) atomic_max_pos_double(&ctl->smax[(prm.slot_in + 1) % 3], m);
        if (any_bad) atomicOr(&ctl->err, DEV_ERR_NUMERIC);
    }
}

}  // namespace ripple
