// Multi-step solver of ONE 2D Euler problem (first-order Rusanov), the
// single-problem kernel of the batch runtime's solo rounds.
//
// One cooperative launch advances the problem K steps; a bounded grid barrier
// separates the steps.  Per launched step the field and batched step kernels
// pay a launch, a pipeline fill and a grid drain (about 8 us at 64^2, so small
// problems were bound by that floor); here a step costs its arithmetic and one
// barrier, and the state of the served sizes (up to 1024^2, 16 MB per buffer)
// stays in L2 between steps.  The step's FP64 work (dt = cfl / smax) is one
// division per CTA, broadcast through shared memory: FP64 issues at 1/64 of
// the FP32 rate on GB300, and a division in every thread cost about 4 us per
// step.  The barrier is one monotonic arrival counter (a release add per CTA,
// acquire polls for the step's target count), with at most one CTA per SM
// arriving.
//
// Work: warps walk units of (strip of 30 columns) x (segment of R rows).  The
// 32 lanes of a warp hold the columns x0 - 1 .. x0 + 30 of the current row:
// lane l evaluates the x face between its left neighbour (shuffled from lane
// l - 1) and itself, the right face of a cell is its right neighbour's left
// face (shuffled back), so lanes 1..30 update their cells with every x face
// evaluated once; along y each lane carries the face below its cell from the
// previous row and prefetches the row two ahead.
//
// The step is the batched step's, term for term: dt = cfl / smax of the input
// state (FP64, from the instance's 3-slot ring), the same Rusanov faces of the
// same left/right states (a face's value depends only on its two states), the
// same cell update (cell_update2), ghost images and wave-speed maximum.  A
// problem's state is therefore bitwise the same whichever kernel advanced
// which of its steps.
#pragma once
#include <cstdint>

#include "batch_kernels.cuh"

namespace ripple {

constexpr int kSoloW = 30;           // cells a warp updates per row
constexpr int kSoloThreads = 1024;   // 32 warps per CTA, one CTA per SM

struct SoloEuler {
    void* buf[2];
    FieldCtl* ctl;
    FieldGeom g;
    int bc;
    int K;                    // steps of this launch
    long long first;          // local step index of the first of them
    int strips, segs, rows;   // units: strips x segs, segment height `rows`
    double cfl, gamma, gm1, inv_dx0, inv_dx1;
    float gamma_f, gm1_f, inv_dx0_f, inv_dx1_f;
    unsigned* bar;            // grid barrier: arrivals of this launch (zero at launch)
    unsigned spin_limit;      // polls of a barrier wait before it gives up
    unsigned* err;            // DEV_ERR_TIMEOUT when a barrier wait ran out
};

template <typename T>
__device__ __forceinline__ void solo_load(const T* __restrict__ in, const FieldGeom& g, int x, int y, T (&q)[4])
{
    const long long base = geom_cell(g, x, y, 0) * g.cell_stride;
#pragma unroll
    for (int m = 0; m < 4; ++m) q[m] = ldcg_t(in + base + (long long)m * g.comp_stride);
}

// Arrive at barrier number b (1, 2, ...) of the launch and wait until every
// CTA has arrived.  Returns false if the wait ran out (bounded polls).  Thread
// 0 arrives after its own earlier writes (release) and the other threads'
// writes (the CTA barrier before it).
__device__ __forceinline__ bool solo_barrier(unsigned* count, unsigned b, unsigned spin_limit, int* sflag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        const unsigned target = b * gridDim.x;
        uint32_t i = 0;
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if (++i > spin_limit) {
                sflag[0] = 1;
                break;
            }
        }
    }
    __syncthreads();
    return sflag[0] == 0;
}

// Registers of a warp's current unit: the rows below, at, above and two above
// the current row, the face below the current row, the admissibility trackers.
template <typename T>
struct SoloUnit {
    int strip, x, xl, y0, y1;
    bool upd, xface;
    T chk;
    bool bad;
    T qc[4], qa[4], qf[4], Fb[4];
};

// Start unit u: its first rows and the face below its first row (none of it
// depends on dt, so the first unit of a step starts before dt is known).
template <typename T>
__device__ __forceinline__ void solo_unit_begin(const FieldGeom& g, int strips, int rows, const T* __restrict__ in,
                                                int u, int lane, T gamma, T gm1, SoloUnit<T>& w)
{
    w.strip = u % strips;
    const int seg = u / strips;
    w.x = w.strip * kSoloW - 1 + lane;
    w.xl = min(w.x, g.n[0]);  // columns past the ghost column load the ghost (unused)
    w.upd = lane >= 1 && lane <= kSoloW && w.x < g.n[0];
    w.xface = lane >= 1 && w.x <= g.n[0];
    w.y0 = seg * rows;
    w.y1 = min(g.n[1], w.y0 + rows);
    w.chk = T(1);
    w.bad = false;
    T qd[4];
    solo_load(in, g, w.xl, w.y0 - 1, qd);
    solo_load(in, g, w.xl, w.y0, w.qc);
    solo_load(in, g, w.xl, w.y0 + 1, w.qa);  // y0 + 1 <= n[1]: at most the ghost row
    if (w.y0 + 2 <= g.n[1]) solo_load(in, g, w.xl, w.y0 + 2, w.qf);
    rusanov<T, 2, 1>(qd, w.qc, gamma, gm1, w.Fb, w.chk, w.upd);
}

// Walk the started unit's rows: faces, update, stores, ghost images.
template <typename T>
__device__ __forceinline__ void solo_unit_walk(const FieldGeom& g, int bc, const T* __restrict__ in,
                                               T* __restrict__ out, T gamma, T gm1, const T (&inv_dx)[3], T dtT,
                                               SoloUnit<T>& w, T& smax)
{
    for (int y = w.y0; y < w.y1; ++y) {
        // rows y + 1 (qa) and y + 2 (qf) are loaded; fetch row y + 3
        T qg[4];
        if (y + 3 <= g.n[1]) solo_load(in, g, w.xl, y + 3, qg);
        T Fa[4], Fl[4], Fr[4], left[4];
        rusanov<T, 2, 1>(w.qc, w.qa, gamma, gm1, Fa, w.chk, w.upd);
#pragma unroll
        for (int m = 0; m < 4; ++m) left[m] = __shfl_up_sync(0xffffffffu, w.qc[m], 1);
        rusanov<T, 2, 0>(left, w.qc, gamma, gm1, Fl, w.chk, w.xface);
#pragma unroll
        for (int m = 0; m < 4; ++m) Fr[m] = __shfl_down_sync(0xffffffffu, Fl[m], 1);
        if (w.upd) {
            T qn[4];
#pragma unroll
            for (int m = 0; m < 4; ++m)
                qn[m] = cell_update2(w.qc[m], Fl[m], Fr[m], w.Fb[m], Fa[m], inv_dx[0], inv_dx[1], dtT);
            const long long base = geom_cell(g, w.x, y, 0) * g.cell_stride;
#pragma unroll
            for (int m = 0; m < 4; ++m) out[base + (long long)m * g.comp_stride] = qn[m];
            bool ok;
            smax = max(smax, wave_sum<T, 2>(qn, gamma, gm1, inv_dx, ok));
            w.bad |= !ok;
            if (w.x < g.h || w.x >= g.n[0] - g.h || y < g.h || y >= g.n[1] - g.h)
                write_ghost_images<T, 2>(out, g, bc, w.x, y, 0, qn);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            w.Fb[m] = Fa[m];
            w.qc[m] = w.qa[m];
            w.qa[m] = w.qf[m];
            w.qf[m] = qg[m];
        }
    }
}

// Launched with blockDim.x a multiple of 32, at most kSoloThreads: the host
// sizes CTAs so that the units spread over as many SMs as possible.
template <typename T>
__global__ void __launch_bounds__(kSoloThreads) solo_euler2d_kernel(const SoloEuler a)
{
    __shared__ int sflag[1];
    __shared__ T s_dt[1];
    __shared__ T s_max[kSoloThreads / 32];
    if (threadIdx.x == 0) sflag[0] = 0;
    FieldCtl* ctl = a.ctl;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    const int warp = blockIdx.x * wpc + wib;
    const int nwarps = gridDim.x * wpc;
    const int units = a.strips * a.segs;
    const T gamma = field_const<T>(a.gamma, a.gamma_f), gm1 = field_const<T>(a.gm1, a.gm1_f);
    const T inv_dx[3] = {field_const<T>(a.inv_dx0, a.inv_dx0_f), field_const<T>(a.inv_dx1, a.inv_dx1_f), T(0)};
    for (int k = 0; k < a.K; ++k) {
        const long long local = a.first + k;
        const int rs = (int)(local % 3);
        const T* __restrict__ in = static_cast<const T*>(a.buf[local & 1]);
        T* __restrict__ out = static_cast<T*>(a.buf[(local & 1) ^ 1]);
        if (threadIdx.x == 0) {
            const double dt = a.cfl / __longlong_as_double((long long)__ldcg(&ctl->smax[rs]));
            s_dt[0] = (T)dt;
            if (blockIdx.x == 0) {
                ctl->t = local == 0 ? dt : ctl->t + dt;
                ctl->dt_last = dt;
                ctl->smax[(rs + 2) % 3] = 0ull;
            }
        }
        SoloUnit<T> w;
        int u = warp;
        if (u < units) solo_unit_begin(a.g, a.strips, a.rows, in, u, lane, gamma, gm1, w);
        __syncthreads();  // s_dt
        const T dtT = s_dt[0];
        T smax = T(0);
        while (u < units) {
            solo_unit_walk(a.g, a.bc, in, out, gamma, gm1, inv_dx, dtT, w, smax);
            // a non-admissible face or new state: the unit's first cell and row
            if (__any_sync(0xffffffffu, w.bad || !(w.chk > T(0))) && lane == 0) {
                record_bad(ctl, BAD_STATE, w.strip * kSoloW, w.y0, 0);
                atomicOr(&ctl->err, DEV_ERR_NUMERIC);
            }
            u += nwarps;
            if (u < units) solo_unit_begin(a.g, a.strips, a.rows, in, u, lane, gamma, gm1, w);
        }
        // CTA maximum of the new wave-speed sums -> the next ring slot (one
        // atomic per CTA, before the CTA's arrival at the barrier)
        T v = smax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) s_max[wib] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            T m = s_max[0];
            for (int i = 1; i < wpc; ++i) m = max(m, s_max[i]);
            atomic_max_pos_double(&ctl->smax[(rs + 1) % 3], (double)m);
        }
        if (k + 1 < a.K && !solo_barrier(a.bar, (unsigned)(k + 1), a.spin_limit, sflag)) {
            if (threadIdx.x == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// The same row walks as the batched step (one launch per global step over
// every active Euler problem): table entries [0, ntiles_e) of the batch are
// walk units instead of tiles, instance-major (BatchEuler::tile_begin is the
// instance's first unit, tiles_x its strips of kSoloW columns, units of
// kBatchWalkRows rows).  A warp takes one unit at a time: the instance's local
// step, its dt (lane 0, FP64, broadcast), the walk, its wave-speed maximum;
// unit 0 of an instance advances t and clears the ring slot after next, as
// tile 0 does in the tiled step.  Results are those of the tiled step bit for
// bit (same faces, same update).
// ---------------------------------------------------------------------------
constexpr int kBatchWalkRows = 16;
constexpr int kBatchWalkThreads = 256;  // threads per CTA of the batched walk kernels (8 warps)
// CTAs per SM the FP32 walk kernels are compiled for: three (80 registers, a
// few bytes of spills) ran the 512-problem step 15 % faster than two (98
// registers); the FP64 kernels need about 150 registers and keep one
template <typename T>
constexpr int batch_walk_min_blocks() { return sizeof(T) == 4 ? 3 : 1; }

// One walk unit of a batched step: local unit lu of instance d at the
// instance's local step `local` (dt by lane 0 in FP64, broadcast; unit 0
// advances t and clears the ring slot after next, as tile 0 does in the tiled
// step), then the unit's wave-speed maximum into the instance's next ring slot.
template <typename T>
__device__ __forceinline__ void batch_walk_unit(const BatchEuler& d, int lu, long long local, int lane)
{
    const int rs = (int)(local % 3);
    FieldCtl* ctl = d.ctl;
    double dt = 0.0;
    if (lane == 0) dt = d.cfl / __longlong_as_double((long long)__ldcg(&ctl->smax[rs]));
    dt = __shfl_sync(0xffffffffu, dt, 0);
    if (lu == 0 && lane == 0) {
        ctl->t = local == 0 ? dt : ctl->t + dt;
        ctl->dt_last = dt;
        ctl->smax[(rs + 2) % 3] = 0ull;
    }
    const T dtT = (T)dt;
    const T gamma = field_const<T>(d.gamma, d.gamma_f), gm1 = field_const<T>(d.gm1, d.gm1_f);
    const T inv_dx[3] = {field_const<T>(d.inv_dx0, d.inv_dx0_f), field_const<T>(d.inv_dx1, d.inv_dx1_f), T(0)};
    const T* in = static_cast<const T*>(d.buf[local & 1]);
    T* out = static_cast<T*>(d.buf[(local & 1) ^ 1]);
    SoloUnit<T> w;
    solo_unit_begin(d.g, d.tiles_x, kBatchWalkRows, in, lu, lane, gamma, gm1, w);
    T smax = T(0);
    solo_unit_walk(d.g, d.bc, in, out, gamma, gm1, inv_dx, dtT, w, smax);
    T v = smax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const bool wbad = __any_sync(0xffffffffu, w.bad || !(w.chk > T(0)));
    if (lane == 0) {
        atomic_max_pos_double(&ctl->smax[(rs + 1) % 3], (double)v);
        if (wbad) {
            record_bad(ctl, BAD_STATE, w.strip * kSoloW, w.y0, 0);
            atomicOr(&ctl->err, DEV_ERR_NUMERIC);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kBatchWalkThreads, batch_walk_min_blocks<T>())
    batch_euler_walk_kernel(const BatchEuler* __restrict__ euler, const int* __restrict__ table,
                            BatchCtl* __restrict__ bctl)
{
    const unsigned long long gstep = __ldcg(&bctl->gstep[0]);
    const int end = __ldcg(&bctl->ntiles_e);
    const int lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpc;
    for (int u = blockIdx.x * wpc + (threadIdx.x >> 5); u < end; u += nwarps) {
        const int inst = __ldg(&table[u]) >> 1;
        const BatchEuler& d = euler[inst];
        const long long local = (long long)gstep - d.start_step;
        if (local < 0 || local >= d.nsteps) continue;
        batch_walk_unit<T>(d, u - d.tile_begin, local, lane);
    }
    __syncwarp();
    batch_finish_launch(bctl, 0);
}

// The walk form of a dependency-driven round (BatchAsync; table entries are
// walk units).  Warps take the round's tasks (round step n, table entry t)
// from its counter, q->chunk at a time, in the step-major order of the tiled
// round.  A unit of step n > 0 first waits (lane 0, bounded) until every unit
// of its instance's step n - 1 is published: done[] counts units, ntiles of
// them per step, and the unit's dt and every cell it reads come from that
// step.  After its walk the warp publishes the unit: the warp barrier orders
// every lane's stores (cells, ghost images, wave-speed maximum, unit 0's ring
// slot) before lane 0's release add, which the waiting lane 0's acquire pairs
// with; the waiting warp's barrier after that acquire orders its lanes' loads
// (L2 loads, no stale L1 lines) after it.  A warp publishes every unit before
// it takes or waits for the next, and the tasks a wait needs precede it in the
// order and were taken by running warps, so the waits end; a wait that runs
// out stops its warp and reports DEV_ERR_TIMEOUT.  Each unit's arithmetic is
// the per-step walk kernel's, so results are those of per-step launches bit
// for bit.
template <typename T>
__global__ void __launch_bounds__(kBatchWalkThreads, batch_walk_min_blocks<T>())
    batch_euler_walk_async_kernel(const BatchEuler* __restrict__ euler, const int* __restrict__ table,
                                  BatchCtl* __restrict__ bctl, BatchAsync* __restrict__ q)
{
    const unsigned long long gstep = __ldcg(&bctl->gstep[0]);
    const int lane = threadIdx.x & 31;
    const int total = q->total, chunk = q->chunk, K = q->K;
    bool ok = true;
    // the current chunk of tasks [c_lo, c_hi), the cached task range [s_lo, s_hi) of round step s_n
    int c_lo = 0, c_hi = 0, s_lo = 0, s_hi = 0, s_n = 0;
    for (;;) {
        if (c_lo == c_hi) {
            int lo = 0;
            if (lane == 0) lo = atomicAdd(&q->next, chunk);
            lo = __shfl_sync(0xffffffffu, lo, 0);
            if (lo >= total) break;
            c_lo = lo;
            c_hi = min(lo + chunk, total);
        }
        const int k = c_lo++;
        if (k < s_lo || k >= s_hi) {
            int lo = 0, hi = K;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(&q->cum[mid]) <= k) lo = mid;
                else hi = mid;
            }
            s_n = lo;
            s_lo = __ldg(&q->cum[lo]);
            s_hi = __ldg(&q->cum[lo + 1]);
        }
        const int t = k - s_lo;
        const int inst = __ldg(&table[t]) >> 1;
        const BatchEuler& d = euler[inst];
        if (s_n > 0) {
            const unsigned need = (unsigned)s_n * (unsigned)d.ntiles;
            int met = 1;
            if (lane == 0) {
                uint32_t i = 0;
                while (ld_acquire_gpu(&q->done[inst]) < need && ++i < kDepSpinLimit) __nanosleep(64);
                met = i < kDepSpinLimit;
            }
            met = __shfl_sync(0xffffffffu, met, 0);
            __syncwarp();
            if (!met) {
                ok = false;
                break;
            }
        }
        batch_walk_unit<T>(d, t - d.tile_begin, (long long)gstep + s_n - d.start_step, lane);
        __syncwarp();
        if (lane == 0) red_release_gpu_add(&q->done[inst], 1u);
    }
    if (!ok && lane == 0) atomicOr(&bctl->err, DEV_ERR_TIMEOUT);
    __syncwarp();
    batch_finish_launch(bctl, 0, (unsigned long long)K);
}

}  // namespace ripple
