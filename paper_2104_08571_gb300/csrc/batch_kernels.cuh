// Batched global step over many independent problems of different sizes.
//
// One launch advances every resident problem by one step: each 2D Euler
// instance by one explicit Rusanov step (the same update as the single-field
// sweep), each eikonal instance by one iteration of its Fast Iterative Method.
// All tiles of all resident problems form one flat tile table that the CTAs
// walk with a fixed stride, so uneven grids share the GPU in one launch.
// Each problem keeps its own dt (its own 3-slot wave-speed ring), its own
// double-buffer parity and its own FIM iteration counter, all derived from the
// device-side global step counter and the step at which the problem joined.
// The last CTA of a launch advances that counter, so K launches can be queued
// (or captured in a CUDA graph) without host involvement.
#pragma once
#include <cstdint>

#include "euler_sweep.cuh"
#include "field.cuh"
#include "fim_tile.cuh"

namespace ripple {

// One resident 2D Euler instance.
struct BatchEuler {
    void* buf[2];
    FieldCtl* ctl;
    FieldGeom g;
    int tiles_x, tile_begin;
    int bc;
    long long start_step, nsteps;
    double gamma, cfl, inv_dx0, inv_dx1;
};

// One resident 2D eikonal instance.
template <typename T>
struct BatchFim {
    FimProblem<T> p;
    int tile_begin;
    long long start_step, max_iters;
    // 0 while running; (k << 2) | 1 once iteration k found nothing active and
    // consolidated the result into buf[0]; (k << 2) | 2 at the iteration cap.
    // Tiles of iteration k still run when another tile of the same launch has
    // already written k here; later iterations skip.
    unsigned long long* status;
    long long* counters;     // [3]: iterations, tile visits, Godunov updates
};

// Device-side control of a batch.  Euler steps and FIM iterations advance on
// separate launches with separate counters, so eikonal problems can iterate
// several times per Euler step.
struct BatchCtl {
    unsigned long long gstep[2];  // completed launches: [0] Euler steps, [1] FIM iterations
    unsigned int done[2];         // CTAs finished in the current launch of each kind
    int ntiles_e;                 // table entries [0, ntiles_e) are Euler tiles
    int ntiles;                   // entries [ntiles_e, ntiles) are eikonal tiles
};

// Tile-table entry: (instance index << 1) | kind, kind 0 = Euler, 1 = eikonal.
// The entry's tile index inside its instance is its position minus the
// instance's tile_begin.

template <typename T, int TX, int TY>
struct BatchSmemEuler {
    T S[4][TY + 2][TX + 2];  // staged tile + 1 ghost layer, component-major
    T FX[4][(TX + 1) * TY];
    T FY[4][TX * (TY + 1)];
};

template <typename T, int LAYOUT, int TX, int TY>
union BatchSmem {
    BatchSmemEuler<T, TX, TY> e;
    FimSmem<T, 2> f;
};

template <typename T, int LAYOUT, int TX, int TY>
__device__ __forceinline__ void batch_euler_tile(BatchSmemEuler<T, TX, TY>& sm, double* red,
                                                 const BatchEuler& d, int lt, long long local)
{
    constexpr int NC = 4, NT = TX * TY;
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const FieldGeom& g = d.g;
    const int x0 = (lt % d.tiles_x) * TX, y0 = (lt / d.tiles_x) * TY;
    const int par = (int)(local & 1);
    const T* __restrict__ in = static_cast<const T*>(d.buf[par]);
    T* __restrict__ out = static_cast<T*>(d.buf[par ^ 1]);
    const int slot = (int)(local % 3);
    const double dt = d.cfl / __longlong_as_double((long long)__ldcg(&d.ctl->smax[slot]));
    const T gamma = (T)d.gamma, gm1 = (T)(d.gamma - 1.0), dtT = (T)dt;
    const T inv_dx[3] = {(T)d.inv_dx0, (T)d.inv_dx1, T(0)};
    if (lt == 0 && tid == 0) {
        d.ctl->t = local == 0 ? dt : d.ctl->t + dt;
        d.ctl->dt_last = dt;
        d.ctl->smax[(slot + 2) % 3] = 0ull;
    }
    // stage the tile with one ghost layer (cells beyond the x/y ghost are not read)
    constexpr int CELLS = (TY + 2) * (TX + 2);
    for (int e = tid; e < NC * CELLS; e += NT) {
        int m, r;
        if (LAYOUT == LAYOUT_SOA) { m = e / CELLS; r = e % CELLS; }
        else { m = e % NC; r = e / NC; }
        const int cy = r / (TX + 2) - 1, cx = r % (TX + 2) - 1;
        const int gx = x0 + cx, gy = y0 + cy;
        T v = T(0);
        if (gx <= g.n[0] && gy <= g.n[1]) v = in[geom_elem(g, gx, gy, 0, m)];
        sm.S[m][cy + 1][cx + 1] = v;
    }
    __syncthreads();
    T chk = T(1);
    // face fluxes: x faces between fx-1 and fx, y faces between fy-1 and fy
    for (int it = tid; it < NFX + NFY; it += NT) {
        T a[NC], b[NC], F[NC];
        if (it < NFX) {
            const int fx = it % (TX + 1), cy = it / (TX + 1);
#pragma unroll
            for (int m = 0; m < NC; ++m) { a[m] = sm.S[m][cy + 1][fx]; b[m] = sm.S[m][cy + 1][fx + 1]; }
            rusanov<T, 2, 0>(a, b, gamma, gm1, F, chk, (x0 + fx <= g.n[0]) && (y0 + cy < g.n[1]));
#pragma unroll
            for (int m = 0; m < NC; ++m) sm.FX[m][it] = F[m];
        } else {
            const int k = it - NFX;
            const int cx = k % TX, fy = k / TX;
#pragma unroll
            for (int m = 0; m < NC; ++m) { a[m] = sm.S[m][fy][cx + 1]; b[m] = sm.S[m][fy + 1][cx + 1]; }
            rusanov<T, 2, 1>(a, b, gamma, gm1, F, chk, (x0 + cx < g.n[0]) && (y0 + fy <= g.n[1]));
#pragma unroll
            for (int m = 0; m < NC; ++m) sm.FY[m][k] = F[m];
        }
    }
    __syncthreads();
    const int gx = x0 + lx, gy = y0 + ly;
    const bool valid = (gx < g.n[0]) & (gy < g.n[1]);
    T smax = T(0);
    bool bad = !(chk > T(0));
    if (valid) {
        T qn[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            T acc = (sm.FX[m][ly * (TX + 1) + lx + 1] - sm.FX[m][ly * (TX + 1) + lx]) * inv_dx[0];
            acc += (sm.FY[m][(ly + 1) * TX + lx] - sm.FY[m][ly * TX + lx]) * inv_dx[1];
            qn[m] = sm.S[m][ly + 1][lx + 1] - dtT * acc;
        }
        const long long base = geom_cell(g, gx, gy, 0) * g.cell_stride;
#pragma unroll
        for (int m = 0; m < NC; ++m) out[base + (long long)m * g.comp_stride] = qn[m];
        bool ok;
        smax = wave_sum<T, 2>(qn, gamma, gm1, inv_dx, ok);
        bad |= !ok;
        if (gx < g.h || gx >= g.n[0] - g.h || gy < g.h || gy >= g.n[1] - g.h)
            write_ghost_images<T, 2>(out, g, d.bc, gx, gy, 0, qn);
    }
    // tile max of the new wave-speed sums -> the instance's next ring slot
    double v = (double)smax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < NT / 32; ++w) m = fmax(m, red[w]);
        atomic_max_pos_double(&d.ctl->smax[(slot + 1) % 3], m);
        if (any_bad) {
            record_bad(d.ctl, BAD_STATE, x0, y0, 0);
            atomicOr(&d.ctl->err, DEV_ERR_NUMERIC);
        }
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void batch_fim_tile(FimSmem<T, 2>& sm, const BatchFim<T>& d, int lt, long long k)
{
    using C = EikTile<2>;
    const int tid = threadIdx.x;
    const FimProblem<T>& a = d.p;
    if (k >= d.max_iters) {
        if (lt == 0 && tid == 0) *d.status = ((unsigned long long)k << 2) | 2ull;
        return;
    }
    const unsigned remaining = __ldcg(&a.count[k % 3]);
    if (remaining == 0u) {
        // converged in the previous iteration: consolidate this tile into buffer 0
        if (__ldcg(&a.cur[(size_t)(k % 2) * a.ntiles + lt]) != 0) {
            const int bx = lt % a.ntx, by = lt / a.ntx;
            for (int c = 0; c < C::CPT; ++c) {
                const int lin = tid + c * C::NT;
                const int gx = bx * C::TS + lin % C::TS, gy = by * C::TS + lin / C::TS;
                if (gx < a.gT.n[0] && gy < a.gT.n[1]) {
                    const long long id = geom_cell(a.gT, gx, gy, 0);
                    a.buf[0][id] = ldcg_t(&a.buf[1][id]);
                }
            }
        }
        if (lt == 0 && tid == 0) {
            d.counters[0] = k;
            *d.status = ((unsigned long long)k << 2) | 1ull;
        }
        return;
    }
    if (lt == 0 && tid == 0) a.count[(k + 2) % 3] = 0u;
    long long visits = 0, updates = 0;
    fim_visit_tile<T, 2>(sm, a, lt, k, visits, updates);
    if (tid == 0 && visits) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&d.counters[1]), (unsigned long long)visits);
        atomicAdd(reinterpret_cast<unsigned long long*>(&d.counters[2]), (unsigned long long)updates);
    }
}

// kind 0: one Euler step of every resident Euler problem; kind 1: one FIM
// iteration of every resident eikonal problem.
template <typename T, int LAYOUT, int TX, int TY>
__global__ void __launch_bounds__(256) batch_step_kernel(const BatchEuler* __restrict__ euler,
                                                         const BatchFim<T>* __restrict__ fim,
                                                         const int* __restrict__ table, BatchCtl* __restrict__ bctl,
                                                         int kind)
{
    static_assert(TX * TY == 256, "the batched step runs 256 threads (the FIM tile size)");
    __shared__ BatchSmem<T, LAYOUT, TX, TY> sm;
    __shared__ double red[8];
    const unsigned long long gstep = __ldcg(&bctl->gstep[kind]);
    const int begin = kind == 0 ? 0 : __ldcg(&bctl->ntiles_e);
    const int end = kind == 0 ? __ldcg(&bctl->ntiles_e) : __ldcg(&bctl->ntiles);
    for (int t = begin + blockIdx.x; t < end; t += gridDim.x) {
        const int entry = __ldg(&table[t]);
        const int idx = entry >> 1;
        if (kind == 0) {
            const BatchEuler& d = euler[idx];
            const long long local = (long long)gstep - d.start_step;
            if (local < 0 || local >= d.nsteps) continue;
            batch_euler_tile<T, LAYOUT, TX, TY>(sm.e, red, d, t - d.tile_begin, local);
        } else {
            const BatchFim<T>& d = fim[idx];
            const long long k = (long long)gstep - d.start_step;
            if (k < 0) continue;
            const unsigned long long st = __ldcg(d.status);
            if (st != 0ull && (unsigned long long)k > (st >> 2)) continue;
            batch_fim_tile<T>(sm.f, d, t - d.tile_begin, k);
        }
    }
    // the last CTA to finish advances this kind's counter
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&bctl->done[kind], 1u) == gridDim.x - 1) {
            bctl->done[kind] = 0u;
            __threadfence();
            atomicAdd(&bctl->gstep[kind], 1ull);
        }
    }
}

}  // namespace ripple
