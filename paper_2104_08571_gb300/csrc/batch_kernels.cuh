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
// (or captured in a CUDA graph) without host involvement.  A dependency-driven
// round (BatchAsync below) runs K steps of every Euler problem in one launch
// of the same kernel instead.
#pragma once
#include <cstdint>

#include "euler_sweep.cuh"
#include "field.cuh"
#include "fim_tile.cuh"

namespace ripple {

// One resident 2D Euler instance.  The TMA maps stage the padded planes of
// buf[0] and buf[1] in boxes of the configured tile shape; they live in
// device memory (64-byte aligned) and are acquired before each use because a
// slot of the descriptor array is reused by later instances.
struct BatchEuler {  // aligned as CUtensorMap (at least 64 bytes)
    CUtensorMap map[2];
    void* buf[2];
    FieldCtl* ctl;
    FieldGeom g;
    int tiles_x, tile_begin, ntiles;
    int bc;
    long long start_step, nsteps;
    double gamma, gm1, cfl, inv_dx0, inv_dx1;  // gm1 = gamma - 1, formed on the host in FP64
    float gamma_f, gm1_f, inv_dx0_f, inv_dx1_f;  // the same rounded to FP32 on the host
};

// A descriptor constant in the field precision: FP32 kernels take the
// host-rounded copy (no conversion on the device's narrow FP64 pipe).
template <typename T>
__device__ __forceinline__ T field_const(double v, float vf)
{
    if constexpr (std::is_same<T, float>::value) return vf;
    else return v;
}

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
    unsigned int err;             // DEV_ERR_TIMEOUT: a bounded wait of a batched launch ran out
};

// Dependency-driven round of the batched Euler step (one persistent launch for
// K steps).  The round's tasks are (round step n, table entry p) in step-major
// order: step n holds the first cum[n + 1] - cum[n] Euler table entries (the
// host orders Euler instances by remaining steps, so the instances still
// stepping at round step n are a prefix).  CTAs take tasks in that order from
// one atomic counter; a task of step n > 0 first waits until its instance has
// completed step n - 1 (done[] counts consumer-warp completions, NCT / 32 per
// tile), because its dt is the CFL limit of the instance's whole state after
// that step.  Every dependency of a task precedes it in the order and tasks
// are taken only by running CTAs, so the waits always end (bounded anyway).
struct BatchAsync {
    int next;            // next task (atomic); the host zeroes it before the launch
    int total;           // tasks of the round: cum[K]
    int K;               // steps of the round
    int chunk;           // tasks a worker (producer warp, or walk warp) takes at once (1..kAsyncChunk: fewer
                         // when a step has few tasks)
    const int* cum;      // [K + 1] first task of each round step
    unsigned* done;      // [Euler instances] consumer-warp completions this round
};

// Tile-table entry: (instance index << 1) | kind, kind 0 = Euler, 1 = eikonal.
// The entry's tile index inside its instance is its position minus the
// instance's tile_begin.

// Shared-memory plan of the batched Euler step: the full/empty mbarriers of
// a ring of NS slots, one header of tile parameters per slot, the staged
// tiles (TMA boxes of the tile plus one ghost layer, all four components;
// each starts on a 128-byte boundary as TMA requires) and two face-flux
// buffers (by tile parity).
template <typename T, int LAYOUT, int TX, int TY>
struct BatchEulerCfg {
    using C = SweepCfg<T, 2, LAYOUT, SCHEME_RUSANOV1, TX, TY>;
    static constexpr int NC = 4, NS = 4;
    static constexpr int NCT = TX * TY;          // consumer threads: one cell each
    static constexpr int NTHREADS = NCT + 32;    // plus one producer warp
    static constexpr int HDRS = 16 * NS;         // after the 2 * NS mbarriers
    static constexpr int SLOT_HDR = 192;         // per-slot tile parameters (BatchTileHdr)
    static constexpr int RING = ((HDRS + NS * SLOT_HDR + 127) / 128) * 128;
    static constexpr int FACES = RING + NS * C::SLOT_BYTES;
    static constexpr int SMEM = FACES + 2 * C::F_BYTES;
    static_assert(NCT == 256, "the batched step updates 256 cells per tile");
    static_assert(RING % 128 == 0 && C::SLOT_BYTES % 128 == 0 && C::F_BYTES % 128 == 0, "TMA destinations");
};

// Everything the consumers need about a staged tile, written by the producer
// before the slot's full barrier completes (the consumers then read no
// descriptor from global memory).  tile < 0 marks the end of the CTA's work.
template <typename T>
struct BatchTileHdr {
    FieldGeom g;
    T* out;          // output buffer of this step
    FieldCtl* ctl;   // the instance's control block
    T gamma, gm1, inv_dx0, inv_dx1, dt;
    int tile, x0, y0, bc, rs;  // rs: the instance's ring slot of this step's input
    int inst;                  // Euler instance index (dependency counter of a dependency-driven round)
};
static_assert(sizeof(BatchTileHdr<double>) <= 192, "tile header fits the slot header");

// The last CTA of a launch to finish advances the step counter of its kind
// (by the steps the launch ran: 1, or K for a dependency-driven round).
__device__ __forceinline__ void batch_finish_launch(BatchCtl* bctl, int kind, unsigned long long steps = 1ull)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&bctl->done[kind], 1u) == gridDim.x - 1) {
            bctl->done[kind] = 0u;
            __threadfence();
            atomicAdd(&bctl->gstep[kind], steps);
        }
    }
}

constexpr uint32_t kDepSpinLimit = 1u << 23;  // dependency waits of a round (x 64 ns sleeps: about 0.5 s)
constexpr int kAsyncChunk = 8;                // most tasks a producer takes from a round's counter at once
constexpr unsigned kPublishRun = 16;          // most completed tiles a consumer warp publishes at once

// Barrier among the 256 consumer threads only (the producer warp runs ahead),
// returning the OR of a predicate over them: every consumer takes the same
// decision at the same barrier.
__device__ __forceinline__ bool consumer_sync_or(bool p)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred o, 1, 256, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p)
        : "memory");
    return r != 0;
}

// One explicit Rusanov step of every resident Euler problem inside its step
// window.  The CTAs walk the Euler part of the tile table with a fixed stride.
// Warp-specialised pipeline: the producer warp (one elected lane) walks the
// CTA's tiles, forms each tile's parameters (dt from the instance's FP64 ring,
// constants in the field's precision) into the slot header and issues the
// slot's TMA load from the instance's own map, up to NS tiles ahead; the 256
// consumer threads wait on the slot's full barrier, compute the tile's faces
// into the face buffer of the tile's parity, meet at one named barrier,
// update one cell each (direct coalesced stores, ghost images), fold the new
// wave speeds per warp into the instance's next ring slot, and release the
// slot through its empty barrier.
// ASYNC: the same pipeline runs a whole dependency-driven round (BatchAsync):
// the producer takes tasks from the round's counter and waits for each task's
// instance to finish the previous step before staging it; every consumer warp
// publishes its part of a tile (fence, then an atomic on done[]).
template <typename T, int LAYOUT, int TX, int TY, bool ASYNC = false>
__global__ void __launch_bounds__(288) batch_euler_kernel(const BatchEuler* __restrict__ euler,
                                                          const int* __restrict__ table,
                                                          BatchCtl* __restrict__ bctl,
                                                          BatchAsync* __restrict__ q = nullptr)
{
    using B = BatchEulerCfg<T, LAYOUT, TX, TY>;
    using C = typename B::C;
    using PV = PlaneView<C, LAYOUT>;
    using Hdr = BatchTileHdr<T>;
    constexpr int NC = 4, NS = B::NS, NCT = B::NCT;
    constexpr int NFX = C::NFX, NFY = C::NFY;
    constexpr int NFXr = ((NFX + 31) / 32) * 32, NFYr = ((NFY + 31) / 32) * 32;
    constexpr int KF = (NFXr + NFYr + NCT - 1) / NCT;
    constexpr int SX = LAYOUT == LAYOUT_SOA ? 1 : NC;
    constexpr int SY = LAYOUT == LAYOUT_SOA ? C::BX : C::BX * NC;
    constexpr int SM = LAYOUT == LAYOUT_SOA ? C::BX * C::BY : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NS;
    auto slot_hdr = [&](unsigned s) { return reinterpret_cast<Hdr*>(smem + B::HDRS + s * B::SLOT_HDR); };
    auto slot_tile = [&](unsigned s) { return reinterpret_cast<T*>(smem + B::RING + s * C::SLOT_BYTES); };
    auto faces = [&](unsigned par) { return reinterpret_cast<T*>(smem + B::FACES + par * C::F_BYTES); };

    const int tid = threadIdx.x;
    const unsigned long long gstep = __ldcg(&bctl->gstep[0]);
    const int end = __ldcg(&bctl->ntiles_e);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCT / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= NCT) {
        // ---------------- producer warp ----------------
        if (tid == NCT) {
            unsigned seq = 0;
            bool ok = true;
            // dependency-driven round: the current chunk of tasks [c_lo, c_hi), the
            // cached task range [s_lo, s_hi) of round step s_n, the last dependency met
            int c_lo = 0, c_hi = 0, s_lo = 0, s_hi = 0, s_n = 0, dep_inst = -1, dep_n = -1;
            // dt of the last (instance, step) a tile was issued for
            int dt_inst = -1;
            long long dt_local = -1;
            double dt = 0.0;
            T dtT = T(0);
            for (int t = blockIdx.x;; t += gridDim.x) {
                const BatchEuler* d = nullptr;
                long long local = 0;
                int inst = 0;
                bool have = false;
                if (!ASYNC) {
                    // next table entry whose instance steps in this launch
                    for (; t < end; t += gridDim.x) {
                        inst = __ldg(&table[t]) >> 1;
                        d = &euler[inst];
                        local = (long long)gstep - d->start_step;
                        if (local >= 0 && local < d->nsteps) break;
                    }
                    have = t < end;
                } else {
                    // next task of the round, taken q->chunk at a time: round step
                    // n (cum[n] <= k < cum[n + 1]) and table entry t = k - cum[n]
                    if (c_lo == c_hi) {
                        const int ch = q->chunk;
                        c_lo = atomicAdd(&q->next, ch);
                        c_hi = min(c_lo + ch, q->total);
                    }
                    if (c_lo < c_hi) {
                        const int k = c_lo++;
                        if (k < s_lo || k >= s_hi) {
                            int lo = 0, hi = q->K;
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (__ldg(&q->cum[mid]) <= k) lo = mid;
                                else hi = mid;
                            }
                            s_n = lo;
                            s_lo = __ldg(&q->cum[lo]);
                            s_hi = __ldg(&q->cum[lo + 1]);
                        }
                        t = k - s_lo;
                        inst = __ldg(&table[t]) >> 1;
                        d = &euler[inst];
                        local = (long long)gstep + s_n - d->start_step;
                        if (s_n > 0 && (inst != dep_inst || s_n != dep_n)) {
                            // the instance's previous step must be complete (its CFL maximum, its halos)
                            const unsigned need = (unsigned)s_n * (unsigned)d->ntiles * (NCT / 32);
                            uint32_t i = 0;
                            while (ld_acquire_gpu(&q->done[inst]) < need && ++i < kDepSpinLimit) __nanosleep(64);
                            if (i >= kDepSpinLimit) ok = false;
                            // other CTAs' stores (generic proxy) before this CTA's TMA reads (async proxy)
                            fence_proxy_async_global();
                            dep_inst = inst;
                            dep_n = s_n;
                        }
                        have = ok;
                    }
                }
                const unsigned s = seq % NS;
                if (seq >= NS && !mbar_wait_bounded(&empty[s], ((seq / NS) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                Hdr* h = slot_hdr(s);
                if (!have) {
                    h->tile = -1;
                    mbar_arrive(&full[s]);
                    ++seq;
                    break;
                }
                const int lt = t - d->tile_begin;
                const int x0 = (lt % d->tiles_x) * TX, y0 = (lt / d->tiles_x) * TY;
                const int rs = (int)(local % 3);
                FieldCtl* ctl = d->ctl;
                if (inst != dt_inst || local != dt_local) {
                    // dt once per (instance, step) run of tiles: an FP64 division
                    dt_inst = inst;
                    dt_local = local;
                    dt = d->cfl / __longlong_as_double((long long)__ldcg(&ctl->smax[rs]));
                    dtT = (T)dt;
                }
                h->g = d->g;
                h->out = static_cast<T*>(d->buf[(local & 1) ^ 1]);
                h->ctl = ctl;
                h->gamma = field_const<T>(d->gamma, d->gamma_f);
                h->gm1 = field_const<T>(d->gm1, d->gm1_f);
                h->inv_dx0 = field_const<T>(d->inv_dx0, d->inv_dx0_f);
                h->inv_dx1 = field_const<T>(d->inv_dx1, d->inv_dx1_f);
                h->dt = dtT;
                h->tile = t;
                h->x0 = x0;
                h->y0 = y0;
                h->bc = d->bc;
                h->rs = rs;
                h->inst = inst;
                if (lt == 0) {
                    ctl->t = local == 0 ? dt : ctl->t + dt;
                    ctl->dt_last = dt;
                    ctl->smax[(rs + 2) % 3] = 0ull;
                }
                const CUtensorMap* map = &d->map[local & 1];
                tensormap_acquire(map);
                const int xs = d->g.lead + d->g.h + x0 - 1 - C::OFF, ys = d->g.h + y0 - 1;
                mbar_arrive_expect_tx(&full[s], (uint32_t)(C::SLOT_ELEMS * sizeof(T)));
                if (LAYOUT == LAYOUT_SOA) tma_load_3d(slot_tile(s), map, xs, ys, 0, &full[s]);
                else tma_load_2d(slot_tile(s), map, xs * NC, ys, &full[s]);
                ++seq;
            }
            // every load this warp issued completes before the CTA exits (bounded)
            for (unsigned sq = seq > NS ? seq - NS : 0; sq < seq; ++sq)
                mbar_wait_bounded(&full[sq % NS], (sq / NS) & 1u);
            if (!ok) atomicOr(&bctl->err, DEV_ERR_TIMEOUT);
        }
        __syncwarp();
        batch_finish_launch(bctl, 0, ASYNC ? (unsigned long long)q->K : 1ull);
        return;
    }

    // ---------------- consumer warps ----------------
    const int lx = tid % TX, ly = tid / TX;
    bool timed_out = false;
    // ASYNC: a warp publishes its parts of tiles late and in runs: the
    // completed tiles of one instance accumulate (pend, npend) and one release
    // publishes them after the faces of a tile of another instance, after
    // kPublishRun tiles, or before the warp blocks waiting for its next tile
    // (so no waiting warp holds unpublished tiles: the waits of a round end).
    int pend = -1;
    unsigned npend = 0;
    auto publish = [&]() {
        __syncwarp();
        if ((tid & 31) == 0) red_release_gpu_add(&q->done[pend], npend);
        pend = -1;
        npend = 0;
    };
    for (unsigned seq = 0;; ++seq) {
        const unsigned s = seq % NS;
        if (ASYNC && pend >= 0) {
            const bool ready = __shfl_sync(0xffffffffu, (tid & 31) == 0 && mbar_try_wait(&full[s], (seq / NS) & 1u), 0);
            if (!ready) publish();
        }
        const bool got = mbar_wait_bounded(&full[s], (seq / NS) & 1u);
        const Hdr& h = *slot_hdr(s);  // shared memory, valid until this warp releases the slot
        const bool stop = !got || h.tile < 0;  // taken by all consumers together at the barrier below
        timed_out |= !got;
        const FieldGeom& g = h.g;
        const int x0 = h.x0, y0 = h.y0;
        const T gamma = h.gamma, gm1 = h.gm1, dtT = h.dt;
        const T inv_dx[3] = {h.inv_dx0, h.inv_dx1, T(0)};
        const T* S = slot_tile(s);
        T* FX = faces(seq & 1u);
        T* FY = FX + NC * NFX;

        // face fluxes: x faces between cells fx-1 | fx, y faces between fy-1 | fy
        T chk = T(1);
#pragma unroll 1
        for (int k = 0; k < (stop ? 0 : KF); ++k) {
            const int it = tid + k * NCT;
            T a[NC], b[NC], F[NC];
            if (it < NFXr) {
                if (it >= NFX) continue;
                const int fx = it % (TX + 1), cy = it / (TX + 1);
                const int o = PV::idx(fx - 1, cy, 0);
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    a[m] = S[o + m * SM];
                    b[m] = S[o + SX + m * SM];
                }
                rusanov<T, 2, 0>(a, b, gamma, gm1, F, chk, (x0 + fx <= g.n[0]) && (y0 + cy < g.n[1]));
#pragma unroll
                for (int m = 0; m < NC; ++m) FX[m * NFX + it] = F[m];
            } else {
                const int kk = it - NFXr;
                if (kk >= NFY) continue;
                const int cx = kk % TX, fy = kk / TX;
                const int o = PV::idx(cx, fy - 1, 0);
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    a[m] = S[o + m * SM];
                    b[m] = S[o + SY + m * SM];
                }
                rusanov<T, 2, 1>(a, b, gamma, gm1, F, chk, (x0 + cx < g.n[0]) && (y0 + fy <= g.n[1]));
#pragma unroll
                for (int m = 0; m < NC; ++m) FY[m * NFY + kk] = F[m];
            }
        }
        __syncwarp();
        if (consumer_sync_or(stop)) break;  // faces of this tile written, unless a consumer stopped
        if (ASYNC && pend >= 0 && (pend != h.inst || npend >= kPublishRun)) publish();
        const int gx = x0 + lx, gy = y0 + ly;
        const bool valid = (gx < g.n[0]) & (gy < g.n[1]);
        T smax = T(0);
        bool bad = !(chk > T(0));
        if (valid) {
            T* __restrict__ out = h.out;
            const int o = PV::idx(lx, ly, 0);
            T qn[NC];
#pragma unroll
            for (int m = 0; m < NC; ++m)
                qn[m] = cell_update2(S[o + m * SM], FX[m * NFX + ly * (TX + 1) + lx], FX[m * NFX + ly * (TX + 1) + lx + 1],
                                     FY[m * NFY + ly * TX + lx], FY[m * NFY + (ly + 1) * TX + lx], inv_dx[0], inv_dx[1],
                                     dtT);
            const long long base = geom_cell(g, gx, gy, 0) * g.cell_stride;
#pragma unroll
            for (int m = 0; m < NC; ++m) out[base + (long long)m * g.comp_stride] = qn[m];
            bool ok;
            smax = wave_sum<T, 2>(qn, gamma, gm1, inv_dx, ok);
            bad |= !ok;
            if (gx < g.h || gx >= g.n[0] - g.h || gy < g.h || gy >= g.n[1] - g.h)
                write_ghost_images<T, 2>(out, g, h.bc, gx, gy, 0, qn);
        }
        // warp max of the new wave-speed sums -> the instance's next ring slot
        T v = smax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        const bool wbad = __any_sync(0xffffffffu, bad);
        if ((tid & 31) == 0) {
            FieldCtl* ctl = h.ctl;
            atomic_max_pos_double(&ctl->smax[(h.rs + 1) % 3], (double)v);
            if (wbad) {
                record_bad(ctl, BAD_STATE, x0, y0, 0);
                atomicOr(&ctl->err, DEV_ERR_NUMERIC);
            }
        }
        // this warp's part of the tile (cells, ghost images, wave speeds) is
        // published later: the warp barrier in publish() orders every lane's
        // stores before lane 0's release, which the acquiring producer pairs with
        if (ASYNC) {
            pend = h.inst;
            ++npend;
        }
        // this warp's reads of the slot (tile and header) are done: release it
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
    }
    if (ASYNC && pend >= 0) publish();
    if (timed_out) atomicOr(&bctl->err, DEV_ERR_TIMEOUT);  // the runtime fails the resident set
    __syncwarp();
    batch_finish_launch(bctl, 0, ASYNC ? (unsigned long long)q->K : 1ull);
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
    fim_visit_tile<T, 2>(sm, a, lt, k, visits, updates, FimFlagBook<T>{a, k});
    if (tid == 0 && visits) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&d.counters[1]), (unsigned long long)visits);
        atomicAdd(reinterpret_cast<unsigned long long*>(&d.counters[2]), (unsigned long long)updates);
    }
}

// The same batched Euler step with the other halo staging: every thread loads
// its share of the tile plus one ghost layer straight from global memory
// (coalesced along x, all loads of a thread issued before its shared-memory
// stores), one tile at a time per CTA.  The autotuner picks between this and
// the TMA pipeline above.
template <typename T, int LAYOUT, int TX, int TY>
__global__ void __launch_bounds__(256) batch_euler_direct_kernel(const BatchEuler* __restrict__ euler,
                                                                 const int* __restrict__ table,
                                                                 BatchCtl* __restrict__ bctl)
{
    constexpr int NC = 4, NT = TX * TY;
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    constexpr int CELLS = (TX + 2) * (TY + 2);
    constexpr int KL = (NC * CELLS + NT - 1) / NT;  // staged elements per thread
    constexpr int NFXr = ((NFX + 31) / 32) * 32, NFYr = ((NFY + 31) / 32) * 32;
    constexpr int KF = (NFXr + NFYr + NT - 1) / NT;
    static_assert(NT == 256, "the batched step runs 256 threads");
    __shared__ T S[NC][TY + 2][TX + 2];
    __shared__ T FX[NC][NFX];
    __shared__ T FY[NC][NFY];
    __shared__ T sp[5];  // tile parameters: gamma, gm1, 1/dx, 1/dy, dt
    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const unsigned long long gstep = __ldcg(&bctl->gstep[0]);
    const int end = __ldcg(&bctl->ntiles_e);
    for (int t = blockIdx.x; t < end; t += gridDim.x) {
        const BatchEuler& d = euler[__ldg(&table[t]) >> 1];
        const long long local = (long long)gstep - d.start_step;
        if (local < 0 || local >= d.nsteps) continue;  // the same for every thread of the CTA
        const FieldGeom g = d.g;
        const int lt = t - d.tile_begin;
        const int x0 = (lt % d.tiles_x) * TX, y0 = (lt / d.tiles_x) * TY;
        const int rs = (int)(local % 3);
        FieldCtl* ctl = d.ctl;
        const T* __restrict__ in = static_cast<const T*>(d.buf[local & 1]);
        T* __restrict__ out = static_cast<T*>(d.buf[(local & 1) ^ 1]);
        T v[KL];
#pragma unroll
        for (int k = 0; k < KL; ++k) {
            const int e = tid + k * NT;
            v[k] = T(0);
            if (e < NC * CELLS) {
                const int m = LAYOUT == LAYOUT_SOA ? e / CELLS : e % NC;
                const int r = LAYOUT == LAYOUT_SOA ? e % CELLS : e / NC;
                const int gx = x0 + r % (TX + 2) - 1, gy = y0 + r / (TX + 2) - 1;
                if (gx <= g.n[0] && gy <= g.n[1]) v[k] = in[geom_elem(g, gx, gy, 0, m)];
            }
        }
#pragma unroll
        for (int k = 0; k < KL; ++k) {
            const int e = tid + k * NT;
            if (e < NC * CELLS) {
                const int m = LAYOUT == LAYOUT_SOA ? e / CELLS : e % NC;
                const int r = LAYOUT == LAYOUT_SOA ? e % CELLS : e / NC;
                S[m][r / (TX + 2)][r % (TX + 2)] = v[k];
            }
        }
        if (tid == 0) {
            const double dt = d.cfl / __longlong_as_double((long long)__ldcg(&ctl->smax[rs]));
            sp[0] = field_const<T>(d.gamma, d.gamma_f);
            sp[1] = field_const<T>(d.gm1, d.gm1_f);
            sp[2] = field_const<T>(d.inv_dx0, d.inv_dx0_f);
            sp[3] = field_const<T>(d.inv_dx1, d.inv_dx1_f);
            sp[4] = (T)dt;
            if (lt == 0) {
                ctl->t = local == 0 ? dt : ctl->t + dt;
                ctl->dt_last = dt;
                ctl->smax[(rs + 2) % 3] = 0ull;
            }
        }
        __syncthreads();
        const T gamma = sp[0], gm1 = sp[1], dtT = sp[4];
        const T inv_dx[3] = {sp[2], sp[3], T(0)};
        T chk = T(1);
#pragma unroll 1
        for (int k = 0; k < KF; ++k) {
            const int it = tid + k * NT;
            T a[NC], b[NC], F[NC];
            if (it < NFXr) {
                if (it >= NFX) continue;
                const int fx = it % (TX + 1), cy = it / (TX + 1);
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    a[m] = S[m][cy + 1][fx];
                    b[m] = S[m][cy + 1][fx + 1];
                }
                rusanov<T, 2, 0>(a, b, gamma, gm1, F, chk, (x0 + fx <= g.n[0]) && (y0 + cy < g.n[1]));
#pragma unroll
                for (int m = 0; m < NC; ++m) FX[m][it] = F[m];
            } else {
                const int kk = it - NFXr;
                if (kk >= NFY) continue;
                const int cx = kk % TX, fy = kk / TX;
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    a[m] = S[m][fy][cx + 1];
                    b[m] = S[m][fy + 1][cx + 1];
                }
                rusanov<T, 2, 1>(a, b, gamma, gm1, F, chk, (x0 + cx < g.n[0]) && (y0 + fy <= g.n[1]));
#pragma unroll
                for (int m = 0; m < NC; ++m) FY[m][kk] = F[m];
            }
        }
        __syncthreads();
        const int gx = x0 + lx, gy = y0 + ly;
        T smax = T(0);
        bool bad = !(chk > T(0));
        if ((gx < g.n[0]) & (gy < g.n[1])) {
            T qn[NC];
#pragma unroll
            for (int m = 0; m < NC; ++m)
                qn[m] = cell_update2(S[m][ly + 1][lx + 1], FX[m][ly * (TX + 1) + lx], FX[m][ly * (TX + 1) + lx + 1],
                                     FY[m][ly * TX + lx], FY[m][(ly + 1) * TX + lx], inv_dx[0], inv_dx[1], dtT);
            const long long base = geom_cell(g, gx, gy, 0) * g.cell_stride;
#pragma unroll
            for (int m = 0; m < NC; ++m) out[base + (long long)m * g.comp_stride] = qn[m];
            bool ok;
            smax = wave_sum<T, 2>(qn, gamma, gm1, inv_dx, ok);
            bad |= !ok;
            if (gx < g.h || gx >= g.n[0] - g.h || gy < g.h || gy >= g.n[1] - g.h)
                write_ghost_images<T, 2>(out, g, d.bc, gx, gy, 0, qn);
        }
        T w = smax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
        const bool wbad = __any_sync(0xffffffffu, bad);
        if ((tid & 31) == 0) {
            atomic_max_pos_double(&ctl->smax[(rs + 1) % 3], (double)w);
            if (wbad) {
                record_bad(ctl, BAD_STATE, x0, y0, 0);
                atomicOr(&ctl->err, DEV_ERR_NUMERIC);
            }
        }
        __syncthreads();  // the next tile overwrites S, FX, FY and sp
    }
    batch_finish_launch(bctl, 0);
}

// One FIM iteration of every resident eikonal problem.
template <typename T>
__global__ void __launch_bounds__(EikTile<2>::NT) batch_fim_kernel(const BatchFim<T>* __restrict__ fim,
                                                        const int* __restrict__ table, BatchCtl* __restrict__ bctl)
{
    __shared__ FimSmem<T, 2> sm;
    const unsigned long long gstep = __ldcg(&bctl->gstep[1]);
    const int begin = __ldcg(&bctl->ntiles_e);
    const int end = __ldcg(&bctl->ntiles);
    for (int t = begin + blockIdx.x; t < end; t += gridDim.x) {
        const BatchFim<T>& d = fim[__ldg(&table[t]) >> 1];
        const long long k = (long long)gstep - d.start_step;
        if (k < 0) continue;
        const unsigned long long st = __ldcg(d.status);
        if (st != 0ull && (unsigned long long)k > (st >> 2)) continue;
        batch_fim_tile<T>(sm, d, t - d.tile_begin, k);
    }
    batch_finish_launch(bctl, 1);
}

}  // namespace ripple
