// Batched and served execution of many independent 2D problems (Euler and
// eikonal) on one GPU: admission by device-memory budget, resident state,
// continuous batching of every resident problem, and completion tickets with
// timestamps.  The paper has no counterpart (its scheduler runs one graph;
// this runtime replaces a request loop).
//
// A scheduler thread per context owns two streams: the compute stream runs
// rounds of up to K Euler steps of the resident set, either one launch of the
// batched step kernel (batch_kernels.cuh) per global step (optionally replayed
// from a CUDA graph) or one dependency-driven launch for the whole round
// (async_queue), each followed by the eikonal FIM iterations; the copy stream
// runs admissions (host -> device copy, layout scatter, padding fill / FIM
// initialisation) and completions (device -> host gather and copy).  Device
// memory comes from the runtime's own stream-ordered pool (on the copy stream),
// counted against the context budget: a request waits while its memory does
// not fit, so problems join and leave the resident set while others keep
// running.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <unordered_map>

#include "batch_kernels.cuh"
#include "euler_solo2d.cuh"
#include "grid_sync.cuh"
#include "runtime.h"

namespace ripple {

template <typename T>
cudaError_t launch_fim_init(const FimProblem<T>& a, int ts, int grid, cudaStream_t s);

// ---------------------------------------------------------------------------
// Kernel table (tile shapes are the autotuner's candidates).
// ---------------------------------------------------------------------------
struct BatchTileShape {
    int tx, ty;
};
constexpr int kNumBatchVariants = 3;
constexpr BatchTileShape kBatchVariants[kNumBatchVariants] = {{32, 8}, {8, 32}, {16, 16}};

// Halo staging of the batched Euler step (an autotuner dimension).
constexpr int kBatchStagingTma = 0;     // producer warp + TMA ring (batch_euler_kernel)
constexpr int kBatchStagingDirect = 1;  // every thread loads from global memory (batch_euler_direct_kernel)
constexpr int kBatchStagingWalk = 2;    // warps walk rows of units, no tile staging (batch_euler_walk_kernel)
constexpr int kNumBatchStagings = 3;

template <typename T, int LAYOUT, int V>
static cudaError_t step_v(int staging, int grid, cudaStream_t s, const BatchEuler* e, const void* f,
                          const int* table, BatchCtl* c, int kind, BatchAsync* q)
{
    constexpr int TX = kBatchVariants[V].tx, TY = kBatchVariants[V].ty;
    using BC = BatchEulerCfg<T, LAYOUT, TX, TY>;
    if (kind != 0)
        batch_fim_kernel<T><<<grid, EikTile<2>::NT, 0, s>>>(static_cast<const BatchFim<T>*>(f), table, c);
    else if (q && staging == kBatchStagingWalk)  // a dependency-driven round over walk units
        batch_euler_walk_async_kernel<T><<<grid, kBatchWalkThreads, 0, s>>>(e, table, c, q);
    else if (q)  // a dependency-driven round over tiles (TMA staging)
        batch_euler_kernel<T, LAYOUT, TX, TY, true><<<grid, BC::NTHREADS, BC::SMEM, s>>>(e, table, c, q);
    else if (staging == kBatchStagingDirect)
        batch_euler_direct_kernel<T, LAYOUT, TX, TY><<<grid, 256, 0, s>>>(e, table, c);
    else if (staging == kBatchStagingWalk)
        batch_euler_walk_kernel<T><<<grid, kBatchWalkThreads, 0, s>>>(e, table, c);
    else
        batch_euler_kernel<T, LAYOUT, TX, TY><<<grid, BC::NTHREADS, BC::SMEM, s>>>(e, table, c);
    return cudaGetLastError();
}
// CTAs per SM of the Euler step kernel of a staging (which also sets the TMA
// kernel's dynamic shared memory limit: called before any launch of it).
template <typename T, int LAYOUT, int V>
static int occ_v(int staging)
{
    constexpr int TX = kBatchVariants[V].tx, TY = kBatchVariants[V].ty;
    int n = 0;
    if (staging == kBatchStagingDirect) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_euler_direct_kernel<T, LAYOUT, TX, TY>, 256, 0);
        return n;
    }
    if (staging == kBatchStagingWalk) {
        // the per-step and the dependency-driven walk kernels share the grid
        int na = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_euler_walk_kernel<T>, kBatchWalkThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&na, batch_euler_walk_async_kernel<T>, kBatchWalkThreads, 0);
        return std::min(n, na);
    }
    using BC = BatchEulerCfg<T, LAYOUT, TX, TY>;
    auto k = batch_euler_kernel<T, LAYOUT, TX, TY, false>;
    auto ka = batch_euler_kernel<T, LAYOUT, TX, TY, true>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, BC::SMEM) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, BC::SMEM) != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, BC::NTHREADS, BC::SMEM);
    return n;
}
template <typename T, int LAYOUT>
static cudaError_t step_l(int v, int staging, int grid, cudaStream_t s, const BatchEuler* e, const void* f,
                          const int* t, BatchCtl* c, int kind, BatchAsync* q)
{
    if (v == 1) return step_v<T, LAYOUT, 1>(staging, grid, s, e, f, t, c, kind, q);
    if (v == 2) return step_v<T, LAYOUT, 2>(staging, grid, s, e, f, t, c, kind, q);
    return step_v<T, LAYOUT, 0>(staging, grid, s, e, f, t, c, kind, q);
}
// One launch: a global step of every Euler (kind 0) or eikonal (kind 1)
// instance, or with q (Euler only) a whole dependency-driven round.
static cudaError_t launch_batch_step(ripple_dtype dt, int layout, int v, int staging, int grid, cudaStream_t s,
                                     const BatchEuler* e, const void* f, const int* t, BatchCtl* c, int kind,
                                     BatchAsync* q = nullptr)
{
    if (dt == RIPPLE_F32)
        return layout == LAYOUT_SOA ? step_l<float, LAYOUT_SOA>(v, staging, grid, s, e, f, t, c, kind, q)
                                    : step_l<float, LAYOUT_AOS>(v, staging, grid, s, e, f, t, c, kind, q);
    return layout == LAYOUT_SOA ? step_l<double, LAYOUT_SOA>(v, staging, grid, s, e, f, t, c, kind, q)
                                : step_l<double, LAYOUT_AOS>(v, staging, grid, s, e, f, t, c, kind, q);
}
// CTAs per SM of the batched FIM iteration kernel.
static int fim_occupancy(ripple_dtype dt)
{
    int n = 0;
    if (dt == RIPPLE_F32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_fim_kernel<float>, EikTile<2>::NT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_fim_kernel<double>, EikTile<2>::NT, 0);
    return std::max(1, n);
}

static int batch_occupancy(ripple_dtype dt, int layout, int v, int staging)
{
    auto pick = [&](auto tag) -> int {
        using T = decltype(tag);
        if (layout == LAYOUT_SOA)
            return v == 1 ? occ_v<T, LAYOUT_SOA, 1>(staging) : v == 2 ? occ_v<T, LAYOUT_SOA, 2>(staging)
                                                                     : occ_v<T, LAYOUT_SOA, 0>(staging);
        return v == 1 ? occ_v<T, LAYOUT_AOS, 1>(staging) : v == 2 ? occ_v<T, LAYOUT_AOS, 2>(staging)
                                                                 : occ_v<T, LAYOUT_AOS, 0>(staging);
    };
    return dt == RIPPLE_F32 ? pick(0.0f) : pick(0.0);
}

// TMA maps of both buffers of an Euler instance, staged in boxes of tile variant v.
static ripple_status encode_batch_maps(BatchEuler& e, ripple_layout layout, ripple_dtype dt, int v)
{
    for (int b = 0; b < 2; ++b) {
        ripple_status st = encode_plane_map(e.buf[b], e.g, layout, dt, 0, 1, kBatchVariants[v].tx,
                                            kBatchVariants[v].ty, &e.map[b]);
        if (st != RIPPLE_OK) return st;
    }
    return RIPPLE_OK;
}

// Fill a uniform admissible Euler state (autotuner sample problems).
template <typename T>
__global__ void fill_uniform_euler(T* buf, const FieldGeom g)
{
    const long long total = (long long)g.px * g.py;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        const T q[4] = {T(1), T(0.5), T(0.25), T(2.65625)};
        for (int m = 0; m < 4; ++m) buf[c * g.cell_stride + m * g.comp_stride] = q[m];
    }
}

// ---------------------------------------------------------------------------
// Runtime state
// ---------------------------------------------------------------------------
using Clock = std::chrono::steady_clock;

constexpr int kSlots = 4096;  // concurrent problems (admitted, resident or completing)
constexpr int kMaxRoundSteps = 4096;  // steps of one dependency-driven round

// A page-locked host arena for request data.  The submitting thread copies a
// pageable request's input into it and the thread that retrieves the ticket
// copies the result out of it, so the scheduler thread's copies to and from
// the device are asynchronous (a copy from or to pageable memory holds the
// calling thread until it is done, and the scheduler thread is the one that
// keeps the GPU busy).  First fit over free blocks, coalesced on release.
struct PinnedArena {
    std::mutex mu;
    char* base = nullptr;
    size_t size = 0;
    bool tried = false;
    std::map<size_t, size_t> free_blocks;  // offset -> bytes

    char* alloc(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        std::lock_guard<std::mutex> lk(mu);
        if (!tried) {
            tried = true;
            if (cudaMallocHost(reinterpret_cast<void**>(&base), kArenaBytes) == cudaSuccess) {
                size = kArenaBytes;
                free_blocks[0] = size;
            } else {
                base = nullptr;
                cudaGetLastError();
            }
        }
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rest = it->second - bytes;
            free_blocks.erase(it);
            if (rest) free_blocks[off + bytes] = rest;
            return base + off;
        }
        return nullptr;
    }
    void release(char* p, size_t bytes)
    {
        if (!p) return;
        bytes = (bytes + 255) / 256 * 256;
        std::lock_guard<std::mutex> lk(mu);
        size_t off = (size_t)(p - base);
        auto next = free_blocks.lower_bound(off);
        if (next != free_blocks.end() && next->first == off + bytes) {
            bytes += next->second;
            free_blocks.erase(next);
        }
        auto it = free_blocks.lower_bound(off);
        if (it != free_blocks.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_blocks[off] = bytes;
    }
    void destroy()
    {
        if (base) cudaFreeHost(base);
        base = nullptr;
        size = 0;
        free_blocks.clear();
    }
    static constexpr size_t kArenaBytes = size_t(512) << 20;
};

struct Inst {
    uint64_t ticket = 0;
    ripple_request req{};
    std::vector<int64_t> src;
    FieldGeom g{}, gs{};
    size_t buf_bytes = 0, sbuf_bytes = 0, scratch_bytes = 0, total_bytes = 0;
    void* buf[2] = {nullptr, nullptr};
    void* sbuf = nullptr;
    void* scratch = nullptr;
    int slot = -1;
    int ntiles = 0, tiles_x = 0, ntx = 0, nty = 0;
    long long start_step = -1;  // Euler: launch index of local step 0 (recomputed on resume)
    long long steps_done = 0;   // Euler steps completed
    bool active = false;        // Euler: stepped in the current rounds
    bool stepped = false;       // taken part in a compute round
    CUtensorMap map[2];         // Euler: TMA maps of buf[0], buf[1] (cached per tile variant and layout)
    int map_key = -1;
    struct GroupEv* gev = nullptr;  // completion of the instance's admission or download group
    char* h_in = nullptr;           // page-locked copy of the input (arena), or null: copied from req.input
    char* h_out = nullptr;          // page-locked stage of the result (arena), or null: copied to req.output
    size_t dense = 0;               // bytes of the input and of the result
    ripple_status result = RIPPLE_OK;
    double t_submit = 0, t_admit = 0, t_start = 0, t_finish = 0;
};

// An event shared by the instances of one admission or download group,
// returned to the runtime's pool when the last of them has seen it.
struct GroupEv {
    cudaEvent_t ev = nullptr;
    int refs = 0;
};

struct Ticket {
    bool done = false;
    ripple_ticket_info info{};
    char* stage = nullptr;  // result in the arena, copied to `out` by the thread that retrieves the ticket
    void* out = nullptr;
    size_t bytes = 0;
};

struct BatchRuntime {
    ripple_ctx ctx = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<Inst*> pending;                      // guarded by mu
    std::unordered_map<uint64_t, Ticket> tickets;   // guarded by mu
    uint64_t next_ticket = 1;                       // guarded by mu
    ripple_batch_config cfg{RIPPLE_SOA, 0, 16, 1, RIPPLE_F32, 4, 0, 0, 0, 4};
    ripple_batch_stats stats{};                     // guarded by mu
    Clock::time_point epoch = Clock::now();
    // scheduler-thread state
    std::vector<Inst*> uploading, resident, downloading;
    cudaStream_t compute = nullptr, copy = nullptr;
    // the runtime's own stream-ordered pool: freed instance memory stays mapped
    // for the next admission (no release to the driver at each synchronisation)
    cudaMemPool_t pool = nullptr;
    cudaEvent_t ev_step = nullptr;
    cudaEvent_t ev_r0 = nullptr, ev_r1 = nullptr;  // timing of a compute round (device_s)
    std::vector<cudaEvent_t> ev_pool;  // events of finished groups, for reuse
    // descriptors of the current admission or download group: pinned host
    // array, its device copy (both kSlots long) and the event after the copy
    unsigned* d_solo_bar = nullptr;  // arrival counter of the multi-step solo launches' grid barrier
    int solo_occ[2] = {0, 0};        // resident CTAs per SM of the solo kernel (FP32, FP64)
    PinnedArena arena;  // request data staged in page-locked memory
    GroupItem* h_items = nullptr;
    GroupItem* d_items = nullptr;
    cudaEvent_t ev_items = nullptr;
    bool started = false;
    // slot arrays: device, and pinned mirrors of status/counters/ctl
    FieldCtl* slot_ctl = nullptr;
    unsigned long long* slot_status = nullptr;
    long long* slot_counters = nullptr;
    FieldCtl* h_ctl = nullptr;
    unsigned long long* h_status = nullptr;
    // written only by the downloads (copy stream): the slot entries of
    // finished instances, read when their group's event has completed
    FieldCtl* out_ctl = nullptr;
    unsigned long long* out_status = nullptr;
    long long* h_counters = nullptr;
    std::vector<int> free_slots;
    // tables
    BatchEuler* d_euler = nullptr;
    void* d_fim = nullptr;
    int* d_table = nullptr;
    BatchCtl* d_bctl = nullptr;
    unsigned* h_berr = nullptr;  // pinned mirror of d_bctl->err
    BatchEuler* h_euler = nullptr;
    void* h_fim = nullptr;
    int* h_table = nullptr;
    int cap_e = 0, cap_f = 0, cap_t = 0;
    // dependency-driven rounds: control block, per-step task offsets, per-instance completions
    BatchAsync* d_async = nullptr;
    int* d_cum = nullptr;      // [kMaxRoundSteps + 1]
    unsigned* d_done = nullptr;
    int cap_done = 0;
    BatchAsync* h_async = nullptr;  // pinned staging of the control block
    int* h_cum = nullptr;           // pinned, [kMaxRoundSteps + 1]
    std::vector<Inst*> euler_order;  // Euler instances in table order (set by rebuild_tables)
    bool dirty = true;
    bool small_only = false;  // batched rounds over the small Euler problems only (solo_round decides)
    bool has_e = false, has_f = false;  // resident kinds (set by rebuild_tables)
    long long gstep_e = 0;  // Euler steps issued (== device counter once they completed)
    long long gstep_f = 0;  // FIM iterations issued
    int grid = 0;        // grid of the per-step launches (occupancy of the configured staging x SMs)
    int grid_async = 0;  // grid of a dependency-driven round (TMA staging)
    int grid_fim = 0;    // grid of the FIM iteration launches (one wave of the FIM kernel)
    std::map<int, cudaGraphExec_t> graphs;  // key: (steps << 2) | has_euler << 1 | has_fim
    int graph_variant = -1, graph_layout = -1, graph_fim = -1, graph_staging = -1, graph_dtype = -1;

    double now() const { return std::chrono::duration<double>(Clock::now() - epoch).count(); }
};

static size_t fim_elem_size(ripple_dtype d) { return d == RIPPLE_F64 ? sizeof(BatchFim<double>) : sizeof(BatchFim<float>); }

static ripple_status rt_alloc(BatchRuntime* rt, size_t bytes, void** p)
{
    *p = nullptr;
    if (fault_injected("alloc")) return fail(RIPPLE_ERR_OOM, "device allocation failed (injected: RIPPLE_FAULT=alloc)");
    bytes = (bytes + 255) / 256 * 256;
    if (!budget_reserve(rt->ctx, bytes)) return RIPPLE_ERR_BUDGET;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, rt->pool, rt->copy);
    if (e != cudaSuccess) {
        rt->ctx->used -= bytes;
        *p = nullptr;
        return cuda_fail(e, "cudaMallocFromPoolAsync");
    }
    return RIPPLE_OK;
}

static void rt_free(BatchRuntime* rt, void* p, size_t bytes)
{
    if (!p) return;
    bytes = (bytes + 255) / 256 * 256;
    cudaFreeAsync(p, rt->copy);
    rt->ctx->used -= bytes;
}

static ripple_status rt_start(BatchRuntime* rt);

// Complete an instance's ticket (rt->mu held).
static void fill_ticket(BatchRuntime* rt, Inst* in, ripple_status st, double t)
{
    in->result = st;
    in->t_finish = t;
    Ticket& tk = rt->tickets[in->ticket];
    tk.done = true;
    tk.info.status = st;
    tk.info.submit_s = in->t_submit;
    tk.info.admit_s = in->t_admit;
    tk.info.start_s = in->t_start;
    tk.info.finish_s = in->t_finish;
    if (in->slot >= 0) {
        if (in->req.kind == RIPPLE_REQ_EULER) {
            tk.info.work = in->req.nsteps;
            tk.info.t = rt->out_ctl[in->slot].t;
        } else {
            tk.info.work = rt->h_counters[in->slot * 3 + 0];
            tk.info.tile_visits = rt->h_counters[in->slot * 3 + 1];
            tk.info.cell_updates = rt->h_counters[in->slot * 3 + 2];
        }
    }
    if (st == RIPPLE_OK) rt->stats.completed++;
    else rt->stats.failed++;
}

static void add_host_time(BatchRuntime* rt, double ripple_batch_stats::*field, double t0)
{
    const double dt = rt->now() - t0;
    std::lock_guard<std::mutex> lk(rt->mu);
    rt->stats.*field += dt;
}

static void finish(BatchRuntime* rt, Inst* in, ripple_status st)
{
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        fill_ticket(rt, in, st, rt->now());
    }
    rt->cv_done.notify_all();
}

// A pooled event for a group of n instances.
static ripple_status group_event(BatchRuntime* rt, int n, GroupEv** out)
{
    *out = nullptr;
    cudaEvent_t ev = nullptr;
    if (!rt->ev_pool.empty()) {
        ev = rt->ev_pool.back();
        rt->ev_pool.pop_back();
    } else {
        RIPPLE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    *out = new GroupEv{ev, n};
    return RIPPLE_OK;
}

// The instance no longer waits on its group's event.
static void drop_event(BatchRuntime* rt, Inst* in)
{
    GroupEv* g = in->gev;
    in->gev = nullptr;
    if (g && --g->refs == 0) {
        rt->ev_pool.push_back(g->ev);
        delete g;
    }
}

static bool group_done(const Inst* in) { return !in->gev || cudaEventQuery(in->gev->ev) == cudaSuccess; }
static void wait_group(const Inst* in)
{
    if (in->gev) cudaEventSynchronize(in->gev->ev);
}

// Free everything an instance holds (stream-ordered after its last use).
static void release(BatchRuntime* rt, Inst* in)
{
    rt_free(rt, in->buf[0], in->buf_bytes);
    rt_free(rt, in->buf[1], in->buf_bytes);
    rt_free(rt, in->sbuf, in->sbuf_bytes);
    rt_free(rt, in->scratch, in->scratch_bytes);
    in->buf[0] = in->buf[1] = in->sbuf = in->scratch = nullptr;
    if (in->slot >= 0) rt->free_slots.push_back(in->slot);
    drop_event(rt, in);
    rt->arena.release(in->h_in, in->dense);
    rt->arena.release(in->h_out, in->dense);
    in->h_in = in->h_out = nullptr;
}

template <typename T>
static FimProblem<T> fim_problem(const Inst* in)
{
    FimProblem<T> a{};
    a.buf[0] = static_cast<T*>(in->buf[0]);
    a.buf[1] = static_cast<T*>(in->buf[1]);
    a.slow = static_cast<const T*>(in->sbuf);
    a.gT = in->g;
    a.gS = in->gs;
    a.ntx = in->ntx;
    a.nty = in->nty;
    a.ntz = 1;
    a.ntiles = in->ntiles;
    a.nsrc = (int)(in->src.size() / 2);
    for (int q = 0; q < a.nsrc; ++q) {
        a.src[q][0] = (int)in->src[2 * q];
        a.src[q][1] = (int)in->src[2 * q + 1];
        a.src[q][2] = 0;
    }
    a.h = in->req.eik.h;
    a.tol = in->req.eik.tol;
    char* base = static_cast<char*>(in->scratch);
    a.count = reinterpret_cast<unsigned*>(base);
    a.act = reinterpret_cast<unsigned*>(base + 64);
    a.cur = reinterpret_cast<unsigned char*>(base + 64 + (size_t)in->ntiles * 12);
    return a;
}

// Allocate and queue the upload of one request.  RIPPLE_ERR_BUDGET: does not fit now.
static ripple_status admit(BatchRuntime* rt, Inst* in)
{
    const ripple_request& r = in->req;
    const ripple_dtype dt = rt->cfg.dtype;
    const size_t es = elem_size(dt);
    const int64_t dims[2] = {r.dims[0], r.dims[1]};
    const size_t dense = (size_t)dims[0] * dims[1] * es * (r.kind == RIPPLE_REQ_EULER ? 4 : 1);
    if (r.kind == RIPPLE_REQ_EULER) {
        in->g = make_field_geom(2, dims, 4, rt->cfg.layout, 1, dt, &in->buf_bytes);
        in->tiles_x = (int)((dims[0] + kBatchVariants[rt->cfg.tile_variant].tx - 1) /
                            kBatchVariants[rt->cfg.tile_variant].tx);
        const int ty = (int)((dims[1] + kBatchVariants[rt->cfg.tile_variant].ty - 1) /
                             kBatchVariants[rt->cfg.tile_variant].ty);
        in->ntiles = in->tiles_x * ty;
        in->total_bytes = 2 * ((in->buf_bytes + 255) / 256 * 256);
    } else {
        in->g = make_field_geom(2, dims, 1, RIPPLE_SOA, 0, dt, &in->buf_bytes);
        in->gs = make_field_geom(2, dims, 1, RIPPLE_SOA, 0, dt, &in->sbuf_bytes);
        constexpr int TS = EikTile<2>::TS;
        in->ntx = (int)((dims[0] + TS - 1) / TS);
        in->nty = (int)((dims[1] + TS - 1) / TS);
        in->ntiles = in->ntx * in->nty;
        // per-tile flags of the batched iterations, or the lists of a solo solve
        in->scratch_bytes = std::max<size_t>(64 + (size_t)in->ntiles * 14, fim_list_scratch_bytes(in->ntiles));
        in->total_bytes = 2 * ((in->buf_bytes + 255) / 256 * 256) + (in->sbuf_bytes + 255) / 256 * 256 +
                          (in->scratch_bytes + 255) / 256 * 256;
    }
    if (dense > in->buf_bytes) return fail(RIPPLE_ERR_INTERNAL, "staging buffer too small");
    if (in->dense != dense) {  // the precision changed after submission: copy directly
        rt->arena.release(in->h_in, in->dense);
        rt->arena.release(in->h_out, in->dense);
        in->h_in = in->h_out = nullptr;
        in->dense = dense;
    }
    if (fault_injected("admit")) return fail(RIPPLE_ERR_OOM, "admission failed (injected: RIPPLE_FAULT=admit)");
    if (rt->free_slots.empty()) return RIPPLE_ERR_BUDGET;
    if (rt->ctx->budget && in->total_bytes > rt->ctx->budget)
        return fail(RIPPLE_ERR_BUDGET, "request larger than the whole memory budget");
    ripple_status st = rt_alloc(rt, in->buf_bytes, &in->buf[0]);
    if (st == RIPPLE_OK) st = rt_alloc(rt, in->buf_bytes, &in->buf[1]);
    if (st == RIPPLE_OK && r.kind == RIPPLE_REQ_EIKONAL) {
        st = rt_alloc(rt, in->sbuf_bytes, &in->sbuf);
        if (st == RIPPLE_OK) st = rt_alloc(rt, in->scratch_bytes, &in->scratch);
    }
    if (st != RIPPLE_OK) {
        rt_free(rt, in->buf[0], in->buf_bytes);
        rt_free(rt, in->buf[1], in->buf_bytes);
        rt_free(rt, in->sbuf, in->sbuf_bytes);
        rt_free(rt, in->scratch, in->scratch_bytes);
        in->buf[0] = in->buf[1] = in->sbuf = in->scratch = nullptr;
        return st;
    }
    in->slot = rt->free_slots.back();
    rt->free_slots.pop_back();
    if (fault_injected("upload")) return fail(RIPPLE_ERR_CUDA, "input upload failed (injected: RIPPLE_FAULT=upload)");
    cudaStream_t s = rt->copy;
    // the second buffer is the dense staging area of the upload
    RIPPLE_CUDA(cudaMemcpyAsync(in->buf[1], in->h_in ? static_cast<const void*>(in->h_in) : r.input, dense,
                                cudaMemcpyHostToDevice, s));
    if (r.kind == RIPPLE_REQ_EULER) {
        // TMA maps of the batched step, encoded while the copies run (the tile
        // shape and layout cannot change while a request is in flight)
        BatchEuler e{};
        e.buf[0] = in->buf[0];
        e.buf[1] = in->buf[1];
        e.g = in->g;
        ripple_status st = encode_batch_maps(e, rt->cfg.layout, dt, rt->cfg.tile_variant);
        if (st != RIPPLE_OK) return st;
        std::memcpy(in->map, e.map, sizeof(in->map));
        in->map_key = rt->cfg.tile_variant * 2 + (rt->cfg.layout == RIPPLE_SOA ? 1 : 0);
    } else {
        const long long total = dims[0] * dims[1];
        const int grid = (int)std::min<long long>((total + 255) / 256, 4LL * rt->ctx->sm_count);
        RIPPLE_CUDA(launch_interior_copy(dt, in->sbuf, in->gs, in->buf[1], LAYOUT_SOA, 0, grid, s));
        RIPPLE_CUDA(cudaMemsetAsync(in->scratch, 0, in->scratch_bytes, s));
        if (dt == RIPPLE_F32) RIPPLE_CUDA(launch_fim_init<float>(fim_problem<float>(in), EikTile<2>::TS, grid, s));
        else RIPPLE_CUDA(launch_fim_init<double>(fim_problem<double>(in), EikTile<2>::TS, grid, s));
    }
    return RIPPLE_OK;
}

// Make the descriptors of a group in the pinned array (after the previous
// group's copy of it has completed) and copy them to the device.
static ripple_status put_items(BatchRuntime* rt, int n, cudaStream_t s)
{
    RIPPLE_CUDA(cudaMemcpyAsync(rt->d_items, rt->h_items, (size_t)n * sizeof(GroupItem), cudaMemcpyHostToDevice, s));
    RIPPLE_CUDA(cudaEventRecord(rt->ev_items, s));
    return RIPPLE_OK;
}

// Device-side preparation of every instance admitted in one scheduler pass,
// after their input copies: two launches over the whole group (Euler: buffer 0
// filled from the dense input with NaN padding, the slot cleared; then the
// boundary images, the first wave-speed maximum, the input check and buffer
// 1's NaN padding; eikonal: the slot cleared), then one event for the group.
static ripple_status admit_group(BatchRuntime* rt, const std::vector<Inst*>& group)
{
    const int n = (int)group.size();
    if (n == 0) return RIPPLE_OK;
    cudaStream_t s = rt->copy;
    RIPPLE_CUDA(cudaEventSynchronize(rt->ev_items));
    long long b0 = 0, b1 = 0;
    for (int i = 0; i < n; ++i) {
        const Inst* in = group[i];
        GroupItem& d = rt->h_items[i];
        d = GroupItem{};
        d.buf = in->buf[0];
        d.other = in->buf[1];
        d.ctl = &rt->slot_ctl[in->slot];
        d.status = &rt->slot_status[in->slot];
        d.counters = &rt->slot_counters[in->slot * 3];
        d.g = in->g;
        d.euler = in->req.kind == RIPPLE_REQ_EULER ? 1 : 0;
        d.gamma = in->req.fv.gamma;
        d.inv_dx0 = d.euler ? 1.0 / in->req.fv.dx[0] : 0.0;
        d.inv_dx1 = d.euler ? 1.0 / in->req.fv.dx[1] : 0.0;
        d.bc = (int)in->req.fv.bc;
        d.blk[0] = b0;
        d.blk[1] = b1;
        const long long nb =
            d.euler ? (in->g.px * in->g.py * in->g.pz + kGroupCellsPerBlock - 1) / kGroupCellsPerBlock : 1;
        b0 += nb;
        if (d.euler) b1 += nb;
    }
    ripple_status st = put_items(rt, n, s);
    if (st != RIPPLE_OK) return st;
    RIPPLE_CUDA(launch_group(rt->cfg.dtype, GROUP_ADMIT_FILL, rt->d_items, n, b0, s));
    RIPPLE_CUDA(launch_group(rt->cfg.dtype, GROUP_ADMIT_PREP, rt->d_items, n, b1, s));
    GroupEv* ge = nullptr;
    st = group_event(rt, n, &ge);
    if (st != RIPPLE_OK) return st;
    const double t = rt->now();
    for (Inst* in : group) {
        in->gev = ge;
        in->t_admit = t;
    }
    RIPPLE_CUDA(cudaEventRecord(ge->ev, s));
    return RIPPLE_OK;
}

// Queue the downloads of a group of finished instances (after the compute
// work recorded in ev_step): one launch gathers every result into its dense
// stage, then one copy per result into the caller's array and one copy per
// slot array of the group's slot range into the pinned mirrors.
static ripple_status start_downloads(BatchRuntime* rt, const std::vector<Inst*>& group)
{
    const int n = (int)group.size();
    if (n == 0) return RIPPLE_OK;
    const ripple_dtype dt = rt->cfg.dtype;
    cudaStream_t s = rt->copy;
    RIPPLE_CUDA(cudaStreamWaitEvent(s, rt->ev_step, 0));
    RIPPLE_CUDA(cudaEventSynchronize(rt->ev_items));
    long long b0 = 0;
    int lo = kSlots, hi = -1;
    for (int i = 0; i < n; ++i) {
        const Inst* in = group[i];
        const bool odd = in->req.kind == RIPPLE_REQ_EULER && (in->req.nsteps & 1);
        GroupItem& d = rt->h_items[i];
        d = GroupItem{};
        d.buf = in->buf[odd ? 1 : 0];
        d.other = in->buf[odd ? 0 : 1];
        d.g = in->g;
        d.euler = in->req.kind == RIPPLE_REQ_EULER ? 1 : 0;
        d.blk[0] = b0;
        b0 += (in->req.dims[0] * in->req.dims[1] + kGroupCellsPerBlock - 1) / kGroupCellsPerBlock;
        lo = std::min(lo, in->slot);
        hi = std::max(hi, in->slot);
    }
    ripple_status st = put_items(rt, n, s);
    if (st != RIPPLE_OK) return st;
    RIPPLE_CUDA(launch_group(dt, GROUP_PACK, rt->d_items, n, b0, s));
    for (int i = 0; i < n; ++i) {
        const Inst* in = group[i];
        const ripple_request& r = in->req;
        const size_t dense = (size_t)(r.dims[0] * r.dims[1]) * elem_size(dt) * (r.kind == RIPPLE_REQ_EULER ? 4 : 1);
        RIPPLE_CUDA(cudaMemcpyAsync(in->h_out ? static_cast<void*>(in->h_out) : r.output, rt->h_items[i].other, dense,
                                    cudaMemcpyDeviceToHost, s));
    }
    const int ns = hi - lo + 1;
    RIPPLE_CUDA(cudaMemcpyAsync(&rt->out_ctl[lo], &rt->slot_ctl[lo], ns * sizeof(FieldCtl), cudaMemcpyDeviceToHost, s));
    RIPPLE_CUDA(cudaMemcpyAsync(&rt->out_status[lo], &rt->slot_status[lo], ns * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, s));
    RIPPLE_CUDA(cudaMemcpyAsync(&rt->h_counters[lo * 3], &rt->slot_counters[lo * 3], ns * 3 * sizeof(long long),
                                cudaMemcpyDeviceToHost, s));
    GroupEv* ge = nullptr;
    st = group_event(rt, n, &ge);
    if (st != RIPPLE_OK) return st;
    for (Inst* in : group) {
        drop_event(rt, in);
        in->gev = ge;
    }
    RIPPLE_CUDA(cudaEventRecord(ge->ev, s));
    return RIPPLE_OK;
}

template <typename T>
static void fill_fim_desc(BatchRuntime* rt, Inst* in, void* h_fim, int idx)
{
    BatchFim<T>* f = static_cast<BatchFim<T>*>(h_fim) + idx;
    f->p = fim_problem<T>(in);
    f->tile_begin = 0;
    f->start_step = in->start_step;
    f->max_iters = in->req.eik.max_iters > 0 ? in->req.eik.max_iters : 1000000;
    f->status = &rt->slot_status[in->slot];
    f->counters = &rt->slot_counters[in->slot * 3];
}

constexpr int kInitDescriptors = 1024;  // Euler and eikonal descriptors allocated at start
constexpr int kInitTiles = 1 << 18;     // tile-table entries allocated at start (1 MB)
constexpr int kInitEvents = 32;         // pooled group events created at start

static ripple_status grow(BatchRuntime* rt, int ne, int nf, int nt)
{
    auto regrow = [&](int need, int& cap, size_t esz, void** d, void** h) -> ripple_status {
        if (need <= cap) return RIPPLE_OK;
        int nc = std::max(need, std::max(64, cap * 2));
        RIPPLE_CUDA(cudaStreamSynchronize(rt->compute));
        if (*d) cudaFree(*d);
        if (*h) cudaFreeHost(*h);
        *d = nullptr;
        *h = nullptr;
        RIPPLE_CUDA(cudaMalloc(d, (size_t)nc * esz));
        RIPPLE_CUDA(cudaMallocHost(h, (size_t)nc * esz));
        cap = nc;
        for (auto& g : rt->graphs) cudaGraphExecDestroy(g.second);
        rt->graphs.clear();
        return RIPPLE_OK;
    };
    ripple_status st = regrow(ne, rt->cap_e, sizeof(BatchEuler), reinterpret_cast<void**>(&rt->d_euler),
                              reinterpret_cast<void**>(&rt->h_euler));
    if (st == RIPPLE_OK) st = regrow(nf, rt->cap_f, fim_elem_size(rt->cfg.dtype), &rt->d_fim, &rt->h_fim);
    if (st == RIPPLE_OK)
        st = regrow(nt, rt->cap_t, sizeof(int), reinterpret_cast<void**>(&rt->d_table),
                    reinterpret_cast<void**>(&rt->h_table));
    return st;
}

// Rebuild the descriptor arrays and the tile table of the resident set.
// Table entries of an instance: its tiles, or with walk staging its walk
// units of kSoloW columns x kBatchWalkRows rows (per-step launches and
// dependency-driven rounds alike).
static bool walk_units(const BatchRuntime* rt) { return rt->cfg.staging == kBatchStagingWalk; }
static int walk_strips(const Inst* in) { return (int)((in->req.dims[0] + kSoloW - 1) / kSoloW); }
static int table_entries(const BatchRuntime* rt, const Inst* in)
{
    if (in->req.kind != RIPPLE_REQ_EULER || !walk_units(rt)) return in->ntiles;
    return walk_strips(in) * (int)((in->req.dims[1] + kBatchWalkRows - 1) / kBatchWalkRows);
}

static ripple_status rebuild_tables(BatchRuntime* rt)
{
    int ne = 0, nf = 0, nt = 0;
    for (Inst* in : rt->resident) {
        if (in->req.kind == RIPPLE_REQ_EULER && !in->active) continue;
        if (in->req.kind != RIPPLE_REQ_EULER && rt->small_only) continue;
        if (in->req.kind == RIPPLE_REQ_EULER) ++ne;
        else ++nf;
        nt += table_entries(rt, in);
    }
    ripple_status st = grow(rt, std::max(ne, 1), std::max(nf, 1), std::max(nt, 1));
    if (st != RIPPLE_OK) return st;
    // the previous launches may still read the pinned mirrors' device copies:
    // the compute stream is idle here (the scheduler synchronises every K steps)
    int ie = 0, jf = 0, t = 0;
    // Euler tiles first, then eikonal tiles (each kind has its own launches)
    std::vector<Inst*> order;
    for (Inst* in : rt->resident)
        if (in->req.kind == RIPPLE_REQ_EULER && in->active) order.push_back(in);
    if (rt->cfg.async_queue) {
        // dependency-driven rounds: most remaining steps first, so the instances
        // still stepping at any step of a round are a prefix of the table (every
        // instance that continues advances by the same K steps: the order holds
        // until the resident set changes)
        std::stable_sort(order.begin(), order.end(), [](const Inst* a, const Inst* b) {
            return a->req.nsteps - a->steps_done > b->req.nsteps - b->steps_done;
        });
    }
    rt->euler_order = order;
    for (Inst* in : rt->resident)
        if (in->req.kind != RIPPLE_REQ_EULER && !rt->small_only) order.push_back(in);
    int nt_e = 0;
    for (Inst* in : order) {
        if (in->req.kind == RIPPLE_REQ_EULER) {
            nt_e += table_entries(rt, in);
            BatchEuler& e = rt->h_euler[ie];
            e.buf[0] = in->buf[0];
            e.buf[1] = in->buf[1];
            e.ctl = &rt->slot_ctl[in->slot];
            e.g = in->g;
            e.tiles_x = walk_units(rt) ? walk_strips(in) : in->tiles_x;
            e.tile_begin = t;
            e.ntiles = table_entries(rt, in);
            e.bc = (int)in->req.fv.bc;
            e.start_step = in->start_step;
            e.nsteps = in->req.nsteps;
            e.gamma = in->req.fv.gamma;
            e.gm1 = in->req.fv.gamma - 1.0;
            e.cfl = in->req.fv.cfl;
            e.inv_dx0 = 1.0 / in->req.fv.dx[0];
            e.inv_dx1 = 1.0 / in->req.fv.dx[1];
            e.gamma_f = (float)e.gamma;
            e.gm1_f = (float)e.gm1;
            e.inv_dx0_f = (float)e.inv_dx0;
            e.inv_dx1_f = (float)e.inv_dx1;
            const int key = rt->cfg.tile_variant * 2 + (rt->cfg.layout == RIPPLE_SOA ? 1 : 0);
            if (in->map_key != key) {
                st = encode_batch_maps(e, rt->cfg.layout, rt->cfg.dtype, rt->cfg.tile_variant);
                if (st != RIPPLE_OK) return st;
                std::memcpy(in->map, e.map, sizeof(in->map));
                in->map_key = key;
            } else {
                std::memcpy(e.map, in->map, sizeof(e.map));
            }
            for (int k = 0; k < e.ntiles; ++k) rt->h_table[t + k] = (ie << 1) | 0;
            ++ie;
        } else {
            if (rt->cfg.dtype == RIPPLE_F32) fill_fim_desc<float>(rt, in, rt->h_fim, jf);
            else fill_fim_desc<double>(rt, in, rt->h_fim, jf);
            if (rt->cfg.dtype == RIPPLE_F32) static_cast<BatchFim<float>*>(rt->h_fim)[jf].tile_begin = t;
            else static_cast<BatchFim<double>*>(rt->h_fim)[jf].tile_begin = t;
            for (int k = 0; k < in->ntiles; ++k) rt->h_table[t + k] = (jf << 1) | 1;
            ++jf;
        }
        t += table_entries(rt, in);
    }
    cudaStream_t s = rt->compute;
    if (ne) RIPPLE_CUDA(cudaMemcpyAsync(rt->d_euler, rt->h_euler, ne * sizeof(BatchEuler), cudaMemcpyHostToDevice, s));
    if (nf)
        RIPPLE_CUDA(cudaMemcpyAsync(rt->d_fim, rt->h_fim, nf * fim_elem_size(rt->cfg.dtype), cudaMemcpyHostToDevice, s));
    if (nt) RIPPLE_CUDA(cudaMemcpyAsync(rt->d_table, rt->h_table, nt * sizeof(int), cudaMemcpyHostToDevice, s));
    const int counts[2] = {nt_e, nt};
    RIPPLE_CUDA(cudaMemcpyAsync(&rt->d_bctl->ntiles_e, counts, sizeof(counts), cudaMemcpyHostToDevice, s));
    RIPPLE_CUDA(cudaStreamSynchronize(s));  // counts live on this stack frame
    rt->has_e = ne > 0;
    rt->has_f = nf > 0;
    rt->dirty = false;
    return RIPPLE_OK;
}

// Queue K units of work on the compute stream; a unit is one Euler step of
// every resident Euler problem followed by F FIM iterations of every resident
// eikonal problem (F = fim_iters_per_step), either kind omitted when absent.
static ripple_status launch_steps(BatchRuntime* rt, int K)
{
    const int layout = rt->cfg.layout == RIPPLE_SOA ? LAYOUT_SOA : LAYOUT_AOS;
    const int F = std::max(1, rt->cfg.fim_iters_per_step);
    auto unit = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (rt->has_e)
            e = launch_batch_step(rt->cfg.dtype, layout, rt->cfg.tile_variant, rt->cfg.staging, rt->grid,
                                  rt->compute, rt->d_euler,
                                  rt->d_fim, rt->d_table, rt->d_bctl, 0);
        for (int f = 0; f < F && rt->has_f && e == cudaSuccess; ++f)
            e = launch_batch_step(rt->cfg.dtype, layout, rt->cfg.tile_variant, rt->cfg.staging, rt->grid_fim,
                                  rt->compute, rt->d_euler,
                                  rt->d_fim, rt->d_table, rt->d_bctl, 1);
        return e;
    };
    const int per_unit = (rt->has_e ? 1 : 0) + (rt->has_f ? F : 0);
    if (!rt->cfg.use_graphs) {
        for (int k = 0; k < K; ++k) RIPPLE_CUDA(unit());
        std::lock_guard<std::mutex> lk(rt->mu);
        rt->stats.launches += (int64_t)K * per_unit;
        return RIPPLE_OK;
    }
    if (rt->graph_variant != rt->cfg.tile_variant || rt->graph_layout != layout || rt->graph_fim != F ||
        rt->graph_staging != rt->cfg.staging || rt->graph_dtype != (int)rt->cfg.dtype) {
        for (auto& g : rt->graphs) cudaGraphExecDestroy(g.second);
        rt->graphs.clear();
        rt->graph_variant = rt->cfg.tile_variant;
        rt->graph_layout = layout;
        rt->graph_staging = rt->cfg.staging;
        rt->graph_dtype = (int)rt->cfg.dtype;
        rt->graph_fim = F;
    }
    // K as a sum of powers of two, each replayed from a captured graph
    for (int bit = 30; bit >= 0; --bit) {
        const int n = 1 << bit;
        if (!(K & n)) continue;
        const int key = (n << 2) | (rt->has_e ? 2 : 0) | (rt->has_f ? 1 : 0);
        auto it = rt->graphs.find(key);
        if (it == rt->graphs.end()) {
            cudaGraph_t g = nullptr;
            RIPPLE_CUDA(cudaStreamBeginCapture(rt->compute, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < n && e == cudaSuccess; ++k) e = unit();
            cudaError_t e2 = cudaStreamEndCapture(rt->compute, &g);
            if (e != cudaSuccess) return cuda_fail(e, "batched step capture");
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            it = rt->graphs.emplace(key, ex).first;
        }
        RIPPLE_CUDA(cudaGraphLaunch(it->second, rt->compute));
        std::lock_guard<std::mutex> lk(rt->mu);
        rt->stats.launches += (int64_t)n * per_unit;
        rt->stats.graph_replays += 1;
    }
    return RIPPLE_OK;
}

// Queue one dependency-driven round on the compute stream: up to K steps of
// every stepped Euler problem in ONE launch (each problem runs r = min(K, its
// remaining steps)), then K x F FIM iterations of the eikonal problems.
// steps[i] receives r of rt->euler_order[i].
static ripple_status launch_round_async(BatchRuntime* rt, int K, std::vector<long long>& steps)
{
    const int ne = (int)rt->euler_order.size();
    if (!rt->d_async) {
        RIPPLE_CUDA(cudaMalloc(&rt->d_async, sizeof(BatchAsync)));
        RIPPLE_CUDA(cudaMalloc(&rt->d_cum, (kMaxRoundSteps + 1) * sizeof(int)));
        RIPPLE_CUDA(cudaMallocHost(&rt->h_async, sizeof(BatchAsync)));
        RIPPLE_CUDA(cudaMallocHost(&rt->h_cum, (kMaxRoundSteps + 1) * sizeof(int)));
    }
    if (ne > rt->cap_done) {
        RIPPLE_CUDA(cudaStreamSynchronize(rt->compute));
        if (rt->d_done) cudaFree(rt->d_done);
        rt->d_done = nullptr;
        const int nc = std::max(ne, std::max(64, rt->cap_done * 2));
        RIPPLE_CUDA(cudaMalloc(&rt->d_done, (size_t)nc * sizeof(unsigned)));
        rt->cap_done = nc;
    }
    // tasks of round step n: the table prefix of the instances with r > n
    steps.assign(ne, 0);
    for (int i = 0; i < ne; ++i)
        steps[i] = std::min<long long>(K, rt->euler_order[i]->req.nsteps - rt->euler_order[i]->steps_done);
    rt->h_cum[0] = 0;
    int m = ne;  // instances with r > n form the prefix [0, m)
    long long tiles = 0;
    for (int i = 0; i < ne; ++i) tiles += table_entries(rt, rt->euler_order[i]);
    for (int n = 0; n < K; ++n) {
        while (m > 0 && steps[m - 1] <= n) {
            --m;
            tiles -= table_entries(rt, rt->euler_order[m]);
        }
        for (int i = 0; i < m; ++i)
            if (steps[i] <= n) return fail(RIPPLE_ERR_INTERNAL, "dependency-driven round: table not ordered");
        if ((long long)rt->h_cum[n] + tiles > INT32_MAX) return fail(RIPPLE_ERR_INVALID, "round too large");
        rt->h_cum[n + 1] = rt->h_cum[n] + (int)tiles;
    }
    BatchAsync& a = *rt->h_async;
    a.next = 0;
    a.total = rt->h_cum[K];
    a.K = K;
    // a step's tasks spread over the workers (the tiled round's CTAs, or the
    // walk round's warps): take them several at a time only when every worker
    // gets that many (a small problem's step stays spread over many workers,
    // so its next step is not held up behind one worker's chunk)
    const bool walk = walk_units(rt);
    const int grid = walk ? rt->grid : rt->grid_async;
    const int workers = walk ? grid * (kBatchWalkThreads / 32) : grid;
    const int per_worker = (int)std::min<long long>(kAsyncChunk, (long long)rt->h_cum[1] / std::max(1, workers));
    a.chunk = std::max(1, per_worker);
    a.cum = rt->d_cum;
    a.done = rt->d_done;
    cudaStream_t s = rt->compute;
    RIPPLE_CUDA(cudaMemcpyAsync(rt->d_cum, rt->h_cum, (K + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    RIPPLE_CUDA(cudaMemcpyAsync(rt->d_async, rt->h_async, sizeof(BatchAsync), cudaMemcpyHostToDevice, s));
    RIPPLE_CUDA(cudaMemsetAsync(rt->d_done, 0, (size_t)std::max(ne, 1) * sizeof(unsigned), s));
    const int layout = rt->cfg.layout == RIPPLE_SOA ? LAYOUT_SOA : LAYOUT_AOS;
    RIPPLE_CUDA(launch_batch_step(rt->cfg.dtype, layout, rt->cfg.tile_variant,
                                  walk ? kBatchStagingWalk : kBatchStagingTma, grid, s, rt->d_euler, rt->d_fim,
                                  rt->d_table, rt->d_bctl, 0, rt->d_async));
    const int F = std::max(1, rt->cfg.fim_iters_per_step);
    long long nf = 0;
    for (long long k = 0; rt->has_f && k < (long long)K * F; ++k, ++nf)
        RIPPLE_CUDA(launch_batch_step(rt->cfg.dtype, layout, rt->cfg.tile_variant, rt->cfg.staging, rt->grid_fim, s,
                                      rt->d_euler, rt->d_fim, rt->d_table, rt->d_bctl, 1));
    std::lock_guard<std::mutex> lk(rt->mu);
    rt->stats.launches += 1 + nf;
    return RIPPLE_OK;
}

// Move finished instances (Euler: all steps done; eikonal: a status word
// set) from the resident set to their downloads.
static void collect_finished(BatchRuntime* rt)
{
    std::vector<Inst*> keep, done;
    for (Inst* in : rt->resident) {
        bool fin = false;
        if (in->req.kind == RIPPLE_REQ_EULER) fin = in->steps_done >= in->req.nsteps;
        else fin = rt->h_status[in->slot] != 0ull;
        (fin ? done : keep).push_back(in);
    }
    rt->resident.swap(keep);
    if (done.empty()) return;
    const double t0 = rt->now();
    rt->dirty = true;
    const ripple_status st = start_downloads(rt, done);
    for (Inst* in : done) {
        if (st == RIPPLE_OK) {
            rt->downloading.push_back(in);
            continue;
        }
        release(rt, in);
        finish(rt, in, st);
        delete in;
    }
    add_host_time(rt, &ripple_batch_stats::host_finish_s, t0);
}

// Solo rounds: while few problems are resident (at most cfg.solo_rounds), each
// round gives the GPU to ONE of them, the oldest (arrival order), on the
// single-problem kernels, whose cost per problem is lower than the batched
// launches' (no work-queue indirection, no per-step launch, no lockstep with a
// larger problem):
//   * an Euler problem takes up to kSoloMaxSteps steps (about a millisecond of
//     work at most) in one launch of the multi-step solver (euler_solo2d.cuh)
//     on its own buffers and control block; its steps are the batched step's
//     bit for bit (buffer parity = step parity, the 3-slot wave-speed ring
//     indexed by the step), so the problem continues in batched rounds when
//     others join;
//   * an eikonal problem is solved whole by the persistent FIM kernel (lists of
//     active tiles), one launch, from its initial state (iterations it ran in
//     batched rounds are discarded: the solve's result does not depend on how
//     its iterations were scheduled, so the bits are the same).
// Requests arriving meanwhile are admitted after the round.  More resident
// problems than that run in batched rounds, where one launch steps all of them.
constexpr long long kSoloMaxSteps = 1024;
// Euler problems of at least this many cells (512^2) run alone when they are
// the oldest: alone a 1024^2 step takes 15 us, in a batched round with others
// 33 us; smaller ones gain from sharing a batched launch
constexpr long long kSoloBigCells = 1LL << 18;

// Solo GPU seconds an Euler step of `cells` cells takes (a fit of the
// multi-step solver on GB300: a fixed barrier and dt cost, then the cells).
static double solo_step_seconds(double cells) { return 3.3e-6 + 12e-12 * cells; }

static ripple_status solo_round(BatchRuntime* rt, bool& handled)
{
    handled = false;
    bool small_only = false;
    Inst* in = nullptr;
    if (rt->cfg.solo_rounds > 0 && !rt->cfg.async_queue && !rt->resident.empty()) {
        // the oldest resident problem (arrival order: shortest-remaining-time-
        // first gave a lower p50 but a higher p99, its largest requests being
        // preempted by every smaller arrival)
        for (Inst* r : rt->resident)
            if (!in || r->t_submit < in->t_submit) in = r;
        // it runs alone while few problems are resident, and always when it is
        // an eikonal problem or a large Euler one (large ones advance faster
        // alone than in lockstep with others); otherwise the small Euler
        // problems share batched rounds
        const bool large = in->req.kind == RIPPLE_REQ_EIKONAL || in->req.dims[0] * in->req.dims[1] >= kSoloBigCells;
        small_only = rt->resident.size() > (size_t)rt->cfg.solo_rounds && !large;
    }
    if (small_only != rt->small_only) {
        rt->small_only = small_only;
        rt->dirty = true;
    }
    if (!in || small_only) return RIPPLE_OK;
    const ripple_dtype dt = rt->cfg.dtype;
    cudaStream_t s = rt->compute;
    FieldCtl* ctl = &rt->slot_ctl[in->slot];
    if (in->req.kind == RIPPLE_REQ_EIKONAL) {
        handled = true;
        RIPPLE_CUDA(cudaEventRecord(rt->ev_r0, s));
        const long long max_iters = in->req.eik.max_iters > 0 ? in->req.eik.max_iters : 1000000;
        ripple_status st =
            dt == RIPPLE_F32 ? fim_solve_lists<float, 2>(fim_problem<float>(in), in->scratch, ctl, max_iters,
                                                         rt->ctx->sm_count, s)
                             : fim_solve_lists<double, 2>(fim_problem<double>(in), in->scratch, ctl, max_iters,
                                                          rt->ctx->sm_count, s);
        if (st != RIPPLE_OK) return st;
        RIPPLE_CUDA(cudaEventRecord(rt->ev_r1, s));
        RIPPLE_CUDA(cudaMemcpyAsync(&rt->h_ctl[in->slot], ctl, sizeof(FieldCtl), cudaMemcpyDeviceToHost, s));
        RIPPLE_CUDA(cudaEventSynchronize(rt->ev_r1));
        RIPPLE_CUDA(cudaStreamSynchronize(s));
        const FieldCtl& c = rt->h_ctl[in->slot];
        const bool capped = (c.err & (DEV_ERR_TIMEOUT | DEV_ERR_BARRIER)) != 0u;
        rt->h_status[in->slot] = ((unsigned long long)c.counters[0] << 2) | (capped ? 2ull : 1ull);
        // the device words the download reads back
        RIPPLE_CUDA(cudaMemcpyAsync(&rt->slot_status[in->slot], &rt->h_status[in->slot], sizeof(unsigned long long),
                                    cudaMemcpyHostToDevice, s));
        RIPPLE_CUDA(cudaMemcpyAsync(&rt->slot_counters[in->slot * 3], ctl->counters, 3 * sizeof(long long),
                                    cudaMemcpyDeviceToDevice, s));
        RIPPLE_CUDA(cudaEventRecord(rt->ev_step, s));
        RIPPLE_CUDA(cudaEventSynchronize(rt->ev_step));
    } else {
        handled = true;
        const ripple_request& r = in->req;
        const long long cells = r.dims[0] * r.dims[1];
        // a launch of about a millisecond at most, so arrivals wait little
        const double est_step = solo_step_seconds((double)cells);
        const long long K = std::min<long long>(
            r.nsteps - in->steps_done, std::max<long long>(8, std::min<long long>(kSoloMaxSteps, (long long)(1e-3 / est_step))));
        SoloEuler a{};
        a.buf[0] = in->buf[0];
        a.buf[1] = in->buf[1];
        a.ctl = ctl;
        a.g = in->g;
        a.bc = (int)r.fv.bc;
        a.K = (int)K;
        a.first = in->steps_done;
        a.cfl = r.fv.cfl;
        a.gamma = r.fv.gamma;
        a.gm1 = r.fv.gamma - 1.0;
        a.inv_dx0 = 1.0 / r.fv.dx[0];
        a.inv_dx1 = 1.0 / r.fv.dx[1];
        a.gamma_f = (float)a.gamma;
        a.gm1_f = (float)a.gm1;
        a.inv_dx0_f = (float)a.inv_dx0;
        a.inv_dx1_f = (float)a.inv_dx1;
        a.bar = rt->d_solo_bar;
        a.spin_limit = grid_spin_limit();
        a.err = &rt->d_bctl->err;
        const int n0 = (int)r.dims[0], n1 = (int)r.dims[1];
        const int per_sm = dt == RIPPLE_F32 ? rt->solo_occ[0] : rt->solo_occ[1];  // at kSoloThreads
        const int sms = rt->ctx->sm_count;
        a.strips = (n0 + kSoloW - 1) / kSoloW;
        // segments as short as one row while the units fit one full CTA per SM
        const long long most = (long long)sms * (kSoloThreads / 32);
        a.rows = (int)std::min<long long>(n1, std::max<long long>(1, ((long long)n1 * a.strips + most - 1) / most));
        a.segs = (n1 + a.rows - 1) / a.rows;
        const long long units = (long long)a.strips * a.segs;
        // CTAs of as few warps as spread the units over every SM (a small
        // problem's step is then short chains on many SMs, not long ones on few)
        const int wpc = (int)std::min<long long>(kSoloThreads / 32, std::max<long long>(1, (units + sms - 1) / sms));
        const int grid = (int)std::max<long long>(
            1, std::min<long long>((units + wpc - 1) / wpc, (long long)std::max(1, per_sm) * sms));
        RIPPLE_CUDA(cudaMemsetAsync(rt->d_solo_bar, 0, 2 * sizeof(unsigned), s));
        RIPPLE_CUDA(cudaEventRecord(rt->ev_r0, s));
        void* args[] = {&a};
        const void* kern = dt == RIPPLE_F32 ? (const void*)solo_euler2d_kernel<float>
                                            : (const void*)solo_euler2d_kernel<double>;
        RIPPLE_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(32 * wpc), args, 0, s));
        RIPPLE_CUDA(cudaEventRecord(rt->ev_r1, s));
        RIPPLE_CUDA(cudaMemcpyAsync(rt->h_berr, &rt->d_bctl->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        RIPPLE_CUDA(cudaEventRecord(rt->ev_step, s));
        RIPPLE_CUDA(cudaEventSynchronize(rt->ev_step));
        if (*rt->h_berr) {
            RIPPLE_CUDA(cudaMemsetAsync(&rt->d_bctl->err, 0, sizeof(unsigned), s));
            return fail(RIPPLE_ERR_TIMEOUT, "a grid barrier wait of a solo round ran out");
        }
        in->steps_done += K;
        // the batched step finds a problem's local step as (global step - start_step)
        in->start_step -= K;
        in->active = true;
        rt->dirty = true;
        std::lock_guard<std::mutex> lk(rt->mu);
        rt->stats.launches += 1;
    }
    in->stepped = true;
    float round_ms = 0.f;
    RIPPLE_CUDA(cudaEventElapsedTime(&round_ms, rt->ev_r0, rt->ev_r1));
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        rt->stats.device_s += 1e-3 * round_ms;
        if (in->req.kind == RIPPLE_REQ_EIKONAL) rt->stats.launches += 1;
    }
    collect_finished(rt);
    return RIPPLE_OK;
}

// One scheduler round of compute: K units over the resident set (K is the
// configured cap, lowered so that no Euler problem runs past its last step),
// or one dependency-driven round (up to K steps of every Euler problem).
static ripple_status compute_round(BatchRuntime* rt)
{
    const double t_enter = rt->now();
    // Active set: resident Euler problems in order of least remaining work
    // (cells x steps) while their cells fit the per-step budget (at least
    // one); eikonal problems always iterate.  A problem that (re)joins the
    // active set continues from its own step count.
    {
        std::vector<Inst*> eu;
        for (Inst* in : rt->resident)
            if (in->req.kind == RIPPLE_REQ_EULER) eu.push_back(in);
        std::stable_sort(eu.begin(), eu.end(), [](const Inst* a, const Inst* b) {
            const double wa = (double)a->req.dims[0] * a->req.dims[1] * (double)(a->req.nsteps - a->steps_done);
            const double wb = (double)b->req.dims[0] * b->req.dims[1] * (double)(b->req.nsteps - b->steps_done);
            return wa < wb;
        });
        const int64_t budget = rt->cfg.active_cells;
        int64_t cells = 0;
        for (Inst* in : eu) {
            const int64_t c = in->req.dims[0] * in->req.dims[1];
            const bool take = !(rt->small_only && c >= kSoloBigCells) &&
                              (budget <= 0 || cells == 0 || cells + c <= budget);
            if (take) cells += c;
            if (take != in->active) {
                in->active = take;
                if (take) in->start_step = rt->gstep_e - in->steps_done;
                rt->dirty = true;
            }
        }
    }
    if (rt->dirty) {
        ripple_status st = rebuild_tables(rt);
        if (st != RIPPLE_OK) return st;
    }
    long long K = std::max(1, rt->cfg.steps_per_sync);
    const bool round_async = rt->cfg.async_queue && rt->has_e;
    std::vector<long long> round_steps;
    if (round_async) {
        long long most = 1;
        for (Inst* in : rt->euler_order) most = std::max(most, in->req.nsteps - in->steps_done);
        K = std::min<long long>(std::min<long long>(K, kMaxRoundSteps), most);
    } else {
        for (Inst* in : rt->resident)
            if (in->req.kind == RIPPLE_REQ_EULER && in->active) K = std::min(K, in->req.nsteps - in->steps_done);
    }
    K = std::max(1LL, K);
    RIPPLE_CUDA(cudaEventRecord(rt->ev_r0, rt->compute));
    ripple_status st = round_async ? launch_round_async(rt, (int)K, round_steps) : launch_steps(rt, (int)K);
    if (st != RIPPLE_OK) return st;
    RIPPLE_CUDA(cudaEventRecord(rt->ev_r1, rt->compute));
    for (Inst* in : rt->resident) in->stepped = true;
    if (rt->has_f)
        RIPPLE_CUDA(cudaMemcpyAsync(rt->h_status, rt->slot_status, kSlots * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, rt->compute));
    RIPPLE_CUDA(cudaMemcpyAsync(rt->h_berr, &rt->d_bctl->err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                rt->compute));
    RIPPLE_CUDA(cudaEventRecord(rt->ev_step, rt->compute));
    const double host_q = rt->now() - t_enter;
    RIPPLE_CUDA(cudaEventSynchronize(rt->ev_step));
    float round_ms = 0.f;
    RIPPLE_CUDA(cudaEventElapsedTime(&round_ms, rt->ev_r0, rt->ev_r1));
    if (*rt->h_berr) {
        RIPPLE_CUDA(cudaMemsetAsync(&rt->d_bctl->err, 0, sizeof(unsigned), rt->compute));
        return fail(RIPPLE_ERR_TIMEOUT, "a bounded wait of a batched launch ran out");
    }
    if (rt->has_e) rt->gstep_e += K;
    if (round_async) {
        for (size_t i = 0; i < rt->euler_order.size(); ++i) rt->euler_order[i]->steps_done += round_steps[i];
    } else {
        for (Inst* in : rt->resident)
            if (in->req.kind == RIPPLE_REQ_EULER && in->active) in->steps_done += K;
    }
    if (rt->has_f) rt->gstep_f += K * std::max(1, rt->cfg.fim_iters_per_step);
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        rt->stats.global_steps = rt->gstep_e;
        rt->stats.fim_iterations = rt->gstep_f;
        rt->stats.device_s += 1e-3 * round_ms;
        rt->stats.host_round_s += host_q;
    }
    collect_finished(rt);
    return RIPPLE_OK;
}

static void scheduler(BatchRuntime* rt)
{
    cudaSetDevice(rt->ctx->device);
    std::vector<Inst*> group;  // admitted in this pass
    double t_adm = 0.0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(rt->mu);
            const bool busy = !rt->resident.empty() || !rt->uploading.empty() || !rt->downloading.empty();
            if (!busy)
                rt->cv_work.wait(lk, [&] { return rt->stop || !rt->pending.empty(); });
            if (rt->stop && rt->resident.empty() && rt->uploading.empty() && rt->downloading.empty()) break;
            t_adm = rt->now();
            // admission: FIFO while memory fits
            while (!rt->pending.empty()) {
                Inst* in = rt->pending.front();
                lk.unlock();
                ripple_status st = admit(rt, in);
                lk.lock();
                if (st == RIPPLE_ERR_BUDGET) {
                    const bool nothing_running =
                        rt->resident.empty() && rt->uploading.empty() && rt->downloading.empty();
                    const bool never_fits = rt->ctx->budget && in->total_bytes > rt->ctx->budget;
                    if (never_fits || nothing_running) {
                        rt->pending.pop_front();
                        lk.unlock();
                        release(rt, in);
                        finish(rt, in, RIPPLE_ERR_BUDGET);
                        delete in;
                        lk.lock();
                        continue;
                    }
                    break;  // wait for memory to free up
                }
                rt->pending.pop_front();
                if (st != RIPPLE_OK) {
                    lk.unlock();
                    release(rt, in);
                    finish(rt, in, st);
                    delete in;
                    lk.lock();
                    continue;
                }
                rt->stats.admitted++;
                rt->uploading.push_back(in);  // counts as running for the admissions that follow
                group.push_back(in);
            }
        }
        if (!group.empty()) {
            const ripple_status st = admit_group(rt, group);
            if (st != RIPPLE_OK) {
                for (Inst* in : group) {
                    rt->uploading.erase(std::find(rt->uploading.begin(), rt->uploading.end(), in));
                    release(rt, in);
                    finish(rt, in, st);
                    delete in;
                }
            }
            group.clear();
            add_host_time(rt, &ripple_batch_stats::host_admit_s, t_adm);
        }
        // uploads that completed join the resident set at the next global step
        for (size_t i = 0; i < rt->uploading.size();) {
            Inst* in = rt->uploading[i];
            if (group_done(in)) {
                drop_event(rt, in);
                // the host mirror of the slot's status word may still hold the
                // previous occupant's (a round that iterates no eikonal problem
                // does not refresh it); the device word was cleared by the
                // admission group, which has completed
                rt->h_status[in->slot] = 0ull;
                rt->arena.release(in->h_in, in->dense);  // the upload has read it
                in->h_in = nullptr;
                in->start_step = in->req.kind == RIPPLE_REQ_EULER ? rt->gstep_e : rt->gstep_f;
                in->steps_done = 0;
                in->active = false;  // the next round's active-set pass decides
                in->t_start = rt->now();
                rt->resident.push_back(in);
                rt->dirty = true;
                rt->uploading.erase(rt->uploading.begin() + i);
            } else {
                ++i;
            }
        }
        // Requests submitted together start together: while nothing resident has
        // stepped yet, the first round waits for the uploads already in flight
        // (they complete in the copy stream's order), at most one second.
        bool fresh = !rt->resident.empty();
        double joined = 1e300;
        for (Inst* in : rt->resident) {
            fresh = fresh && !in->stepped;
            joined = std::min(joined, in->t_start);
        }
        if (fresh && !rt->uploading.empty() && rt->now() - joined < 1.0) {
            wait_group(rt->uploading.front());
            continue;
        }
        if (!rt->resident.empty()) {
            bool solo = false;
            ripple_status st = solo_round(rt, solo);
            if (st == RIPPLE_OK && !solo) st = compute_round(rt);
            if (st != RIPPLE_OK) {
                // a CUDA failure: fail everything resident
                for (Inst* in : rt->resident) {
                    release(rt, in);
                    finish(rt, in, st);
                    delete in;
                }
                rt->resident.clear();
                rt->dirty = true;
            }
        }
        // completions: every ticket of the finished downloads first, then
        // their memory and slots
        {
            std::vector<Inst*> done;
            for (size_t i = 0; i < rt->downloading.size();) {
                Inst* in = rt->downloading[i];
                if (group_done(in)) {
                    done.push_back(in);
                    rt->downloading.erase(rt->downloading.begin() + i);
                } else {
                    ++i;
                }
            }
            if (!done.empty()) {
                const double t0 = rt->now();
                {
                    std::lock_guard<std::mutex> lk(rt->mu);
                    const double t = rt->now();
                    for (Inst* in : done) {
                        ripple_status st = RIPPLE_OK;
                        if (in->req.kind == RIPPLE_REQ_EULER) {
                            const unsigned err = rt->out_ctl[in->slot].err;
                            if (err & DEV_ERR_NUMERIC) st = RIPPLE_ERR_NUMERIC;
                            else if (err) st = RIPPLE_ERR_INTERNAL;
                        } else if ((rt->out_status[in->slot] & 3ull) == 2ull) {
                            st = RIPPLE_ERR_TIMEOUT;
                        }
                        fill_ticket(rt, in, st, t);
                        if (in->h_out) {  // the result waits in the arena for the ticket's retrieval
                            Ticket& tk = rt->tickets[in->ticket];
                            tk.stage = in->h_out;
                            tk.out = in->req.output;
                            tk.bytes = in->dense;
                            in->h_out = nullptr;
                        }
                    }
                }
                rt->cv_done.notify_all();
                for (Inst* in : done) {
                    release(rt, in);
                    delete in;
                }
                add_host_time(rt, &ripple_batch_stats::host_finish_s, t0);
            }
        }
        // nothing to compute: block until the oldest copy group completes (a
        // blocking wait wakes as the copies land; a sleep-and-poll loop's
        // wake-ups depend on the host's load)
        if (rt->resident.empty()) {
            if (!rt->downloading.empty()) wait_group(rt->downloading.front());
            else if (!rt->uploading.empty()) wait_group(rt->uploading.front());
        }
    }
}

static ripple_status rt_start(BatchRuntime* rt)
{
    if (rt->started) return RIPPLE_OK;
    RIPPLE_CUDA(cudaSetDevice(rt->ctx->device));
    RIPPLE_CUDA(cudaStreamCreateWithFlags(&rt->compute, cudaStreamNonBlocking));
    RIPPLE_CUDA(cudaStreamCreateWithFlags(&rt->copy, cudaStreamNonBlocking));
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = rt->ctx->device;
        RIPPLE_CUDA(cudaMemPoolCreate(&rt->pool, &props));
        // keep up to the context budget (all of it when unlimited) mapped between uses
        cuuint64_t keep = rt->ctx->budget ? (cuuint64_t)rt->ctx->budget : ~(cuuint64_t)0;
        RIPPLE_CUDA(cudaMemPoolSetAttribute(rt->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    RIPPLE_CUDA(cudaEventCreateWithFlags(&rt->ev_step, cudaEventDisableTiming));
    RIPPLE_CUDA(cudaEventCreateWithFlags(&rt->ev_items, cudaEventDisableTiming));
    RIPPLE_CUDA(cudaMallocHost(&rt->h_items, kSlots * sizeof(GroupItem)));
    RIPPLE_CUDA(cudaMalloc(&rt->d_solo_bar, 2 * sizeof(unsigned)));
    RIPPLE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rt->solo_occ[0], solo_euler2d_kernel<float>,
                                                              kSoloThreads, 0));
    RIPPLE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rt->solo_occ[1], solo_euler2d_kernel<double>,
                                                              kSoloThreads, 0));
    RIPPLE_CUDA(cudaMalloc(&rt->d_items, kSlots * sizeof(GroupItem)));
    RIPPLE_CUDA(cudaEventCreate(&rt->ev_r0));
    RIPPLE_CUDA(cudaEventCreate(&rt->ev_r1));
    RIPPLE_CUDA(cudaMalloc(&rt->slot_ctl, kSlots * sizeof(FieldCtl)));
    RIPPLE_CUDA(cudaMalloc(&rt->slot_status, kSlots * sizeof(unsigned long long)));
    RIPPLE_CUDA(cudaMalloc(&rt->slot_counters, kSlots * 3 * sizeof(long long)));
    RIPPLE_CUDA(cudaMemset(rt->slot_status, 0, kSlots * sizeof(unsigned long long)));
    RIPPLE_CUDA(cudaMallocHost(&rt->h_ctl, kSlots * sizeof(FieldCtl)));
    RIPPLE_CUDA(cudaMallocHost(&rt->h_status, kSlots * sizeof(unsigned long long)));
    RIPPLE_CUDA(cudaMallocHost(&rt->h_counters, kSlots * 3 * sizeof(long long)));
    RIPPLE_CUDA(cudaMallocHost(&rt->out_ctl, kSlots * sizeof(FieldCtl)));
    RIPPLE_CUDA(cudaMallocHost(&rt->out_status, kSlots * sizeof(unsigned long long)));
    RIPPLE_CUDA(cudaMalloc(&rt->d_bctl, sizeof(BatchCtl)));
    RIPPLE_CUDA(cudaMemset(rt->d_bctl, 0, sizeof(BatchCtl)));
    RIPPLE_CUDA(cudaMallocHost(&rt->h_berr, sizeof(unsigned)));
    *rt->h_berr = 0u;
    rt->free_slots.clear();
    for (int i = kSlots - 1; i >= 0; --i) rt->free_slots.push_back(i);
    const int layout = rt->cfg.layout == RIPPLE_SOA ? LAYOUT_SOA : LAYOUT_AOS;
    const int occ = std::max(1, batch_occupancy(rt->cfg.dtype, layout, rt->cfg.tile_variant, rt->cfg.staging));
    rt->grid = occ * rt->ctx->sm_count;
    rt->grid_fim = fim_occupancy(rt->cfg.dtype) * rt->ctx->sm_count;
    rt->grid_async =
        std::max(1, batch_occupancy(rt->cfg.dtype, layout, rt->cfg.tile_variant, kBatchStagingTma)) * rt->ctx->sm_count;
    rt->gstep_e = 0;
    rt->gstep_f = 0;
    // descriptor tables and group events sized up front: growing them while
    // serving (cudaFree, cudaMallocHost) stalls the scheduler for milliseconds
    {
        const ripple_status st = grow(rt, kInitDescriptors, kInitDescriptors, kInitTiles);
        if (st != RIPPLE_OK) return st;
        for (int i = 0; i < kInitEvents; ++i) {
            cudaEvent_t e = nullptr;
            RIPPLE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            rt->ev_pool.push_back(e);
        }
    }
    rt->started = true;
    rt->th = std::thread(scheduler, rt);
    return RIPPLE_OK;
}

static BatchRuntime* runtime_of(ripple_ctx ctx, bool create)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->batch && create) {
        auto* rt = new BatchRuntime();
        rt->ctx = ctx;
        ctx->batch = rt;
    }
    return static_cast<BatchRuntime*>(ctx->batch);
}

// ---------------------------------------------------------------------------
// Autotuner: time each (halo staging, layout, tile shape) candidate of the
// batched step on sample Euler problems of the given sides and keep the fastest.
// ---------------------------------------------------------------------------
static ripple_status autotune(ripple_ctx ctx, const int64_t* sides, int n, ripple_dtype dt, ripple_batch_config* best,
                              double* ms)
{
    RIPPLE_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s;
    RIPPLE_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    double best_ms = 1e300;
    ripple_status status = RIPPLE_OK;
    for (int sg = 0; sg < kNumBatchStagings && status == RIPPLE_OK; ++sg)
    for (int li = 0; li < 2 && status == RIPPLE_OK; ++li) {
        const ripple_layout lay = li == 0 ? RIPPLE_SOA : RIPPLE_AOS;
        for (int v = 0; v < kNumBatchVariants && status == RIPPLE_OK; ++v) {
            const bool walk = sg == kBatchStagingWalk;  // walk units: the tile shape does not apply
            if (walk && v > 0) {
                if (ms) ms[(sg * 2 + li) * kNumBatchVariants + v] = ms[(sg * 2 + li) * kNumBatchVariants];
                continue;
            }
            std::vector<void*> bufs;
            std::vector<size_t> sizes;
            std::vector<BatchEuler> h(n);
            std::vector<int> table;
            FieldCtl* ctl = nullptr;
            BatchEuler* d_e = nullptr;
            int* d_t = nullptr;
            BatchCtl* d_c = nullptr;
            auto cleanup = [&]() {
                cudaStreamSynchronize(s);
                for (size_t i = 0; i < bufs.size(); ++i) ctx_free(ctx, bufs[i], sizes[i]);
                cudaFree(ctl);
                cudaFree(d_e);
                cudaFree(d_t);
                cudaFree(d_c);
            };
            if (cudaMalloc(&ctl, n * sizeof(FieldCtl)) != cudaSuccess) {
                ctl = nullptr;
                status = fail(RIPPLE_ERR_OOM, "autotune: control blocks");
                break;
            }
            if (cudaMemsetAsync(ctl, 0, n * sizeof(FieldCtl), s) != cudaSuccess) {
                cleanup();
                status = fail(RIPPLE_ERR_CUDA, "autotune: clearing control blocks");
                break;
            }
            for (int i = 0; i < n && status == RIPPLE_OK; ++i) {
                const int64_t dims[2] = {sides[i], sides[i]};
                size_t bytes = 0;
                FieldGeom g = make_field_geom(2, dims, 4, lay, 1, dt, &bytes);
                void* b[2] = {nullptr, nullptr};
                for (int k = 0; k < 2 && status == RIPPLE_OK; ++k) {
                    status = ctx_alloc(ctx, bytes, &b[k]);
                    if (status == RIPPLE_OK) {
                        bufs.push_back(b[k]);
                        sizes.push_back(bytes);
                        if (dt == RIPPLE_F32) fill_uniform_euler<float><<<64, 256, 0, s>>>(static_cast<float*>(b[k]), g);
                        else fill_uniform_euler<double><<<64, 256, 0, s>>>(static_cast<double*>(b[k]), g);
                    }
                }
                const int tx = kBatchVariants[v].tx, ty = kBatchVariants[v].ty;
                h[i].buf[0] = b[0];
                h[i].buf[1] = b[1];
                h[i].ctl = ctl + i;
                h[i].g = g;
                h[i].tiles_x = walk ? (int)((sides[i] + kSoloW - 1) / kSoloW) : (int)((sides[i] + tx - 1) / tx);
                h[i].tile_begin = (int)table.size();
                h[i].bc = RIPPLE_BC_PERIODIC;
                h[i].start_step = 0;
                h[i].nsteps = 1LL << 40;
                h[i].gamma = 1.4;
                h[i].gm1 = 1.4 - 1.0;
                h[i].cfl = 0.4;
                h[i].inv_dx0 = h[i].inv_dx1 = (double)sides[i];
                h[i].gamma_f = (float)h[i].gamma;
                h[i].gm1_f = (float)h[i].gm1;
                h[i].inv_dx0_f = h[i].inv_dx1_f = (float)h[i].inv_dx0;
                if (status == RIPPLE_OK) status = encode_batch_maps(h[i], lay, dt, v);
                const int nt = walk ? h[i].tiles_x * (int)((sides[i] + kBatchWalkRows - 1) / kBatchWalkRows)
                                    : h[i].tiles_x * (int)((sides[i] + ty - 1) / ty);
                for (int k = 0; k < nt; ++k) table.push_back(i << 1);
            }
            if (status != RIPPLE_OK) { cleanup(); break; }
            // smax slot 0 of every sample: any positive value
            std::vector<FieldCtl> hc(n);
            for (int i = 0; i < n; ++i) {
                std::memset(&hc[i], 0, sizeof(FieldCtl));
                const double smax0 = 4.0 * (double)sides[i];
                std::memcpy(&hc[i].smax[0], &smax0, sizeof(double));
            }
            // descriptors, table and control of the sample batch; no launch
            // unless every one of them is in place
            if (cudaMalloc(&d_e, n * sizeof(BatchEuler)) != cudaSuccess) d_e = nullptr;
            if (cudaMalloc(&d_t, table.size() * sizeof(int)) != cudaSuccess) d_t = nullptr;
            if (cudaMalloc(&d_c, sizeof(BatchCtl)) != cudaSuccess) d_c = nullptr;
            if (!d_e || !d_t || !d_c) {
                cleanup();
                status = fail(RIPPLE_ERR_OOM, "autotune: sample descriptors");
                break;
            }
            BatchCtl hb{};
            hb.ntiles_e = (int)table.size();
            hb.ntiles = (int)table.size();
            cudaError_t ce = cudaMemcpyAsync(ctl, hc.data(), n * sizeof(FieldCtl), cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(d_e, h.data(), n * sizeof(BatchEuler), cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(d_t, table.data(), table.size() * sizeof(int), cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_c, &hb, sizeof(BatchCtl), cudaMemcpyHostToDevice, s);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
            if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
            if (ce != cudaSuccess) {
                if (e0) cudaEventDestroy(e0);
                cleanup();
                status = cuda_fail(ce, "autotune: sample set-up");
                break;
            }
            const int lay_i = lay == RIPPLE_SOA ? LAYOUT_SOA : LAYOUT_AOS;
            const int grid = std::max(1, batch_occupancy(dt, lay_i, v, sg)) * ctx->sm_count;
            for (int k = 0; k < 3 && ce == cudaSuccess; ++k)
                ce = launch_batch_step(dt, lay_i, v, sg, grid, s, d_e, nullptr, d_t, d_c, 0);
            cudaEventRecord(e0, s);
            const int reps = 6;
            for (int k = 0; k < reps && ce == cudaSuccess; ++k)
                ce = launch_batch_step(dt, lay_i, v, sg, grid, s, d_e, nullptr, d_t, d_c, 0);
            cudaEventRecord(e1, s);
            cudaStreamSynchronize(s);
            float el = 0.f;
            cudaEventElapsedTime(&el, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cleanup();
            if (ce != cudaSuccess) {
                status = cuda_fail(ce, "autotune launch");
                break;
            }
            const double t = el / reps;
            if (ms) ms[(sg * 2 + li) * kNumBatchVariants + v] = t;
            if (t < best_ms) {
                best_ms = t;
                best->layout = lay;
                best->tile_variant = v;
                best->staging = sg;
            }
        }
    }
    cudaStreamDestroy(s);
    return status;
}

}  // namespace ripple

using namespace ripple;

void batch_runtime_destroy(ripple_ctx ctx)
{
    BatchRuntime* rt = static_cast<BatchRuntime*>(ctx->batch);
    if (!rt) return;
    if (rt->started) {
        {
            std::lock_guard<std::mutex> lk(rt->mu);
            rt->stop = true;
            for (Inst* in : rt->pending) delete in;
            rt->pending.clear();
        }
        rt->cv_work.notify_all();
        rt->th.join();
        cudaStreamSynchronize(rt->copy);
        cudaStreamSynchronize(rt->compute);
        for (auto& g : rt->graphs) cudaGraphExecDestroy(g.second);
        cudaFree(rt->slot_ctl);
        cudaFree(rt->slot_status);
        cudaFree(rt->slot_counters);
        cudaFreeHost(rt->h_ctl);
        cudaFreeHost(rt->h_status);
        cudaFreeHost(rt->h_counters);
        cudaFreeHost(rt->out_ctl);
        cudaFreeHost(rt->out_status);
        cudaFree(rt->d_euler);
        cudaFree(rt->d_fim);
        cudaFree(rt->d_table);
        cudaFree(rt->d_bctl);
        cudaFree(rt->d_async);
        cudaFree(rt->d_cum);
        cudaFree(rt->d_done);
        if (rt->h_async) cudaFreeHost(rt->h_async);
        if (rt->h_cum) cudaFreeHost(rt->h_cum);
        if (rt->h_berr) cudaFreeHost(rt->h_berr);
        cudaFreeHost(rt->h_euler);
        cudaFreeHost(rt->h_fim);
        cudaFreeHost(rt->h_table);
        cudaEventDestroy(rt->ev_step);
        cudaEventDestroy(rt->ev_items);
        for (cudaEvent_t e : rt->ev_pool) cudaEventDestroy(e);
        rt->ev_pool.clear();
        cudaFreeHost(rt->h_items);
        cudaFree(rt->d_solo_bar);
        rt->arena.destroy();
        cudaFree(rt->d_items);
        if (rt->pool) cudaMemPoolDestroy(rt->pool);
        cudaEventDestroy(rt->ev_r0);
        cudaEventDestroy(rt->ev_r1);
        cudaStreamDestroy(rt->compute);
        cudaStreamDestroy(rt->copy);
    }
    delete rt;
    ctx->batch = nullptr;
}

extern "C" {

ripple_status ripple_batch_configure(ripple_ctx ctx, const ripple_batch_config* cfg)
{
    if (!ctx || !cfg) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    if (cfg->layout != RIPPLE_AOS && cfg->layout != RIPPLE_SOA) return fail(RIPPLE_ERR_INVALID, "bad layout");
    if (cfg->tile_variant < 0 || cfg->tile_variant >= kNumBatchVariants) return fail(RIPPLE_ERR_INVALID, "bad tile variant");
    if (cfg->staging < 0 || cfg->staging >= kNumBatchStagings) return fail(RIPPLE_ERR_INVALID, "bad halo staging");
    if (cfg->steps_per_sync < 1) return fail(RIPPLE_ERR_INVALID, "steps_per_sync must be >= 1");
    if (cfg->async_queue != 0 && cfg->async_queue != 1) return fail(RIPPLE_ERR_INVALID, "async_queue must be 0 or 1");
    if (cfg->fim_iters_per_step < 1 || cfg->fim_iters_per_step > 64)
        return fail(RIPPLE_ERR_INVALID, "fim_iters_per_step must be 1..64");
    if (cfg->dtype != RIPPLE_F32 && cfg->dtype != RIPPLE_F64) return fail(RIPPLE_ERR_INVALID, "bad dtype");
    if (cfg->solo_rounds < 0 || cfg->solo_rounds > kSlots) return fail(RIPPLE_ERR_INVALID, "solo_rounds must be 0..4096");
    BatchRuntime* rt = runtime_of(ctx, true);
    std::lock_guard<std::mutex> lk(rt->mu);
    if (rt->started) {
        const bool idle = rt->stats.submitted == rt->stats.completed + rt->stats.failed;
        if (!idle) return fail(RIPPLE_ERR_INVALID, "configure only while no request is in flight");
        if (cfg->dtype != rt->cfg.dtype || cfg->layout != rt->cfg.layout || cfg->tile_variant != rt->cfg.tile_variant ||
            cfg->staging != rt->cfg.staging) {
            // the kernel grid depends on the variant; the scheduler re-reads it
            const int layout = cfg->layout == RIPPLE_SOA ? LAYOUT_SOA : LAYOUT_AOS;
            rt->grid = std::max(1, batch_occupancy(cfg->dtype, layout, cfg->tile_variant, cfg->staging)) * ctx->sm_count;
            rt->grid_fim = fim_occupancy(cfg->dtype) * ctx->sm_count;
            rt->grid_async =
                std::max(1, batch_occupancy(cfg->dtype, layout, cfg->tile_variant, kBatchStagingTma)) * ctx->sm_count;
            if (cfg->dtype != rt->cfg.dtype) {
                // descriptor arrays hold the element type: reallocate on next use
                cudaFree(rt->d_fim);
                cudaFreeHost(rt->h_fim);
                rt->d_fim = nullptr;
                rt->h_fim = nullptr;
                rt->cap_f = 0;
            }
        }
    }
    rt->cfg = *cfg;
    rt->dirty = true;
    return RIPPLE_OK;
}

constexpr size_t kStageCallBytes = size_t(64) << 20;

ripple_status ripple_batch_submit(ripple_ctx ctx, const ripple_request* reqs, int n, uint64_t* tickets)
{
    if (!ctx || (!reqs && n > 0) || (!tickets && n > 0) || n < 0) return fail(RIPPLE_ERR_INVALID, "bad arguments");
    for (int i = 0; i < n; ++i) {
        const ripple_request& r = reqs[i];
        if (r.kind != RIPPLE_REQ_EULER && r.kind != RIPPLE_REQ_EIKONAL) return fail(RIPPLE_ERR_INVALID, "bad kind");
        if (r.dims[0] < 1 || r.dims[1] < 1 || r.dims[0] > 65536 || r.dims[1] > 65536)
            return fail(RIPPLE_ERR_INVALID, "dims out of range");
        if (!r.input || !r.output) return fail(RIPPLE_ERR_INVALID, "NULL input/output");
        if (r.kind == RIPPLE_REQ_EULER) {
            if (r.nsteps < 1) return fail(RIPPLE_ERR_INVALID, "nsteps must be >= 1");
            if (r.fv.scheme != RIPPLE_RUSANOV1) return fail(RIPPLE_ERR_INVALID, "batched Euler runs the Rusanov scheme");
            if (!(r.fv.gamma > 1.0) || !(r.fv.cfl > 0.0) || !(r.fv.dx[0] > 0.0) || !(r.fv.dx[1] > 0.0))
                return fail(RIPPLE_ERR_INVALID, "bad Euler parameters");
            if (r.fv.bc != RIPPLE_BC_PERIODIC && r.fv.bc != RIPPLE_BC_TRANSMISSIVE) return fail(RIPPLE_ERR_INVALID, "bad bc");
        } else {
            if (r.nsrc < 1 || r.nsrc > kMaxSources || !r.sources) return fail(RIPPLE_ERR_INVALID, "need 1..16 sources");
            if (!(r.eik.h > 0.0) || !(r.eik.tol > 0.0)) return fail(RIPPLE_ERR_INVALID, "need h > 0 and tol > 0");
            for (int q = 0; q < r.nsrc; ++q)
                if (r.sources[2 * q] < 0 || r.sources[2 * q] >= r.dims[0] || r.sources[2 * q + 1] < 0 ||
                    r.sources[2 * q + 1] >= r.dims[1])
                    return fail(RIPPLE_ERR_INVALID, "source outside the grid");
        }
    }
    BatchRuntime* rt = runtime_of(ctx, true);
    const double t_in = rt->now();  // latency counts from here, the staging copies included
    ripple_dtype dt;
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        if (!rt->started) {
            ripple_status st = rt_start(rt);
            if (st != RIPPLE_OK) return st;
        }
        dt = rt->cfg.dtype;
    }
    // pageable request data goes through the arena (on this thread); page-locked
    // or registered arrays, data the arena has no room for, and bulk submissions
    // (more than kStageCallBytes: they are admitted together, and a one-thread
    // host copy is slower than the direct pageable copy) are copied directly
    std::vector<char*> st_in(n, nullptr), st_out(n, nullptr);
    std::vector<size_t> st_bytes(n, 0);
    size_t call_bytes = 0;
    for (int i = 0; i < n; ++i) {
        const ripple_request& r = reqs[i];
        st_bytes[i] = (size_t)(r.dims[0] * r.dims[1]) * elem_size(dt) * (r.kind == RIPPLE_REQ_EULER ? 4 : 1);
        call_bytes += st_bytes[i];
    }
    for (int i = 0; i < n && call_bytes <= kStageCallBytes; ++i) {
        const ripple_request& r = reqs[i];
        const size_t dense = st_bytes[i];
        cudaPointerAttributes ai{}, ao{};
        const bool pin_in = cudaPointerGetAttributes(&ai, r.input) == cudaSuccess && ai.type == cudaMemoryTypeHost;
        const bool pin_out = cudaPointerGetAttributes(&ao, r.output) == cudaSuccess && ao.type == cudaMemoryTypeHost;
        cudaGetLastError();
        if (pin_in && pin_out) continue;
        char* a = pin_in ? nullptr : rt->arena.alloc(dense);
        char* b = pin_out ? nullptr : rt->arena.alloc(dense);
        if ((!pin_in && !a) || (!pin_out && !b)) {
            rt->arena.release(a, dense);
            rt->arena.release(b, dense);
            continue;
        }
        if (a) std::memcpy(a, r.input, dense);
        st_in[i] = a;
        st_out[i] = b;
    }
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        const double now = t_in;
        for (int i = 0; i < n; ++i) {
            Inst* in = new Inst();
            in->req = reqs[i];
            in->h_in = st_in[i];
            in->h_out = st_out[i];
            in->dense = st_bytes[i];
            if (reqs[i].kind == RIPPLE_REQ_EIKONAL) {
                in->src.assign(reqs[i].sources, reqs[i].sources + 2 * reqs[i].nsrc);
                in->req.sources = nullptr;
            }
            in->ticket = rt->next_ticket++;
            in->t_submit = now;
            rt->tickets[in->ticket] = Ticket{};
            rt->pending.push_back(in);
            tickets[i] = in->ticket;
            rt->stats.submitted++;
        }
    }
    rt->cv_work.notify_all();
    return RIPPLE_OK;
}

// A retrieved ticket's result, if it waits in the arena: into the caller's
// array (on the retrieving thread), and the arena block back.
static void deliver(BatchRuntime* rt, const Ticket& tk)
{
    if (!tk.stage) return;
    std::memcpy(tk.out, tk.stage, tk.bytes);
    rt->arena.release(tk.stage, tk.bytes);
}

ripple_status ripple_poll(ripple_ctx ctx, uint64_t ticket, ripple_ticket_info* info)
{
    if (!ctx) return fail(RIPPLE_ERR_INVALID, "ctx is NULL");
    BatchRuntime* rt = runtime_of(ctx, false);
    if (!rt) return fail(RIPPLE_ERR_INVALID, "unknown ticket");
    std::unique_lock<std::mutex> lk(rt->mu);
    auto it = rt->tickets.find(ticket);
    if (it == rt->tickets.end()) return fail(RIPPLE_ERR_INVALID, "unknown ticket");
    if (!it->second.done) return RIPPLE_ERR_NOT_READY;
    if (info) *info = it->second.info;
    const Ticket tk = it->second;
    rt->tickets.erase(it);
    lk.unlock();
    deliver(rt, tk);
    return RIPPLE_OK;
}

ripple_status ripple_wait(ripple_ctx ctx, uint64_t ticket, int64_t timeout_ms, ripple_ticket_info* info)
{
    if (!ctx) return fail(RIPPLE_ERR_INVALID, "ctx is NULL");
    BatchRuntime* rt = runtime_of(ctx, false);
    if (!rt) return fail(RIPPLE_ERR_INVALID, "unknown ticket");
    std::unique_lock<std::mutex> lk(rt->mu);
    auto it = rt->tickets.find(ticket);
    if (it == rt->tickets.end()) return fail(RIPPLE_ERR_INVALID, "unknown ticket");
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (!rt->tickets[ticket].done) {
        if (timeout_ms >= 0) {
            if (rt->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !rt->tickets[ticket].done)
                return fail(RIPPLE_ERR_TIMEOUT, "ripple_wait timed out");
        } else {
            rt->cv_done.wait(lk);
        }
    }
    if (info) *info = rt->tickets[ticket].info;
    const Ticket tk = rt->tickets[ticket];
    rt->tickets.erase(ticket);
    lk.unlock();
    deliver(rt, tk);
    return RIPPLE_OK;
}

ripple_status ripple_batch_get_stats(ripple_ctx ctx, ripple_batch_stats* out)
{
    if (!ctx || !out) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    BatchRuntime* rt = runtime_of(ctx, true);
    std::lock_guard<std::mutex> lk(rt->mu);
    *out = rt->stats;
    out->now_s = rt->now();
    return RIPPLE_OK;
}

ripple_status ripple_batch_autotune(ripple_ctx ctx, const int64_t* sides, int n, ripple_dtype dtype,
                                    ripple_batch_config* chosen, double* ms_per_step)
{
    if (!ctx || !sides || n < 1 || !chosen) return fail(RIPPLE_ERR_INVALID, "bad arguments");
    for (int i = 0; i < n; ++i)
        if (sides[i] < 1 || sides[i] > 65536) return fail(RIPPLE_ERR_INVALID, "side out of range");
    ripple_batch_config best = *chosen;
    best.dtype = dtype;
    ripple_status st = autotune(ctx, sides, n, dtype, &best, ms_per_step);
    if (st != RIPPLE_OK) return st;
    *chosen = best;
    return RIPPLE_OK;
}

}  // extern "C"
