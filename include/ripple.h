/*
 * ripple.h -- C ABI of the GB300 (sm_103a) stencil-sweep library.
 *
 * The library implements the data-parallel hot path of Ripple (arXiv
 * 2104.08571): a halo-padded, block-tiled stencil sweep over a multi-component
 * field stored in a polymorphic layout (Section 4.1 tensors with padding,
 * Section 4.2 polymorphic data layout), with the tile plus its ghost cells
 * staged in shared memory (Section 5.4, "in shared" access) and one of two
 * updates applied:
 *   - a finite-volume compressible Euler step (the flux difference of
 *     Section 7.3 inside the solver graph of Section 8, Listing "euler_graph"),
 *   - a Godunov-upwind eikonal relaxation inside a Fast Iterative Method
 *     (Section 7.4, the Hamiltonian |grad phi|^2 - 1/f^2 = 0).
 *
 * Conventions shared by every entry point
 *   - Every function returns a ripple_status; no exception crosses the ABI.
 *     ripple_last_error() returns a thread-local message for the last failure.
 *   - Handles are opaque.  The library owns device memory behind a handle; the
 *     caller owns every host buffer it passes and must destroy handles.
 *     Destroying NULL is RIPPLE_OK.
 *   - dims[0] is x, the fastest-varying axis.  Host/device arrays exchanged
 *     with a field hold interior cells only, in the layout named by the call:
 *       RIPPLE_SOA ("strided"):  a[((c * nz + k) * ny + j) * nx + i]
 *       RIPPLE_AOS ("contiguous"): a[((k * ny + j) * nx + i) * ncomp + c]
 *     with elements of the field's dtype (float for RIPPLE_F32, double for
 *     RIPPLE_F64).
 *   - Euler fields hold the conserved variables in the order
 *     (rho, rho*u_x, rho*u_y[, rho*u_z], E): ncomp = ndim + 2.
 *   - Work is queued on the context's stream (ripple_set_stream).  Calls that
 *     return data to the host synchronise that stream; the others are
 *     asynchronous and report device-side errors (RIPPLE_ERR_NUMERIC,
 *     RIPPLE_ERR_TIMEOUT) at the next synchronising call on that context.
 *   - One context is driven by one host thread at a time, except
 *     ripple_batch_submit / ripple_poll / ripple_wait, which are thread-safe.
 */
#ifndef RIPPLE_H
#define RIPPLE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RIPPLE_API __attribute__((visibility("default")))
#else
#define RIPPLE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RIPPLE_OK = 0,
    RIPPLE_ERR_INVALID = 1,   /* bad argument (shape, halo < stencil radius, dtype, ...) */
    RIPPLE_ERR_OOM = 2,       /* device or host allocation failed */
    RIPPLE_ERR_CUDA = 3,      /* a CUDA runtime/driver call failed */
    RIPPLE_ERR_NOT_READY = 4, /* ripple_poll: request still in flight */
    RIPPLE_ERR_TIMEOUT = 5,   /* a bounded wait (host or device) ran out */
    RIPPLE_ERR_NUMERIC = 6,   /* non-positive or NaN density/pressure was produced */
    RIPPLE_ERR_BUDGET = 7,    /* allocation would exceed the context's memory budget */
    RIPPLE_ERR_INTERNAL = 8   /* library invariant violated */
} ripple_status;

typedef enum { RIPPLE_AOS = 0, RIPPLE_SOA = 1 } ripple_layout;
typedef enum { RIPPLE_F32 = 0, RIPPLE_F64 = 1 } ripple_dtype;
typedef enum { RIPPLE_RUSANOV1 = 0, RIPPLE_MUSCL_HANCOCK_MINMOD = 1, RIPPLE_FORCE_SPLIT = 2 } ripple_scheme;
typedef enum { RIPPLE_BC_PERIODIC = 0, RIPPLE_BC_TRANSMISSIVE = 1 } ripple_bc;

typedef struct ripple_ctx_s* ripple_ctx;
typedef struct ripple_field_s* ripple_field;

/* ------------------------------------------------------------------------ */
/* Context: device, stream, allocator and memory budget.                     */
/* ------------------------------------------------------------------------ */

/*
 * Create a context on CUDA device `device` with a device-memory budget of
 * `mem_budget_bytes` (0 = unlimited).  Field and scratch allocations made
 * through the context count against the budget (RIPPLE_ERR_BUDGET beyond it),
 * following the paper's advice (Section 5.1) to allocate ahead of the
 * computation instead of inside it.  The context owns a CUDA stream until
 * ripple_set_stream replaces it.
 */
RIPPLE_API ripple_status ripple_ctx_create(int device, size_t mem_budget_bytes, ripple_ctx* out);

/* Synchronise, release all scratch memory and the context itself.  Fields
 * created from the context must be destroyed first (RIPPLE_ERR_INVALID
 * otherwise). */
RIPPLE_API ripple_status ripple_ctx_destroy(ripple_ctx ctx);

/* Queue subsequent work on `cuda_stream` (a cudaStream_t, may be e.g. the
 * PyTorch current stream; NULL = the context's own stream).  The caller
 * keeps ownership of a stream it passes. */
RIPPLE_API ripple_status ripple_set_stream(ripple_ctx ctx, void* cuda_stream);

/*
 * Route device allocations through caller callbacks (e.g. the PyTorch caching
 * allocator).  alloc(bytes, user) returns a device pointer aligned to 256 B or
 * NULL; release(ptr, user) frees it.  Passing alloc = NULL restores
 * cudaMalloc/cudaFree.  Must be called before any field is created.
 */
RIPPLE_API ripple_status ripple_set_allocator(ripple_ctx ctx, void* (*alloc)(size_t bytes, void* user),
                                   void (*release)(void* ptr, void* user), void* user);

/* Wait for all work queued on the context's stream; returns the first pending
 * device-side error (RIPPLE_ERR_NUMERIC / RIPPLE_ERR_TIMEOUT) and clears it. */
RIPPLE_API ripple_status ripple_ctx_sync(ripple_ctx ctx);

/* Bytes currently allocated through the context (fields + scratch). */
RIPPLE_API ripple_status ripple_ctx_mem_used(ripple_ctx ctx, size_t* bytes);

/* ------------------------------------------------------------------------ */
/* Fields: halo-padded tensors in AoS or SoA layout (Sections 4.1-4.2).      */
/* ------------------------------------------------------------------------ */

/*
 * Create a field of ndim (2 or 3) axes with dims[d] >= 1 interior cells,
 * `ncomp` (1..5) components per cell, `halo` >= 0 ghost layers on every side
 * of every axis, stored in `layout` with element type `dtype`.  Device memory
 * holds two padded buffers (the double buffer of Section 5.4, in -> out, then
 * swap); the second is allocated on first use by a solver.  Contents start
 * undefined; upload before use.  RIPPLE_ERR_INVALID for dims outside
 * 1..2^20, halo outside 0..8, or more than 2^32 padded cells per buffer;
 * RIPPLE_ERR_OOM / RIPPLE_ERR_BUDGET when the memory is not there.
 */
RIPPLE_API ripple_status ripple_field_create(ripple_ctx ctx, int ndim, const int64_t* dims, int ncomp,
                                  ripple_layout layout, int halo, ripple_dtype dtype,
                                  ripple_field* out);

RIPPLE_API ripple_status ripple_field_destroy(ripple_field field);

/* Copy interior cells from a HOST buffer in `src_layout` into the field
 * (synchronous).  Ghost cells become stale and are refilled by the next solver
 * call. */
RIPPLE_API ripple_status ripple_field_upload(ripple_field field, const void* src, ripple_layout src_layout);

/* Copy interior cells to a HOST buffer in `dst_layout` (synchronous; reports
 * pending device errors like ripple_ctx_sync). */
RIPPLE_API ripple_status ripple_field_download(ripple_field field, void* dst, ripple_layout dst_layout);

/* Same as upload/download, but `src`/`dst` is DEVICE memory of the field's
 * device; asynchronous on the context stream. */
RIPPLE_API ripple_status ripple_field_upload_device(ripple_field field, const void* src, ripple_layout src_layout);
RIPPLE_API ripple_status ripple_field_download_device(ripple_field field, void* dst, ripple_layout dst_layout);

typedef struct {
    int ndim, ncomp, halo;
    ripple_layout layout;
    ripple_dtype dtype;
    int64_t dims[3];     /* interior cells (1 on unused axes) */
    int64_t padded[3];   /* allocated extent per axis, x includes alignment padding */
    int64_t x_lead;      /* padded x index of the first ghost column */
    size_t buffer_bytes; /* bytes of one padded buffer */
    void* current;       /* device pointer of the buffer holding the current state */
} ripple_field_desc;

RIPPLE_API ripple_status ripple_field_describe(ripple_field field, ripple_field_desc* out);

/*
 * Sweep kernel of a field's Euler steps (a tuning choice; every choice gives
 * results within the FP32/FP64 parity bars, and the paper's tiling options of
 * Section 5.4 are its prior art).  variant: -1 = automatic (the default), or
 *   0 = one cell per thread, 32 x 8 tiles; 1 = the same, 32 x 4 tiles;
 *   2 = packed cell pairs, 32 x 8 tiles (FP32); 3 = one warp per 64-cell row,
 *   64 x 14 tiles (FP32 3D MUSCL-Hancock only).
 * zchunk: planes per z work item of 3D sweeps (0 = automatic, 32).
 * RIPPLE_ERR_INVALID for an unknown variant or a negative zchunk; a variant
 * that does not exist for the field's dtype, dimension or scheme makes the
 * next ripple_fv_step fall back to the automatic choice.
 */
RIPPLE_API ripple_status ripple_field_set_sweep(ripple_field field, int variant, int zchunk);

/* ------------------------------------------------------------------------ */
/* Finite-volume Euler step.                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    double gamma;       /* ratio of specific heats (> 1) */
    double cfl;         /* Courant number, dt = cfl / max_cells sum_d (|u_d| + c)/dx_d */
    double dx[3];       /* cell widths per axis (> 0) */
    ripple_scheme scheme;
    ripple_bc bc;
} ripple_fv_params;

typedef struct {
    double t;           /* simulated time advanced by this call (sum of dt, FP64) */
    double dt_last;     /* the last dt used */
    double totals[5];   /* FP64 compensated sums of each conserved variable over interior cells */
    int64_t steps_done; /* steps completed by this call */
} ripple_fv_stats;

/*
 * Advance the Euler field U by `nsteps` explicit steps (Section 8, Listing
 * "euler_graph": wave speeds -> max reduction -> dt -> padding fill -> flux
 * difference update -> swap; the flux difference is that of Section 7.3).
 * RIPPLE_RUSANOV1 and RIPPLE_MUSCL_HANCOCK_MINMOD: the update is unsplit (all
 * axes in one pass) with a Rusanov face flux, first order or MUSCL-Hancock
 * with minmod slopes.  RIPPLE_FORCE_SPLIT is the paper's own solver: a
 * dimensionally split step (update_state_x, then y, then z, each a sweep
 * along one axis with the padding refilled in between) with the FORCE face
 * flux of Section 7.3 (the mean of the Lax-Friedrichs and Richtmyer fluxes),
 * dt from the state at the start of the step by the same rule.  U must have
 * ncomp = ndim + 2 and halo >= 1 (Rusanov, FORCE) or >= 2 (MUSCL-Hancock).  For RIPPLE_F32
 * fields the stencil runs in FP32 while dt and the totals are reduced in
 * FP64; RIPPLE_F64 fields run fully in FP64.
 * With stats != NULL the call synchronises, fills *stats (totals of the final
 * state) and returns RIPPLE_ERR_NUMERIC if any produced state lost
 * positivity.  With stats == NULL the call only queues the work.
 */
RIPPLE_API ripple_status ripple_fv_step(ripple_field U, const ripple_fv_params* params, int64_t nsteps,
                             ripple_fv_stats* stats);

/* ------------------------------------------------------------------------ */
/* Eikonal solve (Fast Iterative Method, Section 7.4).                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double h;            /* grid spacing (cells are h wide on every axis) */
    double tol;          /* a tile converges when no cell changes by tol or more */
    int64_t max_iters;   /* cap on active-list iterations (0 = library default) */
} ripple_eik_params;

typedef struct {
    int64_t iterations;  /* active-list iterations run */
    int64_t tile_visits; /* tile relaxations performed */
    int64_t cell_updates;/* Godunov cell updates performed (tile visits x sweeps x cells) */
} ripple_eik_stats;

/*
 * Solve |grad T| s = 1 on the grid of `slowness` (1 component, any halo) into
 * `T` (1 component, halo >= 1, same dims and dtype), with T = 0 held at the
 * `nsrc` source cells given as ndim coordinates each (x first) in
 * `src_coords`.  Godunov upwind discretisation; outside-domain neighbours are
 * +inf.  The result is the fixed point of T = min(T, G(T)) up to the stopping
 * tolerance.  Returns RIPPLE_ERR_TIMEOUT if max_iters runs out.  Synchronous.
 */
RIPPLE_API ripple_status ripple_eikonal_solve(ripple_field slowness, ripple_field T, const int64_t* src_coords,
                                   int nsrc, const ripple_eik_params* params, ripple_eik_stats* stats);

/* ------------------------------------------------------------------------ */
/* Batched and served execution of independent 2D problems.                  */
/* ------------------------------------------------------------------------ */

/*
 * The paper runs one problem per graph (Section 6 scheduling); this runtime
 * serves many independent problems at once, which the paper does not do.
 * Requests are admitted while their device memory fits the context budget,
 * stay resident until done, and every resident problem advances in ONE launch
 * per global step: a flat work queue over the tiles of all resident problems,
 * each problem with its own dt (Euler) or iteration counter (eikonal).  New
 * requests join while others run (continuous batching).  A scheduler thread
 * per context drives the GPU on its own streams; submit / poll / wait are
 * thread-safe.
 */
typedef enum { RIPPLE_REQ_EULER = 0, RIPPLE_REQ_EIKONAL = 1 } ripple_request_kind;

typedef struct {
    int kind;                 /* ripple_request_kind */
    int64_t dims[2];          /* 2D grid (nx, ny) */
    const void* input;        /* HOST: Euler conserved state (4 components, SoA, dtype of the batch) or
                                 eikonal slowness (1 component); read until the request is admitted */
    void* output;             /* HOST: final Euler state / eikonal travel times, same shape; holds the
                                 result when ripple_poll / ripple_wait retire the ticket (a pageable
                                 array is written by that call, from the runtime's page-locked stage) */
    ripple_fv_params fv;      /* Euler: gamma, cfl, dx, bc; scheme must be RIPPLE_RUSANOV1 */
    int64_t nsteps;           /* Euler: steps to run (>= 1) */
    ripple_eik_params eik;    /* eikonal: h, tol, max_iters */
    const int64_t* sources;   /* eikonal: nsrc (x, y) cell pairs, copied by ripple_batch_submit */
    int nsrc;
} ripple_request;

typedef struct {
    ripple_status status;     /* RIPPLE_OK, _NUMERIC, _TIMEOUT (eikonal cap), _BUDGET (never fits), ... */
    double submit_s, admit_s, start_s, finish_s;  /* runtime clock (seconds since the runtime started) */
    int64_t work;             /* Euler steps / eikonal FIM iterations */
    int64_t tile_visits, cell_updates;            /* eikonal work counters */
    double t;                 /* Euler: simulated time reached */
} ripple_ticket_info;

typedef struct {
    ripple_layout layout;     /* layout of resident Euler states */
    int tile_variant;         /* 0: 32x8, 1: 8x32, 2: 16x16 Euler tiles */
    int steps_per_sync;       /* most global steps queued between scheduler checks (fewer when an
                                 Euler problem ends sooner): latency of joining vs overhead */
    int use_graphs;           /* replay queued steps from captured CUDA graphs */
    ripple_dtype dtype;       /* element type of every request of this context */
    int fim_iters_per_step;   /* eikonal FIM iterations run per Euler global step (1..64) */
    int64_t active_cells;     /* per-step cell budget of stepped Euler problems, chosen by least
                                 remaining work (0 = step every resident problem) */
    int staging;              /* halo staging of the Euler step: 0 = TMA tile loads by a producer warp
                                 into a shared-memory ring; 1 = direct loads by every thread; 2 = no
                                 tiles: warps walk 30-column x 16-row units (x faces by shuffles, the
                                 y face carried); the results are the same bits either way */
    int async_queue;          /* 1 = dependency-driven rounds: ONE persistent launch runs up to
                                 steps_per_sync steps of every stepped Euler problem (each runs
                                 min(steps_per_sync, its remaining steps), so a round does not
                                 shrink when one problem ends); a tile of step n of a problem
                                 starts as soon as that problem has completed step n - 1 (its dt
                                 is the CFL limit of its whole state), with no barrier between
                                 problems or global steps.  With staging 2 the round's tasks are
                                 walk units taken by warps; otherwise tiles staged by TMA (for
                                 staging 1 as well).  0 = one launch per global step (default). */
    int solo_rounds;          /* n > 0 = while at most n problems are resident, each round runs the
                                 oldest of them alone on the single-problem kernels
                                 (Euler: one launch of the multi-step solver, up to about a millisecond
                                 of steps; eikonal: one persistent FIM solve), lowering the latency of
                                 requests served at low load; more resident problems run in batched
                                 rounds.  Results are bitwise those of batched rounds (the solvers
                                 share the per-step arithmetic).  0 = off; 0..4096, default 4. */
} ripple_batch_config;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    int64_t global_steps, launches, graph_replays;
    double now_s;             /* runtime clock now */
    int64_t fim_iterations;   /* eikonal iterations issued */
    double device_s;          /* GPU time of the compute rounds (CUDA events around each round's
                                 launches on the compute stream) */
    double host_admit_s;      /* scheduler-thread time in admissions: allocation, input copies
                                 (synchronous for pageable host arrays), group launches */
    double host_round_s;      /* scheduler-thread time preparing and queueing compute rounds
                                 (tables, launches), without the wait for the GPU */
    double host_finish_s;     /* scheduler-thread time queueing downloads (output copies are
                                 synchronous for pageable host arrays) and completing tickets */
} ripple_batch_stats;

/* Set the batch configuration (defaults: SoA, 32x8, 16 steps per sync, graphs
 * on, F32, 4 FIM iterations per step, no cell budget, TMA staging, one launch
 * per global step, solo rounds up to 4 resident problems).  Only while no request is in flight. */
RIPPLE_API ripple_status ripple_batch_configure(ripple_ctx ctx, const ripple_batch_config* cfg);

/* Queue n requests; tickets_out[i] identifies request i.  Validates every
 * request first (RIPPLE_ERR_INVALID queues nothing).  Never blocks on the GPU.
 * Pageable input arrays are copied here into the runtime's page-locked arena
 * (512 MB per context) when they fit and the call carries at most 64 MB, so
 * the runtime's own copies are asynchronous; page-locked or registered
 * arrays, and the rest, are read by the runtime directly (an input is then
 * read until its request is admitted). */
RIPPLE_API ripple_status ripple_batch_submit(ripple_ctx ctx, const ripple_request* reqs, int n,
                                             uint64_t* tickets_out);

/* RIPPLE_OK and *info filled (ticket retired) once the request finished,
 * RIPPLE_ERR_NOT_READY while it runs, RIPPLE_ERR_INVALID for an unknown ticket.
 * The request's own outcome is info->status.  A result staged in the arena is
 * copied into the request's output array by this call. */
RIPPLE_API ripple_status ripple_poll(ripple_ctx ctx, uint64_t ticket, ripple_ticket_info* info);

/* Block until the request finished (RIPPLE_OK, *info filled, ticket retired) or
 * timeout_ms passed (RIPPLE_ERR_TIMEOUT; timeout_ms < 0 waits forever).  A
 * result staged in the arena is copied into the output array by this call. */
RIPPLE_API ripple_status ripple_wait(ripple_ctx ctx, uint64_t ticket, int64_t timeout_ms, ripple_ticket_info* info);

RIPPLE_API ripple_status ripple_batch_get_stats(ripple_ctx ctx, ripple_batch_stats* out);

/*
 * Autotuner: time the batched step for each halo staging (TMA, direct, walk),
 * layout (SoA, AoS) and tile shape on n sample Euler problems of the given
 * square sides (dtype `dtype`), and return the fastest in *chosen (other fields
 * of *chosen are kept).  ms_per_step (nullable) receives 3 x 2 x 3 timings (the
 * walk staging has no tile shape: its three entries per layout are equal),
 * index (staging * 2 + layout_index) * 3 + tile_variant, SoA = layout index 0.
 * Does not change the context's configuration (pass *chosen to
 * ripple_batch_configure).
 */
RIPPLE_API ripple_status ripple_batch_autotune(ripple_ctx ctx, const int64_t* sides, int n, ripple_dtype dtype,
                                               ripple_batch_config* chosen, double* ms_per_step);

/* ------------------------------------------------------------------------ */
/* Conserved totals for callers that cannot allocate device memory.          */
/* ------------------------------------------------------------------------ */
/* Layout microbenchmarks (Section 7.1 SAXPY, Table saxpy; Section 7.2      */
/* particle update, Table particle_update).  Streaming kernels that          */
/* calibrate the HBM roofline and the cost of the two layouts of Section 4.2 */
/* ("strided" = RIPPLE_SOA, "contiguous" = RIPPLE_AOS).                       */
/* ------------------------------------------------------------------------ */

/*
 * y <- a * x + y over n FP32 elements (Section 7.1).  x and y are DEVICE
 * pointers owned by the caller (4-byte aligned; when they share an alignment
 * modulo 16 bytes the body runs on 16-byte vectors).  Each element is one
 * fused multiply-add rounded once.  Asynchronous on the context's stream.
 * RIPPLE_ERR_INVALID: NULL ctx, n < 0, NULL or misaligned pointers.
 */
RIPPLE_API ripple_status ripple_saxpy(ripple_ctx ctx, int64_t n, float a, const float* x, float* y);

/*
 * One explicit update of n particles (Section 7.2): for d = 0, 1, 2
 *   x_d <- x_d + v_d * dt   (one fused multiply-add, rounded once).
 * `particles` is a DEVICE array of 6n floats owned by the caller, in `layout`:
 *   RIPPLE_AOS ("contiguous"): record r = (x0 x1 x2 v0 v1 v2) at [6r, 6r+6);
 *   RIPPLE_SOA ("strided"):    component d at [d*n, d*n + n), d = x0, x1, x2,
 *                              v0, v1, v2.
 * staged = 0 reads and writes global memory directly; staged = 1 passes
 * 2048-particle chunks through shared memory by asynchronous bulk copies (the
 * paper's shared-memory variants), when the array is 16-byte aligned and n is
 * a multiple of 4 (SoA) or 2 (AoS); otherwise the direct kernel runs.  Both
 * give identical bits.  Asynchronous on the context's stream; a bounded wait
 * that runs out is reported by the next ripple_ctx_sync as RIPPLE_ERR_TIMEOUT.
 * RIPPLE_ERR_INVALID: NULL ctx, n < 0, NULL or misaligned pointer, bad layout.
 */
RIPPLE_API ripple_status ripple_particle_update(ripple_ctx ctx, int64_t n, float dt, float* particles,
                                                ripple_layout layout, int staged);

/* ------------------------------------------------------------------------ */

/*
 * The paper has no counterpart to this entry point.
 *
 * Some callers cannot let a library call cudaMalloc: an application that has
 * given all device memory to its own pool or budget, or a latency-bound loop
 * in which the implicit device synchronisation of cudaMalloc/cudaFree would
 * stall work already queued on the GPU.  This function computes the same FP64
 * compensated per-component sums as the `totals` of ripple_fv_step, over a
 * dense DEVICE array the caller owns, and allocates nothing: its only scratch
 * is a fixed 640 KiB array inside the library's device image, present on every
 * GPU that loads the library until the process exits.
 *
 *   state       device array of interior cells, dims[0] x ... x dims[ndim-1]
 *               (x fastest), `ncomp` components in `layout` (see the
 *               conventions above), elements float (RIPPLE_F32) or double
 *               (RIPPLE_F64).  Read only.
 *   totals_out  device array of `ncomp` doubles, written.
 *   cuda_stream the cudaStream_t to queue on (NULL = legacy default stream).
 * The call is asynchronous on `cuda_stream`; the caller keeps ownership of
 * every pointer.  At most 33,554,432 cells (RIPPLE_ERR_INVALID beyond that,
 * or for ncomp outside 1..5) -- the capacity of the fixed scratch.
 * All calls share the scratch array: calls that overlap on the GPU race and
 * must be serialised by the caller (e.g. by using one stream).  Each call
 * writes every scratch entry it reads, so nothing needs clearing in between.
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.
 */
RIPPLE_API ripple_status ripple_totals_noalloc(const void* state, int ndim, const int64_t* dims, int ncomp,
                                               ripple_layout layout, ripple_dtype dtype, double* totals_out,
                                               void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Library                                                                   */
/* ------------------------------------------------------------------------ */

/* Thread-local description of the last failure on this thread ("" if none). */
RIPPLE_API const char* ripple_last_error(void);

/* Library version string. */
RIPPLE_API const char* ripple_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RIPPLE_H */
