// Host-side runtime structures of the C-ABI library (not part of the ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ripple.h"
#include "euler_sweep.cuh"
#include "field.cuh"

namespace ripple {

void set_error(const std::string& msg);
ripple_status fail(ripple_status st, const std::string& msg);
ripple_status cuda_fail(cudaError_t e, const char* what);

#define RIPPLE_CUDA(call)                                        \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::ripple::cuda_fail(e_, #call); \
    } while (0)

// Tile shapes compiled for the sweep (autotuner candidates).
struct TileShape {
    int tx, ty;
};
// Variants 0, 1: one cell per work item; variant 2 (FP32 only): packed f32x2
// cell pairs (euler_sweep_pair.cuh); variant 3 (FP32 3D MUSCL-Hancock only):
// one warp per 64-cell row of a 64 x 14 tile (euler_sweep_row3.cuh).
constexpr int kNumSweepVariants = 4;
constexpr int kPairVariant = 2;
constexpr int kRowVariant = 3;
constexpr TileShape kSweepVariants[kNumSweepVariants] = {{32, 8}, {32, 4}, {32, 8}, {64, 14}};

// Launch description of one sweep (one explicit step of one field).
struct SweepLaunch {
    const CUtensorMap* map_in;
    const CUtensorMap* map_out;
    void* out;
    FieldCtl* ctl;
    SweepGeom sg;
    SweepParams prm;
    int grid;
    cudaStream_t stream;
};

// Kernel table entry points (one translation unit per element type and dim).
// Return cudaErrorInvalidValue for a combination that is not compiled.
cudaError_t sweep_launch_f32_2d(int layout, int scheme, int v, const SweepLaunch& L);
cudaError_t sweep_launch_f32_3d(int layout, int scheme, int v, const SweepLaunch& L);
cudaError_t sweep_launch_f64_2d(int layout, int scheme, int v, const SweepLaunch& L);
cudaError_t sweep_launch_f64_3d(int layout, int scheme, int v, const SweepLaunch& L);
// Dispatch by element type and dimension (runtime.cu).
cudaError_t sweep_launch(ripple_dtype dt, int dim, int layout, int scheme, int v, const SweepLaunch& L);
int sweep_smem(ripple_dtype dt, int dim, int layout, int scheme, int v);
int sweep_occ(ripple_dtype dt, int dim, int layout, int scheme, int v);

// One eikonal solve by the persistent FIM kernel with lists of active tiles
// (eikonal.cu), queued on s: zeroes `scratch` (fim_list_scratch_bytes bytes)
// and ctl's solver counters, initialises both T buffers and the first list,
// launches the cooperative solve; the result is in buf[0], the iterations,
// tile visits and Godunov updates in ctl->counters[0..2], errors in ctl->err.
template <typename T>
struct FimProblem;
size_t fim_list_scratch_bytes(int ntiles);
template <typename T, int DIM>
ripple_status fim_solve_lists(FimProblem<T> a, void* scratch, FieldCtl* ctl, long long max_iters, int sm_count,
                              cudaStream_t s);

// Dynamic shared memory of a sweep variant (0 if it does not fit).
int sweep_smem_f32_2d(int layout, int scheme, int v);
int sweep_smem_f32_3d(int layout, int scheme, int v);
int sweep_smem_f64_2d(int layout, int scheme, int v);
int sweep_smem_f64_3d(int layout, int scheme, int v);
// Resident CTAs per SM of a sweep variant (0 if it does not fit).
int sweep_occ_f32_2d(int layout, int scheme, int v);
int sweep_occ_f32_3d(int layout, int scheme, int v);
int sweep_occ_f64_2d(int layout, int scheme, int v);
int sweep_occ_f64_3d(int layout, int scheme, int v);

// One sweep of the split FORCE step of an FP32 field on strip walks
// (euler_force_walk.cuh), along axis 0, 1 (or 2 in 3D); defined with the FP32
// sweeps of the same dimension.
struct WalkLaunch {
    const void* in;
    void* out;
    FieldCtl* ctl;
    WalkGeom wg;
    SweepParams prm;
    int grid;
    cudaStream_t stream;
};
cudaError_t force_walk_launch_f32_2d(int layout, int axis, const WalkLaunch& L);
cudaError_t force_walk_launch_f32_3d(int layout, int axis, const WalkLaunch& L);
// Resident CTAs per SM of the walk kernel (0 on error).
int force_walk_occ_f32_2d(int layout, int axis);
int force_walk_occ_f32_3d(int layout, int axis);

// Aux kernels (f32/f64 x 2D/3D), defined in aux.cu.
cudaError_t launch_prep(int dtype, int dim, void* buf, FieldCtl* ctl, const FieldGeom& g, int bc, double gamma,
                        const double inv_dx[3], int slot, int grid, cudaStream_t s);
// Host-side fault injection for tests: RIPPLE_FAULT holds a comma-separated
// list of host steps (alloc, admit, upload) that then fail as if the CUDA call
// behind them had failed.  Nothing reaches the GPU: the failure is made on
// the host, before the call it stands for.
bool fault_injected(const char* step);
// Read and clear the timeout flag of the staged layout microbenchmark kernels.
unsigned layout_bench_take_error(cudaStream_t s);
// Quiet NaN in every non-interior cell of a padded buffer (pad_fill_nan_kernel).
cudaError_t launch_pad_nan(int dtype, void* buf, const FieldGeom& g, int grid, cudaStream_t s);
cudaError_t launch_totals(int dtype, int ncomp, const void* buf, const FieldGeom& g, double* partials, int nblocks,
                          FieldCtl* ctl, cudaStream_t s);
cudaError_t launch_interior_copy(int dtype, void* buf, const FieldGeom& g, void* dense, int dense_layout, int dir,
                                 int grid, cudaStream_t s);
// Grouped admission (op 0: fill buffer 0 and clear the slot, op 1: boundary
// images, wave speeds and buffer 1's padding) and download (op 2: pack) of
// the batch runtime over n device-resident GroupItems (field.cuh).
enum : int { GROUP_ADMIT_FILL = 0, GROUP_ADMIT_PREP = 1, GROUP_PACK = 2 };
cudaError_t launch_group(int dtype, int op, const GroupItem* items, int n, long long blocks, cudaStream_t s);

// Tensor-map cache entry.
struct MapEntry {
    int buffer;  // 0/1
    int kind;    // 0 load (whole padded buffer), 1 store (interior)
    int r, tx, ty;
    CUtensorMap map;
};

struct EikScratch;  // eikonal solver state (eikonal.cu)

}  // namespace ripple

struct ripple_ctx_s {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;  // 0 = unlimited
    std::atomic<size_t> used{0};
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    void* (*alloc_fn)(size_t, void*) = nullptr;
    void (*free_fn)(void*, void*) = nullptr;
    void* alloc_user = nullptr;
    std::atomic<int> nfields{0};
    // scratch owned by the context
    void* staging = nullptr;
    size_t staging_bytes = 0;
    double* partials = nullptr;
    size_t partials_bytes = 0;
    std::mutex mu;
    std::vector<ripple_field> fields;  // live fields (device error words read by ripple_ctx_sync)
    void* batch = nullptr;             // batch/serve runtime (batch.cu)
};

struct ripple_field_s {
    ripple_ctx ctx = nullptr;
    int ndim = 0, ncomp = 0, halo = 0;
    ripple_layout layout = RIPPLE_SOA;
    ripple_dtype dtype = RIPPLE_F32;
    ripple::FieldGeom geom{};
    size_t elems = 0, bytes = 0;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    ripple::FieldCtl* ctl = nullptr;
    std::deque<ripple::MapEntry> maps;  // deque: push_back keeps earlier entries in place
    // Euler bookkeeping
    long long steps_total = 0;  // selects the smax ring slot
    bool pad_nan = false;       // non-interior cells of both buffers set to NaN (before the first step)
    bool prepared = false;      // ghosts + smax of the current buffer valid for:
    double prep_gamma = 0, prep_dx[3] = {0, 0, 0};
    int prep_bc = -1;
    int variant = -1;           // tuned tile variant (-1 = default)
    int zchunk = 0;             // tuned z chunk (0 = automatic)
    ripple::EikScratch* eik = nullptr;
};

// Teardown hooks of the eikonal scratch and the batch runtime.
void eik_scratch_free(ripple_field f);
void batch_runtime_destroy(ripple_ctx ctx);

namespace ripple {
// Reserve `bytes` of the context's budget (atomic); false if it would overflow.
bool budget_reserve(ripple_ctx ctx, size_t bytes);
// Padded geometry of a field (see field.cuh); *bytes = one buffer, 256-byte rounded.
FieldGeom make_field_geom(int ndim, const int64_t* dims, int ncomp, ripple_layout layout, int halo,
                          ripple_dtype dtype, size_t* bytes);
ripple_status ctx_alloc(ripple_ctx ctx, size_t bytes, void** out);
void ctx_free(ripple_ctx ctx, void* p, size_t bytes);
ripple_status ensure_second_buffer(ripple_field f);
// TMA map of a padded buffer of geometry g: kind 0 stages planes of a tile plus
// r ghost cells (box of plane_box), kind 1 stores interior tiles of tx x ty.
ripple_status encode_plane_map(void* buffer, const FieldGeom& g, ripple_layout layout, ripple_dtype dtype, int kind,
                               int r, int tx, int ty, CUtensorMap* out);
const CUtensorMap* field_map(ripple_field f, int buffer, int kind, int r, int tx, int ty, ripple_status* st);
ripple_status take_device_error(ripple_field f);
size_t elem_size(ripple_dtype d);
}  // namespace ripple
