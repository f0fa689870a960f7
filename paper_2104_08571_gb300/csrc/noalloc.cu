// Conserved totals without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a host application that
// has handed all device memory to its own pool or budget, or a latency-bound
// loop for which the implicit device synchronisation of cudaMalloc/cudaFree
// would stall work already queued on the GPU.  This entry point computes the
// same FP64 compensated per-component totals as the statistics of
// ripple_fv_step, but over a dense array the caller owns, and keeps its only
// scratch (the per-block partial sums) in a fixed array in device memory that
// is part of the library image: it calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// Scratch: kMaxPartials blocks x 5 components x (sum, compensation) doubles
// = 655,360 bytes, held by every GPU that loads the library until the process
// exits.  One block sums kCellsPerBlock consecutive cells, so the largest
// accepted array has kMaxPartials * kCellsPerBlock = 33,554,432 cells.
// All calls share the array: calls that overlap on the GPU (different streams,
// or host threads without ordering) race on it and must be serialised by the
// caller.  Each call writes every partial slot it later reads, so nothing
// has to be cleared between calls.
#include <mutex>

#include "runtime.h"

namespace ripple {

// Neumaier compensated accumulation in FP64 (the same scheme as the field
// totals of ripple_fv_step).
struct DenseSum {
    double s, c;
    __device__ void add(double x)
    {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ void merge(const DenseSum& o)
    {
        add(o.s);
        c += o.c;
    }
};

constexpr int kCellsPerBlock = 4096;
constexpr int kMaxPartials = 8192;
constexpr long long kNoallocMaxCells = (long long)kMaxPartials * kCellsPerBlock;
constexpr int kMaxDevices = 64;

// The scratch array.  In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress (see scratch_address below).
static __device__ __align__(256) double g_totals_partials[kMaxPartials * 5 * 2];

// Per-block compensated sums over a chunk of a dense interior array.
template <typename T, int NCOMP>
__global__ void __launch_bounds__(256) dense_totals_partial_kernel(const T* __restrict__ state, long long ncell,
                                                                   int soa, double* __restrict__ partials)
{
    DenseSum acc[NCOMP];
#pragma unroll
    for (int m = 0; m < NCOMP; ++m) acc[m] = DenseSum{0.0, 0.0};
    const long long begin = (long long)blockIdx.x * kCellsPerBlock;
    const long long end = min(begin + kCellsPerBlock, ncell);
    for (long long c = begin + threadIdx.x; c < end; c += blockDim.x) {
#pragma unroll
        for (int m = 0; m < NCOMP; ++m)
            acc[m].add((double)state[soa ? (long long)m * ncell + c : c * NCOMP + m]);
    }
    __shared__ double sh[8][NCOMP][2];
#pragma unroll
    for (int m = 0; m < NCOMP; ++m)
        for (int o = 16; o > 0; o >>= 1) {
            DenseSum other{__shfl_down_sync(0xffffffffu, acc[m].s, o), __shfl_down_sync(0xffffffffu, acc[m].c, o)};
            acc[m].merge(other);
        }
    if ((threadIdx.x & 31) == 0)
        for (int m = 0; m < NCOMP; ++m) {
            sh[threadIdx.x >> 5][m][0] = acc[m].s;
            sh[threadIdx.x >> 5][m][1] = acc[m].c;
        }
    __syncthreads();
    if (threadIdx.x < NCOMP) {
        const int m = threadIdx.x;
        DenseSum b{0.0, 0.0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b.merge(DenseSum{sh[w][m][0], sh[w][m][1]});
        partials[((long long)blockIdx.x * NCOMP + m) * 2 + 0] = b.s;
        partials[((long long)blockIdx.x * NCOMP + m) * 2 + 1] = b.c;
    }
}

// Fixed-order combination of the partials into the caller's output.
__global__ void dense_totals_final_kernel(const double* __restrict__ partials, int nblocks, int ncomp,
                                          double* __restrict__ out)
{
    const int m = threadIdx.x;
    if (m >= ncomp) return;
    DenseSum b{0.0, 0.0};
    for (int blk = 0; blk < nblocks; ++blk)
        b.merge(DenseSum{partials[((long long)blk * ncomp + m) * 2], partials[((long long)blk * ncomp + m) * 2 + 1]});
    out[m] = b.s + b.c;
}

// Device address of the scratch array in the current context, looked up once
// per (device, context) with that device current.  The address belongs to the
// library's module as loaded in one context: a caller that makes its own
// driver context current on the same device, or that resets the device and so
// gets a new primary context, gets a fresh lookup instead of a stale pointer.
typedef CUresult (*PFN_ctx_get_current)(CUcontext*);

static PFN_ctx_get_current ctx_get_current_fn()
{
    static PFN_ctx_get_current fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_ctx_get_current>(p);
    });
    return fn;
}

static ripple_status scratch_address(double** out)
{
    struct Entry {
        int dev;
        CUcontext ctx;
        double* addr;
    };
    static std::mutex mu;
    static Entry cache[kMaxDevices] = {};
    static int ncache = 0;
    int dev = 0;
    RIPPLE_CUDA(cudaGetDevice(&dev));
    auto get = ctx_get_current_fn();
    if (!get) return fail(RIPPLE_ERR_CUDA, "cuCtxGetCurrent is unavailable");
    CUcontext cu = nullptr;
    if (get(&cu) != CUDA_SUCCESS) return fail(RIPPLE_ERR_CUDA, "cuCtxGetCurrent failed");
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < ncache && cu; ++i)
        if (cache[i].dev == dev && cache[i].ctx == cu) {
            *out = cache[i].addr;
            return RIPPLE_OK;
        }
    // set-up for this (device, context): the lookup also binds the device's
    // primary context to this thread if no context was current yet
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_totals_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_totals_partials)");
    if (!cu && (get(&cu) != CUDA_SUCCESS || !cu)) return fail(RIPPLE_ERR_CUDA, "no current CUDA context");
    // keep the table bounded: a context that replaced an earlier one on the
    // same device takes over its entry
    int slot = -1;
    for (int i = 0; i < ncache && slot < 0; ++i)
        if (cache[i].dev == dev) slot = i;
    if (slot < 0) {
        if (ncache == kMaxDevices) return fail(RIPPLE_ERR_INVALID, "too many devices");
        slot = ncache++;
    }
    cache[slot] = Entry{dev, cu, static_cast<double*>(p)};
    *out = cache[slot].addr;
    return RIPPLE_OK;
}

template <typename T>
static cudaError_t launch_dense_totals(const void* state, long long ncell, int ncomp, int soa, double* partials,
                                       int nblocks, double* out, cudaStream_t s)
{
    const T* p = static_cast<const T*>(state);
    switch (ncomp) {
        case 1: dense_totals_partial_kernel<T, 1><<<nblocks, 256, 0, s>>>(p, ncell, soa, partials); break;
        case 2: dense_totals_partial_kernel<T, 2><<<nblocks, 256, 0, s>>>(p, ncell, soa, partials); break;
        case 3: dense_totals_partial_kernel<T, 3><<<nblocks, 256, 0, s>>>(p, ncell, soa, partials); break;
        case 4: dense_totals_partial_kernel<T, 4><<<nblocks, 256, 0, s>>>(p, ncell, soa, partials); break;
        default: dense_totals_partial_kernel<T, 5><<<nblocks, 256, 0, s>>>(p, ncell, soa, partials); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dense_totals_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, ncomp, out);
    return cudaGetLastError();
}

}  // namespace ripple

using namespace ripple;

extern "C" ripple_status ripple_totals_noalloc(const void* state, int ndim, const int64_t* dims, int ncomp,
                                               ripple_layout layout, ripple_dtype dtype, double* totals_out,
                                               void* cuda_stream)
{
    if (!state || !dims || !totals_out) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    if (ndim < 1 || ndim > 3) return fail(RIPPLE_ERR_INVALID, "ndim must be 1..3");
    if (ncomp < 1 || ncomp > 5) return fail(RIPPLE_ERR_INVALID, "ncomp must be 1..5");
    if (layout != RIPPLE_AOS && layout != RIPPLE_SOA) return fail(RIPPLE_ERR_INVALID, "bad layout");
    if (dtype != RIPPLE_F32 && dtype != RIPPLE_F64) return fail(RIPPLE_ERR_INVALID, "bad dtype");
    long long ncell = 1;
    for (int d = 0; d < ndim; ++d) {
        if (dims[d] < 1) return fail(RIPPLE_ERR_INVALID, "dims must be >= 1");
        if (dims[d] > kNoallocMaxCells || ncell > kNoallocMaxCells / dims[d])
            return fail(RIPPLE_ERR_INVALID, "array has more than 33554432 cells, the limit of the fixed scratch "
                                            "of ripple_totals_noalloc");
        ncell *= dims[d];
    }
    double* partials = nullptr;
    ripple_status st = scratch_address(&partials);
    if (st != RIPPLE_OK) return st;
    const int nblocks = (int)((ncell + kCellsPerBlock - 1) / kCellsPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int soa = layout == RIPPLE_SOA;
    cudaError_t e = dtype == RIPPLE_F32
                        ? launch_dense_totals<float>(state, ncell, ncomp, soa, partials, nblocks, totals_out, s)
                        : launch_dense_totals<double>(state, ncell, ncomp, soa, partials, nblocks, totals_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "ripple_totals_noalloc launch");
    return RIPPLE_OK;
}
