// Layout microbenchmarks of the paper's Section 7.1 (SAXPY, Table saxpy) and
// Section 7.2 (three-dimensional particle update, Table particle_update):
// streaming kernels that calibrate the HBM roofline of this part and the cost
// of the two layouts of Section 4.2 ("strided" = SoA, "contiguous" = AoS),
// read straight from global memory or staged through shared memory.
//
// SAXPY:            y <- a x + y                       (12 bytes per element)
// particle update:  x_d <- x_d + v_d dt, d = 0, 1, 2   (24 bytes read, 12 written
//                   per particle; AoS writes back whole 24-byte records)
//
// Direct kernels use 16-byte vector loads/stores with streaming cache hints,
// several vectors in flight per thread, and a grid of whole waves on every SM.
// Staged kernels are the paper's shared-memory variants ("ss", "cs") done the
// way this part allows: bulk asynchronous copies (cp.async.bulk, completion on
// an mbarrier) into a double-buffered shared-memory chunk, the update in
// shared memory, and a bulk asynchronous store back, so the data never passes
// through registers on its way in or out.
#include <cstdint>

#include "runtime.h"
#include "tma.cuh"

namespace ripple {

// Set by a staged kernel whose bounded wait ran out; read (and cleared) by
// ripple_ctx_sync through layout_bench_take_error().
__device__ unsigned g_layout_err = 0u;

__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y)
{
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// y <- a x + y.  Elements [0, head) and [head + 4 n4, n) are scalar (they make
// the vector part start on a 16-byte boundary); the rest is float4.
__global__ void __launch_bounds__(256) saxpy_kernel(long long n, int head, long long n4, float a,
                                                    const float* __restrict__ x, float* __restrict__ y)
{
    constexpr int U = 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const float4* __restrict__ x4 = reinterpret_cast<const float4*>(x + head);
    float4* __restrict__ y4 = reinterpret_cast<float4*>(y + head);
    long long i = t;
    for (; i + (U - 1) * stride < n4; i += U * stride) {
        float4 xv[U], yv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xv[u] = __ldcs(x4 + i + u * stride);
            yv[u] = __ldcs(y4 + i + u * stride);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) __stcs(y4 + i + u * stride, fma4(a, xv[u], yv[u]));
    }
    for (; i < n4; i += stride) __stcs(y4 + i, fma4(a, __ldcs(x4 + i), __ldcs(y4 + i)));
    // scalar head and tail (the whole range when x and y share no 16-byte alignment)
    const long long tail0 = head + 4 * n4;
    if (t < head) y[t] = fmaf(a, x[t], y[t]);
    for (long long e = tail0 + t; e < n; e += stride) y[e] = fmaf(a, x[e], y[e]);
}

// Particle update, SoA ("strided"): p = [x0[n] x1[n] x2[n] v0[n] v1[n] v2[n]].
// vec: every component array starts on a 16-byte boundary and n % 4 == 0.
__global__ void __launch_bounds__(256) particle_soa_kernel(long long n, float dt, float* __restrict__ p, int vec)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (vec) {
        const long long n4 = n / 4;
        for (long long i = t; i < n4; i += stride) {
            float4 xv[3], vv[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                xv[d] = __ldcs(reinterpret_cast<const float4*>(p + d * n) + i);
                vv[d] = __ldcs(reinterpret_cast<const float4*>(p + (3 + d) * n) + i);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) __stcs(reinterpret_cast<float4*>(p + d * n) + i, fma4(dt, vv[d], xv[d]));
        }
    } else {
        for (long long i = t; i < n; i += stride)
#pragma unroll
            for (int d = 0; d < 3; ++d) p[d * n + i] = fmaf(dt, p[(3 + d) * n + i], p[d * n + i]);
    }
}

// Particle update, AoS ("contiguous"): record r = p[6r .. 6r+5] = (x0 x1 x2 v0 v1 v2).
// vec: p starts on a 16-byte boundary; two records (48 bytes) per float4 triple.
__global__ void __launch_bounds__(256) particle_aos_kernel(long long n, float dt, float* __restrict__ p, int vec)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long npair = n / 2;
        float4* __restrict__ q = reinterpret_cast<float4*>(p);
        for (long long i = t; i < npair; i += stride) {
            float4 a = __ldcs(q + 3 * i), b = __ldcs(q + 3 * i + 1), c = __ldcs(q + 3 * i + 2);
            // record 2i: a.x a.y a.z | a.w b.x b.y ; record 2i+1: b.z b.w c.x | c.y c.z c.w
            a.x = fmaf(dt, a.w, a.x);
            a.y = fmaf(dt, b.x, a.y);
            a.z = fmaf(dt, b.y, a.z);
            b.z = fmaf(dt, c.y, b.z);
            b.w = fmaf(dt, c.z, b.w);
            c.x = fmaf(dt, c.w, c.x);
            __stcs(q + 3 * i, a);
            __stcs(q + 3 * i + 1, b);
            __stcs(q + 3 * i + 2, c);
        }
        done = 2 * npair;
    }
    for (long long r = done + t; r < n; r += stride)
#pragma unroll
        for (int d = 0; d < 3; ++d) p[6 * r + d] = fmaf(dt, p[6 * r + 3 + d], p[6 * r + d]);
}

// Staged particle update: chunks of CH particles pass through a double-
// buffered shared-memory stage by bulk copies.  SoA chunk = 6 component runs of
// CH floats (the three positions are stored back); AoS chunk = CH records
// (stored back whole).  Requires 16-byte aligned runs and copy sizes
// (p aligned; n % 4 == 0 for SoA, n % 2 == 0 for AoS).
template <int LAYOUT>
__global__ void __launch_bounds__(256) particle_staged_kernel(long long n, float dt, float* __restrict__ p)
{
    constexpr int CH = 2048;                   // particles per chunk
    constexpr int CHUNK_FLOATS = 6 * CH;       // 48 KB
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    float* stage = reinterpret_cast<float*>(smem + 128);
    const long long nchunks = (n + CH - 1) / CH;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto count_of = [&](long long c) -> int { return (int)min((long long)CH, n - c * CH); };
    auto issue = [&](long long c, int b) {
        const int cnt = count_of(c);
        float* dst = stage + b * CHUNK_FLOATS;
        const uint32_t bytes = (uint32_t)cnt * 4u;
        mbar_arrive_expect_tx(&bars[b], 6u * bytes);
        if (LAYOUT == LAYOUT_SOA) {
            for (int d = 0; d < 6; ++d) bulk_load(dst + d * CH, p + d * n + c * CH, bytes, &bars[b]);
        } else {
            bulk_load(dst, p + 6 * c * CH, 6u * bytes, &bars[b]);
        }
    };
    bool ok = true;
    long long c = blockIdx.x;
    int k = 0;
    if (tid == 0 && c < nchunks) issue(c, 0);
    for (; c < nchunks; c += gridDim.x, ++k) {
        const int b = k & 1;
        const long long cn = c + gridDim.x;
        if (tid == 0 && cn < nchunks) {
            bulk_wait_read<0>();  // the other buffer's store has finished reading it
            issue(cn, b ^ 1);
        }
        if (!mbar_wait_bounded(&bars[b], (uint32_t)((k >> 1) & 1))) ok = false;
        const int cnt = count_of(c);
        float* s = stage + b * CHUNK_FLOATS;
        if (ok) {
            if (LAYOUT == LAYOUT_SOA) {
                for (int j = tid; j < cnt; j += blockDim.x)
#pragma unroll
                    for (int d = 0; d < 3; ++d) s[d * CH + j] = fmaf(dt, s[(3 + d) * CH + j], s[d * CH + j]);
            } else {
                for (int j = tid; j < cnt; j += blockDim.x)
#pragma unroll
                    for (int d = 0; d < 3; ++d) s[6 * j + d] = fmaf(dt, s[6 * j + 3 + d], s[6 * j + d]);
            }
        }
        fence_proxy_async_smem();
        const int any_fail = __syncthreads_or(ok ? 0 : 1);
        if (any_fail) {
            if (tid == 0) atomicOr(&g_layout_err, 1u);
            break;
        }
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)cnt * 4u;
            if (LAYOUT == LAYOUT_SOA) {
                for (int d = 0; d < 3; ++d) bulk_store(p + d * n + c * CH, s + d * CH, bytes);
            } else {
                bulk_store(p + 6 * c * CH, s, 6u * bytes);
            }
            bulk_commit();
        }
    }
    if (tid == 0) {
        bulk_wait<0>();
        if (c < nchunks) {
            // stopped after a failed wait: the loads still in flight (this chunk's,
            // and the next one's if it was issued) complete before the CTA exits
            mbar_wait_bounded(&bars[k & 1], (uint32_t)((k >> 1) & 1));
            if (c + gridDim.x < nchunks) mbar_wait_bounded(&bars[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1));
        }
    }
}

constexpr int kStagedSmem = 128 + 2 * 6 * 2048 * 4;

unsigned layout_bench_take_error(cudaStream_t s)
{
    unsigned h = 0u, z = 0u;
    if (cudaMemcpyFromSymbolAsync(&h, g_layout_err, sizeof(h), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 0u;
    cudaMemcpyToSymbolAsync(g_layout_err, &z, sizeof(z), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return h;
}

}  // namespace ripple

using namespace ripple;

extern "C" {

RIPPLE_API ripple_status ripple_saxpy(ripple_ctx ctx, int64_t n, float a, const float* x, float* y)
{
    if (!ctx || n < 0 || (n > 0 && (!x || !y))) return fail(RIPPLE_ERR_INVALID, "bad saxpy arguments");
    if (n == 0) return RIPPLE_OK;
    const uintptr_t ax = reinterpret_cast<uintptr_t>(x), ay = reinterpret_cast<uintptr_t>(y);
    if (ax % 4 || ay % 4) return fail(RIPPLE_ERR_INVALID, "x and y must be 4-byte aligned floats");
    int head = 0;
    long long n4 = 0;
    if (ax % 16 == ay % 16) {  // a common 16-byte alignment: scalar head, float4 body, scalar tail
        head = (int)std::min<int64_t>(n, (int64_t)(((16 - ax % 16) % 16) / 4));
        n4 = (n - head) / 4;
    }
    const long long units = n4 > 0 ? n4 : n;
    const int grid = (int)std::min<long long>((units + 255) / 256, 8LL * ctx->sm_count);
    saxpy_kernel<<<grid, 256, 0, ctx->stream>>>(n, head, n4, a, x, y);
    RIPPLE_CUDA(cudaGetLastError());
    return RIPPLE_OK;
}

RIPPLE_API ripple_status ripple_particle_update(ripple_ctx ctx, int64_t n, float dt, float* particles,
                                                ripple_layout layout, int staged)
{
    if (!ctx || n < 0 || (n > 0 && !particles)) return fail(RIPPLE_ERR_INVALID, "bad particle arguments");
    if (layout != RIPPLE_AOS && layout != RIPPLE_SOA) return fail(RIPPLE_ERR_INVALID, "bad layout");
    if (n == 0) return RIPPLE_OK;
    const uintptr_t ap = reinterpret_cast<uintptr_t>(particles);
    if (ap % 4) return fail(RIPPLE_ERR_INVALID, "particles must be 4-byte aligned floats");
    const bool soa = layout == RIPPLE_SOA;
    const bool aligned = ap % 16 == 0 && (soa ? n % 4 == 0 : n % 2 == 0);
    if (staged && aligned) {
        static bool configured[2] = {false, false};
        auto k = soa ? particle_staged_kernel<LAYOUT_SOA> : particle_staged_kernel<LAYOUT_AOS>;
        if (!configured[soa ? 1 : 0]) {
            RIPPLE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmem));
            configured[soa ? 1 : 0] = true;
        }
        const long long nchunks = (n + 2047) / 2048;
        const int grid = (int)std::min<long long>(nchunks, 2LL * ctx->sm_count);
        k<<<grid, 256, kStagedSmem, ctx->stream>>>(n, dt, particles);
    } else {
        const int grid = (int)std::min<long long>((n + 255) / 256, 8LL * ctx->sm_count);
        if (soa) particle_soa_kernel<<<grid, 256, 0, ctx->stream>>>(n, dt, particles, aligned ? 1 : 0);
        else particle_aos_kernel<<<grid, 256, 0, ctx->stream>>>(n, dt, particles, ap % 16 == 0 ? 1 : 0);
    }
    RIPPLE_CUDA(cudaGetLastError());
    return RIPPLE_OK;
}

}  // extern "C"
