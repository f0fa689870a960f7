// Fast Iterative Method eikonal solver (the paper's Section 7.4 benchmark,
// Jeong & Whitaker's block FIM) for |grad T| s = 1 on a Cartesian grid.
//
// Design (GB300-native, single persistent cooperative launch):
//   * the grid is cut into tiles (32 x 32 in 2D, 8 x 8 x 8 in 3D); an active
//     tile is relaxed in shared memory with its ghost faces (cross stencil,
//     no corners) by synchronous Jacobi sweeps of the Godunov upwind update
//     T <- min(T, G(T)) until no cell moves by tol or more (or 2 x tile
//     width sweeps);
//   * tiles are double-buffered across the two buffers of the T field: an
//     active tile reads its interior and its neighbours' faces from the
//     buffer each tile currently lives in and writes the other one, so reads
//     and writes of an iteration never overlap and the result does not depend
//     on scheduling (deterministic);
//   * active-list update: a tile that did not converge stays active; a tile
//     whose boundary layer moved by tol or more activates the neighbour
//     across that face;
//   * iterations are separated by a bounded grid barrier (co-residency from
//     the cooperative launch); the run ends when no tile is active, or with
//     DEV_ERR_TIMEOUT when the iteration cap is reached.
// Outside-domain neighbours are +inf; sources stay at 0.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "runtime.h"

namespace ripple {

constexpr int kMaxSources = 16;
constexpr uint32_t kGridSpinLimit = 1u << 26;

struct EikArgs {
    int ntx, nty, ntz, ntiles;
    int nsrc;
    int src[kMaxSources][3];
    double h, tol;
    long long max_iters;
    unsigned* act;         // [3][ntiles]
    unsigned char* cur;    // [2][ntiles]
    unsigned* count;       // [3]
    unsigned* bar;         // [2] grid barrier: arrivals, generation
    FieldCtl* ctl;
};

struct EikScratch {
    size_t bytes = 0;
    void* mem = nullptr;
    int ntiles = 0;
};

template <typename T>
__device__ __forceinline__ T ldcg_t(const T* p);
template <>
__device__ __forceinline__ float ldcg_t<float>(const float* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ double ldcg_t<double>(const double* p) { return __ldcg(p); }

__device__ __forceinline__ float inf_t(float) { return __int_as_float(0x7f800000); }
__device__ __forceinline__ double inf_t(double) { return __longlong_as_double(0x7ff0000000000000ll); }

// Godunov upwind local solver: a[d] = smaller neighbour value along axis d,
// f = s * h.  2D: one-sided if |a0 - a1| >= f, else the two-sided root.
// 3D: sorted a1 <= a2 <= a3, add terms while the candidate exceeds the next.
template <typename T, int DIM>
__device__ __forceinline__ T godunov(T a0, T a1, T a2, T f)
{
    if (DIM == 2) {
        const T lo = fmin(a0, a1);
        const T d = a0 - a1;
        if (!(fabs(d) < f)) return lo + f;
        return T(0.5) * (a0 + a1 + sqrt(T(2) * f * f - d * d));
    } else {
        // sort ascending
        T x = fmin(a0, a1), y = fmax(a0, a1);
        T z = fmax(y, a2);
        y = fmin(y, a2);
        const T x2 = fmin(x, y);
        y = fmax(x, y);
        x = x2;
        T t = x + f;
        if (!(t > y)) return t;
        const T d = x - y;
        t = T(0.5) * (x + y + sqrt(T(2) * f * f - d * d));
        if (!(t > z)) return t;
        // three terms: 3T^2 - 2 S T + (Q - f^2) = 0.  Its discriminant
        // S^2 - 3 (Q - f^2) equals 3 f^2 - sum of squared pairwise differences;
        // the second form has no cancellation between terms of size T^2
        // (which in FP32 would swamp f^2 on fine grids).
        const T dxy = x - y, dxz = x - z, dyz = y - z;
        const T disc = fmax(T(3) * f * f - (dxy * dxy + dxz * dxz + dyz * dyz), T(0));
        return (x + y + z + sqrt(disc)) * (T(1) / T(3));
    }
}

// Bounded sense-reversal grid barrier.  Returns false if the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* sflag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            uint32_t i = 0;
            while (*gen == g0 && ++i < kGridSpinLimit) __nanosleep(32);
            if (i >= kGridSpinLimit) sflag[0] = 1;
        }
        __threadfence();
    }
    __syncthreads();
    return sflag[0] == 0;
}

template <int DIM>
struct EikTile {
    static constexpr int TS = DIM == 2 ? 32 : 8;
    static constexpr int NT = 256;
    static constexpr int CELLS = DIM == 2 ? TS * TS : TS * TS * TS;
    static constexpr int CPT = CELLS / NT;  // cells per thread
    static constexpr int P = TS + 2;        // padded tile side
    static constexpr int PCELLS = DIM == 2 ? P * P : P * P * P;
    static constexpr int MAX_SWEEPS = 2 * TS * (DIM == 3 ? 3 : 1);
};

template <typename T, int DIM>
__global__ void __launch_bounds__(256) fim_kernel(T* __restrict__ buf0, T* __restrict__ buf1,
                                                  const T* __restrict__ slow, const FieldGeom gT,
                                                  const FieldGeom gS, const EikArgs a)
{
    using C = EikTile<DIM>;
    constexpr int TS = C::TS, P = C::P, CPT = C::CPT;
    __shared__ T sa[C::PCELLS];
    __shared__ T sb[C::PCELLS];
    __shared__ T sf[C::CELLS];
    __shared__ int sflag[2];
    __shared__ unsigned side_mask;

    const int tid = threadIdx.x;
    const T INF = inf_t(T(0));
    const T tol = (T)a.tol;
    T* bufs[2] = {buf0, buf1};
    if (tid == 0) sflag[0] = 0;
    __syncthreads();

    long long visits = 0, updates = 0;
    long long k = 0;
    bool timed_out = false;

    // local (tile) index of thread cell c: linear cell = tid + c * NT
    auto cell_xyz = [&](int c, int& x, int& y, int& z) {
        const int lin = tid + c * C::NT;
        x = lin % TS;
        y = (lin / TS) % TS;
        z = DIM == 3 ? lin / (TS * TS) : 0;
    };
    auto pidx = [&](int x, int y, int z) -> int {  // padded smem index, x,y,z in [-1, TS]
        return DIM == 2 ? (y + 1) * P + (x + 1) : ((z + 1) * P + (y + 1)) * P + (x + 1);
    };

    for (;;) {
        const unsigned* act = a.act + (size_t)(k % 3) * a.ntiles;
        unsigned* act_next = a.act + (size_t)((k + 1) % 3) * a.ntiles;
        unsigned* act_clear = a.act + (size_t)((k + 2) % 3) * a.ntiles;
        const unsigned char* cur = a.cur + (size_t)(k % 2) * a.ntiles;
        unsigned char* cur_next = a.cur + (size_t)((k + 1) % 2) * a.ntiles;
        if (blockIdx.x == 0 && tid == 0) a.count[(k + 2) % 3] = 0u;

        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            const unsigned is_active = __ldcg(&act[t]);
            const unsigned char cb = __ldcg(&cur[t]);
            if (tid == 0) {
                act_clear[t] = 0u;
                cur_next[t] = is_active ? (unsigned char)(1 - cb) : cb;
            }
            if (!is_active) continue;
            ++visits;
            const int bx = t % a.ntx, by = (t / a.ntx) % a.nty, bz = DIM == 3 ? t / (a.ntx * a.nty) : 0;
            const int x0 = bx * TS, y0 = by * TS, z0 = bz * TS;
            const T* src_buf = bufs[cb];
            T* dst_buf = bufs[1 - cb];

            // ---- stage the tile: interior from this tile's buffer, faces from the neighbours' ----
            for (int i = tid; i < C::PCELLS; i += C::NT) { sa[i] = INF; sb[i] = INF; }
            __syncthreads();
            T init[CPT];
            bool fixed[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                int x, y, z;
                cell_xyz(c, x, y, z);
                const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
                const bool valid = gx < gT.n[0] && gy < gT.n[1] && gz < gT.n[2];
                T v = INF;
                bool src = false;
                if (valid) {
                    v = ldcg_t(&src_buf[geom_cell(gT, gx, gy, gz)]);
                    sf[tid + c * C::NT] = slow[geom_cell(gS, gx, gy, gz) * gS.cell_stride] * (T)a.h;
                    for (int q = 0; q < a.nsrc; ++q)
                        src |= (a.src[q][0] == gx) & (a.src[q][1] == gy) & (DIM == 2 || a.src[q][2] == gz);
                }
                init[c] = v;
                fixed[c] = !valid || src;
                sa[pidx(x, y, z)] = v;
                sb[pidx(x, y, z)] = v;
            }
            // ghost faces: 2*DIM faces of TS^(DIM-1) cells
            constexpr int FACE = DIM == 2 ? TS : TS * TS;
            for (int i = tid; i < 2 * DIM * FACE; i += C::NT) {
                const int face = i / FACE, r = i % FACE;
                const int axis = face >> 1, side = face & 1;
                int u = r % TS, w = r / TS;  // in-face coordinates
                int lx, ly, lz;
                if (axis == 0) { lx = side ? TS : -1; ly = u; lz = w; }
                else if (axis == 1) { lx = u; ly = side ? TS : -1; lz = w; }
                else { lx = u; ly = w; lz = side ? TS : -1; }
                if (DIM == 2) lz = 0;
                const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
                T v = INF;
                if (gx >= 0 && gy >= 0 && gz >= 0 && gx < gT.n[0] && gy < gT.n[1] && gz < gT.n[2]) {
                    const int nbx = gx / TS, nby = gy / TS, nbz = gz / TS;
                    const int nb = DIM == 2 ? nby * a.ntx + nbx : (nbz * a.nty + nby) * a.ntx + nbx;
                    const unsigned char nbc = __ldcg(&cur[nb]);
                    v = ldcg_t(&bufs[nbc][geom_cell(gT, gx, gy, gz)]);
                }
                sa[pidx(lx, ly, lz)] = v;
                sb[pidx(lx, ly, lz)] = v;
            }
            __syncthreads();

            // ---- Jacobi sweeps in shared memory ----
            T* A = sa;
            T* B = sb;
            bool converged = false;
            int sweeps = 0;
            for (; sweeps < C::MAX_SWEEPS; ++sweeps) {
                bool moved = false;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    if (fixed[c]) continue;
                    int x, y, z;
                    cell_xyz(c, x, y, z);
                    const int id = pidx(x, y, z);
                    const T old = A[id];
                    const T ax = fmin(A[id - 1], A[id + 1]);
                    const T ay = fmin(A[id - P], A[id + P]);
                    const T az = DIM == 3 ? fmin(A[id - P * P], A[id + P * P]) : INF;
                    const T g = godunov<T, DIM>(ax, ay, az, sf[tid + c * C::NT]);
                    const T nv = fmin(old, g);
                    B[id] = nv;
                    moved |= (old - nv) >= tol;
                }
                const int any = __syncthreads_or(moved ? 1 : 0);
                T* tmp = A;
                A = B;
                B = tmp;
                if (!any) {
                    converged = true;
                    ++sweeps;
                    break;
                }
            }
            updates += (long long)sweeps * C::CELLS;

            // ---- write back; boundary-layer changes activate neighbours ----
            if (tid == 0) side_mask = 0u;
            __syncthreads();
            unsigned mask = 0u;
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                int x, y, z;
                cell_xyz(c, x, y, z);
                const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
                const bool valid = gx < gT.n[0] && gy < gT.n[1] && gz < gT.n[2];
                const T v = A[pidx(x, y, z)];
                if (valid) dst_buf[geom_cell(gT, gx, gy, gz)] = v;
                if (valid && (init[c] - v) >= tol) {
                    if (x == 0) mask |= 1u;
                    if (x == TS - 1) mask |= 2u;
                    if (y == 0) mask |= 4u;
                    if (y == TS - 1) mask |= 8u;
                    if (DIM == 3 && z == 0) mask |= 16u;
                    if (DIM == 3 && z == TS - 1) mask |= 32u;
                }
            }
            if (mask) atomicOr(&side_mask, mask);
            __syncthreads();
            if (tid == 0) {
                auto activate = [&](int nb) {
                    if (atomicExch(&act_next[nb], 1u) == 0u) atomicAdd(&a.count[(k + 1) % 3], 1u);
                };
                if (!converged) activate(t);
                const unsigned m = side_mask;
                if ((m & 1u) && bx > 0) activate(t - 1);
                if ((m & 2u) && bx + 1 < a.ntx) activate(t + 1);
                if ((m & 4u) && by > 0) activate(t - a.ntx);
                if ((m & 8u) && by + 1 < a.nty) activate(t + a.ntx);
                if (DIM == 3 && (m & 16u) && bz > 0) activate(t - a.ntx * a.nty);
                if (DIM == 3 && (m & 32u) && bz + 1 < a.ntz) activate(t + a.ntx * a.nty);
            }
            __syncthreads();
        }

        if (!grid_barrier(a.bar, gridDim.x, sflag)) {
            timed_out = true;
            break;
        }
        ++k;
        const unsigned remaining = __ldcg(&a.count[k % 3]);
        if (remaining == 0u) break;
        if (k >= a.max_iters) {
            timed_out = true;
            break;
        }
        // No second barrier: the counter read here, count[k % 3], is next
        // cleared in iteration k + 2, which no CTA starts before every CTA
        // has passed the barrier that ends iteration k + 1.
    }

    if (!timed_out) {
        // consolidate: every tile's current values into buffer 0
        const unsigned char* cur = a.cur + (size_t)(k % 2) * a.ntiles;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            if (__ldcg(&cur[t]) == 0) continue;
            const int bx = t % a.ntx, by = (t / a.ntx) % a.nty, bz = DIM == 3 ? t / (a.ntx * a.nty) : 0;
            for (int c = 0; c < CPT; ++c) {
                int x, y, z;
                cell_xyz(c, x, y, z);
                const int gx = bx * TS + x, gy = by * TS + y, gz = bz * TS + z;
                if (gx < gT.n[0] && gy < gT.n[1] && gz < gT.n[2]) {
                    const long long id = geom_cell(gT, gx, gy, gz);
                    buf0[id] = ldcg_t(&buf1[id]);
                }
            }
        }
    }
    if (tid == 0) {
        atomicAdd((unsigned long long*)&a.ctl->counters[1], (unsigned long long)visits);
        atomicAdd((unsigned long long*)&a.ctl->counters[2], (unsigned long long)updates);
        if (blockIdx.x == 0) a.ctl->counters[0] = k;
        if (timed_out) atomicOr(&a.ctl->err, DEV_ERR_TIMEOUT);
    }
}

// Initialise both buffers (+inf interior, 0 at sources) and the active list.
template <typename T>
__global__ void fim_init_kernel(T* __restrict__ buf0, T* __restrict__ buf1, const FieldGeom g, EikArgs a, int ts)
{
    const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
    const T INF = inf_t(T(0));
    for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
         lin += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(lin % g.n[0]);
        const int j = (int)((lin / g.n[0]) % g.n[1]);
        const int kk = (int)(lin / ((long long)g.n[0] * g.n[1]));
        T v = INF;
        for (int q = 0; q < a.nsrc; ++q)
            if (a.src[q][0] == i && a.src[q][1] == j && (g.ndim == 2 || a.src[q][2] == kk)) v = T(0);
        const long long id = geom_cell(g, i, j, kk);
        buf0[id] = v;
        buf1[id] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned n = 0;
        for (int q = 0; q < a.nsrc; ++q) {
            const int bx = a.src[q][0] / ts, by = a.src[q][1] / ts, bz = g.ndim == 3 ? a.src[q][2] / ts : 0;
            const int t = (bz * a.nty + by) * a.ntx + bx;
            if (a.act[t] == 0u) {
                a.act[t] = 1u;
                ++n;
            }
        }
        a.count[0] = n;
    }
}

void eik_scratch_free_impl(ripple_field f)
{
    if (!f->eik) return;
    ctx_free(f->ctx, f->eik->mem, f->eik->bytes);
    delete f->eik;
    f->eik = nullptr;
}

}  // namespace ripple

using namespace ripple;

void eik_scratch_free(ripple_field f) { eik_scratch_free_impl(f); }

template <typename T, int DIM>
static ripple_status run_fim(ripple_field S, ripple_field Tf, EikArgs& a, int ts)
{
    ripple_ctx ctx = Tf->ctx;
    cudaStream_t s = ctx->stream;
    auto kern = fim_kernel<T, DIM>;
    int per_sm = 0;
    RIPPLE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
    if (per_sm < 1) return fail(RIPPLE_ERR_INTERNAL, "FIM kernel cannot be resident");
    int grid = std::min(per_sm * ctx->sm_count, a.ntiles);
    grid = std::max(grid, 1);
    const long long total = (long long)Tf->geom.n[0] * Tf->geom.n[1] * Tf->geom.n[2];
    int igrid = (int)std::min<long long>((total + 255) / 256, 8LL * ctx->sm_count);
    fim_init_kernel<T><<<igrid, 256, 0, s>>>(static_cast<T*>(Tf->buf[0]), static_cast<T*>(Tf->buf[1]), Tf->geom, a,
                                             ts);
    RIPPLE_CUDA(cudaGetLastError());
    T* b0 = static_cast<T*>(Tf->buf[0]);
    T* b1 = static_cast<T*>(Tf->buf[1]);
    const T* sl = static_cast<const T*>(S->buf[S->cur]);
    FieldGeom gT = Tf->geom, gS = S->geom;
    void* args[] = {&b0, &b1, (void*)&sl, &gT, &gS, &a};
    RIPPLE_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, 0, s));
    Tf->cur = 0;
    return RIPPLE_OK;
}

extern "C" ripple_status ripple_eikonal_solve(ripple_field S, ripple_field Tf, const int64_t* src, int nsrc,
                                              const ripple_eik_params* p, ripple_eik_stats* stats)
{
    if (!S || !Tf || !src || !p) return fail(RIPPLE_ERR_INVALID, "NULL argument");
    if (S->ctx != Tf->ctx) return fail(RIPPLE_ERR_INVALID, "fields of different contexts");
    if (S->ncomp != 1 || Tf->ncomp != 1) return fail(RIPPLE_ERR_INVALID, "eikonal fields have one component");
    if (S->ndim != Tf->ndim || S->dtype != Tf->dtype) return fail(RIPPLE_ERR_INVALID, "field shape/dtype mismatch");
    for (int d = 0; d < 3; ++d)
        if (S->geom.n[d] != Tf->geom.n[d]) return fail(RIPPLE_ERR_INVALID, "field dims differ");
    if (nsrc < 1 || nsrc > kMaxSources) return fail(RIPPLE_ERR_INVALID, "need 1..16 sources");
    if (!(p->h > 0.0) || !(p->tol > 0.0)) return fail(RIPPLE_ERR_INVALID, "need h > 0 and tol > 0");
    const int ndim = Tf->ndim;
    const int ts = ndim == 2 ? EikTile<2>::TS : EikTile<3>::TS;
    EikArgs a{};
    a.ntx = (Tf->geom.n[0] + ts - 1) / ts;
    a.nty = (Tf->geom.n[1] + ts - 1) / ts;
    a.ntz = ndim == 3 ? (Tf->geom.n[2] + ts - 1) / ts : 1;
    a.ntiles = a.ntx * a.nty * a.ntz;
    a.nsrc = nsrc;
    for (int q = 0; q < nsrc; ++q)
        for (int d = 0; d < 3; ++d) {
            const int64_t c = d < ndim ? src[q * ndim + d] : 0;
            if (c < 0 || c >= Tf->geom.n[d]) return fail(RIPPLE_ERR_INVALID, "source outside the grid");
            a.src[q][d] = (int)c;
        }
    a.h = p->h;
    a.tol = p->tol;
    a.max_iters = p->max_iters > 0 ? p->max_iters : 1000000;
    ripple_ctx ctx = Tf->ctx;
    ripple_status st = ensure_second_buffer(Tf);
    if (st != RIPPLE_OK) return st;
    // scratch: act[3][ntiles] u32, cur[2][ntiles] u8, count[3] + barrier[2] u32
    const size_t need = (size_t)a.ntiles * 3 * 4 + (size_t)a.ntiles * 2 + 64;
    if (!Tf->eik || Tf->eik->bytes < need) {
        eik_scratch_free(Tf);
        Tf->eik = new EikScratch();
        st = ctx_alloc(ctx, need, &Tf->eik->mem);
        if (st != RIPPLE_OK) {
            delete Tf->eik;
            Tf->eik = nullptr;
            return st;
        }
        Tf->eik->bytes = need;
        Tf->eik->ntiles = a.ntiles;
    }
    char* base = static_cast<char*>(Tf->eik->mem);
    a.count = reinterpret_cast<unsigned*>(base);
    a.bar = reinterpret_cast<unsigned*>(base + 16);
    a.act = reinterpret_cast<unsigned*>(base + 64);
    a.cur = reinterpret_cast<unsigned char*>(base + 64 + (size_t)a.ntiles * 3 * 4);
    a.ctl = Tf->ctl;
    cudaStream_t s = ctx->stream;
    RIPPLE_CUDA(cudaMemsetAsync(Tf->eik->mem, 0, need, s));
    RIPPLE_CUDA(cudaMemsetAsync(Tf->ctl->counters, 0, sizeof(Tf->ctl->counters), s));
    if (Tf->dtype == RIPPLE_F32)
        st = ndim == 2 ? run_fim<float, 2>(S, Tf, a, ts) : run_fim<float, 3>(S, Tf, a, ts);
    else
        st = ndim == 2 ? run_fim<double, 2>(S, Tf, a, ts) : run_fim<double, 3>(S, Tf, a, ts);
    if (st != RIPPLE_OK) return st;
    FieldCtl host{};
    RIPPLE_CUDA(cudaMemcpyAsync(&host, Tf->ctl, sizeof(FieldCtl), cudaMemcpyDeviceToHost, s));
    RIPPLE_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        stats->iterations = host.counters[0];
        stats->tile_visits = host.counters[1];
        stats->cell_updates = host.counters[2];
    }
    if (host.err) {
        RIPPLE_CUDA(cudaMemsetAsync(&Tf->ctl->err, 0, sizeof(unsigned), s));
        if (host.err & DEV_ERR_TIMEOUT) return fail(RIPPLE_ERR_TIMEOUT, "FIM did not converge within max_iters");
        return fail(RIPPLE_ERR_INTERNAL, "FIM device error");
    }
    return RIPPLE_OK;
}
