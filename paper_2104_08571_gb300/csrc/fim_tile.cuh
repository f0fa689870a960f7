// One visit of one Fast Iterative Method tile (Section 7.4 benchmark; block
// FIM of Jeong & Whitaker), shared by the persistent single-problem solver
// and the batched iteration kernel of the serving runtime.
//
// Which tiles iteration k visits, and which buffer each tile lives in, is the
// business of a bookkeeping policy (per-tile flags or lists of active tiles,
// below).  An active tile is staged in shared memory (its interior from the buffer it
// lives in, the faces of its neighbours from theirs), relaxed by synchronous
// Jacobi sweeps of T <- min(T, G(T)) until no cell moves by tol, and written to
// its other buffer; a tile that did not converge stays active and a boundary
// layer that moved by tol or more activates the neighbour across that face.
#pragma once
#include <cstdint>

#include "field.cuh"

namespace ripple {

constexpr int kMaxSources = 16;

template <typename T>
__device__ __forceinline__ T ldcg_t(const T* p);
template <>
__device__ __forceinline__ float ldcg_t<float>(const float* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ double ldcg_t<double>(const double* p) { return __ldcg(p); }

__device__ __forceinline__ float inf_t(float) { return __int_as_float(0x7f800000); }
__device__ __forceinline__ double inf_t(double) { return __longlong_as_double(0x7ff0000000000000ll); }

// Square root of the local solver: FP32 uses the hardware approximation
// (relative error about 2^-22, far inside the FP32 bar against Fast Marching);
// FP64 keeps the correctly rounded square root.
__device__ __forceinline__ float fim_sqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double fim_sqrt(double x) { return sqrt(x); }

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
        return T(0.5) * (a0 + a1 + fim_sqrt(T(2) * f * f - d * d));
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
        t = T(0.5) * (x + y + fim_sqrt(T(2) * f * f - d * d));
        if (!(t > z)) return t;
        // three terms: 3T^2 - 2 S T + (Q - f^2) = 0.  Its discriminant
        // S^2 - 3 (Q - f^2) equals 3 f^2 - sum of squared pairwise differences;
        // the second form has no cancellation between terms of size T^2
        // (which in FP32 would swamp f^2 on fine grids).
        const T dxy = x - y, dxz = x - z, dyz = y - z;
        const T disc = fmax(T(3) * f * f - (dxy * dxy + dxz * dxz + dyz * dyz), T(0));
        return (x + y + z + fim_sqrt(disc)) * (T(1) / T(3));
    }
}

template <int DIM>
struct EikTile {
    static constexpr int TS = DIM == 2 ? 32 : 8;
    // threads per tile: a tile visit is a chain of Jacobi sweeps, so more threads
    // per 32 x 32 tile (two cells each) shorten every sweep; 8^3 tiles keep 256
    static constexpr int NT = DIM == 2 ? 512 : 256;
    static constexpr int CELLS = DIM == 2 ? TS * TS : TS * TS * TS;
    static constexpr int CPT = CELLS / NT;  // cells per thread
    static constexpr int P = TS + 2;        // padded tile side
    static constexpr int PCELLS = DIM == 2 ? P * P : P * P * P;
    static constexpr int MAX_SWEEPS = 2 * TS * (DIM == 3 ? 3 : 1);
};


// Per-problem state of the FIM iteration.  Two bookkeeping schemes use it:
//   flags (the batched runtime): act[3][ntiles] active flags and cur[2][ntiles]
//     buffer indices, every tile touched by every iteration;
//   lists (the single-problem solver): list[3][ntiles] of the tiles active in
//     each iteration (count[] of them, handed out through take[]), a packed
//     word per tile state[t] = ((k + 1) << 1) | buffer, where k is the last
//     iteration that visited the tile, and mark[t] = 1 + the last iteration
//     the tile was queued for (so a tile enters a list once).
template <typename T>
struct FimProblem {
    T* buf[2];         // the two buffers of the T field
    const T* slow;     // slowness field
    FieldGeom gT, gS;
    int ntx, nty, ntz, ntiles;
    int nsrc;
    int src[kMaxSources][3];
    double h, tol;
    unsigned* act;       // flags: [3][ntiles]
    unsigned char* cur;  // flags: [2][ntiles]
    unsigned* count;     // [3]: tiles activated for each iteration
    int* list;           // lists: [3][ntiles]
    unsigned* state;     // lists: [ntiles]
    unsigned* mark;      // lists: [ntiles]
    unsigned* take;      // lists: [3] next list entry to hand out
};

// Bookkeeping with per-tile flags: every tile is visited (cheaply, if
// inactive) by every iteration, which clears its flag of iteration k + 2 and
// carries its buffer index to iteration k + 1.
template <typename T>
struct FimFlagBook {
    const FimProblem<T>& a;
    long long k;
    __device__ unsigned char buf_of(int t) const { return __ldcg(&a.cur[(size_t)(k % 2) * a.ntiles + t]); }
    __device__ bool begin(int t, unsigned char& cb) const
    {
        const unsigned is_active = __ldcg(&a.act[(size_t)(k % 3) * a.ntiles + t]);
        cb = buf_of(t);
        if (threadIdx.x == 0) {
            a.act[(size_t)((k + 2) % 3) * a.ntiles + t] = 0u;
            a.cur[(size_t)((k + 1) % 2) * a.ntiles + t] = is_active ? (unsigned char)(1 - cb) : cb;
        }
        return is_active != 0u;
    }
    __device__ void activate(int nb) const
    {
        if (atomicExch(&a.act[(size_t)((k + 1) % 3) * a.ntiles + nb], 1u) == 0u) atomicAdd(&a.count[(k + 1) % 3], 1u);
    }
};

// Bookkeeping with lists of active tiles: only listed tiles are visited.  A
// visit of iteration k moves the tile to its other buffer; readers in the same
// iteration still see the old one ((state >> 1) == k + 1 means "moved in this
// iteration"), readers of later iterations the new one.
template <typename T>
struct FimListBook {
    const FimProblem<T>& a;
    long long k;
    __device__ unsigned char buf_of(int t) const
    {
        const unsigned w = __ldcg(&a.state[t]);
        const unsigned char b = (unsigned char)(w & 1u);
        return (w >> 1) == (unsigned)(k + 1) ? (unsigned char)(b ^ 1u) : b;
    }
    __device__ bool begin(int t, unsigned char& cb) const
    {
        cb = buf_of(t);
        __syncthreads();  // every thread has its buffer index before the word changes
        if (threadIdx.x == 0) a.state[t] = ((unsigned)(k + 1) << 1) | (unsigned)(1 - cb);
        return true;
    }
    __device__ void activate(int nb) const
    {
        const unsigned want = (unsigned)(k + 2);
        if (atomicMax(&a.mark[nb], want) < want) {
            const unsigned pos = atomicAdd(&a.count[(k + 1) % 3], 1u);
            a.list[(size_t)((k + 1) % 3) * a.ntiles + pos] = nb;
        }
    }
};

template <typename T, int DIM>
struct FimSmem {
    T sa[EikTile<DIM>::PCELLS];
    T sb[EikTile<DIM>::PCELLS];
    unsigned side_mask;
};

// Visit tile t of problem `a` in iteration k (all threads of the CTA call it)
// with the bookkeeping `book` (FimFlagBook or FimListBook).  Adds one tile
// visit and the Godunov updates performed to the counters.
template <typename T, int DIM, class Book>
__device__ __forceinline__ void fim_visit_tile(FimSmem<T, DIM>& sm, const FimProblem<T>& a, int t, long long k,
                                               long long& visits, long long& updates, const Book& book)
{
    using C = EikTile<DIM>;
    constexpr int TS = C::TS, P = C::P, CPT = C::CPT;
    const int tid = threadIdx.x;
    const T INF = inf_t(T(0));
    const T tol = (T)a.tol;
    const FieldGeom& gT = a.gT;
    const FieldGeom& gS = a.gS;
    T* sa = sm.sa;
    T* sb = sm.sb;

    auto cell_xyz = [&](int c, int& x, int& y, int& z) {  // thread cell c: linear cell tid + c * NT
        const int lin = tid + c * C::NT;
        x = lin % TS;
        y = (lin / TS) % TS;
        z = DIM == 3 ? lin / (TS * TS) : 0;
    };
    auto pidx = [&](int x, int y, int z) -> int {  // padded smem index, x,y,z in [-1, TS]
        return DIM == 2 ? (y + 1) * P + (x + 1) : ((z + 1) * P + (y + 1)) * P + (x + 1);
    };

    unsigned char cb;
    if (!book.begin(t, cb)) return;
    ++visits;
    const int bx = t % a.ntx, by = (t / a.ntx) % a.nty, bz = DIM == 3 ? t / (a.ntx * a.nty) : 0;
    const int x0 = bx * TS, y0 = by * TS, z0 = bz * TS;
    const T* src_buf = a.buf[cb];
    T* dst_buf = a.buf[1 - cb];

    // ---- stage the tile: interior from this tile's buffer, faces from the neighbours' ----
    for (int i = tid; i < C::PCELLS; i += C::NT) { sa[i] = INF; sb[i] = INF; }
    __syncthreads();
    T init[CPT], fh[CPT];
    bool fixed[CPT];
    int cid[CPT];  // padded shared-memory index of each of this thread's cells
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        int x, y, z;
        cell_xyz(c, x, y, z);
        const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
        const bool valid = gx < gT.n[0] && gy < gT.n[1] && gz < gT.n[2];
        T v = INF;
        bool src = false;
        fh[c] = T(0);
        cid[c] = pidx(x, y, z);
        if (valid) {
            v = ldcg_t(&src_buf[geom_cell(gT, gx, gy, gz)]);
            fh[c] = a.slow[geom_cell(gS, gx, gy, gz) * gS.cell_stride] * (T)a.h;
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
            v = ldcg_t(&a.buf[book.buf_of(nb)][geom_cell(gT, gx, gy, gz)]);
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
            const int id = cid[c];
            const T old = A[id];
            const T ax = fmin(A[id - 1], A[id + 1]);
            const T ay = fmin(A[id - P], A[id + P]);
            const T az = DIM == 3 ? fmin(A[id - P * P], A[id + P * P]) : INF;
            const T g = godunov<T, DIM>(ax, ay, az, fh[c]);
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
    if (tid == 0) sm.side_mask = 0u;
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
    if (mask) atomicOr(&sm.side_mask, mask);
    __syncthreads();
    if (tid == 0) {
        auto activate = [&](int nb) { book.activate(nb); };
        if (!converged) activate(t);
        const unsigned m = sm.side_mask;
        if ((m & 1u) && bx > 0) activate(t - 1);
        if ((m & 2u) && bx + 1 < a.ntx) activate(t + 1);
        if ((m & 4u) && by > 0) activate(t - a.ntx);
        if ((m & 8u) && by + 1 < a.nty) activate(t + a.ntx);
        if (DIM == 3 && (m & 16u) && bz > 0) activate(t - a.ntx * a.nty);
        if (DIM == 3 && (m & 32u) && bz + 1 < a.ntz) activate(t + a.ntx * a.nty);
    }
    __syncthreads();
}

}  // namespace ripple
