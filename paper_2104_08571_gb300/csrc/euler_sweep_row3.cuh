// FP32 3D MUSCL-Hancock sweep with one warp per x-row of the tile, sm_103a.
//
// The same step as the other sweep kernels (one launch = one explicit unsplit
// step, out of place; MUSCL-Hancock states, Rusanov faces each evaluated once,
// fused ghost images, CFL maximum and positivity), with the work of a plane
// laid out so that almost every exchange between cells is a register or a
// warp shuffle instead of a shared-memory round trip:
//
//   * a tile is 64 x 14 cells, streamed along z through a chunk of planes;
//     each plane of the tile plus two ghost cells on every side arrives in
//     shared memory by one TMA load (SoA: all components in one 4-D box; AoS:
//     a view of each row as groups of four 20-byte cells) into a 7-slot ring;
//   * warp w = 1..14 owns row w - 1 of the tile, lane l the cells (2l, 2l+1)
//     as a packed f32x2 pair: it forms the x, y and z predicted states of its
//     own cells, its x faces (l's pair of faces is (2l+1/2, 2l+3/2); the left
//     state of cell 2l+2 comes from lane l+1 and the face 2l-1/2 from lane
//     l-1 by shuffles), the y face below its row, the z face above its plane
//     (the predicted states and the face below are carried in registers from
//     the previous plane) and the update of its two cells;
//   * y faces pass between neighbouring warps through one shared row each:
//     warp w writes the high-side y state of its row (RB[w]) and the face
//     below its row (FB[w]); the warp above reads the first, the warp below
//     the second (mbarriers with 32 arrivals, one phase per plane);
//   * warp 0 (the row below the tile) and warp 15 (the row above) are halo
//     warps.  Warp 15 forms the y state of its row and the face above the
//     tile's last row.  Warp 0 forms the y state of its row and takes the
//     tile-edge x work off the row warps: the face x0 - 1/2 and the left state
//     of cell x0 + 64 of every row.  Its outputs go to four buffers (plane
//     iteration mod 4), each with its own mbarrier (EB), so warp 0 runs up to
//     four planes ahead of the slowest row warp: before it writes the buffers
//     of plane z it waits until every thread has released plane z - 4.  Lane
//     0 of warp 0 also issues the TMA loads;
//   * every face and predicted state is formed by the same packed arithmetic
//     wherever it is needed (interior lanes, tile-edge work of the halo
//     warps, the neighbouring tile), so a face shared by two tiles has the
//     same bits in both, the update telescopes and a uniform state stays
//     bit-exact.  The y predicted states of all 16 warps' rows and the y
//     faces of warps 1 .. 15 run through one copy of that code in the plane
//     loop: the loop body's size sets how often warps stall on instruction
//     fetch (a two-plane unrolled body ran 45 % slower).
//
// Every wait is bounded.  A wait first tests its phase without blocking (the
// common case: the data is there); otherwise it polls with a suspend hint.  A
// wait that runs out sets the CTA's abort flag; later waits then return at
// once, so the CTA finishes its loop (stores stay inside the field) and
// reports DEV_ERR_TIMEOUT.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "euler_sweep.cuh"
#include "pair_math.cuh"

namespace ripple {

template <int LAYOUT>
struct Row3Cfg {
    static constexpr int TX = 64, TY = 14;
    static constexpr int NW = TY + 2;   // warps: halo row below, TY row warps, halo row above
    static constexpr int NT = NW * 32;  // 512 threads
    static constexpr int NC = 5, R = 2;
    static constexpr BoxGeom BOX = plane_box(4, NC, LAYOUT == LAYOUT_AOS, R, TX, TY);
    static constexpr int OFF = BOX.off;
    static constexpr int BX = BOX.bx, BY = BOX.by;  // staged plane: 72 x 18 cells
    static constexpr int NS = 7;                  // ring slots
    static constexpr int SLOT_ELEMS = BX * BY * NC;
    static constexpr int SLOT_BYTES = ((SLOT_ELEMS * 4 + 127) / 128) * 128;
    static constexpr int ROW = NC * TX;           // floats of one exchange row, [m][x]
    static constexpr int NE = 4;                  // buffers of warp 0's outputs (plane iteration mod 4)
    // header: mbarriers, reduction scratch, abort flag, step scalars
    static constexpr int BAR_FULL = 0, BAR_EMPTY = NS, BAR_RB = 2 * NS, BAR_FB = 2 * NS + NW;
    static constexpr int BAR_EB = 2 * NS + 2 * NW;
    static constexpr int NBARS = 2 * NS + 2 * NW + NE;
    static constexpr int OFF_RED = NBARS * 8;
    static constexpr int OFF_FLAG = OFF_RED + NW * 8;
    static constexpr int OFF_SDT = OFF_FLAG + 16;
    static constexpr int HDR = ((OFF_SDT + 16 + 127) / 128) * 128;
    static constexpr int OFF_RING = HDR;
    static constexpr int OFF_RY = OFF_RING + NS * SLOT_BYTES;         // y states of rows 0 .. TY-1 (warps 1 .. TY)
    static constexpr int OFF_FY = OFF_RY + TY * ROW * 4;              // faces 0 .. TY of the tile rows
    static constexpr int OFF_E = OFF_FY + (TY + 1) * ROW * 4;         // warp 0's buffers
    // one buffer of warp 0: y state of row -1 [m][x], faces x0 - 1/2 [row][m], left states of x0 + 64 [row][m]
    static constexpr int E_RY = 0, E_FL = ROW, E_LR = ROW + TY * NC, E_FLOATS = ROW + 2 * TY * NC;
    static constexpr int SMEM = OFF_E + ((NE * E_FLOATS * 4 + 127) / 128) * 128;
    static_assert(SMEM <= 227 * 1024, "one CTA per SM");
    static_assert(OFF + R == 4 && BX == 72 && BY == TY + 4, "staged plane: x0 - 4 .. x0 + 67");
    static_assert(BX % 4 == 0, "AoS rows are loaded as groups of four cells");
    // element of cell (x0 + i, y0 + j), component m, in a staged plane
    // (i in [-4, 68), j in [-2, TY + 2)): SoA [m][row][x], AoS [row][x][m]
    __device__ static __forceinline__ int idx(int i, int j, int m)
    {
        if (LAYOUT == LAYOUT_SOA) return (m * BY + j + R) * BX + OFF + R + i;
        return ((j + R) * BX + OFF + R + i) * NC + m;
    }
};

template <int LAYOUT>
__global__ void __launch_bounds__(512, 1)
    euler_sweep_row3_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_out,
                            float* __restrict__ out, FieldCtl* __restrict__ ctl, const SweepGeom sg,
                            const SweepParams prm)
{
    using K = Row3Cfg<LAYOUT>;
    constexpr int TX = K::TX, TY = K::TY, NW = K::NW, NT = K::NT, NC = K::NC, R = K::R, NS = K::NS;
    constexpr int ROW = K::ROW;
    constexpr int SX = LAYOUT == LAYOUT_SOA ? 1 : NC;            // next cell in x
    constexpr int SY = LAYOUT == LAYOUT_SOA ? K::BX : K::BX * NC;  // next row
    constexpr int SM = LAYOUT == LAYOUT_SOA ? K::BX * K::BY : 1;   // next component
    constexpr uint32_t kSlotBytes = (uint32_t)(K::SLOT_ELEMS * sizeof(float));
    (void)map_out;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    double* red = reinterpret_cast<double*>(smem + K::OFF_RED);
    volatile int* flags = reinterpret_cast<volatile int*>(smem + K::OFF_FLAG);
    float* sdt = reinterpret_cast<float*>(smem + K::OFF_SDT);
    float* ring = reinterpret_cast<float*>(smem + K::OFF_RING);
    float* Ry = reinterpret_cast<float*>(smem + K::OFF_RY);
    float* Fy = reinterpret_cast<float*>(smem + K::OFF_FY);
    float* ebuf = reinterpret_cast<float*>(smem + K::OFF_E);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);  // warp-uniform for the compiler
    const int jrow = warp - 1;                               // tile row of this warp: -1 .. TY
    const bool roww = warp >= 1 && warp <= TY;
    const int lx = 2 * lane;  // this lane's cells of the row: lx, lx + 1
    const FieldGeom& g = sg.f;

    // step scalars formed by thread 0 in FP64 and rounded to FP32 once
    if (tid == 0) {
        const double dt = prm.cfl / __longlong_as_double((long long)ctl->smax[prm.slot_in]);
        sdt[0] = (float)dt;
        for (int d = 0; d < 3; ++d) sdt[1 + d] = (float)(0.5 * dt * prm.inv_dx[d]);
        if (blockIdx.x == 0) {
            ctl->t = prm.first ? dt : ctl->t + dt;
            ctl->dt_last = dt;
            ctl->smax[(prm.slot_in + 2) % 3] = 0ull;
        }
        for (int s = 0; s < NS; ++s) {
            mbar_init(&bars[K::BAR_FULL + s], 1);
            mbar_init(&bars[K::BAR_EMPTY + s], NT);
        }
        for (int w = 0; w < NW; ++w) {
            mbar_init(&bars[K::BAR_RB + w], 32);
            mbar_init(&bars[K::BAR_FB + w], 32);
        }
        for (int k = 0; k < K::NE; ++k) mbar_init(&bars[K::BAR_EB + k], 32);
        flags[0] = 0;
        fence_mbar_init();
        prefetch_tensormap(&map_in);
    }
    __syncthreads();
    const f2 gamma = splat<f2>(prm.gamma_f), gm1 = splat<f2>(prm.gm1_f);
    const f2 mdt = splat<f2>(-sdt[0]);
    f2 inv_dx[3], half_dtdx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        inv_dx[d] = splat<f2>(prm.inv_dx_f[d]);
        half_dtdx[d] = splat<f2>(sdt[1 + d]);
    }

    // ---- bounded waits; after the first that runs out, none waits any more ----
    // (a non-blocking test first: most waits find their phase complete, and
    // then cost neither the abort flag's shared-memory load nor a suspend;
    // each later poll may suspend the warp for up to 20 us, and 2^16 polls
    // bound a wait to about a second of polling after the first that suspends)
    auto wait_bar = [&](int b, unsigned parity) {
        if (mbar_test_wait(&bars[b], parity & 1u)) return;
        if (flags[0]) return;
        for (uint32_t i = 0; i < (1u << 16); ++i)
            if (mbar_try_wait_hint(&bars[b], parity & 1u, 20000u)) return;
        flags[0] = 1;
    };

    // ---- TMA ring (thread 0): the planes of the CTA's items, in order ----
    auto item_planes = [&](int item) -> int {
        const int chunk = item % sg.chunks_z;
        return min(sg.zchunk, g.n[2] - chunk * sg.zchunk) + 2 * R;
    };
    int ld_item = blockIdx.x, ld_j = 0;
    unsigned ld_seq = 0;
    auto issue_until = [&](unsigned limit) {  // planes with sequence number < limit
        while (ld_item < sg.items && ld_seq < limit) {
            // after an abort nothing more is issued: every slot then holds at
            // most one copy in flight, which the exit path waits for
            if (flags[0]) return;
            const int slot = (int)(ld_seq % NS);
            // the slot's previous plane must have been released by every thread
            if (ld_seq >= (unsigned)NS) wait_bar(K::BAR_EMPTY + slot, (ld_seq / NS - 1) & 1u);
            if (flags[0]) return;
            const int item = ld_item;
            const int chunk = item % sg.chunks_z;
            const int tile = item / sg.chunks_z;
            const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
            const int xs = g.lead + g.h + x0 - R - K::OFF;  // multiple of 4 cells
            const int ys = g.h + y0 - R;
            const int pz = g.h + chunk * sg.zchunk - R + ld_j;
            float* dst = ring + (size_t)slot * (K::SLOT_BYTES / sizeof(float));
            mbar_arrive_expect_tx(&bars[K::BAR_FULL + slot], kSlotBytes);
            if (LAYOUT == LAYOUT_SOA) tma_load_4d(dst, &map_in, xs, ys, pz, 0, &bars[K::BAR_FULL + slot]);
            else tma_load_4d(dst, &map_in, 0, xs / 4, ys, pz, &bars[K::BAR_FULL + slot]);
            ++ld_seq;
            if (++ld_j == item_planes(item)) {
                ld_j = 0;
                ld_item += gridDim.x;
            }
        }
    };
    unsigned waited = 0;  // planes [0, waited) have landed, as this thread has seen
    auto wait_full = [&](unsigned seq) {
        for (; waited <= seq; ++waited) wait_bar(K::BAR_FULL + (int)(waited % NS), waited / NS);
    };
    auto release = [&](unsigned seq) { mbar_arrive(&bars[K::BAR_EMPTY + (int)(seq % NS)]); };
    auto plane = [&](unsigned seq) -> const float* {
        return ring + (seq % NS) * (unsigned)(K::SLOT_BYTES / sizeof(float));
    };

    auto load_pair = [&](const float* S, int o, f2 (&q)[NC]) {
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            if (LAYOUT == LAYOUT_SOA) q[m] = *reinterpret_cast<const f2*>(S + o + m * SM);
            else q[m] = f2{S[o + m * SM], S[o + SX + m * SM]};
        }
    };
    auto ld2 = [](const float* a) -> f2 { return *reinterpret_cast<const f2*>(a); };
    auto st2 = [](float* a, f2 v) { *reinterpret_cast<f2*>(a) = v; };

    bool bad = false;
    float smax_local = 0.f;
    float chk = 1.f;
    const int my_off = K::idx(lx, jrow, 0);
    // tile-edge rows of warp 0's lanes: the face x0 - 1/2 of row erow0; the
    // left states of cell x0 + 64 of rows erow1 and erow1 + 1
    const int erow0 = min(lane, TY - 1);
    const int erow1 = 2 * min(lane, TY / 2 - 1);

    unsigned seq_base = 0;  // sequence number of the current item's first plane
    unsigned it = 0;        // plane iterations so far (all items)
    f2 zR[NC], Fzm[NC];     // row warps: high z state of the current plane, face below it
#pragma unroll
    for (int m = 0; m < NC; ++m) zR[m] = Fzm[m] = f2{0.f, 0.f};

    for (int item = blockIdx.x; item < sg.items; item += gridDim.x) {
        const int chunk = item % sg.chunks_z;
        const int tile = item / sg.chunks_z;
        const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
        const int z0 = chunk * sg.zchunk;
        const int zn = min(sg.zchunk, g.n[2] - z0);
        const int gx = x0 + lx, gy = y0 + jrow;
        const bool vx0 = roww && gx < g.n[0] && gy < g.n[1];
        const bool vx1 = roww && gx + 1 < g.n[0] && gy < g.n[1];
        const bool near_xy = (x0 < g.h) || (x0 + TX > g.n[0] - g.h) || (y0 < g.h) || (y0 + TY > g.n[1] - g.h);

        // ---- item start: planes z0-2 .. z0+1; z predicted states of z0-1, z0 and the face z0-1/2 ----
        if (tid == 0) issue_until(seq_base + 5);
        wait_full(seq_base + (roww ? 3u : 1u));
        if (roww) {
            f2 q0[NC], q1[NC], q2[NC], q3[NC], L1[NC], R1[NC], L2[NC];
            load_pair(plane(seq_base + 0), my_off, q0);
            load_pair(plane(seq_base + 1), my_off, q1);
            load_pair(plane(seq_base + 2), my_off, q2);
            load_pair(plane(seq_base + 3), my_off, q3);
            muscl<f2, 3, 2>(q0, q1, q2, gm1, half_dtdx[2], L1, R1, chk);
            muscl<f2, 3, 2>(q1, q2, q3, gm1, half_dtdx[2], L2, zR, chk);
            rus<f2, 3, 2>(R1, L2, gamma, gm1, Fzm, chk);
        }
        release(seq_base + 0);
        release(seq_base + 1);

        for (int zl = 0; zl < zn; ++zl, ++it) {
            const int z = z0 + zl;
            const unsigned sz = seq_base + 2 + (unsigned)zl;  // plane z
            const float* S0 = plane(sz);
            const unsigned kb = it & (unsigned)(K::NE - 1);  // warp 0's buffer of this plane
            float* eb = ebuf + kb * K::E_FLOATS;
            if (warp == 0) {
                // warp 0 writes buffer kb of plane z: every thread has released
                // plane z - 4 (so every read of the buffer's last use is done)
                if (sz >= 4u) {
                    const unsigned sp = sz - 4;
                    wait_bar(K::BAR_EMPTY + (int)(sp % NS), sp / NS);
                }
                if (tid == 0) issue_until(sz + 4);  // planes up to z + 3: their slots are free
            }
            wait_full(roww ? sz + 2 : sz);

            if (warp == 0) {
                // ---- halo row below: tile-edge x work of every row ----
                {
                    // cells (x0-1, x0) of row erow0 as a pair, stencil x0-2 .. x0+1: face x0 - 1/2
                    const int o = K::idx(-1, erow0, 0);
                    f2 qm[NC], qc[NC], qp[NC], L[NC], Rh[NC], F[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        const float c_2 = S0[o - SX + m * SM], c_1 = S0[o + m * SM];
                        const float c0 = S0[o + SX + m * SM], c1 = S0[o + 2 * SX + m * SM];
                        qm[m] = f2{c_2, c_1};
                        qc[m] = f2{c_1, c0};
                        qp[m] = f2{c0, c1};
                    }
                    muscl<f2, 3, 0>(qm, qc, qp, gm1, half_dtdx[0], L, Rh, chk);
                    f2 a[NC], b[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        a[m] = f2{Rh[m].x, Rh[m].x};
                        b[m] = f2{L[m].y, L[m].y};
                    }
                    rus<f2, 3, 0>(a, b, gamma, gm1, F, chk);
                    if (lane < TY) {
#pragma unroll
                        for (int m = 0; m < NC; ++m) eb[K::E_FL + lane * NC + m] = F[m].x;
                    }
                }
                {
                    // cell x0 + 64 of rows erow1 and erow1 + 1 as a pair: its left state
                    const int o0 = K::idx(TX - 1, erow1, 0), o1 = o0 + SY;
                    f2 qm[NC], qc[NC], qp[NC], L[NC], Rh[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        qm[m] = f2{S0[o0 + m * SM], S0[o1 + m * SM]};
                        qc[m] = f2{S0[o0 + SX + m * SM], S0[o1 + SX + m * SM]};
                        qp[m] = f2{S0[o0 + 2 * SX + m * SM], S0[o1 + 2 * SX + m * SM]};
                    }
                    muscl<f2, 3, 0>(qm, qc, qp, gm1, half_dtdx[0], L, Rh, chk);
                    if (lane < TY / 2) {
#pragma unroll
                        for (int m = 0; m < NC; ++m) {
                            eb[K::E_LR + erow1 * NC + m] = L[m].x;
                            eb[K::E_LR + (erow1 + 1) * NC + m] = L[m].y;
                        }
                    }
                }
            }
            // ---- every warp: the y predicted states of its row (warp 0: the
            // row below the tile; warp NW - 1: the row above it) ----
            f2 qc[NC], Ly[NC];
            {
                f2 qm[NC], qp[NC], Rh[NC];
                load_pair(S0, my_off - SY, qm);
                load_pair(S0, my_off, qc);
                load_pair(S0, my_off + SY, qp);
                muscl<f2, 3, 1>(qm, qc, qp, gm1, half_dtdx[1], Ly, Rh, chk);
                if (warp < NW - 1) {
                    // the high state goes to the row above: warp 0's buffer
                    // of this plane (with its tile-edge data), or this row's
                    // exchange row
                    float* dst = warp == 0 ? eb + K::E_RY : Ry + jrow * ROW;
#pragma unroll
                    for (int m = 0; m < NC; ++m) st2(dst + m * TX + lx, Rh[m]);
                    mbar_arrive(&bars[warp == 0 ? K::BAR_EB + (int)kb : K::BAR_RB + warp]);
                }
            }
            f2 Fzp[NC];
            if (roww) {
                // z: predicted states of plane z+1, the face z+1/2
                f2 q1[NC], q2[NC], L[NC], Rn[NC];
                load_pair(plane(sz + 1), my_off, q1);
                load_pair(plane(sz + 2), my_off, q2);
                muscl<f2, 3, 2>(qc, q1, q2, gm1, half_dtdx[2], L, Rn, chk);
                rus<f2, 3, 2>(zR, L, gamma, gm1, Fzp, chk);
#pragma unroll
                for (int m = 0; m < NC; ++m) zR[m] = Rn[m];
            }
            f2 Fyl[NC];
            if (warp > 0) {
                // the y face below this row, from the high state of the row below
                // (row -1: warp 0's buffer of this plane; warp NW - 1: the
                // face above the tile's last row)
                const float* below;
                if (warp == 1) {
                    wait_bar(K::BAR_EB + (int)kb, it / K::NE);
                    below = eb + K::E_RY;
                } else {
                    wait_bar(K::BAR_RB + warp - 1, it);
                    below = Ry + (jrow - 1) * ROW;
                }
                f2 a[NC];
#pragma unroll
                for (int m = 0; m < NC; ++m) a[m] = ld2(below + m * TX + lx);
                rus<f2, 3, 1>(a, Ly, gamma, gm1, Fyl, chk);
#pragma unroll
                for (int m = 0; m < NC; ++m) st2(Fy + jrow * ROW + m * TX + lx, Fyl[m]);
                mbar_arrive(&bars[K::BAR_FB + warp]);
            }
            if (roww) {
                f2 dFx[NC];
                {
                    // x: predicted states of the pair, faces lx+1/2 and lx+3/2
                    f2 qm[NC], qp[NC], L[NC], Rh[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        const float cl = S0[my_off - SX + m * SM], cr = S0[my_off + 2 * SX + m * SM];
                        qm[m] = f2{cl, qc[m].x};
                        qp[m] = f2{qc[m].y, cr};
                    }
                    muscl<f2, 3, 0>(qm, qc, qp, gm1, half_dtdx[0], L, Rh, chk);
                    wait_bar(K::BAR_EB + (int)kb, it / K::NE);
                    const float* eL = eb + K::E_LR + jrow * NC;
                    f2 b[NC], F[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        float nx = __shfl_down_sync(0xffffffffu, L[m].x, 1);
                        if (lane == 31) nx = eL[m];
                        b[m] = f2{L[m].y, nx};
                    }
                    rus<f2, 3, 0>(Rh, b, gamma, gm1, F, chk);
                    const float* eF = eb + K::E_FL + jrow * NC;
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        float pv = __shfl_up_sync(0xffffffffu, F[m].y, 1);
                        if (lane == 0) pv = eF[m];
                        dFx[m] = F[m] - f2{pv, F[m].x};
                    }
                }
                // ---- update of plane z ----
                wait_bar(K::BAR_FB + warp + 1, it);
                f2 qn[NC];
                const long long obase = geom_cell(g, gx, gy, z) * g.cell_stride;
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const f2 fyu = ld2(Fy + (jrow + 1) * ROW + m * TX + lx);
                    f2 acc = dFx[m] * inv_dx[0];
                    acc = fma_v(fyu - Fyl[m], inv_dx[1], acc);
                    acc = fma_v(Fzp[m] - Fzm[m], inv_dx[2], acc);
                    qn[m] = fma_v(mdt, acc, qc[m]);
                    Fzm[m] = Fzp[m];
                    if (vx1) {
                        if (LAYOUT == LAYOUT_SOA)
                            *reinterpret_cast<f2*>(out + obase + (long long)m * g.comp_stride) = qn[m];
                        else {
                            out[obase + m] = qn[m].x;
                            out[obase + NC + m] = qn[m].y;
                        }
                    }
                }
                bool ok0, ok1;
                const f2 sw = wave_sum2<3>(qn, gamma, gm1, inv_dx, ok0, ok1);
                smax_local = fmaxf(smax_local, fmaxf(vx0 ? sw.x : 0.f, vx1 ? sw.y : 0.f));
                const bool bad0 = vx0 && !ok0, bad1 = vx1 && !ok1;
                if (bad0 || bad1) {
                    bad = true;
                    record_bad(ctl, BAD_CELL, bad0 ? gx : gx + 1, gy, z);
                }
                if (near_xy || z < g.h || z >= g.n[2] - g.h || (vx0 && !vx1)) {
                    // edge tiles: ghost images; a ragged last column: its single cell
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (!(h == 0 ? vx0 : vx1)) continue;
                        float q1[NC];
#pragma unroll
                        for (int m = 0; m < NC; ++m) q1[m] = h == 0 ? qn[m].x : qn[m].y;
                        if (vx0 && !vx1) {
                            const long long base = geom_cell(g, gx + h, gy, z) * g.cell_stride;
#pragma unroll
                            for (int m = 0; m < NC; ++m) out[base + (long long)m * g.comp_stride] = q1[m];
                        }
                        if (near_xy || z < g.h || z >= g.n[2] - g.h)
                            write_ghost_images<float, 3>(out, g, prm.bc, gx + h, gy, z, q1);
                    }
                }
            }
            if (!(chk > 0.f)) {
                bad = true;
                record_bad(ctl, BAD_STATE, x0, y0, z);
                chk = 1.f;
            }
            release(sz);
        }
        // ---- item end: the last two planes ----
        wait_full(seq_base + (unsigned)zn + 3);
        release(seq_base + (unsigned)zn + 2);
        release(seq_base + (unsigned)zn + 3);
        seq_base += (unsigned)(zn + 2 * R);
    }

    __syncthreads();
    const bool aborted = flags[0] != 0;
    if (tid == 0 && aborted) {
        // let every issued copy land before the CTA's shared memory goes away
        for (unsigned sq = 0; sq < ld_seq; ++sq) {
            if (sq + NS < ld_seq) continue;
            mbar_wait_bounded(&bars[K::BAR_FULL + (int)(sq % NS)], (sq / NS) & 1u);
        }
        atomicOr(&ctl->err, DEV_ERR_TIMEOUT);
    }
    double v = (double)smax_local;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int w = 0; w < NW; ++w) mx = fmax(mx, red[w]);
        atomic_max_pos_double(&ctl->smax[(prm.slot_in + 1) % 3], mx);
        if (any_bad) atomicOr(&ctl->err, DEV_ERR_NUMERIC);
    }
}

}  // namespace ripple
