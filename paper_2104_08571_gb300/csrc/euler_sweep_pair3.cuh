// FP32 3D MUSCL-Hancock sweep on cell pairs with split barriers, sm_103a.
//
// The same step, staging, fusion and packed f32x2 arithmetic as
// euler_sweep_pair_kernel (euler_sweep_pair.cuh), with the plane loop
// rescheduled so that no warp waits for work it does not depend on.
//
// Work per plane z of a tile (pairs of x-adjacent cells, 256 threads):
//   pair warps 0-3 (each thread owns the columns (lx, lx+1) of row ly):
//     one item of y-predicted states of plane z+1 and the z direction
//     (predicted states of plane z+1 from planes z..z+2 and the face z+1/2,
//     registers), then the update of plane z;
//   warps 4-7: the x/y face fluxes of plane z (2 or 3 items each) and the rest
//     of the x/y predicted states of plane z+1 (1 or 2 items each).
// The predicted-state arrays are double buffered (plane parity), so the
// predicted states of plane z+1 are written while the faces of plane z still
// read those of plane z, and the four hand-offs use named barriers in which
// producers only arrive (bar.arrive) and consumers wait (bar.sync):
//   PD[z & 1]  predicted states of plane z complete   (all warps -> warps 4-7)
//   FD         faces of plane z complete               (warps 4-7 -> pair warps)
//   UD         update of plane z read the faces         (pair warps -> warps 4-7)
// Two barriers alternate for PD because the pair warps run one plane ahead on
// it.  The pairing of every arrive with its sync, the absence of lapping and
// of deadlock over any interleaving are checked by a model of this protocol.
// A thread keeps its own cells of plane z from the z direction in registers
// for the update, so plane z is dead once the faces of plane z are complete.
// The updated pairs leave by direct 64-bit stores (each row of a tile is 128
// contiguous bytes per component), which frees the output staging buffers
// for a fifth ring slot: planes are prefetched up to five ahead.
//
// A TMA wait that runs out only records the abort flag: every warp still runs
// the same plane loop (so every barrier still pairs up) and the CTA stops
// together at the next tile's full barrier.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "euler_sweep.cuh"
#include "euler_sweep_pair.cuh"
#include "pair_math.cuh"

namespace ripple {

__device__ __forceinline__ void named_sync(uint32_t id, uint32_t n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(uint32_t id, uint32_t n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <int LAYOUT>
struct Pair3Cfg {
    using PC = PairCfg<3, LAYOUT, SCHEME_MUSCL>;
    using C = typename PC::C;
    static constexpr int NS = 5;  // ring slots: planes z+1..z+5 while the faces of plane z are formed
    static constexpr int SMEM = C::HDR_BYTES + NS * C::SLOT_BYTES + 2 * PC::P_BYTES + PC::F_BYTES;
    static_assert(SMEM <= 113 * 1024, "two CTAs per SM");
    // named barriers (0 is __syncthreads)
    static constexpr uint32_t BAR_PD0 = 1, BAR_PD1 = 2, BAR_UD = 3, BAR_FD = 4;
};

// map_out is part of the sweep launch signature; this kernel stores directly.
template <int LAYOUT>
__global__ void __launch_bounds__(256, 2)
    euler_sweep_pair3_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_out,
                             float* __restrict__ out, FieldCtl* __restrict__ ctl, const SweepGeom sg,
                             const SweepParams prm)
{
    constexpr int DIM = 3;
    using P3 = Pair3Cfg<LAYOUT>;
    using PC = typename P3::PC;
    using C = typename PC::C;
    using PV = PlaneView<C, LAYOUT>;
    constexpr int TX = PC::TX, TY = PC::TY, NC = PC::NC, R = PC::R, NS = P3::NS, NT = PC::NT;
    constexpr int SX = LAYOUT == LAYOUT_SOA ? 1 : NC;
    constexpr int SY = LAYOUT == LAYOUT_SOA ? C::BX : C::BX * NC;
    constexpr int SM = LAYOUT == LAYOUT_SOA ? C::BX * C::BY : 1;
    constexpr int NP = PC::NP;
    static_assert(R == 2 && PC::NXP == 136 && PC::NYP == 160 && PC::NXF == 136 && PC::NYF == 144,
                  "the item assignment below is written for 32 x 8 tiles");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    double* red = reinterpret_cast<double*>(smem + 64);
    int* flags = reinterpret_cast<int*>(smem + 64 + 8 * 16);
    float* ring = reinterpret_cast<float*>(smem + C::HDR_BYTES);
    float* Pbuf = reinterpret_cast<float*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES);
    float* Fs = reinterpret_cast<float*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES + 2 * PC::P_BYTES);
    float* FX = Fs;
    float* FY = Fs + NC * PC::NFX;
    auto PLb = [&](unsigned par) { return Pbuf + par * (PC::P_BYTES / sizeof(float)); };

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);  // warp-uniform for the compiler
    const bool pthr = warp < 4;
    const int lx = 2 * (tid % (TX / 2)), ly = (tid / (TX / 2)) % TY;
    const FieldGeom& g = sg.f;

    // Predicted-state items of a plane (x pairs: cells (2q-1, 2q) of a row,
    // 136 items; y pairs: 160 items).  Pair warp w: y items 32w..32w+31.
    // Warps 4..7: x items 32(w-4)..; warp 6 also the x items 128..135, warp 7
    // the y items 128..159.  Face items of warps 4..7 (x faces: 136 pair
    // items, y faces: 144): 3, 3, 2, 2 per warp.  Lanes past the last item of
    // a kind repeat it.  Item kinds and bases are warp-uniform; each kind has
    // one copy of its code in the plane loop (loops over a warp's items are
    // not unrolled), which keeps the code that warps of different roles run
    // at the same time small.
    const int np_items = pthr ? 1 : (warp >= 6 ? 2 : 1);
    auto p_kind_x = [&](int k) -> bool { return !pthr && (k == 0 || warp == 6); };
    auto p_base = [&](int k) -> int { return pthr ? warp * 32 : k == 0 ? (warp - 4) * 32 : 128; };
    const int nf_items = pthr ? 0 : (warp <= 5 ? 3 : 2);
    auto f_kind_x = [&](int k) -> bool { return k == 0 || (k == 1 && warp == 4); };
    auto f_base = [&](int k) -> int {
        // x: item index; y: item index among the y faces
        if (k == 0) return (warp - 4) * 32;
        if (k == 1) return warp == 4 ? 128 : (warp - 5) * 32;
        return warp == 4 ? 96 : 128;
    };

    // step scalars formed by thread 0 in FP64 and rounded to FP32 once
    float* sdt = reinterpret_cast<float*>(smem + 256);
    if (tid == 0) {
        const double dt = prm.cfl / __longlong_as_double((long long)ctl->smax[prm.slot_in]);
        sdt[0] = (float)dt;
        for (int d = 0; d < 3; ++d) sdt[1 + d] = (float)(0.5 * dt * prm.inv_dx[d]);
        if (blockIdx.x == 0) {
            ctl->t = prm.first ? dt : ctl->t + dt;
            ctl->dt_last = dt;
            ctl->smax[(prm.slot_in + 2) % 3] = 0ull;
        }
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        flags[0] = 0;
        fence_mbar_init();
        prefetch_tensormap(&map_in);
    }
    __syncthreads();
    const f2 gamma = splat<f2>(prm.gamma_f), gm1 = splat<f2>(prm.gm1_f);
    const f2 dtv = splat<f2>(sdt[0]);
    f2 inv_dx[3], half_dtdx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        inv_dx[d] = splat<f2>(prm.inv_dx_f[d]);
        half_dtdx[d] = splat<f2>(sdt[1 + d]);
    }

    // ---- TMA ring (thread 0): planes of the CTA's items in order ----
    auto item_planes = [&](int item) -> int {
        const int chunk = item % sg.chunks_z;
        return min(sg.zchunk, g.n[2] - chunk * sg.zchunk) + 2 * R;
    };
    int ld_item = blockIdx.x, ld_j = 0;
    unsigned ld_seq = 0;
    auto issue_until = [&](unsigned limit) {
        while (ld_item < sg.items && ld_seq < limit) {
            const int item = ld_item;
            const int chunk = item % sg.chunks_z;
            const int tile = item / sg.chunks_z;
            const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
            const int xs = g.lead + g.h + x0 - R - C::OFF;
            const int ys = g.h + y0 - R;
            const int slot = (int)(ld_seq % NS);
            float* dst = ring + (size_t)slot * (C::SLOT_BYTES / sizeof(float));
            mbar_arrive_expect_tx(&bars[slot], (uint32_t)(C::SLOT_ELEMS * sizeof(float)));
            const int pz = g.h + chunk * sg.zchunk - R + ld_j;
            if (LAYOUT == LAYOUT_SOA) tma_load_4d(dst, &map_in, xs, ys, pz, 0, &bars[slot]);
            else tma_load_3d(dst, &map_in, xs * NC, ys, pz, &bars[slot]);
            ++ld_seq;
            if (++ld_j == item_planes(item)) {
                ld_j = 0;
                ld_item += gridDim.x;
            }
        }
    };
    unsigned ready_upto = 0, seq_base = 0;
    auto plane_ptr = [&](unsigned seq) -> const float* {
        return ring + (seq % NS) * (unsigned)(C::SLOT_BYTES / sizeof(float));
    };
    auto wait_planes = [&](unsigned need) {
        bool ok = true;
        for (unsigned sq = ready_upto; sq <= need; ++sq)
            ok &= mbar_wait_bounded(&bars[sq % NS], (uint32_t)((sq / NS) & 1));
        if (need + 1 > ready_upto) ready_upto = need + 1;
        if (!ok) flags[0] = 1;  // recorded; the CTA stops at the next full barrier
    };

    auto load_pair = [&](const float* S, int o, f2 (&q)[NC]) {
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            if (LAYOUT == LAYOUT_SOA) q[m] = *reinterpret_cast<const f2*>(S + o + m * SM);
            else q[m] = f2{S[o + m * SM], S[o + SX + m * SM]};
        }
    };
    auto ld2 = [&](const float* a) -> f2 { return *reinterpret_cast<const f2*>(a); };
    auto st2 = [&](float* a, f2 v) { *reinterpret_cast<f2*>(a) = v; };

    // predicted-state item k of this thread from plane S into buffer P
    auto p_item = [&](int k, const float* S, float* P, float& chk) {
        float* PL = P;
        float* PR = P + NC * NP;
        f2 qm[NC], qc[NC], qp[NC], L[NC], Rr[NC];
        const bool kx = p_kind_x(k);
        int o, pi;
        if (kx) {
            const int it = min(p_base(k) + lane, PC::NXP - 1);
            const int cy = it / PC::XP, c0 = 2 * (it % PC::XP) - 1;
            o = PV::idx(c0 - 1, cy, 0);
            pi = cy * PC::XR + c0 + 1;
        } else {
            const int jj = min(p_base(k) + lane, PC::NYP - 1);
            const int cy = jj / (TX / 2) - 1, cx = 2 * (jj % (TX / 2));
            o = PV::idx(cx, cy, 0);
            pi = PC::NPX + (cy + 1) * TX + cx;
        }
        if (kx) {
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                f2 A, B;
                if (LAYOUT == LAYOUT_SOA) {
                    A = ld2(S + o + m * SM);
                    B = ld2(S + o + 2 + m * SM);
                } else {
                    A = f2{S[o + m * SM], S[o + SX + m * SM]};
                    B = f2{S[o + 2 * SX + m * SM], S[o + 3 * SX + m * SM]};
                }
                qm[m] = A;
                qc[m] = f2{A.y, B.x};
                qp[m] = B;
            }
            muscl<f2, DIM, 0>(qm, qc, qp, gm1, half_dtdx[0], L, Rr, chk);
        } else {
            load_pair(S, o - SY, qm);
            load_pair(S, o, qc);
            load_pair(S, o + SY, qp);
            muscl<f2, DIM, 1>(qm, qc, qp, gm1, half_dtdx[1], L, Rr, chk);
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            st2(PL + m * NP + pi, L[m]);
            st2(PR + m * NP + pi, Rr[m]);
        }
    };

    bool bad = false;
    float smax_local = 0.f;
    bool aborted = false;
    const int my_off = PV::idx(lx, ly, 0);

    for (int item = blockIdx.x; item < sg.items; item += gridDim.x) {
        const int chunk = item % sg.chunks_z;
        const int tile = item / sg.chunks_z;
        const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
        const int z0 = chunk * sg.zchunk;
        const int zn = min(sg.zchunk, g.n[2] - z0);
        const int gx = x0 + lx, gy = y0 + ly;
        const bool vx0 = pthr && (gx < g.n[0]) && (gy < g.n[1]);
        const bool vx1 = pthr && (gx + 1 < g.n[0]) && (gy < g.n[1]);
        const bool near_xy = (x0 < g.h) || (x0 + TX > g.n[0] - g.h) || (y0 < g.h) || (y0 + TY > g.n[1] - g.h);
        float chk = 1.f;

        f2 Fzm[NC], Fzp[NC], zR[NC], qz[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) Fzm[m] = Fzp[m] = zR[m] = qz[m] = f2{0.f, 0.f};

        // ---- item start: every plane of the previous item is dead ----
        __syncthreads();
        if (tid == 0) issue_until(seq_base + NS);  // planes 0..4 (z0-2 .. z0+2)
        // Planes of earlier tiles that this thread never waited for (warps 4-7
        // skip the last two planes of a tile) are complete: the pair warps
        // waited for them before the barrier above.  Skip them: their slots are
        // being reloaded, and a wait on a slot whose mbarrier has since moved two
        // phases on would read the parity of a phase that never completes.
        if (ready_upto < seq_base) ready_upto = seq_base;
        wait_planes(seq_base + 3);
        __syncthreads();
        if (flags[0]) {
            aborted = true;
            break;
        }
        if (pthr) {
            // z: predicted states of plane z0-1 (high face) and z0, the face z0-1/2
            f2 q0[NC], q1[NC], q2[NC], q3[NC], L1[NC], R1[NC], L2[NC];
            load_pair(plane_ptr(seq_base + 0), my_off, q0);
            load_pair(plane_ptr(seq_base + 1), my_off, q1);
            load_pair(plane_ptr(seq_base + 2), my_off, q2);
            load_pair(plane_ptr(seq_base + 3), my_off, q3);
            muscl<f2, DIM, 2>(q0, q1, q2, gm1, half_dtdx[2], L1, R1, chk);
            muscl<f2, DIM, 2>(q1, q2, q3, gm1, half_dtdx[2], L2, zR, chk);
            rus<f2, DIM, 2>(R1, L2, gamma, gm1, Fzm, chk);
        }
        // x/y predicted states of plane z0 into buffer 0
#pragma unroll 1
        for (int k = 0; k < np_items; ++k) p_item(k, plane_ptr(seq_base + R), PLb(0), chk);
        __syncthreads();
        if (tid == 0) issue_until(seq_base + 2 + NS);  // planes 0, 1 are dead: planes 5, 6

        for (int zl = 0; zl < zn; ++zl) {
            const int z = z0 + zl;
            const unsigned jc = (unsigned)(zl + R);
            const bool more = zl + 1 < zn;
            if (pthr) {
                wait_planes(seq_base + jc + 2);
                // predicted states (y) of plane z+1, then the z direction (predicted
                // states of plane z+1, face z+1/2): independent work in one block for
                // the scheduler.  At the last plane of a tile the y item is computed
                // too (plane z+1 is a staged halo plane; nothing reads that buffer
                // any more), but not announced.
                p_item(0, plane_ptr(seq_base + jc + 1), PLb((zl + 1) & 1), chk);
                {
                    f2 q1[NC], q2[NC], L[NC], Rn[NC];
                    load_pair(plane_ptr(seq_base + jc), my_off, qz);
                    load_pair(plane_ptr(seq_base + jc + 1), my_off, q1);
                    load_pair(plane_ptr(seq_base + jc + 2), my_off, q2);
                    muscl<f2, DIM, 2>(qz, q1, q2, gm1, half_dtdx[2], L, Rn, chk);
                    rus<f2, DIM, 2>(zR, L, gamma, gm1, Fzp, chk);
#pragma unroll
                    for (int m = 0; m < NC; ++m) zR[m] = Rn[m];
                }
                if (more) named_arrive(((zl + 1) & 1) ? P3::BAR_PD1 : P3::BAR_PD0, NT);
                named_sync(P3::BAR_FD, NT);
                if (tid == 0) issue_until(seq_base + jc + 1 + NS);  // planes up to z are dead
                // ---- update of plane z ----
                f2 qn[NC];
                const long long obase = geom_cell(g, gx, gy, z) * g.cell_stride;
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const float* fxr = FX + m * PC::NFX + ly * PC::FXR + lx;
                    const f2 fl = ld2(fxr), fn = ld2(fxr + 2);
                    const f2 fr = f2{fl.y, fn.x};
                    const f2 fyl = ld2(FY + m * PC::NFY + ly * TX + lx);
                    const f2 fyh = ld2(FY + m * PC::NFY + (ly + 1) * TX + lx);
                    f2 acc = (fr - fl) * inv_dx[0];
                    acc = fma_v(fyh - fyl, inv_dx[1], acc);
                    acc = fma_v(Fzp[m] - Fzm[m], inv_dx[2], acc);
                    qn[m] = fma_v(f2{-dtv.x, -dtv.y}, acc, qz[m]);
                    // both cells in the domain: one store per component (SoA: an aligned
                    // pair, x of the pair even and rows 16-byte aligned)
                    if (vx1) {
                        if (LAYOUT == LAYOUT_SOA)
                            *reinterpret_cast<f2*>(out + obase + (long long)m * g.comp_stride) = qn[m];
                        else {
                            out[obase + m] = qn[m].x;
                            out[obase + NC + m] = qn[m].y;
                        }
                    }
                    Fzm[m] = Fzp[m];
                }
                if (more) named_arrive(P3::BAR_UD, NT);
                bool ok0, ok1;
                const f2 sw = wave_sum2<DIM>(qn, gamma, gm1, inv_dx, ok0, ok1);
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
                            write_ghost_images<float, DIM>(out, g, prm.bc, gx + h, gy, z, q1);
                    }
                }
            } else {
                if (zl > 0) {
                    named_sync((zl & 1) ? P3::BAR_PD1 : P3::BAR_PD0, NT);  // predicted states of plane z
                    named_sync(P3::BAR_UD, NT);                             // update of plane z-1 done with the faces
                }
                // ---- x/y face fluxes of plane z ----
                const float* P = PLb(zl & 1);
                const float* PL = P;
                const float* PR = P + NC * NP;
#pragma unroll 1
                for (int k = 0; k < nf_items; ++k) {
                    if (f_kind_x(k)) {
                        // x faces (f, f + 1), f = 2q, between cells f - 1 | f and f | f + 1
                        const int it = min(f_base(k) + lane, PC::NXF - 1);
                        const int cy = it / PC::XP, f = 2 * (it % PC::XP);
                        f2 a[NC], b[NC], F[NC];
                        const int i0 = cy * PC::XR + f;
#pragma unroll
                        for (int m = 0; m < NC; ++m) {
                            a[m] = ld2(PR + m * NP + i0);
                            const f2 u = ld2(PL + m * NP + i0), w = ld2(PL + m * NP + i0 + 2);
                            b[m] = f2{u.y, w.x};
                        }
                        rus<f2, DIM, 0>(a, b, gamma, gm1, F, chk);
#pragma unroll
                        for (int m = 0; m < NC; ++m) st2(FX + m * PC::NFX + cy * PC::FXR + f, F[m]);
                    } else {
                        const int jj = min(f_base(k) + lane, PC::NYF - 1);
                        const int fy = jj / (TX / 2), cx = 2 * (jj % (TX / 2));
                        f2 a[NC], b[NC], F[NC];
                        const int il = PC::NPX + fy * TX + cx, ir = il + TX;
#pragma unroll
                        for (int m = 0; m < NC; ++m) {
                            a[m] = ld2(PR + m * NP + il);
                            b[m] = ld2(PL + m * NP + ir);
                        }
                        rus<f2, DIM, 1>(a, b, gamma, gm1, F, chk);
#pragma unroll
                        for (int m = 0; m < NC; ++m) st2(FY + m * PC::NFY + fy * TX + cx, F[m]);
                    }
                }
                named_arrive(P3::BAR_FD, NT);
                // ---- x/y predicted states of plane z+1 (the other buffer) ----
                if (more) {
                    wait_planes(seq_base + jc + 1);
#pragma unroll 1
                    for (int k = 0; k < np_items; ++k) p_item(k, plane_ptr(seq_base + jc + 1), PLb((zl + 1) & 1), chk);
                }
            }
            if (!(chk > 0.f)) {
                bad = true;
                record_bad(ctl, BAD_STATE, x0, y0, z);
                chk = 1.f;
            }
        }
        seq_base += (unsigned)(zn + 2 * R);
    }

    __syncthreads();
    if (tid == 0) {
        if (aborted) {
            for (unsigned sq = ready_upto; sq < ld_seq; ++sq)
                mbar_wait_bounded(&bars[sq % NS], (uint32_t)((sq / NS) & 1));
            atomicOr(&ctl->err, DEV_ERR_TIMEOUT);
        }
    }
    double v = (double)smax_local;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < NT / 32; ++w) m = fmax(m, red[w]);
        atomic_max_pos_double(&ctl->smax[(prm.slot_in + 1) % 3], m);
        if (any_bad) atomicOr(&ctl->err, DEV_ERR_NUMERIC);
    }
}

}  // namespace ripple
