// FP32 Euler sweep on cell pairs (packed f32x2 arithmetic), sm_103a.
//
// Same step, staging and fusion as euler_sweep_kernel (see euler_sweep.cuh):
// one launch = one explicit step, 2.5-D plane streaming through a TMA ring,
// each face flux evaluated once, fused padding fill / CFL max / positivity.
// What changes is the unit of work: every work item is a PAIR of x-adjacent
// cells (or faces), held as f32x2 values, so each multiply, add and fma of
// the reconstruction, predictor, flux and update arithmetic issues once for
// two cells.  128 pair threads each own two neighbouring columns: they run
// the z direction (in phase F) and the update; the x/y predicted states
// (phase P) are pair items over all 256 threads and the x/y face fluxes
// (phase F) pair items of the other 128 threads, which balances the phases.
// The z stencil is read from the resident planes of the ring, so only the
// high-face predicted state and the z face fluxes stay in registers.
// Shared arrays are laid out so that every pair access of the SoA layout is
// one 64-bit shared-memory access.  Tile: 32 x 8 cells.
// Schemes: Rusanov (first order) and MUSCL-Hancock for the unsplit step (3D
// MUSCL-Hancock runs the split-barrier kernel of euler_sweep_pair3.cuh), and
// FORCE for one axis sweep of the split step (prm.axis; faces and update of
// that axis only; dt, t and the CFL maximum are taken by the step's last sweep).
// 2D items are single planes: the ring holds six, and the first-order 2D
// sweeps run three CTAs per SM.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "euler_sweep.cuh"
#include "pair_math.cuh"

namespace ripple {

template <int DIM, int LAYOUT, int SCHEME>
struct PairCfg {
    static constexpr int TX = 32, TY = 8, NT = 256, NPT = 128;
    using C = SweepCfg<float, DIM, LAYOUT, SCHEME, TX, TY>;
    static constexpr int NC = DIM + 2, R = C::R;
    static constexpr int XR = TX + 2;                  // x-predicted cells per row (-1 .. TX)
    static constexpr int NPX = XR * TY;                // x-predicted entries
    static constexpr int NPY = TX * (TY + 2);          // y-predicted entries
    static constexpr int NP = NPX + NPY;
    static constexpr int FXR = TX + 2;                 // x-face row stride (TX + 1 faces, padded even)
    static constexpr int NFX = FXR * TY, NFY = TX * (TY + 1);
    static constexpr int XP = XR / 2;                  // x pairs per row (17)
    static constexpr int NXP = XP * TY, NXPr = ((NXP + 31) / 32) * 32;
    static constexpr int NYP = (TX / 2) * (TY + 2), NYPr = ((NYP + 31) / 32) * 32;
    static constexpr int NXF = XP * TY, NXFr = ((NXF + 31) / 32) * 32;
    static constexpr int NYF = (TX / 2) * (TY + 1), NYFr = ((NYF + 31) / 32) * 32;
    static constexpr int KP = SCHEME == SCHEME_MUSCL ? (NXPr + NYPr + NT - 1) / NT : 0;
    static constexpr int KF = (NXFr + NYFr + (NT - NPT) - 1) / (NT - NPT);  // on the non-pair threads
    static constexpr int P_BYTES = SCHEME == SCHEME_MUSCL ? ((2 * NC * NP * 4 + 127) / 128) * 128 : 0;
    static constexpr int F_BYTES = ((NC * (NFX + NFY) * 4 + 127) / 128) * 128;
    // ring slots: 2D items are single planes, so the ring prefetches whole tiles ahead
    static constexpr int NSR = DIM == 2 ? 6 : C::NS;
    // CTAs per SM: the 2D first-order sweeps (Rusanov, the split FORCE sweep) need
    // fewer registers and their short per-tile work wants more CTAs in flight
    static constexpr int MIN_CTAS = DIM == 2 && SCHEME != SCHEME_MUSCL ? 3 : 2;
    static constexpr int SMEM = C::HDR_BYTES + NSR * C::SLOT_BYTES + 2 * C::OUT_BYTES + P_BYTES + F_BYTES;
    static_assert(C::OFF + R == 4 || LAYOUT == LAYOUT_AOS, "pairs at even x need an even in-slot x offset");
    static_assert(C::BX % 2 == 0 && NP % 2 == 0 && NFX % 2 == 0 && NFY % 2 == 0, "64-bit aligned pairs");
};

// First-order face flux of a scheme along D on cell pairs: Rusanov, or FORCE
// for the split step.
template <int SCHEME, int DIM, int D>
__device__ __forceinline__ void pair_flux1(const f2 (&a)[DIM + 2], const f2 (&b)[DIM + 2], f2 gamma, f2 gm1,
                                           f2 half_dtdx, f2 half_inv_dtdx, f2 (&F)[DIM + 2], float& chk)
{
    if constexpr (SCHEME == SCHEME_FORCE) force<f2, DIM, D>(a, b, gm1, half_dtdx, half_inv_dtdx, F, chk);
    else rus<f2, DIM, D>(a, b, gamma, gm1, F, chk);
}

template <int DIM, int LAYOUT, int SCHEME>
__global__ void __launch_bounds__(256, PairCfg<DIM, LAYOUT, SCHEME>::MIN_CTAS)
    euler_sweep_pair_kernel(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_out,
                            float* __restrict__ out, FieldCtl* __restrict__ ctl, const SweepGeom sg,
                            const SweepParams prm)
{
    using PC = PairCfg<DIM, LAYOUT, SCHEME>;
    using C = typename PC::C;
    using PV = PlaneView<C, LAYOUT>;
    constexpr int TX = PC::TX, TY = PC::TY, NC = PC::NC, R = PC::R, NS = PC::NSR, NT = PC::NT;
    constexpr bool MUSCL = SCHEME == SCHEME_MUSCL;
    constexpr bool FORCE = SCHEME == SCHEME_FORCE;  // one sweep of the split step per launch
    constexpr int SX = LAYOUT == LAYOUT_SOA ? 1 : NC;
    constexpr int SY = LAYOUT == LAYOUT_SOA ? C::BX : C::BX * NC;
    constexpr int SM = LAYOUT == LAYOUT_SOA ? C::BX * C::BY : 1;
    constexpr int NP = PC::NP;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    double* red = reinterpret_cast<double*>(smem + 64);
    int* flags = reinterpret_cast<int*>(smem + 64 + 8 * 16);
    float* ring = reinterpret_cast<float*>(smem + C::HDR_BYTES);
    float* stage = reinterpret_cast<float*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES);
    float* P = reinterpret_cast<float*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES + 2 * C::OUT_BYTES);
    float* Fs = reinterpret_cast<float*>(smem + C::HDR_BYTES + NS * C::SLOT_BYTES + 2 * C::OUT_BYTES + PC::P_BYTES);
    float* PL = P;
    float* PR = P + NC * NP;
    float* FX = Fs;
    float* FY = Fs + NC * PC::NFX;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    // warp index broadcast from lane 0, so the compiler treats it (and every
    // role or item-kind decision derived from it) as warp-uniform
    const int warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const bool pthr = warp < PC::NPT / 32;  // pair warps: each thread owns columns (lx, lx+1) of row ly
    const int lx = 2 * (tid % (TX / 2)), ly = (tid / (TX / 2)) % TY;
    const FieldGeom& g = sg.f;

    // Work items of this thread, the same for every plane and tile: only the
    // staged plane (a ring slot) changes, so their shared-memory offsets are
    // formed once.  Item bases are warp-uniform; the lanes of a partly filled
    // warp past the last item repeat the last item (same operands, same
    // results, same addresses), so no lane-dependent branch is needed.
    // Phase P (predicted states, all warps; the rotation puts the second pass
    // on the non-pair warps): plane offset of the leftmost stencil cell, then
    // the index into the predicted-state arrays.
    int p_src[PC::KP > 0 ? PC::KP : 1], p_dst[PC::KP > 0 ? PC::KP : 1];
#pragma unroll
    for (int k = 0; k < PC::KP; ++k) {
        const int base = (warp * 32 + PC::NPT) % NT + k * NT;
        if (base < PC::NXPr) {
            const int it = min(base + lane, PC::NXP - 1);
            const int cy = it / PC::XP, c0 = 2 * (it % PC::XP) - 1;
            p_src[k] = PV::idx(c0 - 1, cy, 0);
            p_dst[k] = cy * PC::XR + c0 + 1;
        } else {
            const int jj = min(base - PC::NXPr + lane, PC::NYP - 1);
            const int cy = jj / (TX / 2) - 1, cx = 2 * (jj % (TX / 2));
            p_src[k] = PV::idx(cx, cy, 0);
            p_dst[k] = PC::NPX + (cy + 1) * TX + cx;
        }
    }
    // Phase F (x/y face pairs, non-pair warps): source offset (predicted-state
    // index, or plane offset for first order) and face-array index.
    int f_src[PC::KF], f_dst[PC::KF];
#pragma unroll
    for (int k = 0; k < PC::KF; ++k) {
        const int base = (warp - PC::NPT / 32) * 32 + k * (NT - PC::NPT);
        if (base < PC::NXFr) {
            const int it = min(max(base + lane, 0), PC::NXF - 1);
            const int cy = it / PC::XP, f = 2 * (it % PC::XP);
            f_src[k] = MUSCL ? cy * PC::XR + f : PV::idx(f - 2, cy, 0);
            f_dst[k] = cy * PC::FXR + f;
        } else {
            const int jj = min(base - PC::NXFr + lane, PC::NYF - 1);
            const int fy = jj / (TX / 2), cx = 2 * (jj % (TX / 2));
            f_src[k] = MUSCL ? PC::NPX + fy * TX + cx : PV::idx(cx, fy - 1, 0);
            f_dst[k] = fy * TX + cx;
        }
    }

    // step scalars formed by thread 0 in FP64 and rounded to FP32 once
    float* sdt = reinterpret_cast<float*>(smem + 256);
    if (tid == 0) {
        // dt from the max wave-speed sum of the input state, in FP64 once per CTA
        const double dt = prm.cfl / __longlong_as_double((long long)ctl->smax[prm.slot_in]);
        sdt[0] = (float)dt;
        for (int d = 0; d < 3; ++d) {
            sdt[1 + d] = (float)(0.5 * dt * prm.inv_dx[d]);
            sdt[4 + d] = prm.inv_dx[d] > 0.0 ? (float)(0.5 / (dt * prm.inv_dx[d])) : 0.f;  // (dx/dt)/2 (FORCE)
        }
        if (blockIdx.x == 0 && prm.last) {
            ctl->t = prm.first ? dt : ctl->t + dt;
            ctl->dt_last = dt;
            ctl->smax[(prm.slot_in + 2) % 3] = 0ull;
        }
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        flags[0] = 0;
        fence_mbar_init();
        prefetch_tensormap(&map_in);
        prefetch_tensormap(&map_out);
    }
    __syncthreads();
    const f2 gamma = splat<f2>(prm.gamma_f), gm1 = splat<f2>(prm.gm1_f);
    const f2 dtv = splat<f2>(sdt[0]);
    f2 inv_dx[3], half_dtdx[3], half_inv_dtdx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        inv_dx[d] = splat<f2>(prm.inv_dx_f[d]);
        half_dtdx[d] = splat<f2>(sdt[1 + d]);
        half_inv_dtdx[d] = splat<f2>(sdt[4 + d]);
    }
    // axes of this launch: all (unsplit step) or one sweep of the split step
    const bool ax0 = prm.axis < 0 || prm.axis == 0;
    const bool ax1 = prm.axis < 0 || prm.axis == 1;
    const bool ax2 = DIM == 3 && (prm.axis < 0 || prm.axis == 2);


    auto item_planes = [&](int item) -> int {
        if (DIM == 2) return 1;
        const int chunk = item % sg.chunks_z;
        return min(sg.zchunk, g.n[2] - chunk * sg.zchunk) + 2 * R;
    };
    int ld_item = blockIdx.x, ld_j = 0;
    unsigned ld_seq = 0;
    auto issue_until = [&](unsigned limit) {
        while (ld_item < sg.items && ld_seq < limit) {
            const int item = ld_item;
            const int chunk = DIM == 3 ? item % sg.chunks_z : 0;
            const int tile = DIM == 3 ? item / sg.chunks_z : item;
            const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
            const int xs = g.lead + g.h + x0 - R - C::OFF;
            const int ys = g.h + y0 - R;
            const int slot = (int)(ld_seq % NS);
            float* dst = ring + (size_t)slot * (C::SLOT_BYTES / sizeof(float));
            mbar_arrive_expect_tx(&bars[slot], (uint32_t)(C::SLOT_ELEMS * sizeof(float)));
            if (DIM == 3) {
                const int pz = g.h + chunk * sg.zchunk - R + ld_j;
                if (LAYOUT == LAYOUT_SOA) tma_load_4d(dst, &map_in, xs, ys, pz, 0, &bars[slot]);
                else tma_load_3d(dst, &map_in, xs * NC, ys, pz, &bars[slot]);
            } else {
                if (LAYOUT == LAYOUT_SOA) tma_load_3d(dst, &map_in, xs, ys, 0, &bars[slot]);
                else tma_load_2d(dst, &map_in, xs * NC, ys, &bars[slot]);
            }
            ++ld_seq;
            if (++ld_j == item_planes(item)) { ld_j = 0; ld_item += gridDim.x; }
        }
    };

    unsigned ready_upto = 0, seq_base = 0;  // 32-bit plane sequence numbers
    int out_count = 0;
    bool store_pending = false;
    int st_x = 0, st_y = 0, st_z = 0, st_slot = 0;
    bool bad = false;
    float smax_local = 0.f;
    bool aborted = false;

    auto plane_ptr = [&](unsigned seq) -> const float* {
        return ring + (seq % NS) * (unsigned)(C::SLOT_BYTES / sizeof(float));
    };
    auto wait_planes = [&](unsigned need) {
        bool ok = true;
        for (unsigned sq = ready_upto; sq <= need; ++sq)
            ok &= mbar_wait_bounded(&bars[sq % NS], (uint32_t)((sq / NS) & 1));
        ready_upto = need + 1;
        if (!ok) flags[0] = 1;
    };
    auto store_tile = [&]() {
        const float* src = stage + (size_t)st_slot * (C::OUT_BYTES / sizeof(float));
        if (DIM == 3) {
            if (LAYOUT == LAYOUT_SOA) tma_store_4d(&map_out, src, st_x, st_y, st_z, 0);
            else tma_store_3d(&map_out, src, st_x * NC, st_y, st_z);
        } else {
            if (LAYOUT == LAYOUT_SOA) tma_store_3d(&map_out, src, st_x, st_y, 0);
            else tma_store_2d(&map_out, src, st_x * NC, st_y);
        }
        bulk_commit();
    };
    auto producer_step = [&](unsigned free_before) {
        if (tid != 0) return;
        if (store_pending) {
            store_tile();
            store_pending = false;
        }
        bulk_wait_read<1>();
        issue_until(free_before + NS);
    };
    // pair of the x-adjacent cells (o, o + SX) of a staged plane, all components
    auto load_pair = [&](const float* S, int o, f2 (&q)[NC]) {
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            if (LAYOUT == LAYOUT_SOA) q[m] = *reinterpret_cast<const f2*>(S + o + m * SM);
            else q[m] = f2{S[o + m * SM], S[o + SX + m * SM]};
        }
    };
    auto ld2 = [&](const float* a) -> f2 { return *reinterpret_cast<const f2*>(a); };
    auto st2 = [&](float* a, f2 v) { *reinterpret_cast<f2*>(a) = v; };

    for (int item = blockIdx.x; item < sg.items; item += gridDim.x) {
        const int chunk = DIM == 3 ? item % sg.chunks_z : 0;
        const int tile = DIM == 3 ? item / sg.chunks_z : item;
        const int x0 = (tile % sg.tiles_x) * TX, y0 = (tile / sg.tiles_x) * TY;
        const int z0 = chunk * sg.zchunk;
        const int zn = DIM == 3 ? min(sg.zchunk, g.n[2] - z0) : 1;
        const int gx = x0 + lx, gy = y0 + ly;
        const bool vx0 = pthr && (gx < g.n[0]) && (gy < g.n[1]);      // first cell of the pair
        const bool vx1 = pthr && (gx + 1 < g.n[0]) && (gy < g.n[1]);  // second cell
        const bool tma_store_ok = x0 + TX <= g.n[0];
        const bool near_xy = (x0 < g.h) || (x0 + TX > g.n[0] - g.h) || (y0 < g.h) || (y0 + TY > g.n[1] - g.h);
        float chk = 1.f;
        const int my_off = PV::idx(lx, ly, 0);

        f2 Fzm[NC], Fzp[NC], zR[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) Fzm[m] = Fzp[m] = zR[m] = f2{0.f, 0.f};

        // phase P of plane j: x/y predicted pairs -> shared arrays; z pairs in registers
        auto phase_p = [&](unsigned j, int z) {
            const float* S = plane_ptr(seq_base + j);
#pragma unroll
            for (int k = 0; k < PC::KP; ++k) {
                const int base = (warp * 32 + PC::NPT) % NT + k * NT;  // warp-uniform
                if (base < PC::NXPr) {
                    // x pair: cells (2q - 1, 2q) of row cy, read from cell 2q - 2 (even x)
                    f2 qm[NC], qc[NC], qp[NC], L[NC], Rr[NC];
                    const int o = p_src[k];
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
                    const int pi = p_dst[k];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        st2(PL + m * NP + pi, L[m]);
                        st2(PR + m * NP + pi, Rr[m]);
                    }
                } else if (base < PC::NXPr + PC::NYPr) {
                    // y pair: cells (cx, cy), (cx + 1, cy)
                    f2 qm[NC], qc[NC], qp[NC], L[NC], Rr[NC];
                    const int o = p_src[k];
                    load_pair(S, o - SY, qm);
                    load_pair(S, o, qc);
                    load_pair(S, o + SY, qp);
                    muscl<f2, DIM, 1>(qm, qc, qp, gm1, half_dtdx[1], L, Rr, chk);
                    const int pi = p_dst[k];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        st2(PL + m * NP + pi, L[m]);
                        st2(PR + m * NP + pi, Rr[m]);
                    }
                }
            }
        };

        __syncthreads();  // B0
        producer_step(seq_base);

        if (DIM == 3) {
            wait_planes(seq_base + (MUSCL ? 2 * R : 2 * R - 1));
            __syncthreads();
            if (flags[0]) { aborted = true; break; }
            if (pthr) {
                if (!MUSCL) {
                    if (ax2) {
                        f2 q0[NC], q1[NC];
                        load_pair(plane_ptr(seq_base + 0), my_off, q0);
                        load_pair(plane_ptr(seq_base + 1), my_off, q1);
                        pair_flux1<SCHEME, DIM, 2 % DIM>(q0, q1, gamma, gm1, half_dtdx[2], half_inv_dtdx[2], Fzm, chk);
                    }
                } else {
                    f2 q0[NC], q1[NC], q2[NC], q3[NC], L1[NC], R1[NC], L2[NC];
                    load_pair(plane_ptr(seq_base + 0), my_off, q0);
                    load_pair(plane_ptr(seq_base + 1), my_off, q1);
                    load_pair(plane_ptr(seq_base + 2), my_off, q2);
                    load_pair(plane_ptr(seq_base + 3), my_off, q3);
                    muscl<f2, DIM, 2 % DIM>(q0, q1, q2, gm1, half_dtdx[2], L1, R1, chk);
                    muscl<f2, DIM, 2 % DIM>(q1, q2, q3, gm1, half_dtdx[2], L2, zR, chk);
                    rus<f2, DIM, 2 % DIM>(R1, L2, gamma, gm1, Fzm, chk);
                }
            }
        } else {
            wait_planes(seq_base);
        }
        if (MUSCL) phase_p(DIM == 3 ? R : 0, z0);

        for (int zl = 0; zl < zn; ++zl) {
            const int z = z0 + zl;
            const unsigned jc = DIM == 3 ? (unsigned)(zl + R) : 0u;
            __syncthreads();  // B2
            if (flags[0]) { aborted = true; break; }
            producer_step(seq_base + jc);
            const float* S = plane_ptr(seq_base + jc);

            // ---------------- phase F: z work (pair threads), x/y face pairs (others) ----------------
            if (DIM == 3 && pthr) {
                if (!MUSCL) {
                    if (ax2) {
                        f2 q0[NC], q1[NC];
                        load_pair(S, my_off, q0);
                        load_pair(plane_ptr(seq_base + jc + 1), my_off, q1);
                        pair_flux1<SCHEME, DIM, 2 % DIM>(q0, q1, gamma, gm1, half_dtdx[2], half_inv_dtdx[2], Fzp, chk);
                    }
                } else {
                    // predicted states of plane z + 1 and the face z + 1/2
                    f2 q0[NC], q1[NC], q2[NC], L[NC], Rn[NC];
                    load_pair(S, my_off, q0);
                    load_pair(plane_ptr(seq_base + jc + 1), my_off, q1);
                    load_pair(plane_ptr(seq_base + jc + 2), my_off, q2);
                    muscl<f2, DIM, 2 % DIM>(q0, q1, q2, gm1, half_dtdx[2], L, Rn, chk);
                    rus<f2, DIM, 2 % DIM>(zR, L, gamma, gm1, Fzp, chk);
#pragma unroll
                    for (int m = 0; m < NC; ++m) zR[m] = Rn[m];
                }
            }
#pragma unroll
            for (int k = 0; k < PC::KF; ++k) {
                if (pthr) break;
                const int base = (warp - PC::NPT / 32) * 32 + k * (NT - PC::NPT);  // warp-uniform
                if (base < PC::NXFr) {
                    if (FORCE && !ax0) continue;
                    // x faces (f, f + 1), f = 2q, between cells f - 1 | f and f | f + 1
                    f2 a[NC], b[NC], F[NC];
                    if (MUSCL) {
                        const int i0 = f_src[k];  // x-predicted index of cell f - 1
#pragma unroll
                        for (int m = 0; m < NC; ++m) {
                            a[m] = ld2(PR + m * NP + i0);
                            const f2 u = ld2(PL + m * NP + i0), w = ld2(PL + m * NP + i0 + 2);
                            b[m] = f2{u.y, w.x};
                        }
                    } else {
                        const int o = f_src[k];  // cell f - 2: even x
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
                            a[m] = f2{A.y, B.x};
                            b[m] = B;
                        }
                    }
                    pair_flux1<SCHEME, DIM, 0>(a, b, gamma, gm1, half_dtdx[0], half_inv_dtdx[0], F, chk);
                    const int fi = f_dst[k];
#pragma unroll
                    for (int m = 0; m < NC; ++m) st2(FX + m * PC::NFX + fi, F[m]);
                } else if (base < PC::NXFr + PC::NYFr) {
                    if (FORCE && !ax1) continue;
                    f2 a[NC], b[NC], F[NC];
                    if (MUSCL) {
                        const int il = f_src[k], ir = il + TX;
#pragma unroll
                        for (int m = 0; m < NC; ++m) {
                            a[m] = ld2(PR + m * NP + il);
                            b[m] = ld2(PL + m * NP + ir);
                        }
                    } else {
                        const int o = f_src[k];
                        load_pair(S, o, a);
                        load_pair(S, o + SY, b);
                    }
                    pair_flux1<SCHEME, DIM, 1>(a, b, gamma, gm1, half_dtdx[1], half_inv_dtdx[1], F, chk);
                    const int fi = f_dst[k];
#pragma unroll
                    for (int m = 0; m < NC; ++m) st2(FY + m * PC::NFY + fi, F[m]);
                }
            }
            __syncthreads();  // B3

            // ---------------- phase U: pair threads ----------------
            if (pthr) {
                float* st = stage + (size_t)(out_count & 1) * (C::OUT_BYTES / sizeof(float));
                f2 qc[NC];
                load_pair(S, my_off, qc);
                f2 qn[NC];
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const float* fxr = FX + m * PC::NFX + ly * PC::FXR + lx;
                    const f2 fl = ld2(fxr), fn = ld2(fxr + 2);
                    const f2 fr = f2{fl.y, fn.x};
                    const f2 fyl = ld2(FY + m * PC::NFY + ly * TX + lx);
                    const f2 fyh = ld2(FY + m * PC::NFY + (ly + 1) * TX + lx);
                    f2 acc;
                    if constexpr (FORCE) {  // one axis per sweep
                        acc = ax0 ? (fr - fl) * inv_dx[0] : f2{0.f, 0.f};
                        if (ax1) acc = fma_v(fyh - fyl, inv_dx[1], acc);
                        if (ax2) acc = fma_v(Fzp[m] - Fzm[m], inv_dx[2], acc);
                    } else {
                        acc = (fr - fl) * inv_dx[0];
                        acc = fma_v(fyh - fyl, inv_dx[1], acc);
                        if (DIM == 3) acc = fma_v(Fzp[m] - Fzm[m], inv_dx[2], acc);
                    }
                    qn[m] = fma_v(f2{-dtv.x, -dtv.y}, acc, qc[m]);
                    if (tma_store_ok) {
                        if (LAYOUT == LAYOUT_SOA) st2(st + (m * TY + ly) * TX + lx, qn[m]);
                        else {
                            st[(ly * TX + lx) * NC + m] = qn[m].x;
                            st[(ly * TX + lx + 1) * NC + m] = qn[m].y;
                        }
                    }
                }
                if (DIM == 3) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) Fzm[m] = Fzp[m];
                }
                fence_proxy_async_smem();
                // epilogue: wave-speed sums and checks of both cells at once;
                // cells outside the domain (ragged tiles) take no part in either
                bool ok0, ok1;
                const f2 sw = wave_sum2<DIM>(qn, gamma, gm1, inv_dx, ok0, ok1);
                smax_local = fmaxf(smax_local, fmaxf(vx0 ? sw.x : 0.f, vx1 ? sw.y : 0.f));
                const bool bad0 = vx0 && !ok0, bad1 = vx1 && !ok1;
                if (bad0 || bad1) {
                    bad = true;
                    record_bad(ctl, BAD_CELL, bad0 ? gx : gx + 1, gy, z);
                }
                // tile-uniform: ragged tiles store directly; edge tiles write ghost images
                if (!tma_store_ok || near_xy || (DIM == 3 && (z < g.h || z >= g.n[2] - g.h))) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (!(h == 0 ? vx0 : vx1)) continue;
                        float q1[NC];
#pragma unroll
                        for (int m = 0; m < NC; ++m) q1[m] = h == 0 ? qn[m].x : qn[m].y;
                        if (!tma_store_ok) {
                            const long long base = geom_cell(g, gx + h, gy, z) * g.cell_stride;
#pragma unroll
                            for (int m = 0; m < NC; ++m) out[base + (long long)m * g.comp_stride] = q1[m];
                        }
                        if (near_xy || (DIM == 3 && (z < g.h || z >= g.n[2] - g.h)))
                            write_ghost_images<float, DIM>(out, g, prm.bc, gx + h, gy, z, q1);
                    }
                }
            }
            if (tma_store_ok) {
                store_pending = true;
                st_x = x0; st_y = y0; st_z = z; st_slot = out_count & 1;
                ++out_count;
            }
            if (!(chk > 0.f)) {
                bad = true;
                record_bad(ctl, BAD_STATE, x0, y0, z);
                chk = 1.f;
            }
            // ---------------- phase P of the next plane ----------------
            if (DIM == 3 && zl + 1 < zn) {
                wait_planes(seq_base + jc + 1 + R);
                if (MUSCL) phase_p(jc + 1, z + 1);
            }
        }
        if (aborted) break;
        seq_base += DIM == 3 ? (unsigned)(zn + 2 * R) : 1u;
    }

    __syncthreads();
    if (tid == 0) {
        if (store_pending && !aborted) store_tile();
        bulk_wait<0>();
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
        if (prm.last) atomic_max_pos_double(&ctl->smax[(prm.slot_in + 1) % 3], m);
        if (any_bad) atomicOr(&ctl->err, DEV_ERR_NUMERIC);
    }
}

}  // namespace ripple
