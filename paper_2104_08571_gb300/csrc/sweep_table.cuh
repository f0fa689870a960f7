// Compile-time table of Euler sweep kernels for one element type: every
// (dim, layout, scheme, tile variant) combination whose shared memory fits.
#pragma once
#include <type_traits>

#include "euler_sweep_pair.cuh"
#include "euler_sweep_pair3.cuh"
#include "euler_sweep_row3.cuh"
#include "runtime.h"

namespace ripple {

constexpr int kMaxDynSmem = 227 * 1024;

// The kernel behind a table entry: the one-cell kernel, or for the pair
// variant with FP32 fields the packed cell-pair kernel.
template <typename T, int DIM, int LAYOUT, int SCHEME, int V>
struct SweepKernel {
    static constexpr bool pair = V == kPairVariant;
    static constexpr bool row = V == kRowVariant;
    static constexpr int TX = kSweepVariants[V].tx;
    static constexpr int TY = kSweepVariants[V].ty;
    static constexpr bool f32 = std::is_same<T, float>::value;
    // the pair kernels cover every FP32 scheme (the split FORCE step one sweep per
    // launch); the row kernel only the FP32 3D MUSCL-Hancock step
    static constexpr bool exists = row ? (f32 && DIM == 3 && SCHEME == SCHEME_MUSCL) : (!pair || f32);
    // 3D MUSCL-Hancock: the split-barrier schedule (euler_sweep_pair3.cuh)
    static constexpr bool pair3 = pair && DIM == 3 && SCHEME == SCHEME_MUSCL;
    static constexpr int smem()
    {
        if constexpr (row) return Row3Cfg<LAYOUT>::SMEM;
        else if constexpr (pair3) return Pair3Cfg<LAYOUT>::SMEM;
        else if constexpr (pair) return PairCfg<DIM, LAYOUT, SCHEME>::SMEM;
        else return SweepCfg<T, DIM, LAYOUT, SCHEME, TX, TY>::SMEM;
    }
    static constexpr int nt() { return row ? Row3Cfg<LAYOUT>::NT : TX * TY; }
    static auto fn()
    {
        if constexpr (row && exists) return euler_sweep_row3_kernel<LAYOUT>;
        else if constexpr (pair3 && f32) return euler_sweep_pair3_kernel<LAYOUT>;
        else if constexpr (pair && f32) return euler_sweep_pair_kernel<DIM, LAYOUT, SCHEME>;
        else return euler_sweep_kernel<T, DIM, LAYOUT, SCHEME, (row ? 32 : TX), (row ? 8 : TY)>;
    }
};

template <typename T, int DIM, int LAYOUT, int SCHEME, int V>
struct SweepEntry {
    using K = SweepKernel<T, DIM, LAYOUT, SCHEME, V>;
    static constexpr int TX = K::TX;
    static constexpr int TY = K::TY;
    struct SmemOnly {
        static constexpr int SMEM = K::exists ? K::smem() : 0;
        static constexpr int NT = K::nt();
    };
    using C = SmemOnly;
    static constexpr bool fits = K::exists && C::SMEM > 0 && C::SMEM <= kMaxDynSmem;

    static cudaError_t launch(const SweepLaunch& L)
    {
        if constexpr (!fits) {
            return cudaErrorInvalidValue;
        } else {
            auto k = K::fn();
            static bool configured = false;
            if (!configured) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
                if (e != cudaSuccess) return e;
                configured = true;
            }
            k<<<L.grid, C::NT, C::SMEM, L.stream>>>(*L.map_in, *L.map_out, static_cast<T*>(L.out), L.ctl, L.sg,
                                                    L.prm);
            return cudaGetLastError();
        }
    }
    static int smem() { return fits ? C::SMEM : 0; }
    static int occupancy()
    {
        if constexpr (!fits) {
            return 0;
        } else {
            auto k = K::fn();
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
                return 0;
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, C::NT, C::SMEM) != cudaSuccess) return 0;
            return n;
        }
    }
};

template <typename T, int DIM, int LAYOUT, int SCHEME>
struct SweepRow {
    template <int V>
    static cudaError_t launch_v(int v, const SweepLaunch& L)
    {
        if constexpr (V >= kNumSweepVariants) {
            return cudaErrorInvalidValue;
        } else {
            if (v == V) return SweepEntry<T, DIM, LAYOUT, SCHEME, V>::launch(L);
            return launch_v<V + 1>(v, L);
        }
    }
    template <int V>
    static int smem_v(int v)
    {
        if constexpr (V >= kNumSweepVariants) {
            return 0;
        } else {
            if (v == V) return SweepEntry<T, DIM, LAYOUT, SCHEME, V>::smem();
            return smem_v<V + 1>(v);
        }
    }
    template <int V>
    static int occ_v(int v)
    {
        if constexpr (V >= kNumSweepVariants) {
            return 0;
        } else {
            if (v == V) return SweepEntry<T, DIM, LAYOUT, SCHEME, V>::occupancy();
            return occ_v<V + 1>(v);
        }
    }
};

// Dispatch on (layout, scheme) for a fixed dim.
template <typename T, int DIM>
struct SweepDim {
    static cudaError_t launch(int layout, int scheme, int v, const SweepLaunch& L)
    {
        if (layout == LAYOUT_SOA) {
            if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_MUSCL>::template launch_v<0>(v, L);
            if (scheme == SCHEME_FORCE) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_FORCE>::template launch_v<0>(v, L);
            return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_RUSANOV1>::template launch_v<0>(v, L);
        }
        if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_MUSCL>::template launch_v<0>(v, L);
        if (scheme == SCHEME_FORCE) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_FORCE>::template launch_v<0>(v, L);
        return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_RUSANOV1>::template launch_v<0>(v, L);
    }
    static int smem(int layout, int scheme, int v)
    {
        if (layout == LAYOUT_SOA) {
            if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_MUSCL>::template smem_v<0>(v);
            if (scheme == SCHEME_FORCE) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_FORCE>::template smem_v<0>(v);
            return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_RUSANOV1>::template smem_v<0>(v);
        }
        if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_MUSCL>::template smem_v<0>(v);
        if (scheme == SCHEME_FORCE) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_FORCE>::template smem_v<0>(v);
        return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_RUSANOV1>::template smem_v<0>(v);
    }
    static int occ(int layout, int scheme, int v)
    {
        if (layout == LAYOUT_SOA) {
            if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_MUSCL>::template occ_v<0>(v);
            if (scheme == SCHEME_FORCE) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_FORCE>::template occ_v<0>(v);
            return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_RUSANOV1>::template occ_v<0>(v);
        }
        if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_MUSCL>::template occ_v<0>(v);
        if (scheme == SCHEME_FORCE) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_FORCE>::template occ_v<0>(v);
        return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_RUSANOV1>::template occ_v<0>(v);
    }
};

}  // namespace ripple
