// Compile-time table of Euler sweep kernels for one element type: every
// (dim, layout, scheme, tile variant) combination whose shared memory fits.
#pragma once
#include "runtime.h"

namespace ripple {

constexpr int kMaxDynSmem = 227 * 1024;

template <typename T, int DIM, int LAYOUT, int SCHEME, int V>
struct SweepEntry {
    static constexpr int TX = kSweepVariants[V].tx;
    static constexpr int TY = kSweepVariants[V].ty;
    using C = SweepCfg<T, DIM, LAYOUT, SCHEME, TX, TY>;
    static constexpr bool fits = C::SMEM <= kMaxDynSmem;

    static cudaError_t launch(const SweepLaunch& L)
    {
        if constexpr (!fits) {
            return cudaErrorInvalidValue;
        } else {
            auto k = euler_sweep_kernel<T, DIM, LAYOUT, SCHEME, TX, TY>;
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
            auto k = euler_sweep_kernel<T, DIM, LAYOUT, SCHEME, TX, TY>;
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
            return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_RUSANOV1>::template launch_v<0>(v, L);
        }
        if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_MUSCL>::template launch_v<0>(v, L);
        return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_RUSANOV1>::template launch_v<0>(v, L);
    }
    static int smem(int layout, int scheme, int v)
    {
        if (layout == LAYOUT_SOA) {
            if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_MUSCL>::template smem_v<0>(v);
            return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_RUSANOV1>::template smem_v<0>(v);
        }
        if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_MUSCL>::template smem_v<0>(v);
        return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_RUSANOV1>::template smem_v<0>(v);
    }
    static int occ(int layout, int scheme, int v)
    {
        if (layout == LAYOUT_SOA) {
            if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_MUSCL>::template occ_v<0>(v);
            return SweepRow<T, DIM, LAYOUT_SOA, SCHEME_RUSANOV1>::template occ_v<0>(v);
        }
        if (scheme == SCHEME_MUSCL) return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_MUSCL>::template occ_v<0>(v);
        return SweepRow<T, DIM, LAYOUT_AOS, SCHEME_RUSANOV1>::template occ_v<0>(v);
    }
};

}  // namespace ripple
