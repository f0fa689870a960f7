// Bounded grid-wide barrier of the persistent cooperative kernels (the FIM
// solve and the multi-step solo Euler solver).
#pragma once
#include <cstdint>
#include <cstdlib>

namespace ripple {

// Default bound on the polls of a grid-barrier wait (several seconds).  The
// host may lower it (RIPPLE_GRID_SPIN_LIMIT) to exercise the timeout path.
constexpr uint32_t kGridSpinLimit = 1u << 26;

inline unsigned grid_spin_limit()
{
    unsigned limit = kGridSpinLimit;
    if (const char* lim = std::getenv("RIPPLE_GRID_SPIN_LIMIT")) {
        char* end = nullptr;
        const unsigned long v = std::strtoul(lim, &end, 10);
        if (end != lim && v < kGridSpinLimit) limit = (unsigned)v;
    }
    return limit;
}

// Bounded sense-reversal grid barrier over bar[0] (arrivals, reset by the
// last arrival) and bar[1] (generation).  Every CTA of the grid calls it the
// same number of times; sflag (shared memory) records a wait that ran out, and
// the call returns false from then on.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned spin_limit, int* sflag)
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
            while (*gen == g0) {
                if (i++ >= spin_limit) {
                    sflag[0] = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return sflag[0] == 0;
}

}  // namespace ripple
