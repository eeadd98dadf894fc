// Device helpers shared by the persistent (cooperative) kernels.
#pragma once

#include <cstdint>

// Degree bucket (floor(log2(deg + 1))) from which a row counts as heavy: its BFS
// item is shared by all warps of a block instead of one warp.
#define QC_HEAVY_BUCKET 7

namespace qcdev {

enum : int32_t { ST_DONE = 0, ST_NEED_ROWS = 1, ST_TIMEOUT = 2 };

// ~100 ns per spin: more than a second before a wait gives up.
constexpr unsigned long long BARRIER_SPINS = 1ull << 24;

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// bar[0] counts arrivals, bar[1] is the generation.  The spin is bounded: on
// expiry the block records ST_TIMEOUT in *status and returns false; every
// block then leaves at its next barrier.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int32_t *status,
                                             unsigned long long spin_limit = BARRIER_SPINS) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == gen) {
                if (++spins > spin_limit) {
                    atomicExch(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok_s = ok && (*(volatile int32_t *)status != ST_TIMEOUT);
    }
    __syncthreads();
    return ok_s;
}

}  // namespace qcdev
