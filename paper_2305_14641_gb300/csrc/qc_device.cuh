// Device helpers shared by the persistent (cooperative) kernels.
#pragma once

#include <cstdint>

// Degree bucket (floor(log2(deg + 1))) from which a row counts as heavy: its BFS
// item is shared by all warps of a block instead of one warp.
#define QC_HEAVY_BUCKET 7

namespace qcdev {

enum : int32_t { ST_DONE = 0, ST_NEED_ROWS = 1, ST_TIMEOUT = 2 };

// A grid-barrier wait gives up once this much time has passed on the GPU's
// global timer (the longest level of any launch here takes milliseconds).
constexpr unsigned long long BARRIER_TIMEOUT_NS = 2000000000ull;
// Backstop in case the global timer does not advance: polls of >= 100 ns each.
constexpr unsigned long long BARRIER_MAX_POLLS = 1ull << 27;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// bar[0] counts arrivals, bar[1] is the generation.  The wait is bounded: once
// timeout_ns has passed (global timer) the block records ST_TIMEOUT in *status
// and returns false; every block then leaves at its next barrier.  When
// waited_ns is given, thread 0 of a block that waited stores how long it did.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int32_t *status,
                                             unsigned long long timeout_ns = BARRIER_TIMEOUT_NS,
                                             unsigned long long *waited_ns = nullptr) {
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
            const unsigned long long t0 = global_ns();
            unsigned long long polls = 0, now = t0;
            while (*vgen == gen) {
                now = global_ns();
                if (now - t0 > timeout_ns || ++polls > BARRIER_MAX_POLLS) {
                    atomicExch(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
            if (waited_ns) *waited_ns = now - t0;
        }
        __threadfence();
        ok_s = ok && (*(volatile int32_t *)status != ST_TIMEOUT);
    }
    __syncthreads();
    return ok_s;
}

}  // namespace qcdev
