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
// bar[0] counts arrivals over the whole launch and is never reset: the k-th
// barrier (k = 1, 2, ...) opens once the count reaches k x gridDim.x, so a block
// only adds one and waits for that multiple (the launch starts with bar[0] = 0,
// and passes fewer than 2^32 / gridDim.x barriers).  The wait is bounded: once
// timeout_ns has passed (global timer) the block records ST_TIMEOUT in *status
// and returns false; every block then leaves at its next barrier.  When
// waited_ns is given, thread 0 of a block that waited stores how long it did.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int32_t *status,
                                             unsigned long long timeout_ns = BARRIER_TIMEOUT_NS,
                                             unsigned long long *waited_ns = nullptr) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(bar, 1u);
        const unsigned target = ticket - ticket % gridDim.x + gridDim.x;
        int ok = 1;
        if (ticket + 1u != target) {
            volatile unsigned *count = bar;
            const unsigned long long t0 = global_ns();
            unsigned long long polls = 0, now = t0;
            while ((int)(*count - target) < 0) {
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

// Bounds checks of the debug build (compiled with -DQC_DEBUG, library
// libqcgraph_debug.so): every neighbour id a kernel reads from the CSR passes
// through checked_id before it is used as an index.  An id outside [0, n)
// records `code` in the device word qc_debug_word (the first failure wins) and
// is replaced by 0, so the kernel ends normally and the host reports
// QC_ERR_INVALID_GRAPH naming the check, instead of an out-of-range access.
// Release builds compile the checks away.
enum : int32_t {
    DBG_BFS = 1, DBG_PREP = 2, DBG_GGD = 3, DBG_BATCH = 4, DBG_WEIGHTED = 5, DBG_NOALLOC = 6, DBG_SELFTEST = 7
};
#ifdef QC_DEBUG
extern __device__ int32_t qc_debug_word;
__device__ __forceinline__ int checked_id(int id, int n, int32_t code) {
    if ((unsigned)id < (unsigned)n) return id;
    atomicCAS(&qc_debug_word, 0, code);
    return 0;
}
#else
__device__ __forceinline__ int checked_id(int id, int, int32_t) { return id; }
#endif

}  // namespace qcdev
