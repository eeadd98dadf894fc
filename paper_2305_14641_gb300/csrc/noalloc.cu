// Distance histogram without any device allocation.
//
// Some callers cannot let a library allocate GPU memory: an application that
// carves the device memory into a fixed plan at start-up and forbids later
// cudaMalloc calls, a host program that hands the library only the buffers it
// owns (a plugin inside a renderer or a serving process with its own memory
// pool), or code running where an allocation would block or fail (a real-time
// loop, a process at its memory limit).  qc_histogram_static_scratch serves
// them: it computes the same per-node hop-distance histogram as
// qc_graph_histogram, but its working bitsets live in one fixed-size array that
// is part of the library image, so the call itself allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds QC_STATIC_SCRATCH_BYTES of it until the process exits.  Host
// code cannot use the variable's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device looks up the
// real address with cudaGetSymbolAddress, with that device current, and keeps
// it.  All calls share the array and it keeps the last call's contents: every
// call clears what must start at zero, and calls that overlap on the GPU (two
// streams, two threads) race on it.
//
// The kernels here are a plain bitset BFS (one warp per node, one 16-byte
// segment of 128 sources per lane and tile), independent of the tuned kernels
// of the regular path.
#include <cstring>
#include <mutex>

#include "qc_device.cuh"
#include "qc_internal.h"

#define QC_STATIC_SCRATCH_BYTES (16u << 20)
#define QC_STATIC_SCRATCH_MAX_NODES 262144

static __device__ __align__(256) unsigned char qc_static_scratch[QC_STATIC_SCRATCH_BYTES];

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t ONES = ~0ull;

__global__ void sa_first_rows(int32_t n, const int32_t *row_ptr, int32_t *hist) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        hist[v] = 1;
        hist[(size_t)n + v] = row_ptr[v + 1] - row_ptr[v];
    }
}

// Row of node v = sources of the chunk that are v or its neighbours, plus the
// always-set bits (sources >= n, padding word).  One thread per node.
__global__ void sa_init(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t w0,
                        int32_t wn, int32_t stride, int32_t last_word, uint64_t last_mask,
                        uint64_t *vis) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t *row = vis + (size_t)v * stride;
        for (int k = 0; k < stride; ++k) row[k] = (k < wn) ? 0ull : ONES;
        if (last_word >= w0 && last_word < w0 + wn) row[last_word - w0] |= last_mask;
        int k = (v >> 6) - w0;
        if (k >= 0 && k < wn) row[k] |= 1ull << (v & 63);
        for (int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const int u = qcdev::checked_id(col_idx[e], n, qcdev::DBG_NOALLOC);
            k = (u >> 6) - w0;
            if (k >= 0 && k < wn) row[k] |= 1ull << (u & 63);
        }
    }
}

// next = (OR of neighbours' rows) & ~own; out = own | next; hist[level][v] += popc(next).
// hist_row may be null: the pass then only reports (in *flag) whether anything
// is new, for the level just past the caller's last histogram row.
__global__ void sa_level(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                         const ulonglong2 *vin, ulonglong2 *vout, int32_t R, int32_t *hist_row,
                         int32_t *flag) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    bool any_new = false;
    for (int v = warp; v < n; v += nwarps) {
        int count = 0;
        const int beg = row_ptr[v], end = row_ptr[v + 1];
        for (int q0 = 0; q0 < R; q0 += 32) {
            const int q = q0 + lane;
            const bool mine = q < R;
            const ulonglong2 own = mine ? vin[(size_t)v * R + q] : make_ulonglong2(ONES, ONES);
            ulonglong2 acc = make_ulonglong2(0, 0);
            for (int e = beg; e < end; ++e) {
                const int u = qcdev::checked_id(col_idx[e], n, qcdev::DBG_NOALLOC);
                if (mine) {
                    const ulonglong2 x = vin[(size_t)u * R + q];
                    acc.x |= x.x;
                    acc.y |= x.y;
                }
            }
            if (mine) {
                const ulonglong2 nw = make_ulonglong2(acc.x & ~own.x, acc.y & ~own.y);
                vout[(size_t)v * R + q] = make_ulonglong2(own.x | nw.x, own.y | nw.y);
                count += __popcll(nw.x) + __popcll(nw.y);
            }
        }
        count = __reduce_add_sync(FULL, count);
        if (lane == 0 && count) {
            if (hist_row) hist_row[v] += count;
            any_new = true;
        }
    }
    if (__syncthreads_or(any_new) && threadIdx.x == 0) *flag = 1;
}

std::mutex g_mu;
void *g_addr[128];

// The scratch array's device address on the current device (looked up once).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, qc_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" qc_status qc_histogram_static_scratch(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                                 const int32_t *col_idx, int32_t *hist_out,
                                                 int32_t max_levels, int32_t *D_out, void *stream_) {
    if (n < 1 || n > QC_STATIC_SCRATCH_MAX_NODES || nnz < 0 || nnz >= (int64_t(1) << 31) ||
        !row_ptr || (nnz > 0 && !col_idx) || !hist_out || !D_out || max_levels < 2)
        return QC_ERR_INVALID_ARG;
    *D_out = -1;
    cudaStream_t stream = qc_stream(stream_);
    // the array's address is looked up on the current device, so the stream must
    // belong to that device too
    int dev = 0, stream_dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(stream, &stream_dev) != cudaSuccess)
        return QC_ERR_CUDA;
    if (stream_dev != dev) return QC_ERR_INVALID_ARG;
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return QC_ERR_CUDA;

    // layout of the array: [level flag, 256 B] [bitset rows A] [bitset rows B]
    const int64_t W = (n + 63) / 64;
    const size_t avail = QC_STATIC_SCRATCH_BYTES - 256;
    int64_t wc = (int64_t)(avail / (2 * 8 * (size_t)n));
    wc &= ~int64_t(1);                 // whole 16-byte segments
    if (wc < 2) return QC_ERR_INVALID_ARG;
    if (wc > W) wc = W;
    int32_t *flag = reinterpret_cast<int32_t *>(base);
    const int32_t Rmax = (int32_t)((wc + 1) / 2);
    ulonglong2 *visA = reinterpret_cast<ulonglong2 *>(static_cast<unsigned char *>(base) + 256);
    ulonglong2 *visB = visA + (size_t)Rmax * n;

    if (cudaMemsetAsync(hist_out, 0, sizeof(int32_t) * (size_t)max_levels * n, stream) != cudaSuccess)
        return QC_ERR_CUDA;
    const int nb = qc_ceil_div(n, 256) < 1024 ? qc_ceil_div(n, 256) : 1024;
    sa_first_rows<<<nb, 256, 0, stream>>>(n, row_ptr, hist_out);
    if (cudaGetLastError() != cudaSuccess) return QC_ERR_CUDA;
    int32_t D = nnz > 0 ? 1 : 0;
    const int32_t last_word = (int32_t)(W - 1);
    const uint64_t last_mask = (n % 64) ? (ONES << (n % 64)) : 0ull;
    for (int64_t w0 = 0; nnz > 0 && w0 < W; w0 += wc) {
        const int32_t wn = (int32_t)((W - w0) < wc ? (W - w0) : wc);
        const int32_t R = (wn + 1) / 2;
        sa_init<<<qc_ceil_div(n, 128), 128, 0, stream>>>(n, row_ptr, col_idx, (int32_t)w0, wn, 2 * R,
                                                         last_word, last_mask,
                                                         reinterpret_cast<uint64_t *>(visA));
        if (cudaGetLastError() != cudaSuccess) return QC_ERR_CUDA;
        ulonglong2 *in = visA, *out = visB;
        for (int32_t level = 2;; ++level) {
            // The BFS ends with a pass that finds nothing new, one level past D.
            // When that level has no row in hist_out (D = max_levels - 1), the pass
            // runs without a row: if it does find new sources, hist_out is too short.
            const bool past_rows = level >= max_levels;
            if (cudaMemsetAsync(flag, 0, sizeof(int32_t), stream) != cudaSuccess) return QC_ERR_CUDA;
            const int blocks = qc_ceil_div(n, 8) < 4096 ? qc_ceil_div(n, 8) : 4096;
            sa_level<<<blocks, 256, 0, stream>>>(n, row_ptr, col_idx, in, out, R,
                                                 past_rows ? nullptr : hist_out + (size_t)level * n, flag);
            if (cudaGetLastError() != cudaSuccess) return QC_ERR_CUDA;
            int32_t h_flag = 0;
            if (cudaMemcpyAsync(&h_flag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess)
                return QC_ERR_CUDA;
            if (!h_flag) break;
            if (past_rows) return QC_ERR_INVALID_ARG;   // a distance of max_levels or more
            if (level > D) D = level;
            ulonglong2 *t = in;
            in = out;
            out = t;
        }
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) return QC_ERR_CUDA;
    QC_TRY(qc_debug_take(nullptr));
    *D_out = D;
    return QC_OK;
}
