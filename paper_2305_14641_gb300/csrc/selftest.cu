// Self-test of the bounded device wait.  Every persistent kernel of the library
// synchronises its blocks with qcdev::grid_barrier, whose wait gives up after a
// fixed time on the GPU's global timer, records a timeout and lets the kernel return, so a
// block that never arrives ends in QC_ERR_TIMEOUT on the host instead of a hung
// GPU.  This entry point runs that barrier with one block that never arrives.
#include "qc_device.cuh"
#include "qc_internal.h"

#ifdef QC_DEBUG
namespace qcdev {
__device__ int32_t qc_debug_word = 0;
}
#endif

qc_status qc_debug_take(qc_ctx *ctx) {
#ifdef QC_DEBUG
    int32_t w = 0;
    QC_CUDA_TRY(ctx, cudaMemcpyFromSymbol(&w, qcdev::qc_debug_word, sizeof(w)));
    if (w == 0) return QC_OK;
    const int32_t zero = 0;
    QC_CUDA_TRY(ctx, cudaMemcpyToSymbol(qcdev::qc_debug_word, &zero, sizeof(zero)));
    static const char *where[] = {"", "BFS", "graph preparation", "descent", "batched kernel",
                                  "weighted shortest paths", "no-alloc histogram", "self-test"};
    qc_set_error(ctx, "debug build: a neighbour id outside [0, n) reached the %s kernels (check %d)",
                 (w > 0 && w < 8) ? where[w] : "?", w);
    return QC_ERR_INVALID_GRAPH;
#else
    (void)ctx;
    return QC_OK;
#endif
}

namespace {

// Block 0 waits at the barrier; block 1 leaves without arriving.
__global__ void missing_arrival(unsigned *bar, int32_t *status, unsigned long long timeout_ns,
                                unsigned long long *waited_ns) {
    if (blockIdx.x != 0) return;
    qcdev::grid_barrier(bar, status, timeout_ns, waited_ns);
}

}  // namespace

extern "C" qc_status qc_selftest_barrier_timeout(qc_ctx *ctx, int64_t timeout_us, int64_t *waited_ns,
                                                 void *stream_) {
    if (!ctx || timeout_us < 1 || timeout_us > 10000000) return QC_ERR_INVALID_ARG;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_buffer ctl;
    QC_TRY(ctl.allocate(ctx, 8 * sizeof(int32_t), stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(ctl.ptr, 0, ctl.bytes, stream));
    int32_t *status = ctl.as<int32_t>();
    unsigned *bar = reinterpret_cast<unsigned *>(status + 2);
    unsigned long long *waited = reinterpret_cast<unsigned long long *>(status + 4);
    unsigned long long timeout_ns = 1000ull * (unsigned long long)timeout_us;
    void *args[] = {(void *)&bar, (void *)&status, (void *)&timeout_ns, (void *)&waited};
    QC_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void *)missing_arrival, dim3(2), dim3(32), args, 0,
                                                 stream));
    QC_LAUNCHED(ctx);
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h = static_cast<int32_t *>(pin.ptr);
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, status, 6 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    const unsigned long long w = *reinterpret_cast<const unsigned long long *>(h + 4);
    if (waited_ns) *waited_ns = (int64_t)w;
    if (h[0] != qcdev::ST_TIMEOUT) {
        qc_set_error(ctx, "qc_selftest_barrier_timeout: the barrier did not report the missing arrival");
        return QC_ERR_CUDA;
    }
    qc_set_error(ctx, "grid barrier gave up after %.3f ms (limit %.3f ms; one block never arrived)", w * 1e-6,
                 timeout_us * 1e-3);
    return QC_ERR_TIMEOUT;
}

// ---- L2 read bandwidth probe --------------------------------------------------------
// The roofline of an L2-resident kernel: read throughput of a buffer that fits in
// L2, through L2 only (ld.global.cg), either streamed (each thread 16 bytes at a
// time, consecutive across the grid) or as 512-byte segments at pseudo-random
// positions, a warp reading one whole segment per load (16 bytes per lane) with
// four loads in flight, the access pattern of the BFS's neighbour gathers.

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

__global__ void l2_stream(const ulonglong2 *__restrict__ buf, size_t n16, int passes, unsigned long long *sink) {
    unsigned long long acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < passes; ++r)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const ulonglong2 x = __ldcg(buf + i);
            acc ^= x.x ^ x.y;
        }
    if (acc == 0x9e3779b97f4a7c15ull) sink[0] = acc;   // keeps the loads
}

__global__ void l2_segments(const ulonglong2 *__restrict__ buf, uint32_t nseg, int per_warp, unsigned long long *sink) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long acc = 0;
    for (int k = 0; k < per_warp; k += 4) {
        ulonglong2 x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t seg = mix32(warp * 0x9e3779b9U + (uint32_t)(k + j)) % nseg;
            x[j] = __ldcg(buf + (size_t)seg * 32 + lane);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) acc ^= x[j].x ^ x[j].y;
    }
    if (acc == 0x9e3779b97f4a7c15ull) sink[0] = acc;
}

}  // namespace

extern "C" qc_status qc_selftest_l2_read(qc_ctx *ctx, int64_t bytes, int32_t mode, double *gbs, void *stream_) {
    if (!ctx || !gbs || bytes < (1 << 20) || bytes > ((int64_t)1 << 32) || (mode != 0 && mode != 1))
        return QC_ERR_INVALID_ARG;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t n16 = (size_t)bytes / 16;
    qc_buffer buf, sink;
    QC_TRY(buf.allocate(ctx, n16 * 16, stream));
    QC_TRY(sink.allocate(ctx, 64, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(buf.ptr, 0x5a, buf.bytes, stream));
    qc_event_pair ev;
    QC_TRY(ev.create(ctx));
    const int blocks = 4 * ctx->num_sms;
    const uint32_t nseg = (uint32_t)(n16 / 32);
    // about 64 reads of the buffer per timed launch; the first launch warms L2
    const int passes = 64;
    const int per_warp = (int)(((double)passes * n16 * 16) / (512.0 * blocks * 8)) & ~3;
    double moved = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) QC_CUDA_TRY(ctx, cudaEventRecord(ev.a, stream));
        if (mode == 0) {
            l2_stream<<<blocks, 256, 0, stream>>>(buf.as<ulonglong2>(), n16, passes, sink.as<unsigned long long>());
            moved = (double)passes * n16 * 16;
        } else {
            l2_segments<<<blocks, 256, 0, stream>>>(buf.as<ulonglong2>(), nseg, per_warp, sink.as<unsigned long long>());
            moved = (double)per_warp * 512.0 * blocks * 8;
        }
        QC_LAUNCHED(ctx);
        if (rep == 1) QC_CUDA_TRY(ctx, cudaEventRecord(ev.b, stream));
    }
    QC_CUDA_TRY(ctx, cudaEventSynchronize(ev.b));
    float ms = 0.f;
    QC_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ev.a, ev.b));
    *gbs = moved / (ms * 1e-3) / 1e9;
    return QC_OK;
}

// ---- self-test of the debug build's bounds checks ------------------------------------

namespace {

// Passes `id` through the check (never using it as an address) and stores the id
// that comes out.
__global__ void debug_check_kernel(int32_t id, int32_t n, int32_t *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = qcdev::checked_id(id, n, qcdev::DBG_SELFTEST);
}

}  // namespace

extern "C" qc_status qc_selftest_debug_check(qc_ctx *ctx, int32_t id, int32_t n, int32_t *checked_out,
                                             int32_t *debug_build, void *stream_) {
    if (!ctx || !checked_out || !debug_build || n < 1) return QC_ERR_INVALID_ARG;
#ifdef QC_DEBUG
    *debug_build = 1;
#else
    *debug_build = 0;
#endif
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_buffer out;
    QC_TRY(out.allocate(ctx, sizeof(int32_t), stream));
    debug_check_kernel<<<1, 32, 0, stream>>>(id, n, out.as<int32_t>());
    QC_LAUNCHED(ctx);
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(checked_out, out.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    return qc_debug_take(ctx);
}
