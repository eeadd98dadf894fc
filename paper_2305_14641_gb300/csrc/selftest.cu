// Self-test of the bounded device wait.  Every persistent kernel of the library
// synchronises its blocks with qcdev::grid_barrier, whose spin gives up after a
// bounded number of polls, records a timeout and lets the kernel return, so a
// block that never arrives ends in QC_ERR_TIMEOUT on the host instead of a hung
// GPU.  This entry point runs that barrier with one block that never arrives.
#include "qc_device.cuh"
#include "qc_internal.h"

namespace {

// Block 0 waits at the barrier; block 1 leaves without arriving.
__global__ void missing_arrival(unsigned *bar, int32_t *status, unsigned long long spins) {
    if (blockIdx.x != 0) return;
    qcdev::grid_barrier(bar, status, spins);
}

}  // namespace

extern "C" qc_status qc_selftest_barrier_timeout(qc_ctx *ctx, int64_t spin_limit, void *stream_) {
    if (!ctx || spin_limit < 1 || (unsigned long long)spin_limit > qcdev::BARRIER_SPINS)
        return QC_ERR_INVALID_ARG;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_buffer ctl;
    QC_TRY(ctl.allocate(ctx, 4 * sizeof(int32_t), stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(ctl.ptr, 0, ctl.bytes, stream));
    int32_t *status = ctl.as<int32_t>();
    unsigned *bar = reinterpret_cast<unsigned *>(status + 2);
    unsigned long long spins = (unsigned long long)spin_limit;
    void *args[] = {(void *)&bar, (void *)&status, (void *)&spins};
    QC_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void *)missing_arrival, dim3(2), dim3(32), args, 0,
                                                 stream));
    QC_LAUNCHED(ctx);
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h = static_cast<int32_t *>(pin.ptr);
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    if (h[0] != qcdev::ST_TIMEOUT) {
        qc_set_error(ctx, "qc_selftest_barrier_timeout: the barrier did not report the missing arrival");
        return QC_ERR_CUDA;
    }
    qc_set_error(ctx, "grid barrier gave up after %lld spins (one block never arrived)", (long long)spin_limit);
    return QC_ERR_TIMEOUT;
}
