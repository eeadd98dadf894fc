// CSR validation on the device (QC_VALIDATE): the graph must be the sparse form
// of a 0/1 adjacency matrix with an empty diagonal, rows sorted, and symmetric
// unless it is directed.  Also the checks of an installed histogram.
#include "qc_internal.h"

namespace {

enum : int32_t {
    BAD_ROW_PTR = 1,
    BAD_COLUMN = 2,
    BAD_ORDER = 4,      // unsorted row or duplicate edge
    BAD_SELF_LOOP = 8,
    BAD_ASYMMETRIC = 16,
};

// Two kernels, neither of which reads outside row_ptr[0..n] and col_idx[0..nnz)
// whatever the arrays hold.
// check_rows, one thread per row: 0 <= row_ptr[v] <= row_ptr[v+1] <= nnz (which,
// over all v, makes row_ptr non-decreasing within [0, nnz]); thread 0 checks the
// two ends.
__global__ void check_rows(int32_t n, int64_t nnz, const int32_t *row_ptr, int32_t *err) {
    int bad = 0;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz)) bad |= BAD_ROW_PTR;
    for (int v = tid; v < n; v += gridDim.x * blockDim.x) {
        const int beg = row_ptr[v], end = row_ptr[v + 1];
        if (beg < 0 || beg > end || (int64_t)end > nnz) bad |= BAD_ROW_PTR;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(err, bad);
}

// check_edges, one thread per edge (so a hub's row costs no more than others):
// the edge's row v is found by binary search in row_ptr (within [0, n) whatever
// row_ptr holds; where row_ptr is invalid the row may be wrong, and then
// check_rows has already flagged it), then its column is in range, not v, above
// the previous column of the row, and (symmetric) v appears in the column's row,
// by binary search between that row's bounds once they are checked.
__global__ void check_edges(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx, bool symmetric,
                            int32_t *err) {
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;                      // the last v with row_ptr[v] <= e
        while (lo < hi) {
            const int mid = lo + ((hi - lo + 1) >> 1);
            if ((int64_t)row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int v = lo;
        const int u = col_idx[e];
        if (u < 0 || u >= n) { bad |= BAD_COLUMN; continue; }
        if (u == v) bad |= BAD_SELF_LOOP;
        if (e > 0 && e > (int64_t)row_ptr[v] && col_idx[e - 1] >= u) bad |= BAD_ORDER;
        if (!symmetric) continue;
        const int64_t ulo = row_ptr[u], uend = row_ptr[u + 1];
        if (ulo < 0 || uend < ulo || uend > nnz) { bad |= BAD_ROW_PTR; continue; }
        int a = (int)ulo, b = (int)uend - 1;
        bool found = false;
        while (a <= b) {
            const int mid = a + ((b - a) >> 1);
            const int x = col_idx[mid];
            if (x == v) { found = true; break; }
            if (x < v) a = mid + 1; else b = mid - 1;
        }
        if (!found) bad |= BAD_ASYMMETRIC;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(err, bad);
}

// Both checks into err (zeroed by the caller).
qc_status launch_csr_checks(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                            bool symmetric, int32_t *err, cudaStream_t stream) {
    const int rb = qc_ceil_div(n, 256) < 2 * ctx->num_sms ? qc_ceil_div(n, 256) : 2 * ctx->num_sms;
    check_rows<<<rb, 256, 0, stream>>>(n, nnz, row_ptr, err);
    QC_LAUNCHED(ctx);
    if (nnz > 0) {
        const int64_t eb64 = (nnz + 255) / 256;
        const int eb = eb64 < 8 * (int64_t)ctx->num_sms ? (int)eb64 : 8 * ctx->num_sms;
        check_edges<<<eb, 256, 0, stream>>>(n, nnz, row_ptr, col_idx, symmetric, err);
        QC_LAUNCHED(ctx);
    }
    return QC_OK;
}

// After a queued check (qc_validate_csr_queue): if it found anything, every row
// is made empty, so the kernels queued behind it read no column id and no row
// bound outside the arrays; the caller discards their results and reports the
// verdict.
__global__ void empty_rows_if_bad(int32_t n, int32_t *row_ptr, const int32_t *err) {
    if (*(volatile const int32_t *)err == 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) row_ptr[i] = 0;
}

enum : int32_t {
    BAD_H0 = 1,         // h(0, v) != 1
    BAD_H1 = 2,         // h(1, v) != out-degree
    BAD_NEGATIVE = 4,
    BAD_SUM = 8,        // more than n nodes at finite distance
    LAST_ROW_USED = 16, // some node has h(D, v) > 0 (required)
};

// One thread per node: the identities every histogram of this graph satisfies.
__global__ void check_hist(int32_t n, const int32_t *row_ptr, const int32_t *hist, int32_t D, int32_t *err) {
    int bad = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        long long sum = 0;
        for (int d = 0; d <= D; ++d) {
            const int h = hist[(size_t)d * n + v];
            if (h < 0) bad |= BAD_NEGATIVE;
            sum += h;
        }
        if (hist[v] != 1) bad |= BAD_H0;
        if (D >= 1 && hist[(size_t)n + v] != row_ptr[v + 1] - row_ptr[v]) bad |= BAD_H1;
        if (sum > n) bad |= BAD_SUM;
        if (hist[(size_t)D * n + v] > 0) bad |= LAST_ROW_USED;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(err, bad);
}

}  // namespace

qc_status qc_validate_hist(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *hist,
                           int32_t D, cudaStream_t stream) {
    if ((nnz == 0) != (D == 0)) {
        qc_set_error(ctx, "invalid histogram: D = %d for a graph with %lld edges", D, (long long)nnz);
        return QC_ERR_INVALID_GRAPH;
    }
    qc_buffer err;
    QC_TRY(err.allocate(ctx, sizeof(int32_t), stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), stream));
    const int blocks = qc_ceil_div(n, 256) < 4 * ctx->num_sms ? qc_ceil_div(n, 256) : 4 * ctx->num_sms;
    check_hist<<<blocks, 256, 0, stream>>>(n, row_ptr, hist, D, err.as<int32_t>());
    QC_LAUNCHED(ctx);
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h = static_cast<int32_t *>(pin.ptr);
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    const int32_t e = h[0];
    if ((e & ~LAST_ROW_USED) || !(e & LAST_ROW_USED)) {
        qc_set_error(ctx, "invalid histogram (flags 0x%x):%s%s%s%s%s", e, (e & BAD_H0) ? " h(0) != 1;" : "",
                     (e & BAD_H1) ? " h(1) != degree;" : "", (e & BAD_NEGATIVE) ? " negative count;" : "",
                     (e & BAD_SUM) ? " more than n nodes;" : "",
                     (e & LAST_ROW_USED) ? "" : " row D is empty;");
        return QC_ERR_INVALID_GRAPH;
    }
    return QC_OK;
}

qc_status qc_csr_verdict(qc_ctx *ctx, int32_t flags) {
    if (!flags) return QC_OK;
    qc_set_error(ctx, "invalid CSR (flags 0x%x):%s%s%s%s%s", flags,
                 (flags & BAD_ROW_PTR) ? " row_ptr not 0-based, non-decreasing and ending at nnz;" : "",
                 (flags & BAD_COLUMN) ? " column id out of range;" : "",
                 (flags & BAD_ORDER) ? " row not strictly ascending;" : "",
                 (flags & BAD_SELF_LOOP) ? " self-loop;" : "",
                 (flags & BAD_ASYMMETRIC) ? " not symmetric;" : "");
    return QC_ERR_INVALID_GRAPH;
}

qc_status qc_validate_csr_queue(qc_ctx *ctx, int32_t n, int64_t nnz, int32_t *row_ptr, const int32_t *col_idx,
                                bool symmetric, int32_t *err, cudaStream_t stream) {
    QC_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, sizeof(int32_t), stream));
    QC_TRY(launch_csr_checks(ctx, n, nnz, row_ptr, col_idx, symmetric, err, stream));
    const int eb = qc_ceil_div(n + 1, 256) < 2 * ctx->num_sms ? qc_ceil_div(n + 1, 256) : 2 * ctx->num_sms;
    empty_rows_if_bad<<<eb, 256, 0, stream>>>(n, row_ptr, err);
    QC_LAUNCHED(ctx);
    return QC_OK;
}

qc_status qc_validate_csr(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, bool symmetric, cudaStream_t stream) {
    qc_buffer err;
    QC_TRY(err.allocate(ctx, sizeof(int32_t), stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), stream));
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t &h_err = *static_cast<int32_t *>(pin.ptr);
    QC_TRY(launch_csr_checks(ctx, n, nnz, row_ptr, col_idx, symmetric, err.as<int32_t>(), stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(&h_err, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    return qc_csr_verdict(ctx, h_err);
}
