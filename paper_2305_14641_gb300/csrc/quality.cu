// Clustering quality measures of the paper's evaluation (Section 4.2) on the
// device, for label vectors that are already on the GPU (as qc_ggd_labels and the
// batched and served forms leave them):
//   Modularity  Q = inside / w - gamma sum_c (sum of degrees in c)^2 / w^2, with
//               inside the CSR entries whose two ends share a cluster and w the
//               degree total (Newman's form; 2m for an undirected graph);
//   ARI         (index - expected) / (max - expected) over pair counts of the
//               contingency table (Hubert & Arabie 1985);
//   FMI         TP / sqrt((TP + FP)(TP + FN)) over pairs;
//   NMI         MI / sqrt(H(truth) H(labels)), natural logarithms.
// Every count and pair sum is an exact 64-bit integer; only the entropies and
// the mutual information are accumulated in binary64 (with the device's log).
// The host forms the final ratios from those sums.
#include <cmath>
#include <vector>

#include "qc_internal.h"

namespace {

enum : int32_t { BAD_LABEL = 1, BAD_TRUTH = 2 };

// Mark the labels in use (labels are node ids: roots of the descent).
__global__ void q_mark(int32_t n, const int32_t *labels, int32_t *cid, int32_t *err) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int l = labels[v];
        if ((unsigned)l >= (unsigned)n) {
            atomicOr(err, BAD_LABEL);
            continue;
        }
        cid[l] = 1;
    }
}

// Compact cluster ids in any order (the measures do not depend on the numbering).
__global__ void q_compact(int32_t n, int32_t *cid, int32_t *count) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x)
        cid[l] = cid[l] ? atomicAdd(count, 1) : -1;
}

// Per node: cluster sizes, degree sums, truth sizes and the contingency table.
__global__ void q_count(int32_t n, const int32_t *row_ptr, const int32_t *labels, const int32_t *truth,
                        int32_t n_truth, const int32_t *cid, unsigned long long *size, unsigned long long *degsum,
                        unsigned long long *tsize, unsigned long long *table, int32_t *err) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int l = labels[v];
        if ((unsigned)l >= (unsigned)n) continue;
        const int c = cid[l];
        atomicAdd(size + c, 1ull);
        if (row_ptr) atomicAdd(degsum + c, (unsigned long long)(row_ptr[v + 1] - row_ptr[v]));
        if (truth) {
            const int t = truth[v];
            if ((unsigned)t >= (unsigned)n_truth) {
                atomicOr(err, BAD_TRUTH);
                continue;
            }
            atomicAdd(tsize + t, 1ull);
            atomicAdd(table + (size_t)c * n_truth + t, 1ull);
        }
    }
}

// CSR entries whose two ends carry the same label (one warp per row).
__global__ void q_inside(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *labels,
                         unsigned long long *inside) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long cnt = 0;
    for (int v = warp; v < n; v += nwarps) {
        const int lv = labels[v];
        for (int e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) {
            const int u = col_idx[e];
            if ((unsigned)u < (unsigned)n && labels[u] == lv) ++cnt;
        }
    }
    for (int off = 16; off; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (lane == 0 && cnt) atomicAdd(inside, cnt);
}

__device__ __forceinline__ unsigned long long pairs(unsigned long long x) { return x * (x - 1) / 2; }

// Sums over an array of counts: sum x^2 or sum C(x, 2) (exact), and, with a
// total, the entropy term -sum (x / total) log(x / total).
__global__ void q_sums(int64_t m, const unsigned long long *x, int square, unsigned long long *sum, double total,
                       double *entropy) {
    unsigned long long s = 0;
    double h = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long v = x[i];
        s += square ? v * v : pairs(v);
        if (entropy && v) {
            const double p = (double)v / total;
            h -= p * log(p);
        }
    }
    for (int off = 16; off; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        h += __shfl_xor_sync(0xffffffffu, h, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (s) atomicAdd(sum, s);
        if (entropy && h != 0.0) atomicAdd(entropy, h);
    }
}

// Mutual information: sum_ij (n_ij / n) log(n n_ij / (a_i b_j)), a = cluster sizes, b = truth sizes.
__global__ void q_mutual(int32_t C, int32_t n_truth, const unsigned long long *table, const unsigned long long *size,
                         const unsigned long long *tsize, double n, double *mi) {
    double acc = 0.0;
    const int64_t m = (int64_t)C * n_truth;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long v = table[i];
        if (!v) continue;
        const int c = (int)(i / n_truth), t = (int)(i - (int64_t)c * n_truth);
        const double p = (double)v / n;
        acc += p * log((double)v * n / ((double)size[c] * (double)tsize[t]));
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(mi, acc);
}

}  // namespace

extern "C" qc_status qc_quality(qc_ctx *ctx, const qc_graph *g, int32_t n, const int32_t *labels,
                                const int32_t *truth, int32_t n_truth, double gamma, qc_quality_result *out,
                                void *stream_) {
    if (!ctx || !out || !labels || n < 1 || (g && (g->n != n || g->ctx != ctx)) || (truth && n_truth < 1) ||
        !std::isfinite(gamma))
        return QC_ERR_INVALID_ARG;
    const int32_t *row_ptr = g ? g->row_ptr.as<int32_t>() : nullptr;
    const int32_t *col_idx = g ? g->col_idx.as<int32_t>() : nullptr;
    const double nan = std::nan("");
    out->modularity = out->ari = out->fmi = out->nmi = nan;
    out->clusters = 0;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int blocks = qc_ceil_div(n, 256) < 4 * ctx->num_sms ? qc_ceil_div(n, 256) : 4 * ctx->num_sms;
    // control: [0] error flags, [1] clusters; then 64-bit sums
    qc_buffer ctl, cid;
    QC_TRY(ctl.allocate(ctx, 256, stream));
    QC_TRY(cid.allocate(ctx, sizeof(int32_t) * (size_t)n, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(ctl.ptr, 0, ctl.bytes, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(cid.ptr, 0, cid.bytes, stream));
    int32_t *err = ctl.as<int32_t>(), *count = err + 1;
    q_mark<<<blocks, 256, 0, stream>>>(n, labels, cid.as<int32_t>(), err);
    QC_LAUNCHED(ctx);
    q_compact<<<blocks, 256, 0, stream>>>(n, cid.as<int32_t>(), count);
    QC_LAUNCHED(ctx);
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h = static_cast<int32_t *>(pin.ptr);
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, err, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    if (h[0] & BAD_LABEL) {
        qc_set_error(ctx, "qc_quality: a label outside [0, n)");
        return QC_ERR_INVALID_ARG;
    }
    const int32_t C = h[1];
    out->clusters = C;
    // sums: [0] inside, [1] sum deg_c^2, [2] sum C(n_ij, 2), [3] sum C(a_i, 2), [4] sum C(b_j, 2);
    // doubles: [5] H(labels), [6] H(truth), [7] MI
    unsigned long long *sums = reinterpret_cast<unsigned long long *>(ctl.as<char>() + 64);
    double *dsum = reinterpret_cast<double *>(sums + 5);
    qc_buffer size, degsum, tsize, table;
    QC_TRY(size.allocate(ctx, 8 * (size_t)C, stream));
    QC_TRY(degsum.allocate(ctx, 8 * (size_t)C, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(size.ptr, 0, size.bytes, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(degsum.ptr, 0, degsum.bytes, stream));
    if (truth) {
        if ((double)C * (double)n_truth > (double)(1ll << 31)) {
            qc_set_error(ctx, "qc_quality: %d clusters x %d true classes is too large a table", C, n_truth);
            return QC_ERR_INVALID_ARG;
        }
        QC_TRY(tsize.allocate(ctx, 8 * (size_t)n_truth, stream));
        QC_TRY(table.allocate(ctx, 8 * (size_t)C * n_truth, stream));
        QC_CUDA_TRY(ctx, cudaMemsetAsync(tsize.ptr, 0, tsize.bytes, stream));
        QC_CUDA_TRY(ctx, cudaMemsetAsync(table.ptr, 0, table.bytes, stream));
    }
    q_count<<<blocks, 256, 0, stream>>>(n, row_ptr, labels, truth, n_truth, cid.as<int32_t>(),
                                        size.as<unsigned long long>(), degsum.as<unsigned long long>(),
                                        tsize.as<unsigned long long>(), table.as<unsigned long long>(), err);
    QC_LAUNCHED(ctx);
    const int cb = qc_ceil_div(C, 256) < 4 * ctx->num_sms ? qc_ceil_div(C, 256) : 4 * ctx->num_sms;
    if (row_ptr) {
        q_inside<<<qc_ceil_div(n, 8) < 8 * ctx->num_sms ? qc_ceil_div(n, 8) : 8 * ctx->num_sms, 256, 0, stream>>>(
            n, row_ptr, col_idx, labels, sums + 0);
        QC_LAUNCHED(ctx);
        q_sums<<<cb, 256, 0, stream>>>(C, degsum.as<unsigned long long>(), 1, sums + 1, 0.0, nullptr);
        QC_LAUNCHED(ctx);
    }
    if (truth) {
        const int64_t m = (int64_t)C * n_truth;
        const int tb = (int)std::min<int64_t>((m + 255) / 256, 4 * (int64_t)ctx->num_sms);
        q_sums<<<tb, 256, 0, stream>>>(m, table.as<unsigned long long>(), 0, sums + 2, 0.0, nullptr);
        QC_LAUNCHED(ctx);
        q_sums<<<cb, 256, 0, stream>>>(C, size.as<unsigned long long>(), 0, sums + 3, (double)n, dsum + 0);
        QC_LAUNCHED(ctx);
        const int nb = qc_ceil_div(n_truth, 256) < 4 * ctx->num_sms ? qc_ceil_div(n_truth, 256) : 4 * ctx->num_sms;
        q_sums<<<nb, 256, 0, stream>>>(n_truth, tsize.as<unsigned long long>(), 0, sums + 4, (double)n, dsum + 1);
        QC_LAUNCHED(ctx);
        q_mutual<<<tb, 256, 0, stream>>>(C, n_truth, table.as<unsigned long long>(), size.as<unsigned long long>(),
                                         tsize.as<unsigned long long>(), (double)n, dsum + 2);
        QC_LAUNCHED(ctx);
    }
    unsigned long long *hs = reinterpret_cast<unsigned long long *>(static_cast<char *>(pin.ptr) + 64);
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(hs, sums, 8 * 8, cudaMemcpyDeviceToHost, stream));
    h[1] = 0;
    if (row_ptr)   // w: the degree total, the CSR's last row pointer
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(h + 1, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    if (h[0] & BAD_TRUTH) {
        qc_set_error(ctx, "qc_quality: a true class outside [0, n_truth)");
        return QC_ERR_INVALID_ARG;
    }
    const double *hd = reinterpret_cast<const double *>(hs + 5);
    if (row_ptr) {
        const double w = (double)h[1];
        out->modularity = w == 0.0 ? 0.0 : (double)hs[0] / w - gamma * (double)hs[1] / (w * w);
    }
    if (truth) {
        const double index = (double)hs[2], a = (double)hs[4], b = (double)hs[3];   // a: truth, b: labels
        const double total = (double)n * ((double)n - 1.0) / 2.0;
        const double expected = total > 0.0 ? a * b / total : 0.0;
        const double maximum = (a + b) / 2.0;
        out->ari = maximum == expected ? 1.0 : (index - expected) / (maximum - expected);
        out->fmi = (a == 0.0 || b == 0.0) ? 0.0 : index / std::sqrt(b * a);
        const double hl = hd[0], ht = hd[1], mi = hd[2];
        out->nmi = (hl == 0.0 || ht == 0.0) ? (hl == ht ? 1.0 : 0.0) : mi / std::sqrt(ht * hl);
    }
    return QC_OK;
}
