// Context, memory accounting, error reporting, graph upload.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "qc_internal.h"

void qc_set_error(qc_ctx *ctx, const char *fmt, ...) {
    if (!ctx) return;
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    ctx->last_error = buf;
}

qc_status qc_mem_alloc(qc_ctx *ctx, size_t bytes, cudaStream_t stream, void **out) {
    *out = nullptr;
    if (bytes == 0) return QC_OK;
    size_t before = ctx->in_use.fetch_add(bytes);
    if (ctx->budget && before + bytes > ctx->budget) {
        ctx->in_use.fetch_sub(bytes);
        qc_set_error(ctx, "memory budget exceeded: %zu bytes in use + %zu requested > budget %zu",
                     before, bytes, ctx->budget);
        return QC_ERR_BUDGET;
    }
    void *p = nullptr;
    if (ctx->custom_alloc) {
        p = ctx->alloc.alloc(bytes, stream, ctx->alloc.user);
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (!p) {
        ctx->in_use.fetch_sub(bytes);
        qc_set_error(ctx, "device allocation of %zu bytes failed", bytes);
        return QC_ERR_OOM;
    }
    *out = p;
    return QC_OK;
}

void qc_mem_free(qc_ctx *ctx, void *ptr, size_t bytes, cudaStream_t stream) {
    if (!ptr) return;
    if (ctx->custom_alloc) ctx->alloc.free(ptr, bytes, stream, ctx->alloc.user);
    else cudaFreeAsync(ptr, stream);
    ctx->in_use.fetch_sub(bytes);
}

qc_ctx::~qc_ctx() {
    for (void *p : pinned_free) cudaFreeHost(p);
    for (cudaStream_t s : all_streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
}

cudaError_t qc_stream_acquire(qc_ctx *ctx, int priority, cudaStream_t *out) {
    {
        std::lock_guard<std::mutex> lk(ctx->streams_mu);
        for (size_t i = 0; i < ctx->spare_streams.size(); ++i)
            if (ctx->spare_streams[i].first == priority) {
                *out = ctx->spare_streams[i].second;
                ctx->spare_streams.erase(ctx->spare_streams.begin() + (std::ptrdiff_t)i);
                return cudaSuccess;
            }
    }
    cudaStream_t s = nullptr;
    const cudaError_t e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, priority);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(ctx->streams_mu);
    ctx->all_streams.push_back(s);
    *out = s;
    return cudaSuccess;
}

void qc_stream_release(qc_ctx *ctx, cudaStream_t s, int priority) {
    if (!s) return;
    std::lock_guard<std::mutex> lk(ctx->streams_mu);
    ctx->spare_streams.emplace_back(priority, s);
}

qc_status qc_pinned::acquire() {
    {
        std::lock_guard<std::mutex> lk(ctx->pinned_mu);
        if (!ctx->pinned_free.empty()) {
            ptr = ctx->pinned_free.back();
            ctx->pinned_free.pop_back();
            return QC_OK;
        }
    }
    QC_CUDA_TRY(ctx, cudaMallocHost(&ptr, QC_PINNED_BYTES));
    return QC_OK;
}

qc_pinned::~qc_pinned() {
    if (!ptr) return;
    std::lock_guard<std::mutex> lk(ctx->pinned_mu);
    ctx->pinned_free.push_back(ptr);
}

qc_status qc_event_pair::create(qc_ctx *ctx) {
    QC_CUDA_TRY(ctx, cudaEventCreate(&a));
    QC_CUDA_TRY(ctx, cudaEventCreate(&b));
    return QC_OK;
}

thread_local float qc_thread_sm_share = 0.f;

void qc_record_kernel(qc_ctx *ctx, const char *kernel, double ms, double model_bytes, double min_bytes) {
    std::lock_guard<std::mutex> lk(ctx->stats_mu);
    qc_kernel_stats &st = ctx->stats[kernel];
    st.launches += 1;
    st.total_ms += ms;
    st.model_bytes += model_bytes;
    st.min_bytes += min_bytes;
}

// Words of sources per BFS chunk.  Every level of a chunk ends at a grid barrier
// after a tail of the last rows, a cost that does not grow with the chunk's
// width, while a row's gather reads R contiguous 16-byte segments per
// neighbour, so wide chunks stay efficient after their bitsets leave L2.
// Measured on GB300 (SBM graphs of mean degree 20, n = 2^15 .. 2^19), the
// fastest width keeps the two bitset buffers near eight times L2, between 64
// and 256 words; below that the per-level fixed cost dominates (sizing the
// buffers to half of L2 ran 2-3x slower at n >= 2^18).  With the two-hop
// set-up, whose cost grows slowly with the width, n = 2^18 solves in 78.4 ms
// at 256 words against 82.7 ms at 128 (four times L2) and 111 ms at 64.  The
// width is a multiple of 64 words (whole 32-segment tiles) chosen so that the
// chunks split the W words evenly.  QCGRAPH_CHUNK_WORDS overrides the choice (tests
// use it to force many chunks).
int32_t qc_bfs_chunk_words(const qc_ctx *ctx, int32_t n) {
    const int64_t W = ((int64_t)n + 63) / 64;
    int64_t wc;
    if (const char *env = getenv("QCGRAPH_CHUNK_WORDS")) {
        wc = atoll(env);
        if (wc < 1) wc = 1;
    } else {
        const size_t l2 = ctx->l2_bytes ? ctx->l2_bytes : (size_t)96 << 20;
        int64_t target = (int64_t)(8 * l2 / (2 * 8 * (size_t)(n > 0 ? n : 1)));
        target = std::min<int64_t>(std::max<int64_t>(target, 64), 256);
        const int64_t chunks = (W + target - 1) / target;
        wc = ((W + chunks - 1) / chunks + 63) / 64 * 64;
    }
    if (wc > 512) wc = 512;
    if (wc > W) wc = W;
    return (int32_t)(wc > 0 ? wc : 1);
}

extern "C" {

qc_status qc_context_set_timing(qc_ctx *ctx, int enable) {
    if (!ctx) return QC_ERR_INVALID_ARG;
    ctx->timing = enable != 0;
    return QC_OK;
}

qc_status qc_context_kernel_stats(qc_ctx *ctx, const char *kernel, qc_kernel_stats *out, int reset) {
    if (!ctx || !kernel || !out) return QC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->stats_mu);
    auto it = ctx->stats.find(kernel);
    *out = it == ctx->stats.end() ? qc_kernel_stats{0, 0.0, 0.0, 0.0} : it->second;
    if (reset && it != ctx->stats.end()) ctx->stats.erase(it);
    return QC_OK;
}

uint64_t qc_context_launch_count(const qc_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

const char *qc_status_string(qc_status s) {
    switch (s) {
    case QC_OK: return "ok";
    case QC_ERR_INVALID_ARG: return "invalid argument";
    case QC_ERR_INVALID_GRAPH: return "invalid graph";
    case QC_ERR_OOM: return "out of device memory";
    case QC_ERR_BUDGET: return "memory budget exceeded";
    case QC_ERR_CUDA: return "CUDA error";
    case QC_ERR_TIMEOUT: return "device wait timed out";
    case QC_ERR_CANCELLED: return "cancelled";
    case QC_ERR_NOT_READY: return "not ready";
    }
    return "unknown status";
}

const char *qc_last_error(const qc_ctx *ctx) {
    if (!ctx) return "";
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    return ctx->last_error.c_str();
}

qc_status qc_context_create(int device, size_t mem_budget_bytes, const qc_allocator *alloc,
                            qc_ctx **out) {
    if (!out || device < 0) return QC_ERR_INVALID_ARG;
    *out = nullptr;
    if (alloc && (!alloc->alloc || !alloc->free)) return QC_ERR_INVALID_ARG;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device >= count) {
        cudaGetLastError();
        return QC_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return QC_ERR_CUDA;
    qc_ctx *ctx = new qc_ctx();
    ctx->device = device;
    ctx->budget = mem_budget_bytes;
    if (alloc) {
        ctx->alloc = *alloc;
        ctx->custom_alloc = true;
    }
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    ctx->num_sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, device);
    ctx->l2_bytes = (size_t)v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ctx->smem_optin = (size_t)v;
    if (!alloc) {
        // keep freed blocks in the stream-ordered pool instead of returning them to
        // the driver at every synchronisation (a process-local pool setting)
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    *out = ctx;
    return QC_OK;
}

void qc_context_destroy(qc_ctx *ctx) { delete ctx; }

size_t qc_context_bytes_in_use(const qc_ctx *ctx) { return ctx ? ctx->in_use.load() : 0; }

qc_status qc_graph_create(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, uint32_t flags, void *stream_, qc_graph **out) {
    qc_range range("qc.graph_create");
    if (!ctx || !out) return QC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || nnz < 0 || nnz >= (int64_t(1) << 31) || !row_ptr || (nnz > 0 && !col_idx)) {
        qc_set_error(ctx, "qc_graph_create: n=%d nnz=%lld out of range or null CSR", n,
                     (long long)nnz);
        return QC_ERR_INVALID_ARG;
    }
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const bool on_device = flags & QC_PTR_DEVICE;
    qc_graph *g = new qc_graph();
    g->ctx = ctx;
    g->n = n;
    g->nnz = nnz;
    g->directed = (flags & QC_DIRECTED) != 0;
    qc_status st = g->row_ptr.allocate(ctx, sizeof(int32_t) * (size_t)(n + 1), stream);
    if (st == QC_OK) st = g->col_idx.allocate(ctx, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), stream);
    if (st != QC_OK) {
        delete g;
        return st;
    }
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(g->row_ptr.ptr, row_ptr, sizeof(int32_t) * (size_t)(n + 1), kind, stream);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(g->col_idx.ptr, col_idx, sizeof(int32_t) * (size_t)nnz, kind, stream);
    if (e != cudaSuccess) {
        qc_set_error(ctx, "qc_graph_create: copy failed: %s", cudaGetErrorString(e));
        delete g;
        return QC_ERR_CUDA;
    }
    if (flags & QC_VALIDATE) {
        st = qc_validate_csr(ctx, n, nnz, g->row_ptr.as<int32_t>(), g->col_idx.as<int32_t>(), !g->directed,
                             stream);
        if (st != QC_OK) {
            delete g;
            return st;
        }
    }
    *out = g;
    return QC_OK;
}

void qc_graph_destroy(qc_graph *g) { delete g; }

void qc_graph_drop_histogram(qc_graph *g) {
    if (!g) return;
    g->hist.release();
    g->hist_rows = 0;
    g->hist_valid = false;
    g->D = 0;
}

int32_t qc_graph_num_nodes(const qc_graph *g) { return g ? g->n : 0; }
int64_t qc_graph_num_edges(const qc_graph *g) { return g ? g->nnz : 0; }

qc_status qc_graph_histogram(qc_graph *g, int32_t *hist_out, int32_t *D_out, void *stream_) {
    if (!g || !D_out) return QC_ERR_INVALID_ARG;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(g->ctx, cudaSetDevice(g->ctx->device));
    if (!g->hist_valid) QC_TRY(qc_bfs_histogram(g, stream));
    *D_out = g->D;
    if (hist_out)
        QC_CUDA_TRY(g->ctx, cudaMemcpyAsync(hist_out, g->hist.ptr,
                                            sizeof(int32_t) * (size_t)(g->D + 1) * (size_t)g->n,
                                            cudaMemcpyDeviceToDevice, stream));
    QC_CUDA_TRY(g->ctx, cudaStreamSynchronize(stream));
    return QC_OK;
}

qc_status qc_graph_set_histogram(qc_graph *g, const int32_t *hist, int32_t D, uint32_t flags, void *stream_) {
    if (!g || !hist) return QC_ERR_INVALID_ARG;
    qc_ctx *ctx = g->ctx;
    if (D < 0 || D >= g->n) {
        qc_set_error(ctx, "qc_graph_set_histogram: D = %d outside [0, n) for n = %d", D, g->n);
        return QC_ERR_INVALID_ARG;
    }
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_buffer nb;
    const size_t bytes = sizeof(int32_t) * (size_t)(D + 1) * (size_t)g->n;
    QC_TRY(nb.allocate(ctx, bytes, stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(nb.ptr, hist, bytes,
                                     (flags & QC_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     stream));
    if (flags & QC_VALIDATE)
        QC_TRY(qc_validate_hist(ctx, g->n, g->nnz, g->row_ptr.as<int32_t>(), nb.as<int32_t>(), D, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));   // a host source may be freed on return
    g->hist = std::move(nb);
    g->hist_rows = D + 1;
    g->D = D;
    g->hist_valid = true;
    return QC_OK;
}

qc_status qc_potential(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out,
                       void *stream_) {
    if (!g || !sigmas || n_sigma < 1 || !V_out) {
        if (g) qc_set_error(g->ctx, "qc_potential: null pointer or n_sigma < 1");
        return QC_ERR_INVALID_ARG;
    }
    for (int32_t s = 0; s < n_sigma; ++s)
        if (!qc_sigma_ok(sigmas[s])) {
            qc_set_error(g->ctx, "qc_potential: sigma[%d] = %g is not finite and > 0", s, sigmas[s]);
            return QC_ERR_INVALID_ARG;
        }
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(g->ctx, cudaSetDevice(g->ctx->device));
    if (!g->hist_valid) QC_TRY(qc_bfs_enqueue(g, stream));
    const qc_status st = qc_potential_from_hist(g, sigmas, n_sigma, V_out, stream);
    bool redone = false;
    const qc_status settled = qc_bfs_settle(g, stream, &redone);
    if (st != QC_OK) return st;
    if (settled != QC_OK) return settled;
    return redone ? qc_potential_from_hist(g, sigmas, n_sigma, V_out, stream) : QC_OK;
}

// Descent and roots queued on `stream`; roots per sigma counted into roots_dev.
// keys: V's descent keys when the potential kernel wrote them, else null.
static qc_status ggd_enqueue(qc_graph *g, const double *V, int32_t n_sigma, int32_t *labels_out,
                             int32_t *roots_dev, cudaStream_t stream, const long long *keys = nullptr) {
    qc_ctx *ctx = g->ctx;
    QC_CUDA_TRY(ctx, cudaMemsetAsync(roots_dev, 0, sizeof(int32_t) * (size_t)n_sigma, stream));
    return qc_descend(ctx, g->n, g->row_ptr.as<int32_t>(), g->col_idx.as<int32_t>(),
                      g->prepared ? g->order.as<int32_t>() : nullptr, V, n_sigma, labels_out, roots_dev, stream,
                      keys);
}

static qc_status read_roots(qc_ctx *ctx, const qc_buffer &roots, int32_t *n_clusters_out, cudaStream_t stream) {
    if (!n_clusters_out) return QC_OK;
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(n_clusters_out, roots.ptr, roots.bytes, cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    return qc_debug_take(ctx);
}

qc_status qc_ggd_labels(qc_graph *g, const double *V, int32_t n_sigma, int32_t *labels_out,
                        int32_t *n_clusters_out, void *stream_) {
    qc_range range("qc.ggd");
    if (!g || !V || n_sigma < 1 || !labels_out) {
        if (g) qc_set_error(g->ctx, "qc_ggd_labels: null pointer or n_sigma < 1");
        return QC_ERR_INVALID_ARG;
    }
    cudaStream_t stream = qc_stream(stream_);
    qc_ctx *ctx = g->ctx;
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_buffer roots;
    QC_TRY(roots.allocate(ctx, sizeof(int32_t) * (size_t)n_sigma, stream));
    QC_TRY(ggd_enqueue(g, V, n_sigma, labels_out, roots.as<int32_t>(), stream));
    return read_roots(ctx, roots, n_clusters_out, stream);
}

// Algorithm 4: the BFS (when the histogram is not cached), potentials, descent
// and roots are queued back to back; the BFS's outcome is read once at the end.
qc_status qc_solve(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out,
                   int32_t *labels_out, int32_t *n_clusters_out, void *stream_) {
    qc_range range("qc.solve");
    if (!g || !sigmas || n_sigma < 1 || !labels_out) {
        if (g) qc_set_error(g->ctx, "qc_solve: null pointer or n_sigma < 1");
        return QC_ERR_INVALID_ARG;
    }
    for (int32_t s = 0; s < n_sigma; ++s)
        if (!qc_sigma_ok(sigmas[s])) {
            qc_set_error(g->ctx, "qc_solve: sigma[%d] = %g is not finite and > 0", s, sigmas[s]);
            return QC_ERR_INVALID_ARG;
        }
    cudaStream_t stream = qc_stream(stream_);
    qc_ctx *ctx = g->ctx;
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_buffer Vtmp, roots;
    double *V = V_out;
    if (!V) {
        QC_TRY(Vtmp.allocate(ctx, sizeof(double) * (size_t)n_sigma * (size_t)g->n, stream));
        V = Vtmp.as<double>();
    }
    QC_TRY(roots.allocate(ctx, sizeof(int32_t) * (size_t)n_sigma, stream));
    // the potential kernel writes the descent's keys too
    qc_buffer keys;
    QC_TRY(keys.allocate(ctx, sizeof(long long) * (size_t)n_sigma * (size_t)g->n, stream));
    long long *K = keys.as<long long>();
    qc_status st = QC_OK;
    if (!g->hist_valid) st = qc_bfs_enqueue(g, stream);
    if (st == QC_OK) st = qc_potential_from_hist(g, sigmas, n_sigma, V, stream, K);
    if (st == QC_OK) {
        qc_range r2("qc.ggd");
        st = ggd_enqueue(g, V, n_sigma, labels_out, roots.as<int32_t>(), stream, K);
    }
    bool redone = false;
    const qc_status settled = qc_bfs_settle(g, stream, &redone);
    if (st != QC_OK) return st;
    if (settled != QC_OK) return settled;
    if (redone) {
        QC_TRY(qc_potential_from_hist(g, sigmas, n_sigma, V, stream, K));
        QC_TRY(ggd_enqueue(g, V, n_sigma, labels_out, roots.as<int32_t>(), stream, K));
    }
    return read_roots(ctx, roots, n_clusters_out, stream);
}


qc_status qc_cluster(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                     uint32_t flags, const double *sigmas, int32_t n_sigma, int32_t *labels_out,
                     int32_t *n_clusters_out, void *stream_) {
    qc_range range("qc.cluster");
    if (!ctx) return QC_ERR_INVALID_ARG;
    if (!sigmas || n_sigma < 1 || !labels_out) {
        qc_set_error(ctx, "qc_cluster: null pointer or n_sigma < 1");
        return QC_ERR_INVALID_ARG;
    }
    for (int32_t s = 0; s < n_sigma; ++s)
        if (!qc_sigma_ok(sigmas[s])) {
            qc_set_error(ctx, "qc_cluster: sigma[%d] = %g is not finite and > 0", s, sigmas[s]);
            return QC_ERR_INVALID_ARG;
        }
    cudaStream_t stream = qc_stream(stream_);
    qc_graph *g = nullptr;
    // the upload, then the validation queued without a wait: the work behind it
    // runs on an emptied CSR if the check fails, and the verdict is read with the
    // results
    QC_TRY(qc_graph_create(ctx, n, nnz, row_ptr, col_idx, flags & ~(uint32_t)QC_VALIDATE, stream_, &g));
    std::unique_ptr<qc_graph, void (*)(qc_graph *)> hold(g, qc_graph_destroy);
    const bool validate = (flags & QC_VALIDATE) != 0;
    qc_buffer verdict;
    if (validate) {
        QC_TRY(verdict.allocate(ctx, sizeof(int32_t), stream));
        QC_TRY(qc_validate_csr_queue(ctx, n, nnz, g->row_ptr.as<int32_t>(), g->col_idx.as<int32_t>(), !g->directed,
                                     verdict.as<int32_t>(), stream));
    }
    const size_t cells = (size_t)n_sigma * (size_t)n;
    qc_buffer V, labels, roots, keys;
    QC_TRY(V.allocate(ctx, sizeof(double) * cells, stream));
    QC_TRY(keys.allocate(ctx, sizeof(long long) * cells, stream));
    QC_TRY(labels.allocate(ctx, sizeof(int32_t) * cells, stream));
    QC_TRY(roots.allocate(ctx, sizeof(int32_t) * (size_t)n_sigma, stream));
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    // the pinned block: the verdict in its first word, the cluster counts after it
    int32_t *h_verdict = static_cast<int32_t *>(pin.ptr);
    int32_t *h_counts = h_verdict + 4;
    const bool counts_pinned = n_clusters_out && sizeof(int32_t) * ((size_t)n_sigma + 4) <= QC_PINNED_BYTES;
    // potentials, descent and both copies out, queued behind the BFS
    auto queue = [&]() -> qc_status {
        QC_TRY(qc_potential_from_hist(g, sigmas, n_sigma, V.as<double>(), stream, keys.as<long long>()));
        {
            qc_range r2("qc.ggd");
            QC_TRY(ggd_enqueue(g, V.as<double>(), n_sigma, labels.as<int32_t>(), roots.as<int32_t>(), stream,
                               keys.as<long long>()));
        }
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(labels_out, labels.ptr, labels.bytes, cudaMemcpyDefault, stream));
        if (counts_pinned)
            QC_CUDA_TRY(ctx, cudaMemcpyAsync(h_counts, roots.ptr, roots.bytes, cudaMemcpyDeviceToHost, stream));
        return QC_OK;
    };
    h_verdict[0] = 0;
    qc_status st = qc_bfs_enqueue(g, stream);
    if (st == QC_OK) st = queue();
    if (st == QC_OK && validate)
        st = cudaMemcpyAsync(h_verdict, verdict.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) == cudaSuccess
                 ? QC_OK
                 : QC_ERR_CUDA;
    bool redone = false;
    const qc_status settled = qc_bfs_settle(g, stream, &redone);   // waits for all of the above
    if (st != QC_OK) return st;
    if (validate) {
        QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));   // returns at once where the settle has waited
        QC_TRY(qc_csr_verdict(ctx, h_verdict[0]));
    }
    if (settled != QC_OK) return settled;
    if (redone) QC_TRY(queue());
    if (n_clusters_out && !counts_pinned)
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(n_clusters_out, roots.ptr, roots.bytes, cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    QC_TRY(qc_debug_take(ctx));
    if (counts_pinned) memcpy(n_clusters_out, h_counts, roots.bytes);
    return QC_OK;
}

}  // extern "C"
