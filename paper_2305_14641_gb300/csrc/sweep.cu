// A solve plan for one graph and a fixed list of sigma values: Algorithm 4 for
// every sigma (the all-source BFS and histogram behind Algorithm 1, the
// potentials of Eq. 7, Graph Gradient Descent of Algorithm 2 and the roots of
// Algorithm 3), queued once into CUDA graphs together with every buffer it
// uses, and replayed.
//
// Two graphs are captured: `full` recomputes everything from the resident CSR
// (histogram rows zeroed, the BFS of every source chunk, potentials, descent,
// roots, and the BFS's outcome and the root counts copied to pinned host
// memory); `sweep` reuses the plan's histogram (potentials, descent, roots).
// The BFS learns the largest distance D on the device and the potential kernel
// reads it from there, so nothing in a replay waits for the host.  After a full
// replay the host reads the outcome once: a BFS that ran out of histogram rows
// is captured again with more rows and replayed; one whose grid barrier timed
// out returns QC_ERR_TIMEOUT.
//
// Where a capture is refused (a driver without cooperative kernel nodes, for
// instance) the plan queues the same work directly on each run.
#include <cstring>
#include <vector>

#include "qc_device.cuh"
#include "qc_internal.h"

struct qc_sweep {
    qc_graph *g = nullptr;
    qc_ctx *ctx = nullptr;
    std::vector<double> sigmas;
    int32_t S = 0;
    double *V = nullptr;          // potentials [S][n] (the caller's, or V_own)
    int32_t *labels = nullptr;    // labels [S][n] (the caller's)
    qc_buffer V_own, hist, out, roots, parent, keys, dtab;
    qc_bfs_scratch bs;
    int32_t rows = 0;             // histogram rows
    std::vector<double> tab;      // potential tables over `rows` distances
    int32_t *pinned = nullptr;    // [0..1] BFS outcome, [8 ..) roots per sigma
    cudaStream_t cap = nullptr;   // private stream: allocation and capture
    cudaEvent_t done = nullptr;   // recorded after every run (waited for on destruction)
    cudaGraphExec_t full = nullptr, sweep = nullptr;
    uint64_t kernels_full = 0, kernels_sweep = 0;   // kernels inside each graph
    bool captured = false;        // replays use the graphs
    bool have_hist = false;       // a full run has filled the histogram
    int32_t D = -1;
    ~qc_sweep();
};

namespace {

using qcdev::ST_NEED_ROWS;
using qcdev::ST_TIMEOUT;

void drop_graphs(qc_sweep *p) {
    if (p->full) cudaGraphExecDestroy(p->full);
    if (p->sweep) cudaGraphExecDestroy(p->sweep);
    p->full = p->sweep = nullptr;
    p->captured = false;
}

// Potentials, descent and roots from the plan's histogram, root counts to pinned memory.
qc_status queue_sweep(qc_sweep *p, cudaStream_t s) {
    qc_ctx *ctx = p->ctx;
    qc_graph *g = p->g;
    QC_TRY(qc_potential_launch(ctx, g->n, p->hist.as<int32_t>(), p->rows - 1, p->out.as<int32_t>() + 1, p->S, p->tab,
                               p->dtab.as<double>(), p->V, p->keys.as<long long>(), s));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(p->roots.ptr, 0, p->roots.bytes, s));
    QC_TRY(qc_descend_into(ctx, g->n, g->row_ptr.as<int32_t>(), g->col_idx.as<int32_t>(), g->order.as<int32_t>(),
                           p->V, p->S, p->labels, p->roots.as<int32_t>(), p->parent.as<int32_t>(),
                           p->keys.as<long long>(), s, true));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(p->pinned + 8, p->roots.ptr, p->roots.bytes, cudaMemcpyDeviceToHost, s));
    return QC_OK;
}

// Everything from the CSR: zero the histogram rows the BFS adds into, the BFS of
// every chunk (outcome words reset by the first), then the sweep.
qc_status queue_full(qc_sweep *p, cudaStream_t s) {
    qc_ctx *ctx = p->ctx;
    qc_graph *g = p->g;
    const int32_t n = g->n, W = (n + 63) / 64;
    QC_CUDA_TRY(ctx, cudaMemsetAsync(p->hist.as<int32_t>() + 2 * (size_t)n, 0,
                                     sizeof(int32_t) * (size_t)(p->rows - 2) * (size_t)n, s));
    for (int32_t w0 = 0; w0 < W; w0 += p->bs.wc)
        QC_TRY(qc_bfs_launch(g, p->bs, w0, 2, p->hist.as<int32_t>(), p->rows, p->out.as<int32_t>(), w0 == 0, nullptr,
                             s));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(p->pinned, p->out.ptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    return queue_sweep(p, s);
}

// Histogram rows, their tables (and a device copy when they do not travel inline).
qc_status size_rows(qc_sweep *p, int32_t rows) {
    qc_ctx *ctx = p->ctx;
    const int32_t n = p->g->n;
    p->rows = rows;
    QC_TRY(p->hist.allocate(ctx, sizeof(int32_t) * (size_t)rows * (size_t)n, p->cap));
    qc_potential_tables(p->sigmas.data(), p->S, rows, p->tab);
    p->dtab.release();
    if (!qc_potential_tables_inline(p->S, rows)) {
        QC_TRY(p->dtab.allocate(ctx, sizeof(double) * p->tab.size(), p->cap));
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(p->dtab.ptr, p->tab.data(), p->dtab.bytes, cudaMemcpyHostToDevice, p->cap));
    }
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(p->cap));
    return QC_OK;
}

// Capture one graph of queued work; false (and no graph) when the capture is refused.
bool capture(qc_sweep *p, qc_status (*queue)(qc_sweep *, cudaStream_t), cudaGraphExec_t *exec, uint64_t *kernels) {
    qc_ctx *ctx = p->ctx;
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const uint64_t before = ctx->launches.load();
    const qc_status st = queue(p, p->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
    *kernels = ctx->launches.load() - before;
    ctx->launches.fetch_sub(*kernels);            // captured, not launched
    bool ok = st == QC_OK && e == cudaSuccess && graph;
    if (ok) ok = cudaGraphInstantiate(exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        *exec = nullptr;
        cudaGetLastError();
    }
    return ok;
}

qc_status capture_all(qc_sweep *p) {
    drop_graphs(p);
    p->captured = capture(p, queue_full, &p->full, &p->kernels_full) &&
                  capture(p, queue_sweep, &p->sweep, &p->kernels_sweep);
    if (!p->captured) drop_graphs(p);
    return QC_OK;
}

}  // namespace

static qc_status sweep_run(qc_sweep *p, int32_t reuse_histogram, int32_t *n_clusters_out, cudaStream_t stream);

qc_sweep::~qc_sweep() {
    if (done) {
        cudaEventSynchronize(done);
        cudaEventDestroy(done);
    }
    drop_graphs(this);
    V_own.release();
    hist.release();
    out.release();
    roots.release();
    parent.release();
    keys.release();
    dtab.release();
    bs.release();
    if (cap) {
        cudaStreamSynchronize(cap);
        qc_stream_release(ctx, cap, 0);
    }
    if (pinned) cudaFreeHost(pinned);
}

extern "C" {

qc_status qc_sweep_create(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out, int32_t *labels_out,
                          void *stream_, qc_sweep **out) {
    if (!g || !sigmas || n_sigma < 1 || !labels_out || !out) return QC_ERR_INVALID_ARG;
    qc_ctx *ctx = g->ctx;
    for (int32_t s = 0; s < n_sigma; ++s)
        if (!qc_sigma_ok(sigmas[s])) {
            qc_set_error(ctx, "qc_sweep_create: sigma[%d] = %g is not finite and > 0", s, sigmas[s]);
            return QC_ERR_INVALID_ARG;
        }
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaStream_t stream = qc_stream(stream_);
    qc_sweep *p = new qc_sweep;
    p->g = g;
    p->ctx = ctx;
    p->sigmas.assign(sigmas, sigmas + n_sigma);
    p->S = n_sigma;
    p->labels = labels_out;
    auto fail = [&](qc_status st) {
        delete p;
        return st;
    };
    if (qc_stream_acquire(ctx, 0, &p->cap) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void **)&p->pinned, sizeof(int32_t) * (8 + (size_t)n_sigma)) != cudaSuccess) {
        qc_set_error(ctx, "qc_sweep_create: stream, event or pinned memory not available");
        return fail(QC_ERR_CUDA);
    }
    // the caller's earlier work on the graph (its upload) comes first
    if (cudaEventRecord(p->done, stream) != cudaSuccess || cudaStreamWaitEvent(p->cap, p->done, 0) != cudaSuccess)
        return fail(QC_ERR_CUDA);
    const int32_t n = g->n;
    qc_status st;
    if ((st = qc_graph_prepare(g, p->cap)) != QC_OK) return fail(st);
    if (!g->prep_checked) {
        if (cudaMemcpyAsync(p->pinned, g->prep_ctl.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, p->cap) != cudaSuccess ||
            cudaStreamSynchronize(p->cap) != cudaSuccess)
            return fail(QC_ERR_CUDA);
        if ((st = qc_graph_prepare_status(g, p->pinned[0])) != QC_OK) return fail(st);
    }
    if (!V_out) {
        if ((st = p->V_own.allocate(ctx, sizeof(double) * (size_t)n_sigma * n, p->cap)) != QC_OK) return fail(st);
        p->V = p->V_own.as<double>();
    } else {
        p->V = V_out;
    }
    if ((st = p->out.allocate(ctx, sizeof(int32_t) * 8, p->cap)) != QC_OK ||
        (st = p->roots.allocate(ctx, sizeof(int32_t) * (size_t)n_sigma, p->cap)) != QC_OK ||
        (st = p->parent.allocate(ctx, sizeof(int32_t) * (size_t)n_sigma * n, p->cap)) != QC_OK ||
        (st = p->keys.allocate(ctx, sizeof(long long) * (size_t)n_sigma * n, p->cap)) != QC_OK)
        return fail(st);
    if (g->nnz > 0 && (st = qc_bfs_scratch_init(g, p->bs, p->cap)) != QC_OK) return fail(st);
    // rows: the graph's known depth when it has a histogram (the last pass, which
    // finds nothing, needs a row too), else 32; more are added when a run needs them
    int32_t rows = g->hist_valid && !g->bfs_queued ? g->D + 2 : 32;
    rows = rows < 2 ? 2 : (rows > n + 1 ? n + 1 : rows);
    if ((st = size_rows(p, rows)) != QC_OK) return fail(st);
    if (g->nnz > 0) capture_all(p);
    *out = p;
    return QC_OK;
}

qc_status qc_sweep_run(qc_sweep *p, int32_t reuse_histogram, int32_t *n_clusters_out, void *stream_) {
    if (!p) return QC_ERR_INVALID_ARG;
    qc_ctx *ctx = p->ctx;
    if (reuse_histogram && !p->have_hist) {
        qc_set_error(ctx, "qc_sweep_run: no histogram yet (run once with reuse_histogram = 0)");
        return QC_ERR_INVALID_ARG;
    }
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaStream_t stream = qc_stream(stream_);
    const qc_status st = sweep_run(p, reuse_histogram, n_clusters_out, stream);
    cudaEventRecord(p->done, stream);
    return st;
}

qc_status qc_sweep_info(const qc_sweep *p, int32_t *D, int32_t *captured, int64_t *kernels_per_run) {
    if (!p) return QC_ERR_INVALID_ARG;
    if (D) *D = p->have_hist ? p->D : -1;
    if (captured) *captured = p->captured ? 1 : 0;
    if (kernels_per_run) *kernels_per_run = (int64_t)p->kernels_full;
    return QC_OK;
}

void qc_sweep_destroy(qc_sweep *p) { delete p; }

}  // extern "C"

static qc_status sweep_run(qc_sweep *p, int32_t reuse_histogram, int32_t *n_clusters_out, cudaStream_t stream) {
    qc_ctx *ctx = p->ctx;
    qc_graph *g = p->g;
    if (g->nnz == 0) {
        // no edges: every node is its own cluster; the single-graph path has nothing to wait for
        const qc_status st = qc_solve(g, p->sigmas.data(), p->S, p->V, p->labels, n_clusters_out, stream);
        p->have_hist = st == QC_OK;
        p->D = 0;
        return st;
    }
    if (reuse_histogram) {
        if (p->captured) {
            QC_CUDA_TRY(ctx, cudaGraphLaunch(p->sweep, stream));
            ctx->launches.fetch_add(p->kernels_sweep);
        } else {
            QC_TRY(queue_sweep(p, stream));
        }
    } else {
        qc_range range("qc.sweep_full");
        while (true) {
            if (p->captured) {
                QC_CUDA_TRY(ctx, cudaGraphLaunch(p->full, stream));
                ctx->launches.fetch_add(p->kernels_full);
            } else {
                QC_TRY(queue_full(p, stream));
            }
            QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
            QC_TRY(qc_debug_take(ctx));
            if (p->pinned[0] == ST_TIMEOUT) {
                p->have_hist = false;
                qc_set_error(ctx, "qc_sweep_run: BFS grid barrier timed out");
                return QC_ERR_TIMEOUT;
            }
            if (p->pinned[0] != ST_NEED_ROWS) break;
            // deeper than the rows allow: twice the rows, captured again
            int32_t rows = p->rows * 2 > p->pinned[1] + 1 ? p->rows * 2 : p->pinned[1] + 1;
            if (rows > g->n + 1) rows = g->n + 1;
            QC_TRY(size_rows(p, rows));
            if (p->captured) capture_all(p);
        }
        p->have_hist = true;
        p->D = p->pinned[1] - 1;
    }
    if (n_clusters_out) {
        QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        std::memcpy(n_clusters_out, p->pinned + 8, sizeof(int32_t) * (size_t)p->S);
    }
    return QC_OK;
}
