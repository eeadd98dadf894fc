// Internal declarations shared by the translation units of libqcgraph.so.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qcgraph.h"

// ---- context -------------------------------------------------------------------

struct qc_tune_key {
    int kind;        // which kernel family
    int n_bucket;    // log2 bucket of the node count
    int deg_bucket;  // log2 bucket of the mean degree
    bool operator<(const qc_tune_key &o) const {
        if (kind != o.kind) return kind < o.kind;
        if (n_bucket != o.n_bucket) return n_bucket < o.n_bucket;
        return deg_bucket < o.deg_bucket;
    }
};

struct qc_ctx {
    int device = 0;
    size_t budget = 0;                    // 0 = no cap
    std::atomic<size_t> in_use{0};
    qc_allocator alloc{};
    bool custom_alloc = false;
    int num_sms = 0;
    size_t l2_bytes = 0;
    size_t smem_optin = 0;
    mutable std::mutex err_mu;
    std::string last_error;
    std::mutex tune_mu;
    std::map<qc_tune_key, int> tune;      // autotuned choice per (kind, size bucket)
    std::atomic<uint64_t> launches{0};    // kernels launched on this context
    std::atomic<bool> timing{false};
    std::mutex stats_mu;
    std::map<std::string, qc_kernel_stats> stats;
    std::mutex pinned_mu;
    std::vector<void *> pinned_free;       // 64 KiB pinned host blocks ready for reuse
    std::atomic<float> coop_sm_share{1.0f};  // share of SMs the cooperative kernels fill
    std::mutex streams_mu;
    std::vector<std::pair<int, cudaStream_t>> spare_streams;   // (priority, stream) not in use
    std::vector<cudaStream_t> all_streams;                       // every stream the context made
    ~qc_ctx();
};

// Streams the library makes (sweep and batch plans, servers) belong to the context
// and live until it is destroyed: memory allocated stream-ordered on one of them (a
// graph prepared by a plan, say) can be given back on it whenever its owner goes.
// A released stream returns to the context's spares (non-blocking, by priority).
cudaError_t qc_stream_acquire(qc_ctx *ctx, int priority, cudaStream_t *out);
void qc_stream_release(qc_ctx *ctx, cudaStream_t s, int priority);

// A pinned host block of QC_PINNED_BYTES for small device<->host transfers,
// taken from the context's pool and given back on destruction.
#define QC_PINNED_BYTES (64u << 10)
struct qc_pinned {
    qc_ctx *ctx;
    void *ptr = nullptr;
    explicit qc_pinned(qc_ctx *c) : ctx(c) {}
    qc_pinned(const qc_pinned &) = delete;
    qc_pinned &operator=(const qc_pinned &) = delete;
    qc_status acquire();
    ~qc_pinned();
};

// Two CUDA events for timing one launch.
struct qc_event_pair {
    cudaEvent_t a = nullptr, b = nullptr;
    qc_status create(qc_ctx *ctx);
    ~qc_event_pair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// An NVTX range around one phase of the method (graph upload, preparation,
// BFS, potential, descent, batch run, shortest paths), for profilers that read
// NVTX (ncu --nvtx, Nsight Systems).  Without such a tool attached a push or
// pop costs a function call.
struct qc_range {
    explicit qc_range(const char *name) { nvtxRangePushA(name); }
    ~qc_range() { nvtxRangePop(); }
    qc_range(const qc_range &) = delete;
    qc_range &operator=(const qc_range &) = delete;
};

// Count one launch (and surface launch-configuration errors).
#define QC_LAUNCHED(ctx)                                                                \
    do {                                                                                \
        (ctx)->launches.fetch_add(1, std::memory_order_relaxed);                        \
        QC_CUDA_TRY((ctx), cudaGetLastError());                                         \
    } while (0)

void qc_record_kernel(qc_ctx *ctx, const char *kernel, double ms, double model_bytes, double min_bytes = 0.0);

void qc_set_error(qc_ctx *ctx, const char *fmt, ...);

// Scratch and resident memory go through these so that the budget is honoured.
qc_status qc_mem_alloc(qc_ctx *ctx, size_t bytes, cudaStream_t stream, void **out);
void qc_mem_free(qc_ctx *ctx, void *ptr, size_t bytes, cudaStream_t stream);

// A scratch buffer released when it goes out of scope (stream-ordered).
struct qc_buffer {
    qc_ctx *ctx = nullptr;
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    qc_buffer() = default;
    qc_buffer(const qc_buffer &) = delete;
    qc_buffer &operator=(const qc_buffer &) = delete;
    qc_buffer(qc_buffer &&o) noexcept { *this = std::move(o); }
    qc_buffer &operator=(qc_buffer &&o) noexcept {
        release();
        ctx = o.ctx; ptr = o.ptr; bytes = o.bytes; stream = o.stream;
        o.ptr = nullptr; o.bytes = 0;
        return *this;
    }
    ~qc_buffer() { release(); }
    qc_status allocate(qc_ctx *c, size_t b, cudaStream_t s) {
        release();
        ctx = c; stream = s; bytes = b;
        if (b == 0) return QC_OK;
        qc_status st = qc_mem_alloc(c, b, s, &ptr);
        if (st != QC_OK) { ptr = nullptr; bytes = 0; }
        return st;
    }
    void release() {
        if (ptr) qc_mem_free(ctx, ptr, bytes, stream);
        ptr = nullptr; bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

#define QC_CUDA_TRY(ctx, expr)                                                          \
    do {                                                                                \
        cudaError_t qc_e_ = (expr);                                                     \
        if (qc_e_ != cudaSuccess) {                                                     \
            qc_set_error((ctx), "%s:%d: %s: %s", __FILE__, __LINE__, #expr,             \
                         cudaGetErrorString(qc_e_));                                    \
            return QC_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

#define QC_TRY(expr)                                                                    \
    do {                                                                                \
        qc_status qc_s_ = (expr);                                                       \
        if (qc_s_ != QC_OK) return qc_s_;                                               \
    } while (0)

// ---- graph --------------------------------------------------------------------

struct qc_graph {
    qc_ctx *ctx = nullptr;
    std::mutex use_mu;       // held by a serving worker while it runs the graph's single-graph path
    int32_t n = 0;
    int64_t nnz = 0;
    bool directed = false;   // row v = out-neighbours (QC_DIRECTED)
    qc_buffer row_ptr;       // int32[n+1]
    qc_buffer col_idx;       // int32[nnz]
    bool weighted = false;   // qc_graph_set_weights was called
    qc_buffer weights;       // double[nnz], aligned with col_idx
    // cached all-source BFS result
    bool hist_valid = false;
    int32_t D = 0;           // largest finite hop distance
    int32_t hist_rows = 0;   // allocated rows of hist
    qc_buffer hist;          // int32[hist_rows][n], level-major
    bool bfs_queued = false; // a BFS was queued and its outcome not yet read (qc_bfs_settle)
    qc_buffer bfs_out;       // int32[8]: BFS outcome, [0] state, [1] highest level reached
    // preparation (see prep.cu), computed once
    bool prepared = false;
    bool prep_checked = false;   // the components launch's status has been read
    qc_buffer prep_ctl;      // int32[8]: status and grid barrier of that launch; [6..7] sum of degree^2
    qc_buffer comp;          // int32[n] component = smallest node id in it
    qc_buffer wcomp;         // int32[W] component of a whole 64-source word, or -1
    qc_buffer wmajor;        // int32[W] the component holding most of a mixed word's sources
    qc_buffer wmask;         // uint64[W] bits of the word's sources in that component
    qc_buffer order;         // int32[n] nodes, heaviest degree bucket first
    qc_buffer oinfo;         // int4[n]: {node, row start, row end, 0} at each order position
};

// prep.cu
// Queues the preparation kernels without waiting; the components launch's
// status stays on the device until qc_graph_prepare_status reads it (the BFS
// reads it in the same wait as its own status).
qc_status qc_graph_prepare(qc_graph *g, cudaStream_t stream);
// QC_OK or QC_ERR_TIMEOUT from the last preparation, given its status word as
// copied to the host after a wait.
qc_status qc_graph_prepare_status(qc_graph *g, int32_t host_status);
// hist[0][v] = 1, hist[1][v] = deg(v)
qc_status qc_fill_first_rows(qc_graph *g, cudaStream_t stream);
// bfs.cu helper shared with the batched paths
double qc_bfs_level_model_bytes(int64_t n, int64_t nnz, int64_t wn);
// context.cu: words of sources per BFS chunk (also sizes the server's memory estimate)
int32_t qc_bfs_chunk_words(const qc_ctx *ctx, int32_t n);

// ---- entry points implemented per translation unit ---------------------------------

// bfs.cu: scratch of one all-source BFS (every chunk reuses it).
struct qc_bfs_scratch {
    int32_t wc = 0, R_max = 0, T_max = 0;   // source words per chunk, row segments, tiles
    bool masks = false;                     // variant: change masks
    int32_t mask_ratio = 0;
    int32_t two_hop = 1;                    // levels 1-2 from the CSR: 0 never, 1 sparse graphs, 2 always
    qc_buffer visA, visB, sat, ctl, wl, fmask;
    qc_buffer cursor;                       // two-hop set-up over several chunks: 2 x int32[n]
    // Gives every buffer back (stream-ordered on the stream each was allocated on,
    // so call it while those streams exist).
    void release() {
        visA.release();
        visB.release();
        sat.release();
        ctl.release();
        wl.release();
        fmask.release();
        cursor.release();
    }
};
qc_status qc_bfs_scratch_init(qc_graph *g, qc_bfs_scratch &bs, cudaStream_t stream);
// prep.cu: device address of the sum over nodes of degree^2 (written by the preparation)
const unsigned long long *qc_graph_deg2(const qc_graph *g);
// Queue one launch of the BFS kernel: the chunk of source words from w0, from
// level `start` (2 = fresh), adding into hist[rows][n], outcome in out[0..1]
// (reset first when reset_out).  The graph must be prepared.
qc_status qc_bfs_launch(qc_graph *g, qc_bfs_scratch &bs, int32_t w0, int32_t start, int32_t *hist, int32_t rows,
                        int32_t *out, bool reset_out, unsigned long long *stamps, cudaStream_t stream);
// bfs.cu: all-source bitset BFS + histogram into g->hist (sets D, hist_valid),
// waiting for every launch.
qc_status qc_bfs_histogram(qc_graph *g, cudaStream_t stream);
// The same BFS with every launch queued and nothing waited for (timing mode and
// graphs without edges still wait): g->hist is valid for work queued behind it on
// `stream`, but D is known on the device only (g->bfs_out[1] - 1) until
// qc_bfs_settle reads the outcome.  Every call that queues it settles before it
// returns.
qc_status qc_bfs_enqueue(qc_graph *g, cudaStream_t stream);
// Wait for `stream` and read a queued BFS's outcome: sets D, or returns its
// error; when a launch ran out of histogram rows the BFS is run again (waiting)
// and *redone is set, so that work queued on the old rows must be queued again.
qc_status qc_bfs_settle(qc_graph *g, cudaStream_t stream, bool *redone);

// potential.cu: V[s][v] from the cached histogram; keys (optional): the descent's
// order-preserving keys of V, node-major int64[n][n_sigma], written alongside.
qc_status qc_potential_from_hist(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V,
                                 cudaStream_t stream, long long *keys = nullptr);
// Host weight tables for one sigma, d = 0..len-1 (identical expression to the
// definition: w = exp(-d^2 / (2 sigma^2)), u = d^2 w).
void qc_weight_table(double sigma, int32_t len, double *w, double *u);
// Check sigma: finite and > 0.
bool qc_sigma_ok(double sigma);
// Tables of the potential kernel for sigmas over distances 0..L-1: w[s][d], then
// u[s][d], then den[s] = 2 sigma^2.
void qc_potential_tables(const double *sigmas, int32_t n_sigma, int32_t L, std::vector<double> &tab);
// Whether such tables travel as a kernel parameter (else they are read from a device copy).
bool qc_potential_tables_inline(int32_t n_sigma, int32_t L);
// Queue the potential kernel over hist[Dmax+1][n] (D_dev: the BFS's outcome words
// + 1 when D is known on the device only, else null); dtab: device copy of tab
// when the tables do not travel inline; keys as for qc_potential_from_hist.
qc_status qc_potential_launch(qc_ctx *ctx, int32_t n, const int32_t *hist, int32_t Dmax, const int32_t *D_dev,
                              int32_t n_sigma, const std::vector<double> &tab, const double *dtab, double *V,
                              long long *keys, cudaStream_t stream);

// ggd.cu: parents and roots.
// order: nodes heaviest first (the graph's preparation) or NULL for 0..n-1.
// keys (optional): V's keys already written by the potential kernel (V is then not read).
qc_status qc_descend(qc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *order, const double *V, int32_t n_sigma, int32_t *labels,
                     int32_t *n_roots_dev, cudaStream_t stream, const long long *keys = nullptr);
// The same with caller-provided scratch: parent int32[n_sigma][n], keys int64[n][n_sigma]
// (filled from V here unless keys_ready).
qc_status qc_descend_into(qc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                          const int32_t *order, const double *V, int32_t n_sigma, int32_t *labels,
                          int32_t *n_roots_dev, int32_t *parent, long long *keys, cudaStream_t stream,
                          bool keys_ready = false);

// batch.cu: the graph-per-CTA kernel without a plan (used by the serving loop)
struct qc_cta_launch;
int32_t qc_cta_max_nodes();
size_t qc_cta_bytes_per_node();
qc_status qc_cta_launch_async(qc_ctx *ctx, int32_t m, qc_graph *const *graphs, const double *sigmas,
                              int32_t *const *labels, int max_sms, cudaStream_t stream, qc_cta_launch **out);
// counts: device int32[m]; flags: device int32[m + 1] (see batch.cu)
int32_t *qc_cta_counts(qc_cta_launch *L);
int32_t *qc_cta_flags(qc_cta_launch *L);
void qc_cta_launch_free(qc_cta_launch *L);

// validate.cu
// One launch checks the whole CSR (row_ptr included) and waits for the verdict.
qc_status qc_validate_csr(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr_dev,
                          const int32_t *col_idx_dev, bool symmetric, cudaStream_t stream);
// The same check queued without waiting: err (device int32) receives its flags,
// and if it found anything every row of row_ptr_dev is then made empty, so that
// the work queued behind it stays inside the arrays; the caller reads err once
// its work has finished and reports qc_csr_verdict of it.
qc_status qc_validate_csr_queue(qc_ctx *ctx, int32_t n, int64_t nnz, int32_t *row_ptr_dev,
                                const int32_t *col_idx_dev, bool symmetric, int32_t *err, cudaStream_t stream);
qc_status qc_csr_verdict(qc_ctx *ctx, int32_t flags);
qc_status qc_validate_hist(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr_dev,
                           const int32_t *hist_dev, int32_t D, cudaStream_t stream);

// selftest.cu: in the debug build, the first failed bounds check since the last
// call (read and cleared after the work queued so far has finished; the
// caller has already waited for it); QC_ERR_INVALID_GRAPH naming it, else
// QC_OK.  Always QC_OK in release builds.
qc_status qc_debug_take(qc_ctx *ctx);

static inline cudaStream_t qc_stream(void *s) { return static_cast<cudaStream_t>(s); }

static inline int qc_ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Share of the SMs the calling thread's cooperative launches may fill, when set
// (> 0); else the context's share applies.  The serving loop's workers set it per
// request.
extern thread_local float qc_thread_sm_share;

// SMs' worth of blocks a cooperative (persistent) kernel may fill.
static inline int qc_coop_sms(const qc_ctx *ctx) {
    const float share = qc_thread_sm_share > 0.f ? qc_thread_sm_share : ctx->coop_sm_share.load();
    const int s = (int)(share * (float)ctx->num_sms);
    return s < 1 ? 1 : (s > ctx->num_sms ? ctx->num_sms : s);
}
