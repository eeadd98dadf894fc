/*
 * qcgraph — graph Quantum Clustering on one GB300 (sm_103a).
 *
 * C ABI of libqcgraph.so.  Plain pointers and sizes only; every call returns a
 * qc_status and no exception crosses the boundary.  Details of the last error
 * of a context are in qc_last_error().
 *
 * The method (arXiv 2305.14641, Section 3.1, Algorithms 1-4):
 *   dist(i, j)  hop distance between nodes i and j of an undirected,
 *               unweighted graph (infinite when unreachable; such pairs add
 *               nothing to the sums below);
 *   V(i)        = (1 / (2 sigma^2)) * sum_j d^2 e^{-d^2/(2 sigma^2)}
 *                                   / sum_j e^{-d^2/(2 sigma^2)},  d = dist(i, j),
 *               j over all nodes including i (Eq. 7 last line, Algorithm 1);
 *   parent(i)   the lowest-potential neighbour of i (smallest node id among
 *               equal minima) when its V is strictly below V(i), else i
 *               (Algorithm 2 with the prose that follows Algorithm 4);
 *   label(i)    the root reached from i by following parents (Algorithm 3),
 *               reported as that root's node id.
 *
 * Conventions for every call:
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are asynchronous on it unless they write host memory, in
 *     which case they synchronise that stream before returning.
 *   - Arrays marked "device" must be device memory of the context's GPU and stay
 *     valid until the work queued on `stream` has completed.  The caller owns
 *     every array it passes; the library never frees them.
 *   - Outputs go into caller-provided buffers.  The library allocates its own
 *     scratch through the context's allocator (see qc_allocator).
 *   - An object made on a stream (a graph, a batch plan) allocates its memory
 *     stream-ordered on that stream and gives it back on the same stream when it
 *     is destroyed, so the stream must outlive the object.  Streams the library
 *     makes itself (for sweep and batch plans and servers) belong to the context
 *     and live until qc_context_destroy, so a graph that such a plan or server
 *     prepared can be destroyed after it.
 *   - There is no CPU fallback: without a usable GPU every call that needs one
 *     returns QC_ERR_CUDA.
 */
#ifndef QCGRAPH_H
#define QCGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QC_OK = 0,
    QC_ERR_INVALID_ARG = 1,    /* a null pointer, a size out of range, sigma <= 0 or NaN */
    QC_ERR_INVALID_GRAPH = 2,  /* CSR fails validation (see QC_VALIDATE) */
    QC_ERR_OOM = 3,            /* the allocator returned no memory */
    QC_ERR_BUDGET = 4,         /* the request would exceed the context's memory budget */
    QC_ERR_CUDA = 5,           /* a CUDA runtime error, or no usable GPU */
    QC_ERR_TIMEOUT = 6,        /* a device-side wait gave up (its time limit ran out) */
    QC_ERR_CANCELLED = 7,      /* a served request was cancelled */
    QC_ERR_NOT_READY = 8       /* a served request has not completed yet */
} qc_status;

typedef struct qc_ctx qc_ctx;
typedef struct qc_graph qc_graph;
typedef struct qc_batch qc_batch;
typedef struct qc_server qc_server;
typedef struct qc_sweep qc_sweep;

/* Device-memory provider.  alloc returns `bytes` of device memory usable on
 * `stream` (NULL on failure); free returns it.  Both may be called from any
 * thread that calls into the library, and from the serving thread.  Passing
 * NULL for the allocator selects cudaMallocAsync / cudaFreeAsync. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} qc_allocator;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the scratch
 * and resident-graph memory the library holds at once (0 = no cap); a call that
 * would exceed it returns QC_ERR_BUDGET and allocates nothing.  `alloc` is
 * copied; NULL selects the stream-ordered CUDA allocator.
 * Errors: QC_ERR_INVALID_ARG (out == NULL, device < 0), QC_ERR_CUDA. */
qc_status qc_context_create(int device, size_t mem_budget_bytes, const qc_allocator *alloc,
                            qc_ctx **out);
/* Destroy a context.  All graphs, batches and servers made from it must have
 * been destroyed first. */
void qc_context_destroy(qc_ctx *ctx);
/* Bytes the context currently holds through its allocator. */
size_t qc_context_bytes_in_use(const qc_ctx *ctx);
/* Per-kernel timing, for measurement.  When enabled, the library brackets every
 * launch of its dominant kernels with CUDA events on the launching stream and
 * accumulates their durations with two byte counts per launch:
 *   model_bytes  the pull-all model of the BFS: per level pass over a chunk of
 *                wn source words, 8 wn (E + 3N) bitset bytes + the CSR + one
 *                histogram row (an upper bound: saturated rows are skipped);
 *   min_bytes    the bytes the launch must move between HBM and the GPU at
 *                the least: its inputs read once (CSR, node order and row
 *                bounds, components, per-word masks), its histogram rows
 *                written once, and, for each level, the bitset rows still
 *                open at that level (read and written, 32 bytes per 16-byte
 *                segment, counted on the device) beyond what L2 can hold.
 * Names: "bfs_level" per launch, "bfs_pass_<l>" per level from device
 * timestamps.  Off by default; it adds one counter update per warp and item
 * run to the BFS. */
typedef struct {
    uint64_t launches;
    double total_ms;        /* sum of event-measured launch durations */
    double model_bytes;     /* sum of modelled pull-all bytes */
    double min_bytes;       /* sum of compulsory HBM bytes */
} qc_kernel_stats;
qc_status qc_context_set_timing(qc_ctx *ctx, int enable);
/* kernel: "bfs_level" (the bitset BFS level step).  reset != 0 clears the
 * counters after reading them. */
qc_status qc_context_kernel_stats(qc_ctx *ctx, const char *kernel, qc_kernel_stats *out, int reset);
/* Number of kernels the library has launched on this context so far. */
uint64_t qc_context_launch_count(const qc_ctx *ctx);
/* Static text for a status code. */
const char *qc_status_string(qc_status s);
/* Message of the most recent error on this context ("" if none).  Valid until
 * the next call on the context. */
const char *qc_last_error(const qc_ctx *ctx);

/* ---- one graph ------------------------------------------------------------ */

enum {
    QC_PTR_DEVICE = 1u, /* row_ptr / col_idx are device pointers (else host) */
    QC_VALIDATE = 2u,   /* check the CSR: row_ptr[0] = 0, non-decreasing, row_ptr[n] =
                           nnz; column ids in [0, n); rows strictly ascending (sorted,
                           no duplicates); no self-loops; symmetric (undirected) unless
                           QC_DIRECTED */
    QC_DIRECTED = 4u    /* the graph is directed: row v lists v's out-neighbours */
};

/* Upload an unweighted graph in CSR form (the paper's adjacency matrix input
 * of Algorithms 1 and 4, held sparse): node v's neighbours are
 * col_idx[row_ptr[v] .. row_ptr[v+1]-1].  row_ptr: int32[n+1]; col_idx:
 * int32[nnz].  Undirected graphs store each edge in both rows.  With
 * QC_DIRECTED row v holds the edges v -> u (graph(v, u) of Algorithm 1): the
 * distance dist(i, j) is then the length of the shortest directed path from i
 * to j, and the descent of Algorithm 2 looks at out-neighbours.  The library copies
 * the arrays into device memory it owns; the copy stays resident until
 * qc_graph_destroy.  Without QC_VALIDATE the CSR is trusted: an invalid one
 * gives undefined results (out-of-range ids may fault the GPU).
 * Errors: QC_ERR_INVALID_ARG (n < 1, nnz < 0, nnz >= 2^31, null pointers),
 * QC_ERR_INVALID_GRAPH (validation failed), QC_ERR_BUDGET, QC_ERR_OOM,
 * QC_ERR_CUDA. */
qc_status qc_graph_create(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, uint32_t flags, void *stream,
                          qc_graph **out);
void qc_graph_destroy(qc_graph *g);
/* Release the cached histogram (the next qc_potential / qc_graph_histogram runs
 * the BFS again). */
void qc_graph_drop_histogram(qc_graph *g);
int32_t qc_graph_num_nodes(const qc_graph *g);
int64_t qc_graph_num_edges(const qc_graph *g);

/* Per-node hop-distance histogram (Algorithm 1 depends on node i only through
 * the multiset {dist(i, j)}): hist[d][v] = #{j : dist(v, j) = d} for d = 0..D,
 * D the largest finite distance in the graph.  Runs the all-source bitset BFS
 * the first time (the result is cached in the graph and reused by later
 * qc_potential calls for any sigma).
 * hist_out: device int32[(D+1) * n] row-major (level-major) or NULL to query D
 * only.  D_out: host, required.  Synchronises `stream` (D is a host output).
 * Errors: QC_ERR_INVALID_ARG, QC_ERR_BUDGET, QC_ERR_OOM, QC_ERR_CUDA. */
qc_status qc_graph_histogram(qc_graph *g, int32_t *hist_out, int32_t *D_out, void *stream);

/* Edge weights for the weighted reading of Section 3.1 (an edge's distance is
 * its weight; between any two nodes, the length of the lightest path, summed
 * hop by hop in binary64).  w: double[nnz] aligned with col_idx (w[e] is the
 * weight of the edge in position e), host memory or (QC_PTR_DEVICE) device
 * memory; the library keeps a copy with the graph.  With QC_VALIDATE the
 * weights must be finite and > 0, and equal in both rows of an undirected edge.
 * The weights serve qc_potential_weighted only; the hop-distance calls ignore
 * them.  Errors: QC_ERR_INVALID_ARG, QC_ERR_INVALID_GRAPH, QC_ERR_BUDGET,
 * QC_ERR_OOM, QC_ERR_CUDA. */
qc_status qc_graph_set_weights(qc_graph *g, const double *w, uint32_t flags, void *stream);

/* Install a histogram computed earlier (qc_graph_histogram of the same graph,
 * saved and reloaded), so that potentials for new sigma values need no BFS: the
 * checkpoint of a sigma sweep.  hist: int32[(D+1) * n], level-major as
 * qc_graph_histogram writes it, host memory or (QC_PTR_DEVICE) device memory;
 * the library copies it.  0 <= D < n.  With QC_VALIDATE the rows are checked on
 * the device against what the graph fixes: h(0, v) = 1, h(1, v) = out-degree,
 * entries >= 0, sum over d <= n, row D not all zero, and D = 0 exactly when the
 * graph has no edges.
 * Errors: QC_ERR_INVALID_ARG (null pointers, D out of range),
 * QC_ERR_INVALID_GRAPH (validation failed), QC_ERR_BUDGET, QC_ERR_OOM,
 * QC_ERR_CUDA. */
qc_status qc_graph_set_histogram(qc_graph *g, const int32_t *hist, int32_t D, uint32_t flags,
                                 void *stream);

/* Potential V for every node and every sigma (Eq. 7 last line, Algorithm 1),
 * in binary64, summed over distances in ascending order from the histogram.
 * sigmas: host double[n_sigma], each finite and > 0.  V_out: device
 * double[n_sigma * n], V_out[s * n + v].
 * Errors: QC_ERR_INVALID_ARG (n_sigma < 1, bad sigma, null), QC_ERR_BUDGET,
 * QC_ERR_OOM, QC_ERR_CUDA. */
qc_status qc_potential(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out,
                       void *stream);

/* The potential with the distance of Section 3.1 taken literally from the
 * adjacency matrix instead of hop counts: 0 from a node to itself, the edge
 * weight (1 here) to a neighbour, and M, a value above every weight that the
 * paper does not fix, to every other node, connected or not.  Node v then has
 * deg(v) terms at distance 1 and n - 1 - deg(v) at distance M; no BFS runs.
 * Same arithmetic, layout and errors as qc_potential; M must be finite and > 1
 * (QC_ERR_INVALID_ARG otherwise). */
qc_status qc_potential_adjacency(qc_graph *g, const double *sigmas, int32_t n_sigma, double M,
                                 double *V_out, void *stream);

/* Graph Gradient Descent and cluster centers (Algorithms 2 and 3) for n_sigma
 * potential vectors.  V: device double[n_sigma * n] (as written by
 * qc_potential), free of NaN (a NaN gives unspecified parents).  labels_out: device int32[n_sigma * n], the root node id each
 * node descends to.  n_clusters_out: host int32[n_sigma] (number of roots) or
 * NULL; when given, the call synchronises `stream`.
 * Errors: QC_ERR_INVALID_ARG, QC_ERR_BUDGET, QC_ERR_OOM, QC_ERR_CUDA. */
qc_status qc_ggd_labels(qc_graph *g, const double *V, int32_t n_sigma, int32_t *labels_out,
                        int32_t *n_clusters_out, void *stream);

/* Algorithm 1 over weighted distances (qc_graph_set_weights first): for every
 * node i and sigma, V = (sum_j d^2 e^{-d^2/2sigma^2} / sum_j e^{-d^2/2sigma^2}) /
 * (2 sigma^2) with d = dist(i, j) the lightest-path length from i (along arcs
 * for a directed graph), j over the nodes i reaches, i itself included.  All-
 * source shortest paths run on the device in blocks of sources; the sums use
 * binary64 with the device's exp (for an undirected graph each pair's terms
 * once for both nodes, and the e^{...} sum exactly in integers but for one
 * truncation per term), so V agrees with a sequential host evaluation to
 * within 1e-12 relative and is the same on every run.  V_out: device double[n_sigma * n].  Descent: qc_ggd_labels on V_out.
 * Errors: QC_ERR_INVALID_ARG (no weights, bad sigma), QC_ERR_BUDGET,
 * QC_ERR_OOM, QC_ERR_CUDA (including weights that let lengths fall without
 * end), QC_ERR_TIMEOUT. */
qc_status qc_potential_weighted(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out,
                                void *stream);

/* Algorithm 4 in one call: qc_potential then qc_ggd_labels.  V_out may be NULL
 * (the potentials then live in library scratch).  Same arguments and errors as
 * those two calls. */
qc_status qc_solve(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out,
                   int32_t *labels_out, int32_t *n_clusters_out, void *stream);

/* Algorithm 4 from a CSR to labels in one call, for a graph that is not kept:
 * qc_graph_create (arguments and flags as there: host arrays unless
 * QC_PTR_DEVICE, QC_VALIDATE, QC_DIRECTED), then the BFS and histogram, the
 * potential for every sigma, the descent and the roots, with the labels copied
 * to labels_out: int32[n_sigma][n], host or device memory (any address the CUDA
 * copy engines can write).  n_clusters_out: host int32[n_sigma] or NULL.  The
 * work after the upload is queued back to back and the call waits once at the
 * end, so on return labels_out holds the result and the library holds nothing
 * of the graph.  QC_VALIDATE's check is queued too, ahead of the rest: if it
 * fails, the work behind it runs on the graph with every row emptied (so it
 * stays inside the arrays), the call returns QC_ERR_INVALID_GRAPH, and
 * labels_out and n_clusters_out then hold nothing meaningful.
 * Errors: those of qc_graph_create and qc_solve. */
qc_status qc_cluster(qc_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                     uint32_t flags, const double *sigmas, int32_t n_sigma, int32_t *labels_out,
                     int32_t *n_clusters_out, void *stream);

/* ---- one graph, a fixed sigma sweep, replayed ---------------------------------- */

/* A solve plan for one graph and a fixed list of sigma values: Algorithm 4 for
 * each sigma (the hop-distance histogram of every node behind Algorithm 1, the
 * potentials of Eq. 7, Graph Gradient Descent of Algorithm 2 and the roots of
 * Algorithm 3), queued once into CUDA graphs together with every buffer the
 * work uses, and replayed by qc_sweep_run.  The plan keeps a histogram of its
 * own (the graph's cached one is neither read nor changed).
 * sigmas: host double[n_sigma], each finite and > 0 (copied).  V_out: device
 * double[n_sigma * n] or NULL (the potentials then stay in plan memory);
 * labels_out: device int32[n_sigma * n], root node ids, V_out[s * n + v] and
 * labels_out[s * n + v] as qc_potential / qc_ggd_labels write them; both must
 * stay valid while the plan exists.  The graph must outlive the plan.  Runs of
 * one plan must not overlap on the GPU.  Creation synchronises `stream`.
 * Errors: QC_ERR_INVALID_ARG, QC_ERR_BUDGET, QC_ERR_OOM, QC_ERR_CUDA. */
qc_status qc_sweep_create(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out, int32_t *labels_out,
                          void *stream, qc_sweep **out);
/* One run.  reuse_histogram = 0: everything from the resident CSR (the BFS,
 * then potentials, descent and roots for every sigma); the call waits for the
 * run to read the BFS's outcome (a BFS deeper than the plan's histogram rows is
 * run again with more rows).  reuse_histogram != 0: potentials, descent and
 * roots from the histogram of the plan's last full run (QC_ERR_INVALID_ARG if
 * there was none); asynchronous on `stream` unless n_clusters_out is given.
 * n_clusters_out: host int32[n_sigma] (roots per sigma) or NULL.
 * Errors: QC_ERR_INVALID_ARG, QC_ERR_TIMEOUT (a device-side wait gave up),
 * QC_ERR_CUDA. */
qc_status qc_sweep_run(qc_sweep *p, int32_t reuse_histogram, int32_t *n_clusters_out, void *stream);
/* D of the last full run (-1 before one); whether runs replay captured CUDA
 * graphs (1) or queue the same kernels directly (0, where a capture is
 * refused); the kernels one full run executes.  Any pointer may be NULL. */
qc_status qc_sweep_info(const qc_sweep *p, int32_t *D, int32_t *captured, int64_t *kernels_per_run);
void qc_sweep_destroy(qc_sweep *p);

/* ---- quality of a clustering ------------------------------------------------------ */

/* The measures of the paper's evaluation (Section 4.2) for a label vector on the
 * device.  labels: device int32[n], each a node id in [0, n) (root ids, as
 * qc_ggd_labels writes them).  g: the clustered graph (undirected, n nodes, made
 * on ctx), or NULL to skip modularity.  truth: device int32[n] of true
 * classes in [0, n_truth), or NULL to skip ARI, FMI and NMI.  Results (host,
 * NaN where skipped):
 *   modularity  Q = inside / w - gamma sum_c (degree sum of c)^2 / w^2 (inside =
 *               CSR entries within a cluster, w = the degree total: Newman's form);
 *   ari         the Adjusted Rand Index (Hubert & Arabie) over pair counts of
 *               the contingency table;
 *   fmi         TP / sqrt((TP + FP)(TP + FN)) over pairs;
 *   nmi         MI / sqrt(H(truth) H(labels)), natural logarithms;
 *   clusters    distinct labels.
 * Counts and pair sums are exact integers on the device; the entropies and
 * the mutual information are binary64 sums.  Synchronises `stream`.
 * Errors: QC_ERR_INVALID_ARG (nulls, a graph of another size or context, a
 * label or class out of range, a contingency table over 2^31 cells),
 * QC_ERR_BUDGET, QC_ERR_OOM, QC_ERR_CUDA. */
typedef struct {
    double modularity, ari, fmi, nmi;
    int32_t clusters;
} qc_quality_result;
qc_status qc_quality(qc_ctx *ctx, const qc_graph *g, int32_t n, const int32_t *labels, const int32_t *truth,
                     int32_t n_truth, double gamma, qc_quality_result *out, void *stream);

/* ---- many graphs ------------------------------------------------------------ */

/* A batch plan: Algorithm 4 for n_graphs graphs, graph k clustered with
 * sigma_per_graph[k] (host), its labels written to labels_out + label_offsets[k]
 * (labels_out: device int32, label_offsets: host int64[n_graphs]; the caller
 * sizes labels_out so that every graph's n labels fit).  The plan packs the
 * graphs' descriptors once, picks tile shapes with the context's autotuner,
 * and captures the whole solve (one persistent kernel over all graphs, then
 * descent and roots) into a CUDA graph.  The graphs must outlive the plan.
 * n_clusters_out of qc_batch_run: host int32[n_graphs] or NULL (when given,
 * the call synchronises `stream`).
 * Errors: QC_ERR_INVALID_ARG, QC_ERR_BUDGET, QC_ERR_OOM, QC_ERR_CUDA,
 * QC_ERR_TIMEOUT (a device-side wait gave up). */
qc_status qc_batch_create(qc_ctx *ctx, int32_t n_graphs, qc_graph *const *graphs,
                          const double *sigma_per_graph, int32_t *labels_out,
                          const int64_t *label_offsets, void *stream, qc_batch **out);
qc_status qc_batch_run(qc_batch *b, int32_t *n_clusters_out, void *stream);
void qc_batch_destroy(qc_batch *b);
/* The configuration the plan runs: threads per CTA, source words per chunk and
 * the mean degree below which a thread instead of a warp takes a node (the
 * autotuner's choice, or QCGRAPH_BATCH_CONFIG="threads,words[,degree]" from the
 * environment when that names candidates).  All are 0 when no graph of the
 * plan fits the graph-per-CTA kernel.  sparse_degree may be NULL.
 * Errors: QC_ERR_INVALID_ARG. */
qc_status qc_batch_config(const qc_batch *b, int32_t *threads, int32_t *chunk_words, int32_t *sparse_degree);

/* One-shot form: create a plan, run it once, destroy it. */
qc_status qc_solve_batch(qc_ctx *ctx, int32_t n_graphs, qc_graph *const *graphs,
                         const double *sigma_per_graph, int32_t *labels_out,
                         const int64_t *label_offsets, void *stream);

/* ---- serving ------------------------------------------------------------------ */

typedef struct {
    size_t mem_budget_bytes;   /* admission budget for resident requests (0 = the context's,
                                  or 100 GB if the context has none) */
    int32_t max_active;        /* most requests on the GPU at once (0 = 256) */
    int32_t streams;           /* batched launches in flight at once (0 = 4) */
    int32_t large_workers;     /* threads running the single-graph path (0 = 4) */
    float large_sm_share;      /* share of the SMs the single-graph path's persistent
                                  kernels may fill, leaving the rest to batched launches
                                  (0 = 0.4); applies to the whole context until
                                  qc_server_destroy restores its previous share, so
                                  give a server a context of its own */
    int32_t divide_share;      /* 1: a large request gets large_sm_share divided by the
                                  number of large requests running at that moment (a lone
                                  one gets all of it); 0: each gets large_sm_share */
} qc_server_config;

typedef struct {
    uint64_t submitted, completed, cancelled, failed;
    uint64_t steps;            /* batched launches the scheduler issued */
    uint64_t large_solved;     /* requests solved one by one on the large-graph worker */
    size_t bytes_resident;     /* admitted requests' estimated bytes right now */
    size_t peak_bytes_resident;
    int32_t active, queued;
    int32_t peak_in_flight;    /* most batched launches on the GPU at once */
} qc_server_stats;

/* Per-request times on the host clock (milliseconds from submission). */
typedef struct {
    double admit_ms;           /* admitted to the GPU */
    double start_ms;           /* its GPU work issued (batched launch, or taken by a large-graph worker) */
    double done_ms;            /* result available (the request's latency) */
    int32_t n;
    int64_t nnz;
    int32_t batch_size;        /* requests in the launch that carried it (0: large-graph worker) */
} qc_request_info;

/* A serving loop on its own host threads: submitted requests wait in FIFO
 * order until their memory estimate fits the budget and a slot is free.
 * Admitted requests up to the graph-per-CTA limit (2048 nodes) are grouped
 * into one launch of the batched kernel per scheduler step; several such
 * launches run at once on separate streams, so requests that arrive while
 * others are on the GPU start without waiting for them (continuous batching).
 * Larger requests go to worker threads that run the single-graph path on
 * low-priority streams, their persistent kernels limited to a share of the SMs
 * so that batched launches keep running beside them.
 * A request's result does not depend on what it shares the GPU with.
 * cfg may be NULL for defaults. */
qc_status qc_server_create(qc_ctx *ctx, const qc_server_config *cfg, qc_server **out);
/* Queue one request: a host CSR (copied before the call returns; same layout
 * and checks as qc_graph_create with QC_VALIDATE) and its sigma.
 * req_id: host, receives the request id.
 * Errors: QC_ERR_INVALID_ARG, QC_ERR_INVALID_GRAPH, QC_ERR_BUDGET (the request
 * alone exceeds the budget).  The full CSR check runs here for graphs of up to
 * 2048 nodes; larger graphs get row_ptr checked here and the rest checked on
 * the GPU when they are admitted, in which case an invalid graph is reported
 * as the request's own status (QC_ERR_INVALID_GRAPH from poll / wait). */
qc_status qc_server_submit(qc_server *s, int32_t n, int64_t nnz, const int32_t *row_ptr,
                           const int32_t *col_idx, double sigma, uint64_t *req_id);
/* Queue one request on a graph already resident on the GPU (qc_graph_create on
 * the server's context) and its sigma: the form of Algorithm 4's input that
 * keeps the CSR, and after the first request the graph's histogram, on the
 * device across requests, so a later sigma on the same graph needs no BFS.  The
 * graph is only read (several requests on one graph run one after another on
 * the single-graph path); it must outlive its requests, and the caller must not
 * use it while they are pending.
 * Errors: QC_ERR_INVALID_ARG (null, bad sigma, a graph of another context),
 * QC_ERR_BUDGET. */
qc_status qc_server_submit_graph(qc_server *s, qc_graph *g, double sigma, uint64_t *req_id);
/* Non-blocking: *done = 1 and labels_out (host int32[n], root node ids),
 * *n_clusters and *info filled when the request has completed, else *done = 0.
 * labels_out, n_clusters and info may each be NULL.  A completed request's
 * result is released after it has been read.  Returns the request's own error
 * status if it failed, QC_ERR_INVALID_ARG for an unknown id. */
qc_status qc_server_poll(qc_server *s, uint64_t req_id, int32_t *labels_out,
                         int32_t *n_clusters, qc_request_info *info, int *done);
/* Blocking form of poll: waits up to timeout_ms (< 0: no limit); returns
 * QC_ERR_NOT_READY if the time ran out. */
qc_status qc_server_wait(qc_server *s, uint64_t req_id, int64_t timeout_ms,
                         int32_t *labels_out, int32_t *n_clusters, qc_request_info *info);
/* Cancel a queued or active request (its memory is released at the next step). */
qc_status qc_server_cancel(qc_server *s, uint64_t req_id);
qc_status qc_server_get_stats(qc_server *s, qc_server_stats *out);
/* Stop the loop (cancelling what is left) and free everything it holds. */
void qc_server_destroy(qc_server *s);

/* ---- self-test of the bounded device wait ----------------------------------------- */

/* The paper has no counterpart to this call.  Every persistent kernel of the
 * library synchronises its blocks with a grid barrier whose wait gives up once
 * 2 s have passed on the GPU's global timer, records a timeout and returns, so
 * that a block that never arrives surfaces as QC_ERR_TIMEOUT instead of a hung
 * GPU.  This call launches that barrier with two blocks, one of which leaves
 * without arriving, and a limit of timeout_us microseconds (1 .. 10^7).
 * waited_ns: host, receives how long the waiting block waited (GPU global
 * timer), or NULL.
 * Returns QC_ERR_TIMEOUT (with qc_last_error describing it) when the wait gave
 * up as designed; the context stays usable.  QC_ERR_CUDA if the barrier failed
 * to notice the missing block, QC_ERR_INVALID_ARG for a bad limit. */
qc_status qc_selftest_barrier_timeout(qc_ctx *ctx, int64_t timeout_us, int64_t *waited_ns, void *stream);

/* ---- self-test of the weighted path's exponential --------------------------------- */

/* The paper has no counterpart to this call.  The weighted potential evaluates
 * exp(-t) for every pair and sigma with a routine of its own that runs on the
 * integer pipe (GB300 issues binary64 operations at a small fraction of its
 * integer rate); this call runs it elementwise on caller data so that it can be
 * checked against a reference exp:
 *   QC_ARITH_EXP_NEG  out[i] = exp(-x[i]) (Tang's table-driven method in 64-bit
 *                     fixed point; about 1 ulp; 0 from x = 745 on);
 *                     x[i] >= 0 and not NaN; y unused (may be null).
 * x, out: device binary64[n], caller-owned, stream-ordered on `stream`.
 * QC_ERR_INVALID_ARG for another op, n < 0, or a null x or out with n > 0. */
enum { QC_ARITH_EXP_NEG = 0 };
qc_status qc_selftest_arith(qc_ctx *ctx, int32_t op, const double *x, const double *y, double *out, int64_t n,
                            void *stream);

/* ---- self-test of the debug build ------------------------------------------------------ */

/* The paper has no counterpart to this call.  The library has a debug build
 * (libqcgraph_debug.so, the same sources compiled with QC_DEBUG) in which every
 * neighbour id a kernel reads from the CSR is checked against [0, n) before it
 * is used: a failed check is recorded in a device word, the id is replaced by
 * 0, and the next call that waits for the GPU returns QC_ERR_INVALID_GRAPH
 * naming the kernel, instead of the GPU reading out of bounds.  Release builds
 * leave the checks out.  This call passes `id` through that check (it is never
 * used as an address) and returns what came out in *checked_out (id itself, or
 * 0 in the debug build when id is outside [0, n)); *debug_build says which
 * build answered.  Returns QC_ERR_INVALID_GRAPH when the check failed (debug
 * build only), QC_OK otherwise.  Errors: QC_ERR_INVALID_ARG, QC_ERR_CUDA. */
qc_status qc_selftest_debug_check(qc_ctx *ctx, int32_t id, int32_t n, int32_t *checked_out, int32_t *debug_build,
                                  void *stream);

/* ---- L2 read bandwidth probe ---------------------------------------------------------- */

/* The paper has no counterpart to this call.  It measures the read throughput of
 * a device buffer of `bytes` bytes (1 MiB .. 4 GiB; below the L2 size it stays
 * resident there) read through L2 only: mode 0 streams it (16 bytes per thread,
 * consecutive across the grid), mode 1 reads 512-byte segments at pseudo-random
 * positions, one warp per segment and four in flight, the pattern of the BFS's
 * neighbour gathers.  The buffer is read about 64 times in one timed launch
 * after a warming one; *gbs receives the bytes read per second / 1e9.  It serves
 * as the roofline of kernels whose working set lives in L2.
 * Errors: QC_ERR_INVALID_ARG, QC_ERR_BUDGET, QC_ERR_OOM, QC_ERR_CUDA. */
qc_status qc_selftest_l2_read(qc_ctx *ctx, int64_t bytes, int32_t mode, double *gbs, void *stream);

/* ---- histogram without device allocation ---------------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that may not
 * allocate device memory at all (a host application that fixes its GPU memory
 * plan at start-up and forbids later cudaMalloc calls, a plugin that may only
 * use buffers its host hands it, a loop that cannot afford an allocation).
 *
 * Same result as qc_graph_histogram, computed with no context and no
 * allocation: the working bitsets live in a 16 MiB array that is part of the
 * library (every GPU that loads the library holds it until the process exits).
 * row_ptr / col_idx: device int32 CSR of an undirected graph, as
 * qc_graph_create with QC_VALIDATE accepts it (not checked here).  hist_out:
 * device int32[max_levels * n], level-major; every row is written (rows past D
 * are zero).  D_out: host, receives D (-1 on failure).  Synchronises `stream`.
 *
 * max_levels: rows of hist_out; D + 1 rows suffice (D the largest finite
 * distance), so a graph with a path of n nodes needs at most n rows.
 *
 * Set-up: the first call on a device (with that device current) looks up the
 * array's device address; make that first call outside any stream capture.
 * `stream` must belong to the current device.
 * All calls share the one array: calls that overlap on the GPU (other streams
 * or threads) race and give wrong results.
 * Errors: QC_ERR_INVALID_ARG (n < 1 or n > 262144, max_levels < 2 or fewer
 * than D + 1, null pointers, a stream of another device), QC_ERR_CUDA. */
qc_status qc_histogram_static_scratch(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                      const int32_t *col_idx, int32_t *hist_out,
                                      int32_t max_levels, int32_t *D_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QCGRAPH_H */
