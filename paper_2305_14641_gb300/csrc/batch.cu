// Many graphs at once: Algorithm 4 for every graph of a batch in one
// persistent kernel, captured into a CUDA graph.
//
// Each CTA takes graphs from a queue (largest first) and runs the whole method
// for one graph before taking the next:
//   1. connected components by hook-and-shortcut label propagation in shared
//      memory (sources in another component start marked, as in the single-graph
//      BFS, so complete rows are skipped);
//   2. the all-source bitset BFS, a chunk of c source words at a time, with the
//      chunk's bitset columns of every node held in shared memory (two buffers of
//      n x c words): one warp per node ORs its neighbours' words, lanes over the
//      neighbour list (a thread per node for graphs of low mean degree); per-node
//      counts of new sources go to a per-CTA histogram in global memory, level by
//      level;
//   3. the potential of Eq. 7 / Algorithm 1 from the histogram with host-computed
//      binary64 weights for the graph's sigma (same expressions and ascending-
//      distance order as the single-graph path);
//   4. Graph Gradient Descent (strict descent, lowest-id tie-break) and roots by
//      path halving, both in shared memory; labels and the root count go out.
// A graph whose BFS needs more than L_cap levels is flagged and finished by the
// single-graph path on the host side.  Graphs too large for a CTA's shared
// memory take the single-graph path too.
//
// The plan picks the CTA size, the chunk width c and the thread-per-node degree
// threshold with a small autotuner that times the candidates on the batch
// itself and caches the winner per (largest n, mean degree) bucket in the
// context.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <numeric>
#include <vector>

#include "qc_device.cuh"
#include "qc_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t ONES = ~0ull;
constexpr int MAXC = 8;            // most source words per chunk (held per lane in registers)
constexpr int L_CAP = 32;          // histogram rows per graph in the batched kernel
constexpr int SPARSE_DEGREE = 24;  // default: below this mean degree a thread, not a warp, takes a node
constexpr int SPARSE_CANDIDATES[3] = {12, 24, 48};   // the autotuner's choices for that threshold
// Larger graphs take the single-graph path: one CTA walks all n/64 source words
// of its graph, so its time grows as n^2 x degree while the multi-CTA path
// spreads a large graph over the whole GPU.
constexpr int CTA_MAX_N = 2048;

struct CtaGraph {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    int32_t *labels;
    int32_t n;
    int32_t directed;              // row v = out-neighbours: components are the weak ones
    double den;                    // 2 sigma^2
};

struct CtaParams {
    const CtaGraph *graphs;
    const int32_t *order;          // work order, largest first
    int32_t n_graphs;
    int32_t *queue;                // next position in order
    const double *tables;          // [graph][w: L_CAP][u: L_CAP]
    int32_t n_max;
    int32_t c;                     // source words per chunk
    int32_t sparse_degree;         // graphs of lower mean degree: a thread per node
    int32_t *hist;                 // [gridDim.x][L_CAP][n_max]
    int32_t *n_clusters;           // [n_graphs]
    int32_t *overflow;             // [n_graphs + 1]: per graph, and [n_graphs] = any
};

__device__ __forceinline__ unsigned long long or_reduce64(unsigned long long x) {
    const unsigned lo = __reduce_or_sync(FULL, (unsigned)x);
    const unsigned hi = __reduce_or_sync(FULL, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Bits of word gw that start set for a node of component cv.
__device__ __forceinline__ uint64_t cta_preset(int n, int gw, int cv, const int32_t *L, const int32_t *wc) {
    uint64_t m;
    const int w = wc[gw];
    if (w >= 0) {
        m = (w == cv) ? 0ull : ONES;
    } else {
        m = 0ull;
        const int s0 = 64 * gw, cnt = min(64, n - s0);
        for (int b = 0; b < cnt; ++b)
            if (L[s0 + b] != cv) m |= 1ull << b;
    }
    const int tail = n - 64 * gw;
    if (tail < 64) m |= ONES << tail;
    return m;
}

__device__ void solve_graph(const CtaParams &P, const int g, unsigned char *smem) {
    const CtaGraph G = P.graphs[g];
    const int n = G.n;
    const int W = (n + 63) / 64;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    const int32_t *rp = G.row_ptr;
    const int32_t *ci = G.col_idx;
    int32_t *L = reinterpret_cast<int32_t *>(smem);                       // n
    int32_t *wc = L + n;                                                  // W
    uint64_t *colA = reinterpret_cast<uint64_t *>(smem + 16 * (((size_t)4 * (n + W) + 15) / 16));
    uint64_t *colB = colA + (size_t)n * P.c;
    int32_t *hist = P.hist + (size_t)blockIdx.x * L_CAP * P.n_max;
    __shared__ int s_flag;

    // 1. components: L[v] names a node of v's component with id <= v
    for (int v = tid; v < n; v += nthr) {
        int m = v;
        for (int e = rp[v]; e < rp[v + 1]; ++e) m = min(m, qcdev::checked_id(ci[e], n, qcdev::DBG_BATCH));
        L[v] = m;
    }
    __syncthreads();
    volatile int32_t *VL = L;
    while (true) {
        for (int v = tid; v < n; v += nthr) {
            int x = VL[v], y = VL[x];
            while (x != y) {
                x = y;
                y = VL[x];
            }
            VL[v] = x;
        }
        __syncthreads();
        bool changed = false;
        for (int v = wid; v < n; v += nw) {
            const int a = VL[v];
            for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
                const int b = VL[qcdev::checked_id(ci[e], n, qcdev::DBG_BATCH)];
                if (b < a) {
                    if (atomicMin(L + a, b) > b) changed = true;
                } else if (G.directed && a < b) {
                    if (atomicMin(L + b, a) > a) changed = true;
                }
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    for (int k = tid; k < W; k += nthr) {
        const int s0 = 64 * k, cnt = min(64, n - s0), c0 = L[s0];
        bool same = true;
        for (int b = 1; b < cnt && same; ++b) same = L[s0 + b] == c0;
        wc[k] = same ? c0 : -1;
    }
    for (int v = tid; v < n; v += nthr) {
        hist[v] = 1;
        hist[n + v] = rp[v + 1] - rp[v];
    }
    __syncthreads();

    // 2. BFS, chunk by chunk
    const bool sparse = (long long)rp[n] < (long long)P.sparse_degree * n;   // short rows: a thread per node
    int rows_ready = 2;       // hist rows zeroed / written so far
    int D = (rp[n] > 0) ? 1 : 0;
    bool overflow = false;
    for (int c0 = 0; c0 < W && rp[n] > 0 && !overflow; c0 += P.c) {
        const int cw = min(P.c, W - c0);
        // level 1 in colA: preset bits, then v and its neighbours
        for (int i = tid; i < n * cw; i += nthr) {
            const int v = i / cw, k = i - v * cw;
            colA[(size_t)v * P.c + k] = cta_preset(n, c0 + k, L[v], L, wc);
        }
        __syncthreads();
        for (int v = wid; v < n; v += nw) {
            const int beg = rp[v], end = rp[v + 1];
            for (int e = beg + lane; e <= end; e += 32) {
                const int u = (e == end) ? v : qcdev::checked_id(ci[e], n, qcdev::DBG_BATCH);
                const int k = (u >> 6) - c0;
                if (k >= 0 && k < cw)
                    atomicOr((unsigned long long *)&colA[(size_t)v * P.c + k], 1ull << (u & 63));
            }
        }
        __syncthreads();
        for (int level = 2;; ++level) {
            if (level >= L_CAP) {
                overflow = true;
                break;
            }
            if (level >= rows_ready) {
                for (int v = tid; v < n; v += nthr) hist[(size_t)level * n + v] = 0;
                rows_ready = level + 1;
                __syncthreads();
            }
            const uint64_t *in = (level & 1) ? colB : colA;
            uint64_t *out = (level & 1) ? colA : colB;
            bool any_new = false;
            if (sparse) {
                // one thread per node: no cross-lane reductions for short rows
                for (int v = tid; v < n; v += nthr) {
                    uint64_t own[MAXC], acc[MAXC];
                    bool full = true;
#pragma unroll
                    for (int k = 0; k < MAXC; ++k) {
                        own[k] = (k < cw) ? in[(size_t)v * P.c + k] : ONES;
                        acc[k] = 0ull;
                        full = full && own[k] == ONES;
                    }
                    if (!full) {
                        for (int e = rp[v]; e < rp[v + 1]; ++e) {
                            const uint64_t *nrow = in + (size_t)qcdev::checked_id(ci[e], n, qcdev::DBG_BATCH) * P.c;
#pragma unroll
                            for (int k = 0; k < MAXC; ++k)
                                if (k < cw) acc[k] |= nrow[k];
                        }
                    }
                    int cnt = 0;
#pragma unroll
                    for (int k = 0; k < MAXC; ++k) {
                        if (k < cw) {
                            const uint64_t nwd = acc[k] & ~own[k];
                            out[(size_t)v * P.c + k] = own[k] | nwd;
                            cnt += __popcll(nwd);
                        }
                    }
                    if (cnt) {
                        hist[(size_t)level * n + v] += cnt;
                        any_new = true;
                    }
                }
            } else
            for (int v = wid; v < n; v += nw) {
                uint64_t own[MAXC], acc[MAXC];
                bool full = true;
#pragma unroll
                for (int k = 0; k < MAXC; ++k) {
                    own[k] = (k < cw) ? in[(size_t)v * P.c + k] : ONES;
                    acc[k] = 0ull;
                    full = full && own[k] == ONES;
                }
                if (!full) {
                    const int beg = rp[v], end = rp[v + 1];
                    for (int e = beg + lane; e < end; e += 32) {
                        const uint64_t *nrow = in + (size_t)qcdev::checked_id(ci[e], n, qcdev::DBG_BATCH) * P.c;
#pragma unroll
                        for (int k = 0; k < MAXC; ++k)
                            if (k < cw) acc[k] |= nrow[k];
                    }
#pragma unroll
                    for (int k = 0; k < MAXC; ++k)
                        if (k < cw) acc[k] = or_reduce64(acc[k]);
                }
                int cnt = 0;
#pragma unroll
                for (int k = 0; k < MAXC; ++k) {
                    if (k < cw) {
                        const uint64_t nwd = acc[k] & ~own[k];
                        if (lane == k) out[(size_t)v * P.c + k] = own[k] | nwd;
                        cnt += __popcll(nwd);
                    }
                }
                if (lane == 0 && cnt) {
                    hist[(size_t)level * n + v] += cnt;
                    any_new = true;
                }
            }
            if (!__syncthreads_or(any_new)) {
                D = max(D, level - 1);
                break;
            }
        }
    }
    if (overflow) {
        if (tid == 0) {
            P.overflow[g] = 1;
            P.overflow[P.n_graphs] = 1;
        }
        __syncthreads();
        return;
    }

    // 3. potential (keys of non-negative doubles order like the doubles)
    long long *key = reinterpret_cast<long long *>(colA);
    int32_t *parent = reinterpret_cast<int32_t *>(colB);
    const double *w = P.tables + (size_t)g * 2 * L_CAP;
    const double *u = w + L_CAP;
    for (int v = tid; v < n; v += nthr) {
        double s1 = 0.0, s2 = 0.0;
        for (int d = 0; d <= D; ++d) {
            const int h = hist[(size_t)d * n + v];
            if (h == 0) continue;
            s1 = __dadd_rn(s1, __dmul_rn((double)h, u[d]));
            s2 = __dadd_rn(s2, __dmul_rn((double)h, w[d]));
        }
        key[v] = __double_as_longlong(__ddiv_rn(__ddiv_rn(s1, s2), G.den));
    }
    __syncthreads();
    // 4. descent and roots
    if (sparse) {
        for (int v = tid; v < n; v += nthr) {
            long long bk = 0;
            int best = -1;
            for (int e = rp[v]; e < rp[v + 1]; ++e) {
                const int x = qcdev::checked_id(ci[e], n, qcdev::DBG_BATCH);
                const long long k = key[x];
                if (best < 0 || k < bk || (k == bk && x < best)) {
                    bk = k;
                    best = x;
                }
            }
            parent[v] = (best >= 0 && bk < key[v]) ? best : v;
        }
    } else
    for (int v = wid; v < n; v += nw) {
        long long bk = 0;
        int best = -1;
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const int x = qcdev::checked_id(ci[e], n, qcdev::DBG_BATCH);
            const long long k = key[x];
            if (best < 0 || k < bk || (k == bk && x < best)) {
                bk = k;
                best = x;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const long long ok = __shfl_xor_sync(FULL, bk, off);
            const int ob = __shfl_xor_sync(FULL, best, off);
            if (ob >= 0 && (best < 0 || ok < bk || (ok == bk && ob < best))) {
                bk = ok;
                best = ob;
            }
        }
        if (lane == 0) parent[v] = (best >= 0 && bk < key[v]) ? best : v;
    }
    __syncthreads();
    volatile int32_t *P_ = parent;
    int roots = 0;
    for (int v = tid; v < n; v += nthr) {
        int x = v;
        while (true) {
            const int px = P_[x];
            if (px == x) break;
            const int gx = P_[px];
            if (gx != px) P_[x] = gx;
            x = gx;
        }
        G.labels[v] = x;
        roots += (x == v);
    }
    roots = __reduce_add_sync(FULL, roots);
    if (tid == 0) s_flag = 0;
    __syncthreads();
    if (lane == 0 && roots) atomicAdd(&s_flag, roots);
    __syncthreads();
    if (tid == 0) P.n_clusters[g] = s_flag;
    __syncthreads();
}

__global__ void batch_kernel(const CtaParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int pos;
    while (true) {
        if (threadIdx.x == 0) pos = atomicAdd(P.queue, 1);
        __syncthreads();
        const int i = pos;
        __syncthreads();
        if (i >= P.n_graphs) break;
        solve_graph(P, P.order[i], smem);
    }
}

size_t smem_bytes(int n_max, int c) {
    const int W = (n_max + 63) / 64;
    return 16 * (((size_t)4 * (n_max + W) + 15) / 16) + 2 * 8 * (size_t)n_max * c;
}

}  // namespace

struct qc_batch {
    qc_ctx *ctx = nullptr;
    int32_t n_graphs = 0;
    std::vector<qc_graph *> graphs;
    std::vector<double> sigmas;
    int32_t *labels = nullptr;
    std::vector<int64_t> offsets;
    std::vector<int32_t> big;        // graphs that take the single-graph path
    int32_t n_cta = 0;               // graphs in the batched kernel
    qc_buffer descs, order, tables, hist, counts, flags, queue;
    int threads = 256, c = 1, grid = 1, sparse_degree = SPARSE_DEGREE;
    size_t smem = 0;
    int32_t n_max = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int32_t> cta_index;  // batch index of each kernel graph
    ~qc_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) {
            cudaStreamSynchronize(cap_stream);
            qc_stream_release(ctx, cap_stream, 0);
        }
    }
};

static qc_status batch_enqueue(qc_batch *b, cudaStream_t s, int threads, int c, int sparse_degree) {
    qc_ctx *ctx = b->ctx;
    const size_t smem = smem_bytes(b->n_max, c);
    QC_CUDA_TRY(ctx, cudaFuncSetAttribute((const void *)batch_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)batch_kernel,
                                                                   threads, smem));
    if (per_sm < 1) return QC_ERR_INVALID_ARG;
    int grid = per_sm * ctx->num_sms;
    if (grid > b->n_cta) grid = b->n_cta;
    if (grid > b->grid) grid = b->grid;         // hist scratch is sized for b->grid CTAs
    CtaParams P;
    P.graphs = b->descs.as<CtaGraph>();
    P.order = b->order.as<int32_t>();
    P.n_graphs = b->n_cta;
    P.queue = b->queue.as<int32_t>();
    P.tables = b->tables.as<double>();
    P.n_max = b->n_max;
    P.c = c;
    P.sparse_degree = sparse_degree;
    P.hist = b->hist.as<int32_t>();
    P.n_clusters = b->counts.as<int32_t>();
    P.overflow = b->flags.as<int32_t>();
    QC_CUDA_TRY(ctx, cudaMemsetAsync(b->queue.ptr, 0, sizeof(int32_t), s));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(b->flags.ptr, 0, b->flags.bytes, s));
    batch_kernel<<<grid, threads, smem, s>>>(P);
    QC_LAUNCHED(ctx);
    return QC_OK;
}

// ---- one-shot launch for the serving loop (no plan, no capture) --------------------

struct qc_cta_launch {
    qc_buffer descs, order, tables, hist, counts, flags, queue;
    int32_t m = 0;
};

int32_t qc_cta_max_nodes() { return CTA_MAX_N; }

size_t qc_cta_bytes_per_node() { return sizeof(int32_t) * L_CAP; }

// Enqueue the batched kernel for m graphs (each n <= qc_cta_max_nodes()) on
// `stream`.  labels[i]: device int32[n_i].  The returned record owns the
// launch's device buffers; keep it until the stream has passed the launch.
// Per graph, counts[i] and flags[i] (1 = needs the single-graph path) are in
// L->counts / L->flags.  max_sms caps the SMs' worth of CTAs the launch may
// fill (0 = all).
qc_status qc_cta_launch_async(qc_ctx *ctx, int32_t m, qc_graph *const *graphs, const double *sigmas,
                              int32_t *const *labels, int max_sms, cudaStream_t stream, qc_cta_launch **out) {
    auto *L = new qc_cta_launch();
    std::unique_ptr<qc_cta_launch> guard(L);
    L->m = m;
    int32_t n_max = 1;
    std::vector<CtaGraph> d(m);
    std::vector<double> tab((size_t)m * 2 * L_CAP);
    for (int32_t i = 0; i < m; ++i) {
        qc_graph *g = graphs[i];
        n_max = std::max(n_max, g->n);
        d[i].row_ptr = g->row_ptr.as<int32_t>();
        d[i].col_idx = g->col_idx.as<int32_t>();
        d[i].labels = labels[i];
        d[i].n = g->n;
        d[i].directed = g->directed ? 1 : 0;
        d[i].den = 2.0 * (sigmas[i] * sigmas[i]);
        qc_weight_table(sigmas[i], L_CAP, tab.data() + (size_t)i * 2 * L_CAP,
                        tab.data() + (size_t)i * 2 * L_CAP + L_CAP);
    }
    std::vector<int32_t> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return d[a].n > d[b].n; });
    int c = 1;
    while (c < MAXC && smem_bytes(n_max, 2 * c) + 1024 <= 100 * 1024 && c < (n_max + 63) / 64) c *= 2;
    const size_t smem = smem_bytes(n_max, c);
    QC_CUDA_TRY(ctx, cudaFuncSetAttribute((const void *)batch_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)batch_kernel, 256, smem));
    const int sms = (max_sms > 0 && max_sms < ctx->num_sms) ? max_sms : ctx->num_sms;
    int grid = std::max(1, std::min(per_sm * sms, m));
    QC_TRY(L->descs.allocate(ctx, sizeof(CtaGraph) * m, stream));
    QC_TRY(L->tables.allocate(ctx, sizeof(double) * tab.size(), stream));
    QC_TRY(L->order.allocate(ctx, sizeof(int32_t) * m, stream));
    QC_TRY(L->counts.allocate(ctx, sizeof(int32_t) * m, stream));
    QC_TRY(L->flags.allocate(ctx, sizeof(int32_t) * (m + 1), stream));
    QC_TRY(L->queue.allocate(ctx, sizeof(int32_t), stream));
    QC_TRY(L->hist.allocate(ctx, sizeof(int32_t) * (size_t)grid * L_CAP * n_max, stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(L->descs.ptr, d.data(), L->descs.bytes, cudaMemcpyHostToDevice, stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(L->tables.ptr, tab.data(), L->tables.bytes, cudaMemcpyHostToDevice, stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(L->order.ptr, ord.data(), L->order.bytes, cudaMemcpyHostToDevice, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(L->queue.ptr, 0, sizeof(int32_t), stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(L->flags.ptr, 0, L->flags.bytes, stream));
    // the host vectors above are pageable: these copies complete before returning
    CtaParams P;
    P.graphs = L->descs.as<CtaGraph>();
    P.order = L->order.as<int32_t>();
    P.n_graphs = m;
    P.queue = L->queue.as<int32_t>();
    P.tables = L->tables.as<double>();
    P.n_max = n_max;
    P.c = c;
    P.sparse_degree = SPARSE_DEGREE;
    P.hist = L->hist.as<int32_t>();
    P.n_clusters = L->counts.as<int32_t>();
    P.overflow = L->flags.as<int32_t>();
    batch_kernel<<<grid, 256, smem, stream>>>(P);
    QC_LAUNCHED(ctx);
    *out = guard.release();
    return QC_OK;
}

void qc_cta_launch_free(qc_cta_launch *L) { delete L; }
int32_t *qc_cta_counts(qc_cta_launch *L) { return L->counts.as<int32_t>(); }
int32_t *qc_cta_flags(qc_cta_launch *L) { return L->flags.as<int32_t>(); }

extern "C" {

qc_status qc_batch_create(qc_ctx *ctx, int32_t n_graphs, qc_graph *const *graphs,
                          const double *sigma_per_graph, int32_t *labels_out,
                          const int64_t *label_offsets, void *stream_, qc_batch **out) {
    if (!ctx || !out || n_graphs < 1 || !graphs || !sigma_per_graph || !labels_out || !label_offsets)
        return QC_ERR_INVALID_ARG;
    *out = nullptr;
    for (int32_t k = 0; k < n_graphs; ++k) {
        if (!graphs[k] || graphs[k]->ctx != ctx || label_offsets[k] < 0) {
            qc_set_error(ctx, "qc_batch_create: graph %d is null, from another context, or has a "
                              "negative label offset", k);
            return QC_ERR_INVALID_ARG;
        }
        if (!qc_sigma_ok(sigma_per_graph[k])) {
            qc_set_error(ctx, "qc_batch_create: sigma[%d] = %g is not finite and > 0", k,
                         sigma_per_graph[k]);
            return QC_ERR_INVALID_ARG;
        }
    }
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    auto *b = new qc_batch();
    std::unique_ptr<qc_batch> guard(b);
    b->ctx = ctx;
    b->n_graphs = n_graphs;
    b->graphs.assign(graphs, graphs + n_graphs);
    b->sigmas.assign(sigma_per_graph, sigma_per_graph + n_graphs);
    b->labels = labels_out;
    b->offsets.assign(label_offsets, label_offsets + n_graphs);
    int64_t sum_nnz = 0, sum_n = 0;
    for (int32_t k = 0; k < n_graphs; ++k) {
        if (graphs[k]->n > CTA_MAX_N) {
            b->big.push_back(k);
            continue;
        }
        b->cta_index.push_back(k);
        b->n_max = std::max(b->n_max, graphs[k]->n);
        sum_nnz += graphs[k]->nnz;
        sum_n += graphs[k]->n;
    }
    b->n_cta = (int32_t)b->cta_index.size();
    if (b->n_cta > 0) {
        const int32_t m = b->n_cta;
        // descriptors, weights, work order (largest estimated work first)
        std::vector<CtaGraph> d(m);
        std::vector<double> tab((size_t)m * 2 * L_CAP);
        std::vector<double> cost(m);
        for (int32_t i = 0; i < m; ++i) {
            const int32_t k = b->cta_index[i];
            qc_graph *g = graphs[k];
            d[i].row_ptr = g->row_ptr.as<int32_t>();
            d[i].col_idx = g->col_idx.as<int32_t>();
            d[i].labels = labels_out + label_offsets[k];
            d[i].n = g->n;
            d[i].directed = g->directed ? 1 : 0;
            const double s = sigma_per_graph[k];
            d[i].den = 2.0 * (s * s);
            qc_weight_table(s, L_CAP, tab.data() + (size_t)i * 2 * L_CAP,
                            tab.data() + (size_t)i * 2 * L_CAP + L_CAP);
            cost[i] = (double)((g->n + 63) / 64) * (double)(g->nnz + g->n);
        }
        std::vector<int32_t> ord(m);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t c) { return cost[a] > cost[c]; });
        QC_TRY(b->descs.allocate(ctx, sizeof(CtaGraph) * m, stream));
        QC_TRY(b->tables.allocate(ctx, sizeof(double) * tab.size(), stream));
        QC_TRY(b->order.allocate(ctx, sizeof(int32_t) * m, stream));
        QC_TRY(b->counts.allocate(ctx, sizeof(int32_t) * m, stream));
        QC_TRY(b->flags.allocate(ctx, sizeof(int32_t) * (m + 1), stream));
        QC_TRY(b->queue.allocate(ctx, sizeof(int32_t), stream));
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(b->descs.ptr, d.data(), b->descs.bytes, cudaMemcpyHostToDevice, stream));
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(b->tables.ptr, tab.data(), b->tables.bytes, cudaMemcpyHostToDevice,
                                         stream));
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(b->order.ptr, ord.data(), b->order.bytes, cudaMemcpyHostToDevice,
                                         stream));
        QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));   // host vectors go out of scope
        // histogram scratch for the most CTAs any candidate runs
        b->grid = 4 * ctx->num_sms;
        if (b->grid > m) b->grid = m;
        QC_TRY(b->hist.allocate(ctx, sizeof(int32_t) * (size_t)b->grid * L_CAP * b->n_max, stream));

        // autotune: candidates (threads, chunk words) that fit the shared memory
        const double mean_deg = sum_n ? (double)sum_nnz / (double)sum_n : 0.0;
        qc_tune_key key{1, (int)std::ceil(std::log2((double)b->n_max + 1)),
                        (int)std::floor(std::log2(mean_deg + 1.0))};
        int choice = -1;
        {
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            auto it = ctx->tune.find(key);
            if (it != ctx->tune.end()) choice = it->second;
        }
        const int W_max = (b->n_max + 63) / 64;
        std::vector<std::pair<int, int>> cands;
        for (int threads : {256, 512})
            for (int c : {1, 2, 4, 8}) {
                if (c > 1 && c / 2 >= W_max) continue;   // a wider chunk than any graph needs
                if (smem_bytes(b->n_max, c) + 1024 > ctx->smem_optin) continue;
                cands.push_back({threads, c});
            }
        if (cands.empty()) {
            qc_set_error(ctx, "qc_batch_create: no kernel configuration fits n = %d", b->n_max);
            return QC_ERR_INVALID_ARG;
        }
        // a choice is stored as shape index + 16 x threshold index
        const int n_sd = (int)(sizeof(SPARSE_CANDIDATES) / sizeof(SPARSE_CANDIDATES[0]));
        // QCGRAPH_BATCH_CONFIG="threads,chunk_words[,sparse_degree]" fixes the choice when
        // it names candidates (reproducible profiling), else the autotuner decides
        if (const char *env = getenv("QCGRAPH_BATCH_CONFIG")) {
            int t = 0, c = 0, sd = SPARSE_DEGREE;
            const int got = sscanf(env, "%d,%d,%d", &t, &c, &sd);
            int sdi = -1;
            for (int j = 0; j < n_sd; ++j)
                if (SPARSE_CANDIDATES[j] == sd) sdi = j;
            if (got >= 2 && sdi >= 0)
                for (size_t i = 0; i < cands.size(); ++i)
                    if (cands[i].first == t && cands[i].second == c) choice = (int)i + 16 * sdi;
        }
        if (choice < 0 || choice % 16 >= (int)cands.size() || choice / 16 >= n_sd) {
            // first the tile shape at the default threshold, then the threshold for that shape
            qc_event_pair ev;
            QC_TRY(ev.create(ctx));
            auto time_one = [&](int t, int c, int sd, float *ms) -> qc_status {
                *ms = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {       // first run warms up
                    QC_CUDA_TRY(ctx, cudaEventRecord(ev.a, stream));
                    if (batch_enqueue(b, stream, t, c, sd) != QC_OK) {
                        *ms = 1e30f;
                        return QC_OK;
                    }
                    QC_CUDA_TRY(ctx, cudaEventRecord(ev.b, stream));
                    QC_CUDA_TRY(ctx, cudaEventSynchronize(ev.b));
                    QC_CUDA_TRY(ctx, cudaEventElapsedTime(ms, ev.a, ev.b));
                }
                return QC_OK;
            };
            int default_sdi = 0;
            for (int j = 0; j < n_sd; ++j)
                if (SPARSE_CANDIDATES[j] == SPARSE_DEGREE) default_sdi = j;
            float best = 1e30f;
            int shape = 0;
            for (size_t i = 0; i < cands.size(); ++i) {
                float ms = 0.f;
                QC_TRY(time_one(cands[i].first, cands[i].second, SPARSE_DEGREE, &ms));
                if (ms < best) {
                    best = ms;
                    shape = (int)i;
                }
            }
            int sdi = default_sdi;
            for (int j = 0; j < n_sd; ++j) {
                if (j == default_sdi) continue;
                float ms = 0.f;
                QC_TRY(time_one(cands[shape].first, cands[shape].second, SPARSE_CANDIDATES[j], &ms));
                if (ms < best) {
                    best = ms;
                    sdi = j;
                }
            }
            choice = shape + 16 * sdi;
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            ctx->tune[key] = choice;
        }
        b->threads = cands[choice % 16].first;
        b->c = cands[choice % 16].second;
        b->sparse_degree = SPARSE_CANDIDATES[choice / 16];
        // capture the batched solve
        QC_CUDA_TRY(ctx, qc_stream_acquire(ctx, 0, &b->cap_stream));
        QC_CUDA_TRY(ctx, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        qc_status st = batch_enqueue(b, b->cap_stream, b->threads, b->c, b->sparse_degree);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (st != QC_OK) return st;
        QC_CUDA_TRY(ctx, e);
        b->graph = graph;
        QC_CUDA_TRY(ctx, cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    *out = guard.release();
    return QC_OK;
}

qc_status qc_batch_run(qc_batch *b, int32_t *n_clusters_out, void *stream_) {
    qc_range range("qc.batch_run");
    if (!b) return QC_ERR_INVALID_ARG;
    qc_ctx *ctx = b->ctx;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h = static_cast<int32_t *>(pin.ptr);
    std::vector<int32_t> redo(b->big);
    if (b->n_cta > 0) {
        QC_CUDA_TRY(ctx, cudaGraphLaunch(b->exec, stream));
        QC_LAUNCHED(ctx);
        // any graph that ran out of histogram rows?
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, b->flags.as<int32_t>() + b->n_cta, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, stream));
        QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        QC_TRY(qc_debug_take(ctx));
        if (h[0]) {
            std::vector<int32_t> f(b->n_cta);
            QC_CUDA_TRY(ctx, cudaMemcpy(f.data(), b->flags.ptr, sizeof(int32_t) * b->n_cta,
                                        cudaMemcpyDeviceToHost));
            for (int32_t i = 0; i < b->n_cta; ++i)
                if (f[i]) redo.push_back(b->cta_index[i]);
        }
        if (n_clusters_out) {
            std::vector<int32_t> cnt(b->n_cta);
            QC_CUDA_TRY(ctx, cudaMemcpyAsync(cnt.data(), b->counts.ptr, sizeof(int32_t) * b->n_cta,
                                             cudaMemcpyDeviceToHost, stream));
            QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
            for (int32_t i = 0; i < b->n_cta; ++i) n_clusters_out[b->cta_index[i]] = cnt[i];
        }
    }
    // graphs the batched kernel does not take: the single-graph path, one by one
    for (int32_t k : redo) {
        int32_t nc = 0;
        QC_TRY(qc_solve(b->graphs[k], &b->sigmas[k], 1, nullptr, b->labels + b->offsets[k],
                        n_clusters_out ? &nc : nullptr, stream_));
        if (n_clusters_out) n_clusters_out[k] = nc;
    }
    return QC_OK;
}

void qc_batch_destroy(qc_batch *b) { delete b; }

qc_status qc_batch_config(const qc_batch *b, int32_t *threads, int32_t *chunk_words, int32_t *sparse_degree) {
    if (!b || !threads || !chunk_words) return QC_ERR_INVALID_ARG;
    *threads = b->n_cta > 0 ? b->threads : 0;
    *chunk_words = b->n_cta > 0 ? b->c : 0;
    if (sparse_degree) *sparse_degree = b->n_cta > 0 ? b->sparse_degree : 0;
    return QC_OK;
}

qc_status qc_solve_batch(qc_ctx *ctx, int32_t n_graphs, qc_graph *const *graphs,
                         const double *sigma_per_graph, int32_t *labels_out,
                         const int64_t *label_offsets, void *stream) {
    qc_batch *b = nullptr;
    QC_TRY(qc_batch_create(ctx, n_graphs, graphs, sigma_per_graph, labels_out, label_offsets, stream, &b));
    qc_status st = qc_batch_run(b, nullptr, stream);
    qc_batch_destroy(b);
    return st;
}

}  // extern "C"
