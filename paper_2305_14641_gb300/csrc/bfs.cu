// All-source hop-distance BFS on 64-source bitsets, fused with the per-node
// distance histogram.
//
// Method: Algorithm 1 needs, for every node i, the multiset of hop distances
// {dist(i, j)} (Section 3.1, hop reading).  In an undirected graph
// dist(s, v) = dist(v, s), so running a BFS from every source s and counting, at
// node v, how many sources reach v at level d gives v's own histogram h_v(d)
// without any cross-node reduction.
//
// Layout: sources are packed 64 to a uint64 word; the BFS handles a chunk of
// `wn` consecutive words (64*wn sources) at a time.  vis[v] is a row of
// `stride` words (stride even, so a row is whole 16-byte segments) holding the
// sources already known to be within the current level of v.  Two rows per node
// (vis_in, vis_out) ping-pong between levels.
//
// Level step (pull): a source s first reaches v at level l+1 exactly when s is
// within level l of some neighbour u and not within level l of v:
//     next[v] = (OR_{u in N(v)} vis_l[u]) & ~vis_l[v],   vis_{l+1}[v] = vis_l[v] | next[v]
//     hist[l+1][v] += popcount(next[v])
// Bits of sources >= n (the tail of the last word) and the padding word of an
// odd-length row start set, so they never count and a row that has met every
// source reads as all ones ("saturated").  A saturated row never changes again:
// sat[v] records the level at which v's row saturated and later levels skip v
// without touching its row.
#include <cstdlib>
#include <cstring>

#include "qc_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t ONES = ~0ull;
constexpr int NOT_SAT = 0x7fffffff;

struct LevelArgs {
    int32_t n;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const ulonglong2 *vis_in;   // [n][R]
    ulonglong2 *vis_out;        // [n][R]
    int32_t R;                  // 16-byte segments per row (= stride / 2)
    int32_t *sat;               // [n] level at which the row saturated, NOT_SAT if not yet
    int32_t level;              // the level being produced (>= 2)
    int32_t *hist_row;          // hist[level][*]
    int32_t *level_new;         // set to 1 when any node gained a source at this level
};

__device__ __forceinline__ bool seg_full(ulonglong2 a) { return (a.x & a.y) == ONES; }

// One warp per node (grid-stride).  Lanes are split into 32/G neighbour slots of
// G lanes; lane (slot, q) reads segment q + k*G (k < SPL) of every neighbour the
// slot takes.  G = 32 for rows of 32 segments or more (one neighbour at a time,
// each lane SPL segments); smaller rows read 32/G neighbours at once.
template <int G, int SPL>
__global__ void __launch_bounds__(256, (SPL >= 8 ? 1 : (SPL >= 4 ? 2 : 4))) bfs_pull_level(const LevelArgs a) {
    constexpr int SLOTS = 32 / G;
    const int lane = threadIdx.x & 31;
    const int slot = lane / G;
    const int q0 = lane % G;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    bool any_new = false;
    for (int v = warp; v < a.n; v += nwarps) {
        const int sv = a.sat[v];
        if (sv <= a.level - 2) continue;                 // saturated in both buffers
        ulonglong2 *out_row = a.vis_out + (size_t)v * a.R;
        if (sv == a.level - 1) {                          // saturated last level: copy ones
            if (slot == 0) {
#pragma unroll
                for (int k = 0; k < SPL; ++k) {
                    const int q = q0 + k * G;
                    if (q < a.R) out_row[q] = make_ulonglong2(ONES, ONES);
                }
            }
            continue;
        }
        const ulonglong2 *in_row = a.vis_in + (size_t)v * a.R;
        ulonglong2 own[SPL], acc[SPL];
        bool act[SPL];
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            const int q = q0 + k * G;
            own[k] = (q < a.R) ? in_row[q] : make_ulonglong2(ONES, ONES);
            acc[k] = make_ulonglong2(0, 0);
            act[k] = !seg_full(own[k]);
        }
        const int beg = a.row_ptr[v], end = a.row_ptr[v + 1];
        for (int j0 = beg; j0 < end; j0 += 32) {
            const int cnt = min(32, end - j0);
            const int myu = (lane < cnt) ? a.col_idx[j0 + lane] : 0;
            const int rounds = (cnt + SLOTS - 1) / SLOTS;
            for (int m = 0; m < rounds; ++m) {
                const int t = m * SLOTS + slot;
                const int u = __shfl_sync(FULL, myu, t < 32 ? t : 31);
                if (t < cnt) {
                    const ulonglong2 *nrow = a.vis_in + (size_t)u * a.R;
#pragma unroll
                    for (int k = 0; k < SPL; ++k) {
                        const int q = q0 + k * G;
                        if (act[k] && q < a.R) {
                            const ulonglong2 x = nrow[q];
                            acc[k].x |= x.x;
                            acc[k].y |= x.y;
                        }
                    }
                }
            }
            // stop once every segment of this slot has found all its missing sources
            bool more = false;
#pragma unroll
            for (int k = 0; k < SPL; ++k) {
                act[k] = act[k] && !seg_full(make_ulonglong2(acc[k].x | own[k].x, acc[k].y | own[k].y));
                more |= act[k];
            }
            if (!__any_sync(FULL, more)) break;
        }
        // combine the slots' partial ORs
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
#pragma unroll
            for (int off = G; off < 32; off <<= 1) {
                acc[k].x |= __shfl_xor_sync(FULL, acc[k].x, off);
                acc[k].y |= __shfl_xor_sync(FULL, acc[k].y, off);
            }
        }
        int count = 0;
        bool full = true;
        if (slot == 0) {
#pragma unroll
            for (int k = 0; k < SPL; ++k) {
                const int q = q0 + k * G;
                if (q < a.R) {
                    const ulonglong2 nw = make_ulonglong2(acc[k].x & ~own[k].x, acc[k].y & ~own[k].y);
                    const ulonglong2 o = make_ulonglong2(own[k].x | nw.x, own[k].y | nw.y);
                    out_row[q] = o;
                    count += __popcll(nw.x) + __popcll(nw.y);
                    full = full && seg_full(o);
                }
            }
        }
        count = __reduce_add_sync(FULL, count);
        full = __all_sync(FULL, full);
        if (lane == 0) {
            if (count) {
                a.hist_row[v] += count;
                any_new = true;
            }
            if (full) a.sat[v] = a.level;
        }
    }
    if (__syncthreads_or(any_new) && threadIdx.x == 0) *a.level_new = 1;
}

// Level 1 straight from the CSR: v's row holds v itself and its neighbours that
// fall in the chunk, plus the always-set bits (sources >= n, padding word).
// One thread per node; only that thread touches the row.
__global__ void bfs_init_chunk(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                               int32_t w0, int32_t wn, int32_t stride, int32_t last_word,
                               uint64_t last_mask, uint64_t *vis, int32_t *sat) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t *row = vis + (size_t)v * stride;
        for (int k = 0; k < stride; ++k) row[k] = (k < wn) ? 0ull : ONES;
        if (last_word >= w0 && last_word < w0 + wn) row[last_word - w0] |= last_mask;
        int k = (v >> 6) - w0;
        if (k >= 0 && k < wn) row[k] |= 1ull << (v & 63);
        for (int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const int u = col_idx[e];
            k = (u >> 6) - w0;
            if (k >= 0 && k < wn) row[k] |= 1ull << (u & 63);
        }
        bool full = true;
        for (int q = 0; q < stride; ++q) full = full && (row[q] == ONES);
        sat[v] = full ? 1 : NOT_SAT;
    }
}

// hist[0][v] = 1 (v itself), hist[1][v] = deg(v).
__global__ void bfs_hist_first_rows(int32_t n, const int32_t *row_ptr, int32_t *hist) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        hist[v] = 1;
        hist[(size_t)n + v] = row_ptr[v + 1] - row_ptr[v];
    }
}

typedef void (*pull_fn)(const LevelArgs);

pull_fn pick_pull(int R, int *G_out) {
    if (R <= 1) { *G_out = 1; return bfs_pull_level<1, 1>; }
    if (R <= 2) { *G_out = 2; return bfs_pull_level<2, 1>; }
    if (R <= 4) { *G_out = 4; return bfs_pull_level<4, 1>; }
    if (R <= 8) { *G_out = 8; return bfs_pull_level<8, 1>; }
    if (R <= 16) { *G_out = 16; return bfs_pull_level<16, 1>; }
    *G_out = 32;
    if (R <= 32) return bfs_pull_level<32, 1>;
    if (R <= 64) return bfs_pull_level<32, 2>;
    if (R <= 128) return bfs_pull_level<32, 4>;
    return bfs_pull_level<32, 8>;
}

// Grow hist to hold at least `rows` levels (new rows zeroed), keeping the old rows.
qc_status ensure_hist_rows(qc_graph *g, int32_t rows, cudaStream_t stream) {
    if (rows <= g->hist_rows) return QC_OK;
    int32_t want = g->hist_rows ? g->hist_rows : 16;
    while (want < rows) want *= 2;
    if (want > g->n + 1) want = g->n + 1 > rows ? g->n + 1 : rows;
    qc_buffer nb;
    const size_t row_bytes = sizeof(int32_t) * (size_t)g->n;
    QC_TRY(nb.allocate(g->ctx, row_bytes * (size_t)want, stream));
    QC_CUDA_TRY(g->ctx, cudaMemsetAsync(nb.ptr, 0, nb.bytes, stream));
    if (g->hist_rows)
        QC_CUDA_TRY(g->ctx, cudaMemcpyAsync(nb.ptr, g->hist.ptr, row_bytes * (size_t)g->hist_rows,
                                            cudaMemcpyDeviceToDevice, stream));
    g->hist = std::move(nb);
    g->hist_rows = want;
    return QC_OK;
}

}  // namespace

// Modelled algorithmic bytes of one level launch over a chunk of wn source words
// (pull over every node): per node and word, gather the row word of each
// neighbour, read the node's own word and write it back, plus one write of the
// next-frontier word (8 wn (E + 3N)); the CSR once (4(N+1) + 4E); one histogram
// row (4N).
static double bfs_level_model_bytes(int64_t n, int64_t nnz, int64_t wn) {
    return 8.0 * (double)wn * (double)(nnz + 3 * n) + 4.0 * (double)(n + 1) + 4.0 * (double)nnz +
           4.0 * (double)n;
}

// Words of sources handled per chunk: as many as keep both bitset buffers within
// about half of L2 (they are re-read once per neighbour per level), at most 512.
// QCGRAPH_CHUNK_WORDS overrides the choice (tests use it to force many chunks).
static int32_t choose_chunk_words(const qc_graph *g) {
    const int64_t W = (g->n + 63) / 64;
    if (const char *env = getenv("QCGRAPH_CHUNK_WORDS")) {
        int64_t forced = atoll(env);
        if (forced >= 1) return (int32_t)(forced < W ? forced : W);
    }
    const size_t target = g->ctx->l2_bytes ? g->ctx->l2_bytes / 2 : (size_t)48 << 20;
    int64_t wc = (int64_t)(target / (2 * 8 * (size_t)g->n));
    if (wc < 2) wc = 2;
    if (wc > 512) wc = 512;
    if (wc > W) wc = W;
    return (int32_t)wc;
}

qc_status qc_bfs_histogram(qc_graph *g, cudaStream_t stream) {
    qc_ctx *ctx = g->ctx;
    const int32_t n = g->n;
    const int64_t W = (n + 63) / 64;
    const int32_t wc = choose_chunk_words(g);
    const int32_t R_max = (wc + 1) / 2;
    g->hist_valid = false;
    g->D = g->nnz > 0 ? 1 : 0;
    QC_TRY(ensure_hist_rows(g, 2, stream));
    const int threads = 256;
    const int node_blocks = qc_ceil_div(n, threads) < 4 * ctx->num_sms ? qc_ceil_div(n, threads)
                                                                         : 4 * ctx->num_sms;
    bfs_hist_first_rows<<<node_blocks, threads, 0, stream>>>(n, g->row_ptr.as<int32_t>(),
                                                           g->hist.as<int32_t>());
    QC_LAUNCHED(ctx);
    if (g->nnz == 0) {
        g->hist_valid = true;
        return QC_OK;
    }
    qc_buffer visA, visB, sat, flags;
    const size_t vis_bytes = sizeof(ulonglong2) * (size_t)R_max * (size_t)n;
    QC_TRY(visA.allocate(ctx, vis_bytes, stream));
    QC_TRY(visB.allocate(ctx, vis_bytes, stream));
    QC_TRY(sat.allocate(ctx, sizeof(int32_t) * (size_t)n, stream));
    const int32_t max_levels = n + 2;
    QC_TRY(flags.allocate(ctx, sizeof(int32_t) * (size_t)max_levels, stream));
    int32_t *h_flag = nullptr;
    QC_CUDA_TRY(ctx, cudaMallocHost(&h_flag, sizeof(int32_t)));
    struct PinnedGuard { int32_t *p; ~PinnedGuard() { cudaFreeHost(p); } } guard{h_flag};

    const bool timing = ctx->timing.load();
    cudaEvent_t ev[2] = {nullptr, nullptr};
    struct EventGuard {
        cudaEvent_t *e;
        ~EventGuard() { for (int i = 0; i < 2; ++i) if (e[i]) cudaEventDestroy(e[i]); }
    } ev_guard{ev};
    if (timing) {
        QC_CUDA_TRY(ctx, cudaEventCreate(&ev[0]));
        QC_CUDA_TRY(ctx, cudaEventCreate(&ev[1]));
    }
    const int32_t last_word = (int32_t)(W - 1);
    const uint64_t last_mask = (n % 64) ? (ONES << (n % 64)) : 0ull;
    int dev_blocks_per_sm = 0;
    for (int64_t w0 = 0; w0 < W; w0 += wc) {
        const int32_t wn = (int32_t)((W - w0) < wc ? (W - w0) : wc);
        const int32_t R = (wn + 1) / 2;
        bfs_init_chunk<<<qc_ceil_div(n, 128), 128, 0, stream>>>(
            n, g->row_ptr.as<int32_t>(), g->col_idx.as<int32_t>(), (int32_t)w0, wn, 2 * R,
            last_word, last_mask, visA.as<uint64_t>(), sat.as<int32_t>());
        QC_LAUNCHED(ctx);
        QC_CUDA_TRY(ctx, cudaMemsetAsync(flags.ptr, 0, flags.bytes, stream));
        int G = 32;
        pull_fn fn = pick_pull(R, &G);
        if (!dev_blocks_per_sm) {
            QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dev_blocks_per_sm,
                                                                           (const void *)fn, 256, 0));
            if (dev_blocks_per_sm < 1) dev_blocks_per_sm = 1;
        }
        const int warps_needed = n;
        int blocks = qc_ceil_div(warps_needed, 8);
        const int cap_blocks = dev_blocks_per_sm * ctx->num_sms;
        if (blocks > cap_blocks) blocks = cap_blocks;
        ulonglong2 *in = visA.as<ulonglong2>(), *out = visB.as<ulonglong2>();
        for (int32_t level = 2; level <= n; ++level) {
            QC_TRY(ensure_hist_rows(g, level + 1, stream));
            LevelArgs a;
            a.n = n;
            a.row_ptr = g->row_ptr.as<int32_t>();
            a.col_idx = g->col_idx.as<int32_t>();
            a.vis_in = in;
            a.vis_out = out;
            a.R = R;
            a.sat = sat.as<int32_t>();
            a.level = level;
            a.hist_row = g->hist.as<int32_t>() + (size_t)level * n;
            a.level_new = flags.as<int32_t>() + level;
            if (timing) QC_CUDA_TRY(ctx, cudaEventRecord(ev[0], stream));
            fn<<<blocks, 256, 0, stream>>>(a);
            QC_LAUNCHED(ctx);
            if (timing) QC_CUDA_TRY(ctx, cudaEventRecord(ev[1], stream));
            QC_CUDA_TRY(ctx, cudaMemcpyAsync(h_flag, a.level_new, sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, stream));
            QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
            if (timing) {
                float ms = 0.f;
                QC_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ev[0], ev[1]));
                qc_record_kernel(ctx, "bfs_level", ms, bfs_level_model_bytes(n, g->nnz, wn));
            }
            if (!*h_flag) break;
            if (level > g->D) g->D = level;
            ulonglong2 *t = in;
            in = out;
            out = t;
        }
    }
    g->hist_valid = true;
    return QC_OK;
}
