// Per-graph preparation, computed once and kept with the graph:
//   comp[v]   connected component of v, as the smallest node id in it;
//   wcomp[k]  the component shared by all valid sources of 64-source word k,
//             or -1 when the word mixes components;
//   wmajor[k], wmask[k]  the component holding most of word k's sources and
//             the bits of those sources;
//   order[i]  nodes by decreasing degree bucket (floor(log2(deg + 1))), so that
//             dealing them round-robin to warps spreads the heavy rows;
//             order[n] = how many lead the order with degree >= 2^QC_HEAVY_BUCKET - 1
//             (the BFS gives those rows to whole blocks);
//   oinfo[i]  {order[i], row start, row end, 0}, so that a BFS item's node and
//             row arrive in one load instead of two dependent ones.
// Sources in another component than v can never reach v: the BFS marks them
// as already seen in v's row from the start, so a row is complete ("all ones")
// as soon as v's own component has reached it.  For a directed graph the
// components are the weakly connected ones: still a bound on reachability, but
// a row may then never complete.
#include <algorithm>

#include "qc_device.cuh"
#include "qc_internal.h"

namespace {

// Union-find over the labels L (a node's label chain ends at its tree's root).
// uf_link is a lock-free union: a root is attached below a smaller root by
// compare-and-swap, so every root is the smallest id of its tree.
__device__ __forceinline__ void uf_link(int32_t *L, int u, int v) {
    volatile int32_t *VL = L;
    int p1 = VL[u], p2 = VL[v];
    while (p1 != p2) {
        const int high = max(p1, p2), low = min(p1, p2);
        const int ph = VL[high];
        if (ph == low) break;
        if (ph == high && atomicCAS(L + high, high, low) == high) break;
        p1 = VL[VL[high]];
        p2 = VL[low];
    }
}

__device__ __forceinline__ void uf_compress(int32_t *L, int n, int tid, int nthreads) {
    volatile int32_t *VL = L;
    for (int v = tid; v < n; v += nthreads) {
        int x = VL[v];
        while (VL[x] != x) x = VL[x];
        VL[v] = x;
    }
}

__device__ __forceinline__ int degree_bucket(int deg) { return 31 - __clz(deg + 1); }

// Per 64-source word: wcomp = the one component of all its sources, or -1; the
// component holding most of them (wmajor) and their bits (wmask), so that the
// BFS presets the row of a node in that component with one mask and walks the
// word bit by bit only for nodes of the word's minor components.
// One warp per word: a vote settles the common case of a word inside one
// component; lane 0 counts the components of a mixed word.
__device__ void word_components(int32_t n, int32_t W, const int32_t *comp, int32_t *wcomp, int32_t *wmajor,
                                unsigned long long *wmask) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k = warp; k < W; k += nwarps) {
        const int s0 = 64 * k;
        const int cnt = min(64, n - s0);
        const int c0 = comp[s0];
        const bool same = (lane >= cnt || comp[s0 + lane] == c0) && (lane + 32 >= cnt || comp[s0 + 32 + lane] == c0);
        const bool whole = __all_sync(0xffffffffu, same);
        if (lane == 0) {
            if (whole) {
                wcomp[k] = c0;
                wmajor[k] = c0;
                wmask[k] = cnt == 64 ? ~0ull : ((1ull << cnt) - 1);
            } else {
                int best = c0, best_count = 0;
                unsigned long long best_mask = 0ull, seen = 0ull;
                for (int b = 0; b < cnt; ++b) {
                    if ((seen >> b) & 1ull) continue;
                    const int c = comp[s0 + b];
                    unsigned long long m = 0ull;
                    for (int b2 = b; b2 < cnt; ++b2)
                        if (comp[s0 + b2] == c) m |= 1ull << b2;
                    seen |= m;
                    const int pc = __popcll(m);
                    if (pc > best_count) {
                        best = c;
                        best_count = pc;
                        best_mask = m;
                    }
                }
                wcomp[k] = -1;
                wmajor[k] = best;
                wmask[k] = best_mask;
            }
        }
        __syncwarp();
    }
}

struct PrepParams {
    int32_t n, W;
    const int32_t *row_ptr, *col_idx;
    int32_t *L;                     // [n] union-find labels (scratch)
    int32_t *ctl;                   // [0] status, [2..3] barrier, [4] largest component, [6..7] sum deg^2
    int32_t directed;
    int32_t *comp, *wcomp, *wmajor;
    unsigned long long *wmask;
    // scattered degree order (null order: another kernel writes it)
    int32_t *bins;                  // [64] zeroed: counts per bucket, then each bucket's next position
    int32_t *order;                 // [n + 1]
    int4 *info;                     // [n]
};

// The whole preparation in one cooperative launch, phases separated by grid
// barriers:
//   A. labels L[v] = v; per-bucket degree counts; the sum of squared degrees;
//   B. every node links to its first two neighbours; the bucket counts become
//      each bucket's first position (heaviest bucket first);
//   C. compression; every node takes a position in its bucket (the scattered order);
//   D. the label shared by most of 64 evenly spaced nodes names the largest
//      component found so far; info[i] for every order position;
//   E. nodes outside that component link to their remaining neighbours (in a
//      directed graph every node links all its arcs);
//   F. comp[v] = the root of v's tree, the smallest id of its component;
//   G. the words' components.
// Components by sampled union-find after Sutton et al., "Optimizing Parallel
// Graph Connectivity Computation via Subgraph Sampling" (2018).
__global__ void __launch_bounds__(256) prep_fused(const PrepParams p) {
    unsigned *bar = reinterpret_cast<unsigned *>(p.ctl + 2);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const int n = p.n;
    __shared__ int32_t local[32];
    __shared__ int s_lab[64], s_cnt[64];
    // A
    if (threadIdx.x < 32) local[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long sq = 0;
    for (int v = tid; v < n; v += nthreads) {
        p.L[v] = v;
        const int d = p.row_ptr[v + 1] - p.row_ptr[v];
        if (p.order) atomicAdd(&local[degree_bucket(d)], 1);
        sq += (unsigned long long)d * (unsigned long long)d;
    }
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
    if ((threadIdx.x & 31) == 0 && sq) atomicAdd(reinterpret_cast<unsigned long long *>(p.ctl + 6), sq);
    __syncthreads();
    if (p.order && threadIdx.x < 32 && local[threadIdx.x]) atomicAdd(&p.bins[threadIdx.x], local[threadIdx.x]);
    if (!qcdev::grid_barrier(bar, p.ctl)) return;
    // B
    for (int v = tid; v < n; v += nthreads) {
        const int beg = p.row_ptr[v], end = p.row_ptr[v + 1];
        for (int e = beg; e < end && e < beg + 2; ++e)
            uf_link(p.L, v, qcdev::checked_id(p.col_idx[e], n, qcdev::DBG_PREP));
    }
    if (p.order && tid == 0) {
        int acc = 0;
        for (int b = 31; b >= 0; --b) {
            p.bins[32 + b] = acc;
            acc += p.bins[b];
            if (b == QC_HEAVY_BUCKET) p.order[n] = acc;
        }
    }
    if (!qcdev::grid_barrier(bar, p.ctl)) return;
    // C
    uf_compress(p.L, n, tid, nthreads);
    if (p.order) {
        // one counter update per bucket and warp (most nodes share a few buckets,
        // and a counter update per node serialised on them)
        const int lane_c = threadIdx.x & 31;
        for (int v0 = tid - lane_c; v0 < n; v0 += nthreads) {
            const int v = v0 + lane_c;
            const int b = v < n ? degree_bucket(p.row_ptr[v + 1] - p.row_ptr[v]) : 32;
            const unsigned same = __match_any_sync(0xffffffffu, b);
            const int leader = __ffs(same) - 1;
            int at = 0;
            if (b < 32 && lane_c == leader) at = atomicAdd(&p.bins[32 + b], __popc(same));
            at = __shfl_sync(0xffffffffu, at, leader);
            if (b < 32) p.order[at + __popc(same & ((1u << lane_c) - 1u))] = v;
        }
    }
    if (!qcdev::grid_barrier(bar, p.ctl)) return;
    // D
    if (blockIdx.x == 0) {
        if (threadIdx.x < 64) s_lab[threadIdx.x] = p.L[(int)(((long long)threadIdx.x * (n - 1)) / 63)];
        __syncthreads();
        if (threadIdx.x < 64) {
            int c = 0;
            for (int i = 0; i < 64; ++i) c += (s_lab[i] == s_lab[threadIdx.x]);
            s_cnt[threadIdx.x] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int best = 0;
            for (int i = 1; i < 64; ++i)
                if (s_cnt[i] > s_cnt[best]) best = i;
            p.ctl[4] = p.directed ? -1 : s_lab[best];
        }
    }
    if (p.order)
        for (int i = tid; i < n; i += nthreads) {
            const int v = p.order[i];
            p.info[i] = make_int4(v, p.row_ptr[v], p.row_ptr[v + 1], 0);
        }
    if (!qcdev::grid_barrier(bar, p.ctl)) return;
    // E: a warp tests 32 consecutive nodes with one load and walks, lanes
    // across the row, the rows of those outside that component (a warp per
    // node, one label load after another, made this the longest phase)
    const int giant = *(volatile int32_t *)(p.ctl + 4);
    const int lane = threadIdx.x & 31;
    for (int v0 = tid - lane; v0 < n; v0 += nthreads) {
        const int vl = v0 + lane;
        unsigned rest = __ballot_sync(0xffffffffu, vl < n && *(volatile int32_t *)(p.L + vl) != giant);
        while (rest) {
            const int v = v0 + __ffs(rest) - 1;
            rest &= rest - 1;
            const int end = p.row_ptr[v + 1];
            for (int e = p.row_ptr[v] + 2 + lane; e < end; e += 32)
                uf_link(p.L, v, qcdev::checked_id(p.col_idx[e], n, qcdev::DBG_PREP));
        }
    }
    if (!qcdev::grid_barrier(bar, p.ctl)) return;
    // F
    for (int v = tid; v < n; v += nthreads) {
        const volatile int32_t *VL = p.L;
        int x = VL[v];
        while (VL[x] != x) x = VL[x];
        p.comp[v] = x;
    }
    if (!qcdev::grid_barrier(bar, p.ctl)) return;
    // G
    word_components(n, p.W, p.comp, p.wcomp, p.wmajor, p.wmask);
    if (tid == 0) p.ctl[1] = 1;
}

// Degree order, stable: nodes by decreasing degree bucket and, within a bucket,
// by increasing id.  Graphs whose ids follow their communities (as generated
// graphs and many real ones do) then keep neighbouring rows close in the BFS's
// work lists, so the rows a level gathers for nearby items are reused from L2
// before they are evicted.  Taken when the BFS's two bitset buffers exceed L2
// (measured on GB300: the SBM of 262,144 nodes, 2 x 256 MiB of bitsets, solves
// in 92.8 instead of 99.9 ms; the DC-SBM of 16,384 nodes, 2 x 32 MiB, is 4 %
// slower in the stable order, so it keeps the scattered one).  Block i of the grid owns the nodes [i chunk, (i + 1) chunk):
// order_counts counts its nodes per bucket, order_offsets turns the counts into
// first positions (heaviest bucket first, then block by block), and order_place
// writes each block's nodes in id order.
__global__ void order_counts(int32_t n, int32_t chunk, const int32_t *row_ptr, int32_t *counts) {
    __shared__ int32_t c[32];
    if (threadIdx.x < 32) c[threadIdx.x] = 0;
    __syncthreads();
    const int v0 = blockIdx.x * chunk, v1 = min(n, v0 + chunk);
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x)
        atomicAdd(&c[degree_bucket(row_ptr[v + 1] - row_ptr[v])], 1);
    __syncthreads();
    if (threadIdx.x < 32) counts[blockIdx.x * 32 + threadIdx.x] = c[threadIdx.x];
}

// One block of 32 warps; warp b scans bucket b over the nb blocks, then the
// buckets are stacked heaviest first; *n_heavy = nodes in buckets >= QC_HEAVY_BUCKET.
__global__ void __launch_bounds__(1024) order_offsets(int32_t nb, const int32_t *counts, int32_t *offsets,
                                                      int32_t *n_heavy) {
    __shared__ int32_t total[32];
    const int lane = threadIdx.x & 31, b = threadIdx.x >> 5;
    int run = 0;
    for (int i0 = 0; i0 < nb; i0 += 32) {
        const int i = i0 + lane;
        const int c = i < nb ? counts[i * 32 + b] : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (i < nb) offsets[i * 32 + b] = run + incl - c;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) total[b] = run;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int bb = 31; bb >= 0; --bb) {
            const int t = total[bb];
            total[bb] = acc;
            acc += t;
            if (bb == QC_HEAVY_BUCKET) *n_heavy = acc;
        }
    }
    __syncthreads();
    for (int i = lane; i < nb; i += 32) offsets[i * 32 + b] += total[b];
}

// 256 threads: the block's nodes 256 at a time; a node's place is its bucket's
// next position plus the nodes of that bucket before it in this step (earlier
// warps, then earlier lanes of its warp).
__global__ void __launch_bounds__(256) order_place(int32_t n, int32_t chunk, const int32_t *row_ptr,
                                                  const int32_t *offsets, int32_t *order) {
    __shared__ int32_t base[32];
    __shared__ int32_t wcount[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < 32) base[threadIdx.x] = offsets[blockIdx.x * 32 + threadIdx.x];
    const int v0 = blockIdx.x * chunk, v1 = min(n, v0 + chunk);
    for (int s = v0; s < v1; s += 256) {
        const int v = s + threadIdx.x;
        const bool ok = v < v1;
        const int b = ok ? degree_bucket(row_ptr[v + 1] - row_ptr[v]) : 32;
        const unsigned same = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(same & ((1u << lane) - 1u));
        wcount[w][lane] = 0;
        __syncthreads();
        if (ok && rank == 0) wcount[w][b] = __popc(same);
        __syncthreads();
        if (ok) {
            int before = 0;
            for (int ww = 0; ww < w; ++ww) before += wcount[ww][b];
            order[base[b] + before + rank] = v;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            int tot = 0;
            for (int ww = 0; ww < 8; ++ww) tot += wcount[ww][threadIdx.x];
            base[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}

// info[i] = {order[i], its row start, its row end, 0}: one 16-byte load gives a
// BFS item everything it needs before it reads the neighbour ids.
__global__ void order_info(int32_t n, const int32_t *row_ptr, const int32_t *order, int4 *info) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = order[i];
        info[i] = make_int4(v, row_ptr[v], row_ptr[v + 1], 0);
    }
}

__global__ void first_rows(int32_t n, const int32_t *row_ptr, int32_t *hist) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        hist[v] = 1;
        hist[(size_t)n + v] = row_ptr[v + 1] - row_ptr[v];
    }
}

}  // namespace

qc_status qc_fill_first_rows(qc_graph *g, cudaStream_t stream) {
    qc_ctx *ctx = g->ctx;
    const int nb = qc_ceil_div(g->n, 256) < 4 * ctx->num_sms ? qc_ceil_div(g->n, 256) : 4 * ctx->num_sms;
    first_rows<<<nb, 256, 0, stream>>>(g->n, g->row_ptr.as<int32_t>(), g->hist.as<int32_t>());
    QC_LAUNCHED(ctx);
    return QC_OK;
}

qc_status qc_graph_prepare(qc_graph *g, cudaStream_t stream) {
    if (g->prepared) return QC_OK;
    qc_range range("qc.prepare");
    qc_ctx *ctx = g->ctx;
    const int32_t n = g->n;
    const int32_t W = (n + 63) / 64;
    QC_TRY(g->comp.allocate(ctx, sizeof(int32_t) * (size_t)n, stream));
    QC_TRY(g->wcomp.allocate(ctx, sizeof(int32_t) * (size_t)W, stream));
    QC_TRY(g->wmajor.allocate(ctx, sizeof(int32_t) * (size_t)W, stream));
    QC_TRY(g->wmask.allocate(ctx, sizeof(unsigned long long) * (size_t)W, stream));
    QC_TRY(g->order.allocate(ctx, sizeof(int32_t) * (size_t)(n + 1), stream));
    QC_TRY(g->oinfo.allocate(ctx, sizeof(int4) * (size_t)n, stream));
    qc_buffer L, bins;
    QC_TRY(L.allocate(ctx, sizeof(int32_t) * (size_t)n, stream));
    const int32_t *rp = g->row_ptr.as<int32_t>();
    const int32_t *ci = g->col_idx.as<int32_t>();
    // the scattered degree order is written inside the fused launch; the stable one
    // (bitsets beyond L2) by its own kernels afterwards
    const double bitset_bytes = 2.0 * 8.0 * (double)n * (double)qc_bfs_chunk_words(ctx, n);
    const bool stable = bitset_bytes > (double)ctx->l2_bytes;
    const int ob = std::max(1, std::min(qc_ceil_div(n, 256), 4 * ctx->num_sms));
    QC_TRY(bins.allocate(ctx, sizeof(int32_t) * (stable ? 64 * (size_t)ob : 64), stream));
    QC_TRY(g->prep_ctl.allocate(ctx, sizeof(int32_t) * 8, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(g->prep_ctl.ptr, 0, g->prep_ctl.bytes, stream));
    if (!stable) QC_CUDA_TRY(ctx, cudaMemsetAsync(bins.ptr, 0, bins.bytes, stream));
    {
        // one thread per node is all the link phases use; more blocks only make each
        // grid barrier dearer
        int per_sm = 0;
        QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)prep_fused, 256, 0));
        const int wb = qc_ceil_div(n, 256) < 8 * ctx->num_sms ? qc_ceil_div(n, 256) : 8 * ctx->num_sms;
        int blocks = per_sm * qc_coop_sms(ctx);
        if (blocks > wb) blocks = wb;
        if (blocks < 1) blocks = 1;
        PrepParams pp;
        pp.n = n;
        pp.W = W;
        pp.row_ptr = rp;
        pp.col_idx = ci;
        pp.L = L.as<int32_t>();
        pp.ctl = g->prep_ctl.as<int32_t>();
        pp.directed = g->directed ? 1 : 0;
        pp.comp = g->comp.as<int32_t>();
        pp.wcomp = g->wcomp.as<int32_t>();
        pp.wmajor = g->wmajor.as<int32_t>();
        pp.wmask = g->wmask.as<unsigned long long>();
        pp.bins = stable ? nullptr : bins.as<int32_t>();
        pp.order = stable ? nullptr : g->order.as<int32_t>();
        pp.info = stable ? nullptr : g->oinfo.as<int4>();
        void *args[] = {(void *)&pp};
        QC_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void *)prep_fused, dim3(blocks), dim3(256), args, 0,
                                                     stream));
        QC_LAUNCHED(ctx);
        g->prep_checked = false;
    }
    if (stable) {
        // stable degree order: blocks own contiguous ranges of node ids
        const int chunk = qc_ceil_div(n, ob);
        int32_t *counts = bins.as<int32_t>(), *offsets = counts + 32 * (size_t)ob;
        order_counts<<<ob, 256, 0, stream>>>(n, chunk, rp, counts);
        QC_LAUNCHED(ctx);
        order_offsets<<<1, 1024, 0, stream>>>(ob, counts, offsets, g->order.as<int32_t>() + n);
        QC_LAUNCHED(ctx);
        order_place<<<ob, 256, 0, stream>>>(n, chunk, rp, offsets, g->order.as<int32_t>());
        QC_LAUNCHED(ctx);
        const int nb = qc_ceil_div(n, 256) < 4 * ctx->num_sms ? qc_ceil_div(n, 256) : 4 * ctx->num_sms;
        order_info<<<nb, 256, 0, stream>>>(n, rp, g->order.as<int32_t>(), g->oinfo.as<int4>());
        QC_LAUNCHED(ctx);
    }
    g->prepared = true;
    return QC_OK;
}

const unsigned long long *qc_graph_deg2(const qc_graph *g) {
    return reinterpret_cast<const unsigned long long *>(g->prep_ctl.as<int32_t>() + 6);
}

qc_status qc_graph_prepare_status(qc_graph *g, int32_t host_status) {
    if (g->prep_checked) return QC_OK;
    if (host_status == qcdev::ST_TIMEOUT) {
        qc_set_error(g->ctx, "connected components: grid barrier timed out");
        g->prepared = false;          // prepare again next time
        return QC_ERR_TIMEOUT;
    }
    g->prep_checked = true;
    return QC_OK;
}
