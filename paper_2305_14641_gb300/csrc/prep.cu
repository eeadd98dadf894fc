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
#include "qc_device.cuh"
#include "qc_internal.h"

namespace {

// Connected components by hooking and shortcutting (after Shiloach & Vishkin),
// all iterations in one cooperative launch.  L[v] always names a node of v's
// component with id <= v, and labels only decrease:
//   hook:     for every edge (v, u) with a = L[v] > b = L[u]: L[a] = min(L[a], b);
//   shortcut: L[v] = L[L[v]] until L[v] is a root (L[L[v]] = L[v]).
// An iteration in which no hook lowers a label leaves every edge's two ends with
// the same root label, which is then the smallest id of the component.
// A directed graph lists each edge in one row only, so there the hook runs in
// both directions (a < b: L[b] = min(L[b], a)) and the result is the weakly
// connected components, which bound what any node can reach.
// ctl: [0] status, [1] iterations run, [2..3] barrier, [8 + it] "a hook changed
// something in iteration it".
__global__ void __launch_bounds__(256) cc_persistent(int32_t n, const int32_t *row_ptr,
                                                     const int32_t *col_idx, int32_t *L, int32_t *ctl,
                                                     int32_t max_iters, int32_t resume, int32_t directed) {
    unsigned *bar = reinterpret_cast<unsigned *>(ctl + 2);
    const int lane = threadIdx.x & 31;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const int warp = tid >> 5;
    const int nwarps = nthreads >> 5;
    if (!resume) {
        // start at the smallest neighbour when smaller (Jaiganesh & Burtscher, ECL-CC, 2018)
        for (int v = tid; v < n; v += nthreads) {
            int m = v;
            const int end = row_ptr[v + 1];
            for (int e = row_ptr[v]; e < end; ++e) m = min(m, col_idx[e]);
            L[v] = m;
        }
        if (!qcdev::grid_barrier(bar, ctl)) return;
    }
    volatile int32_t *VL = L;
    for (int it = 0; it < max_iters; ++it) {
        // shortcut
        for (int v = tid; v < n; v += nthreads) {
            int x = VL[v];
            int y = VL[x];
            while (x != y) {
                x = y;
                y = VL[x];
            }
            VL[v] = x;
        }
        if (!qcdev::grid_barrier(bar, ctl)) return;
        // hook
        bool changed = false;
        for (int v = warp; v < n; v += nwarps) {
            const int a = VL[v];
            const int end = row_ptr[v + 1];
            for (int e = row_ptr[v] + lane; e < end; e += 32) {
                const int b = VL[col_idx[e]];
                if (b < a) {
                    if (atomicMin(L + a, b) > b) changed = true;
                } else if (directed && a < b) {
                    if (atomicMin(L + b, a) > a) changed = true;
                }
            }
        }
        if (__syncthreads_or(changed) && threadIdx.x == 0) ctl[8 + it] = 1;
        if (!qcdev::grid_barrier(bar, ctl)) return;
        if (*(volatile int32_t *)(ctl + 8 + it) == 0) {
            if (tid == 0) ctl[1] = it + 1;
            return;
        }
    }
    if (tid == 0) {
        ctl[1] = max_iters;
        ctl[0] = qcdev::ST_NEED_ROWS;     // not converged yet: run again
    }
}

// Final labels: the root of each node's label chain.
__global__ void cc_flatten(int32_t n, const int32_t *L, int32_t *comp) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int x = L[v];
        while (L[x] != x) x = L[x];
        comp[v] = x;
    }
}

// Per 64-source word: wcomp = the one component of all its sources, or -1; the
// component holding most of them (wmajor) and their bits (wmask), so that the
// BFS presets the row of a node in that component with one mask and walks the
// word bit by bit only for nodes of the word's minor components.
__global__ void word_components(int32_t n, int32_t W, const int32_t *comp, int32_t *wcomp, int32_t *wmajor,
                                unsigned long long *wmask) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < W; k += gridDim.x * blockDim.x) {
        const int s0 = 64 * k;
        const int cnt = min(64, n - s0);
        int best = comp[s0], best_count = 0;
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
        wcomp[k] = (best_count == cnt) ? best : -1;
        wmajor[k] = best;
        wmask[k] = best_mask;
    }
}

__device__ __forceinline__ int degree_bucket(int deg) { return 31 - __clz(deg + 1); }

__global__ void bucket_count(int32_t n, const int32_t *row_ptr, int32_t *counts) {
    __shared__ int32_t local[32];
    if (threadIdx.x < 32) local[threadIdx.x] = 0;
    __syncthreads();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        atomicAdd(&local[degree_bucket(row_ptr[v + 1] - row_ptr[v])], 1);
    __syncthreads();
    if (threadIdx.x < 32 && local[threadIdx.x]) atomicAdd(&counts[threadIdx.x], local[threadIdx.x]);
}

// cursor[b] = number of nodes in buckets above b (heaviest bucket first);
// *n_heavy = nodes in buckets >= QC_HEAVY_BUCKET (a prefix of the order).
__global__ void bucket_scan(const int32_t *counts, int32_t *cursor, int32_t *n_heavy) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 31; b >= 0; --b) {
            cursor[b] = acc;
            acc += counts[b];
            if (b == QC_HEAVY_BUCKET) *n_heavy = acc;
        }
    }
}

__global__ void bucket_scatter(int32_t n, const int32_t *row_ptr, int32_t *cursor, int32_t *order) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        order[atomicAdd(&cursor[degree_bucket(row_ptr[v + 1] - row_ptr[v])], 1)] = v;
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
    qc_buffer p, bins;
    QC_TRY(p.allocate(ctx, sizeof(int32_t) * (size_t)n, stream));
    QC_TRY(bins.allocate(ctx, sizeof(int32_t) * 64, stream));
    const int tb = 256;
    const int nb = qc_ceil_div(n, tb) < 4 * ctx->num_sms ? qc_ceil_div(n, tb) : 4 * ctx->num_sms;
    const int wb = qc_ceil_div(n, 8) < 8 * ctx->num_sms ? qc_ceil_div(n, 8) : 8 * ctx->num_sms;
    const int32_t *rp = g->row_ptr.as<int32_t>();
    const int32_t *ci = g->col_idx.as<int32_t>();
    {
        int per_sm = 0;
        QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)cc_persistent,
                                                                       256, 0));
        int blocks = per_sm * qc_coop_sms(ctx);
        if (blocks > wb) blocks = wb;
        if (blocks < 1) blocks = 1;
        qc_buffer ctl;
        const int32_t max_iters = 512;
        QC_TRY(ctl.allocate(ctx, sizeof(int32_t) * (8 + max_iters), stream));
        qc_pinned pin(ctx);
        QC_TRY(pin.acquire());
        int32_t *h = static_cast<int32_t *>(pin.ptr);
        int32_t resume = 0;
        while (true) {
            QC_CUDA_TRY(ctx, cudaMemsetAsync(ctl.ptr, 0, ctl.bytes, stream));
            int32_t n_ = n, iters = max_iters, directed = g->directed ? 1 : 0;
            int32_t *L = p.as<int32_t>(), *c = ctl.as<int32_t>();
            void *args[] = {&n_, (void *)&rp, (void *)&ci, &L, &c, &iters, &resume, &directed};
            QC_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void *)cc_persistent, dim3(blocks), dim3(256),
                                                         args, 0, stream));
            QC_LAUNCHED(ctx);
            QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, ctl.ptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
            QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
            if (h[0] == qcdev::ST_TIMEOUT) {
                qc_set_error(ctx, "connected components: grid barrier timed out");
                return QC_ERR_TIMEOUT;
            }
            if (h[0] == qcdev::ST_DONE) break;
            resume = 1;
        }
    }
    cc_flatten<<<nb, tb, 0, stream>>>(n, p.as<int32_t>(), g->comp.as<int32_t>());
    QC_LAUNCHED(ctx);
    word_components<<<qc_ceil_div(W, 128), 128, 0, stream>>>(n, W, g->comp.as<int32_t>(), g->wcomp.as<int32_t>(),
                                                            g->wmajor.as<int32_t>(),
                                                            g->wmask.as<unsigned long long>());
    QC_LAUNCHED(ctx);
    QC_CUDA_TRY(ctx, cudaMemsetAsync(bins.ptr, 0, bins.bytes, stream));
    bucket_count<<<nb, tb, 0, stream>>>(n, rp, bins.as<int32_t>());
    QC_LAUNCHED(ctx);
    bucket_scan<<<1, 32, 0, stream>>>(bins.as<int32_t>(), bins.as<int32_t>() + 32,
                                      g->order.as<int32_t>() + n);
    QC_LAUNCHED(ctx);
    bucket_scatter<<<nb, tb, 0, stream>>>(n, rp, bins.as<int32_t>() + 32, g->order.as<int32_t>());
    QC_LAUNCHED(ctx);
    order_info<<<nb, tb, 0, stream>>>(n, rp, g->order.as<int32_t>(), g->oinfo.as<int4>());
    QC_LAUNCHED(ctx);
    g->prepared = true;
    return QC_OK;
}
