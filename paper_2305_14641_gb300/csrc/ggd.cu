// Graph Gradient Descent (Algorithm 2 with the prose that follows Algorithm 4)
// and cluster centers (Algorithm 3).
//
// parent(v): among v's neighbours take the smallest V, the smallest node id on
// ties; v moves there only if that V is strictly below its own, else it stays
// its own center.  Strict descent makes every parent chain strictly decreasing
// in V, so chains end at roots (parent(r) = r) and never cycle.
//
// Comparisons run on order-preserving 64-bit integer keys of the doubles
// (IEEE order, -0 and +0 equal), which the integer pipe compares far faster
// than GB300's binary64 pipe; for NaN-free V the outcome of every comparison
// is the same as comparing the doubles.  Keys are laid out node-major,
// K[v * S + s], so one neighbour's S keys are one contiguous run.
//
// Parents: one warp per node (a block per node of degree >= 127); lanes scan
// the neighbours keeping the best (key, id) for up to 16 sigma values, then a
// butterfly over the lanes (and, for a block, shared memory) combines them (the
// result does not depend on the scan order).
//
// Roots: every (sigma, node) thread walks its chain with path halving
// (parent[x] <- parent[parent[x]]) in a scratch parent array; concurrent walkers
// only ever replace a pointer by another ancestor of the same node, so any
// interleaving still ends at the same root.  The root goes to a separate label
// array: a halving write by another walker may still replace parent[v] after v
// found its root, so the parent array itself is not the answer.
#include "qc_device.cuh"
#include "qc_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ long long order_key(double x) {
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ull) b = 0;          // -0 compares equal to +0
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

// K[v * S + s] = key(V[s * n + v]) through 32 x 32 shared-memory tiles.
__global__ void key_transpose(int32_t n, int32_t S, const double *__restrict__ V, long long *__restrict__ K) {
    __shared__ long long tile[32][33];
    const int v0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int s = s0 + r, v = v0 + threadIdx.x;
        if (s < S && v < n) tile[r][threadIdx.x] = order_key(V[(size_t)s * n + v]);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int v = v0 + r, s = s0 + threadIdx.x;
        if (s < S && v < n) K[(size_t)v * S + s] = tile[threadIdx.x][r];
    }
}

// (k, u) precedes (bk, best): smaller key, then smaller id; best < 0 = none yet.
__device__ __forceinline__ bool better(long long k, int u, long long bk, int best) {
    return best < 0 || k < bk || (k == bk && u < best);
}

// Best (key, id) over the neighbours of one node for this lane's sigma: the
// neighbour ids [beg, end) in 32-id chunks first, first + step, ... (step > 1 when
// several warps share the row).  Lane = (slot, sigma): SG lanes per slot, one sigma
// each; the 32/SG slots take every (32/SG)-th neighbour of a chunk.  Neighbour ids
// come 32 at a time from one coalesced load and are broadcast by shuffle; each lane
// keeps U key loads in flight.  log2(32/SG) butterfly steps combine the slots, so
// lanes of slot 0 end with the warp's best.
template <int SG>
__device__ __forceinline__ void scan_row(int32_t n, const int32_t *__restrict__ col_idx,
                                         const long long *__restrict__ K, int32_t S, int s, bool sok, int beg,
                                         int end, int first, int step, long long &bk, int &best) {
    constexpr int SLOTS = 32 / SG;
    constexpr int U = 8;
    const int lane = threadIdx.x & 31;
    const int slot = lane / SG;
    for (int j0 = beg + 32 * first; j0 < end; j0 += 32 * step) {
        const int cnt = min(32, end - j0);
        const int myu = (lane < cnt) ? qcdev::checked_id(col_idx[j0 + lane], n, qcdev::DBG_GGD) : 0;
        for (int m = 0; m < cnt; m += SLOTS * U) {
            long long x[U];
            int uu[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int t = m + k * SLOTS + slot;
                uu[k] = __shfl_sync(FULL, myu, t & 31);
                x[k] = (sok && t < cnt) ? K[(size_t)uu[k] * S + s] : 0;
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const int t = m + k * SLOTS + slot;
                if (sok && t < cnt && better(x[k], uu[k], bk, best)) {
                    bk = x[k];
                    best = uu[k];
                }
            }
        }
    }
#pragma unroll
    for (int off = SG; off < 32; off <<= 1) {
        const long long ok = __shfl_xor_sync(FULL, bk, off);
        const int ob = __shfl_xor_sync(FULL, best, off);
        if (ob >= 0 && better(ok, ob, bk, best)) {
            bk = ok;
            best = ob;
        }
    }
}

// Parents for sigma values s0 .. s0 + sn - 1 (sn <= SG).  Nodes go in `order`
// (heaviest first) when given: its first order[n] rows (degree >= 127) take a
// whole block each, whose 8 warps split the row and meet in shared memory; every
// other row takes one warp.
template <int SG>
__global__ void __launch_bounds__(256, 4) ggd_parent_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                                                         const int32_t *__restrict__ col_idx,
                                                         const long long *__restrict__ K, int32_t S,
                                                         int32_t s0, int32_t sn,
                                                         const int32_t *__restrict__ order,
                                                         int32_t *__restrict__ parent) {
    constexpr int WARPS = 8;
    __shared__ long long red_k[WARPS][SG];
    __shared__ int red_b[WARPS][SG];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int slot = lane / SG;
    const int sl = lane % SG;
    const bool sok = sl < sn;
    const int s = s0 + sl;
    const int heavy = order ? order[n] : 0;
    for (int i = blockIdx.x; i < heavy; i += gridDim.x) {
        const int v = order[i];
        long long bk = 0;
        int best = -1;
        scan_row<SG>(n, col_idx, K, S, s, sok, row_ptr[v], row_ptr[v + 1], wib, WARPS, bk, best);
        if (slot == 0) {
            red_k[wib][sl] = bk;
            red_b[wib][sl] = best;
        }
        __syncthreads();
        if (wib == 0 && slot == 0 && sok) {
            for (int w = 1; w < WARPS; ++w) {
                const int ob = red_b[w][sl];
                if (ob >= 0 && better(red_k[w][sl], ob, bk, best)) {
                    bk = red_k[w][sl];
                    best = ob;
                }
            }
            const long long own = K[(size_t)v * S + s];
            parent[(size_t)s * n + v] = (best >= 0 && bk < own) ? best : v;
        }
        __syncthreads();
    }
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = heavy + warp; i < n; i += nwarps) {
        const int v = order ? order[i] : i;
        long long bk = 0;
        int best = -1;
        scan_row<SG>(n, col_idx, K, S, s, sok, row_ptr[v], row_ptr[v + 1], 0, 1, bk, best);
        if (slot == 0 && sok) {
            const long long own = K[(size_t)v * S + s];
            parent[(size_t)s * n + v] = (best >= 0 && bk < own) ? best : v;
        }
    }
}

__global__ void find_roots_kernel(int32_t n, int32_t *parent, int32_t *__restrict__ labels,
                                  int32_t *n_roots) {
    const int s = blockIdx.y;
    volatile int32_t *P = parent + (size_t)s * n;
    int roots = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int x = v;
        while (true) {
            const int px = P[x];
            if (px == x) break;
            const int gx = P[px];
            if (gx != px) P[x] = gx;
            x = gx;
        }
        if (x == v) ++roots;
        labels[(size_t)s * n + v] = x;
    }
    roots = __reduce_add_sync(FULL, roots);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd(n_roots + s, roots);
}

typedef void (*parent_fn)(int32_t, const int32_t *, const int32_t *, const long long *, int32_t,
                          int32_t, int32_t, const int32_t *, int32_t *);

parent_fn pick_parent(int sn) {
    if (sn <= 1) return ggd_parent_kernel<1>;
    if (sn <= 2) return ggd_parent_kernel<2>;
    if (sn <= 4) return ggd_parent_kernel<4>;
    if (sn <= 8) return ggd_parent_kernel<8>;
    return ggd_parent_kernel<16>;
}

}  // namespace

qc_status qc_descend_into(qc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                          const int32_t *order, const double *V, int32_t n_sigma, int32_t *labels,
                          int32_t *n_roots_dev, int32_t *parent, long long *keys, cudaStream_t stream,
                          bool keys_ready) {
    if (!keys_ready) {
        key_transpose<<<dim3(qc_ceil_div(n, 32), qc_ceil_div(n_sigma, 32)), dim3(32, 8), 0, stream>>>(
            n, n_sigma, V, keys);
        QC_LAUNCHED(ctx);
    }
    const int wblocks = qc_ceil_div(n, 8) < 16 * ctx->num_sms ? qc_ceil_div(n, 8) : 16 * ctx->num_sms;
    for (int32_t s0 = 0; s0 < n_sigma; s0 += 16) {
        const int32_t sn = (n_sigma - s0) < 16 ? (n_sigma - s0) : 16;
        pick_parent(sn)<<<wblocks, 256, 0, stream>>>(n, row_ptr, col_idx, keys, n_sigma, s0, sn, order, parent);
        QC_LAUNCHED(ctx);
    }
    const int blocks = qc_ceil_div(n, 256) < 2 * ctx->num_sms ? qc_ceil_div(n, 256) : 2 * ctx->num_sms;
    find_roots_kernel<<<dim3(blocks, n_sigma), 256, 0, stream>>>(n, parent, labels, n_roots_dev);
    QC_LAUNCHED(ctx);
    return QC_OK;
}

qc_status qc_descend(qc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *order, const double *V, int32_t n_sigma, int32_t *labels,
                     int32_t *n_roots_dev, cudaStream_t stream, const long long *keys) {
    qc_buffer parent, own_keys;
    QC_TRY(parent.allocate(ctx, sizeof(int32_t) * (size_t)n * (size_t)n_sigma, stream));
    if (!keys) QC_TRY(own_keys.allocate(ctx, sizeof(long long) * (size_t)n * (size_t)n_sigma, stream));
    return qc_descend_into(ctx, n, row_ptr, col_idx, order, V, n_sigma, labels, n_roots_dev,
                           parent.as<int32_t>(), keys ? const_cast<long long *>(keys) : own_keys.as<long long>(),
                           stream, keys != nullptr);
}
