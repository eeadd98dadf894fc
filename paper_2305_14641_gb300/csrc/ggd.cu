// Graph Gradient Descent (Algorithm 2 with the prose that follows Algorithm 4)
// and cluster centers (Algorithm 3).
//
// parent(v): among v's neighbours take the smallest V, the smallest node id on
// ties; v moves there only if that V is strictly below its own, else it stays
// its own center.  Strict descent makes every parent chain strictly decreasing
// in V, so chains end at roots (parent(r) = r) and never cycle.
//
// Roots: every (sigma, node) thread walks its chain with path halving
// (parent[x] <- parent[parent[x]]) in a scratch parent array; concurrent walkers
// only ever replace a pointer by another ancestor of the same node, so any
// interleaving still ends at the same root.  The root goes to a separate label
// array: a halving write by another walker may still replace parent[v] after v
// found its root, so the parent array itself is not the answer.
#include "qc_internal.h"

namespace {

__global__ void ggd_parent_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col_idx, const double *__restrict__ V,
                                  int32_t *__restrict__ parent) {
    const int s = blockIdx.y;
    const double *Vs = V + (size_t)s * n;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double vv = Vs[v];
        int best = -1;
        double bv = 0.0;
        const int end = row_ptr[v + 1];
        for (int e = row_ptr[v]; e < end; ++e) {
            const int u = col_idx[e];
            const double x = Vs[u];
            if (best < 0 || x < bv || (x == bv && u < best)) {
                best = u;
                bv = x;
            }
        }
        parent[(size_t)s * n + v] = (best >= 0 && bv < vv) ? best : v;
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
    roots = __reduce_add_sync(0xffffffffu, roots);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd(n_roots + s, roots);
}

}  // namespace

qc_status qc_descend(qc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     const double *V, int32_t n_sigma, int32_t *labels, int32_t *n_roots_dev,
                     cudaStream_t stream) {
    const int blocks = qc_ceil_div(n, 256) < 2 * ctx->num_sms ? qc_ceil_div(n, 256) : 2 * ctx->num_sms;
    dim3 grid(blocks, n_sigma);
    qc_buffer parent;
    QC_TRY(parent.allocate(ctx, sizeof(int32_t) * (size_t)n * (size_t)n_sigma, stream));
    ggd_parent_kernel<<<grid, 256, 0, stream>>>(n, row_ptr, col_idx, V, parent.as<int32_t>());
    QC_LAUNCHED(ctx);
    find_roots_kernel<<<grid, 256, 0, stream>>>(n, parent.as<int32_t>(), labels, n_roots_dev);
    QC_LAUNCHED(ctx);
    return QC_OK;
}
