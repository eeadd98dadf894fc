// The potential of Eq. 7 (last line) / Algorithm 1, evaluated from the distance
// histogram:
//     sum1 = sum_d h_v(d) * d^2 e^{-d^2/(2 sigma^2)},  sum2 = sum_d h_v(d) * e^{-d^2/(2 sigma^2)}
//     V_v  = (sum1 / sum2) / (2 sigma^2)
// Binary64 throughout.  The factors e^{-d^2/(2 sigma^2)} and d^2 e^{...} are
// computed once per (sigma, d) on the host with the C library's exp, so the
// device never evaluates an exponential; the device adds the terms in
// ascending d starting from 0.0 with explicitly rounded multiplies and adds
// (no fused multiply-add) and divides with IEEE round-to-nearest.
#include <cmath>
#include <vector>

#include "qc_internal.h"

bool qc_sigma_ok(double sigma) { return std::isfinite(sigma) && sigma > 0.0; }

void qc_weight_table(double sigma, int32_t len, double *w, double *u) {
    for (int32_t d = 0; d < len; ++d) {
        const double d2 = (double)((int64_t)d * d);
        w[d] = std::exp(-d2 / (2.0 * (sigma * sigma)));
        u[d] = d2 * w[d];
    }
}

namespace {

// One thread per (sigma, node); hist is level-major so a warp reads 32
// consecutive counts per level.  tables: w[s][d], u[s][d] for d = 0..D, den[s] = 2 sigma^2.
// The largest distance: D, or (when the BFS that fills hist is still queued ahead
// on the stream) the one the BFS recorded, D_dev[0] - 1, at most D.
__device__ __forceinline__ int32_t distance_bound(int32_t D, const int32_t *D_dev) {
    return D_dev ? max(0, min(D, *D_dev - 1)) : D;
}

__global__ void potential_kernel(int32_t n, int32_t Dmax, const int32_t *D_dev, const int32_t *__restrict__ hist,
                                 const double *__restrict__ w, const double *__restrict__ u,
                                 const double *__restrict__ den, double *__restrict__ V) {
    const int s = blockIdx.y;
    const double *ws = w + (size_t)s * (Dmax + 1);
    const double *us = u + (size_t)s * (Dmax + 1);
    const int32_t D = distance_bound(Dmax, D_dev);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double sum1 = 0.0, sum2 = 0.0;
        for (int d = 0; d <= D; ++d) {
            const int c = hist[(size_t)d * n + v];
            if (c == 0) continue;          // adds +0.0 to non-negative sums: no change
            const double h = (double)c;
            sum1 = __dadd_rn(sum1, __dmul_rn(h, us[d]));
            sum2 = __dadd_rn(sum2, __dmul_rn(h, ws[d]));
        }
        V[(size_t)s * n + v] = __ddiv_rn(__ddiv_rn(sum1, sum2), den[s]);
    }
}

// Small tables travel as a kernel parameter (no copy, no synchronisation): 16
// sigma values over 32 distances fit.
constexpr int INLINE_DOUBLES = 1040;
struct InlineTables {
    double t[INLINE_DOUBLES];      // w[s][d], then u[s][d], then den[s]
};

__global__ void potential_kernel_inline(int32_t n, int32_t Dmax, const int32_t *D_dev, int32_t S,
                                        const int32_t *__restrict__ hist,
                                        const __grid_constant__ InlineTables tab, double *__restrict__ V) {
    const int s = blockIdx.y;
    const int L = Dmax + 1;
    const double *ws = tab.t + s * L;
    const double *us = tab.t + S * L + s * L;
    const double den = tab.t[2 * S * L + s];
    const int32_t D = distance_bound(Dmax, D_dev);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double sum1 = 0.0, sum2 = 0.0;
        for (int d = 0; d <= D; ++d) {
            const int c = hist[(size_t)d * n + v];
            if (c == 0) continue;
            const double h = (double)c;
            sum1 = __dadd_rn(sum1, __dmul_rn(h, us[d]));
            sum2 = __dadd_rn(sum2, __dmul_rn(h, ws[d]));
        }
        V[(size_t)s * n + v] = __ddiv_rn(__ddiv_rn(sum1, sum2), den);
    }
}

// Distance 0 to itself, 1 to each of deg(v) neighbours, M to the other
// n - 1 - deg(v) nodes, summed in that ascending order.  tab: per sigma w0, w1,
// wM, u0, u1, uM, den.
__global__ void potential_adjacency_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                                           const __grid_constant__ InlineTables tab, double *__restrict__ V) {
    const int s = blockIdx.y;
    const double *t = tab.t + 7 * s;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int deg = row_ptr[v + 1] - row_ptr[v];
        const double h[3] = {1.0, (double)deg, (double)(n - 1 - deg)};
        double sum1 = 0.0, sum2 = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (h[k] == 0.0) continue;
            sum1 = __dadd_rn(sum1, __dmul_rn(h[k], t[3 + k]));
            sum2 = __dadd_rn(sum2, __dmul_rn(h[k], t[k]));
        }
        V[(size_t)s * n + v] = __ddiv_rn(__ddiv_rn(sum1, sum2), t[6]);
    }
}

}  // namespace

extern "C" qc_status qc_potential_adjacency(qc_graph *g, const double *sigmas, int32_t n_sigma, double M,
                                            double *V_out, void *stream_) {
    if (!g || !sigmas || n_sigma < 1 || !V_out) return QC_ERR_INVALID_ARG;
    qc_ctx *ctx = g->ctx;
    if (!std::isfinite(M) || !(M > 1.0)) {
        qc_set_error(ctx, "qc_potential_adjacency: M = %g must be finite and > 1", M);
        return QC_ERR_INVALID_ARG;
    }
    for (int32_t s = 0; s < n_sigma; ++s)
        if (!qc_sigma_ok(sigmas[s])) {
            qc_set_error(ctx, "qc_potential_adjacency: sigma[%d] = %g is not finite and > 0", s, sigmas[s]);
            return QC_ERR_INVALID_ARG;
        }
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const double dist[3] = {0.0, 1.0, M};
    const int per = INLINE_DOUBLES / 7;
    for (int32_t s0 = 0; s0 < n_sigma; s0 += per) {
        const int32_t sn = (n_sigma - s0) < per ? (n_sigma - s0) : per;
        InlineTables it;
        for (int32_t s = 0; s < sn; ++s) {
            const double sigma = sigmas[s0 + s];
            for (int k = 0; k < 3; ++k) {
                const double d2 = dist[k] * dist[k];
                it.t[7 * s + k] = std::exp(-d2 / (2.0 * (sigma * sigma)));
                it.t[7 * s + 3 + k] = d2 * it.t[7 * s + k];
            }
            it.t[7 * s + 6] = 2.0 * (sigma * sigma);
        }
        dim3 grid(qc_ceil_div(g->n, 256) < 2 * ctx->num_sms ? qc_ceil_div(g->n, 256) : 2 * ctx->num_sms, sn);
        potential_adjacency_kernel<<<grid, 256, 0, stream>>>(g->n, g->row_ptr.as<int32_t>(), it,
                                                             V_out + (size_t)s0 * g->n);
        QC_LAUNCHED(ctx);
    }
    return QC_OK;
}

void qc_potential_tables(const double *sigmas, int32_t n_sigma, int32_t L, std::vector<double> &tab) {
    tab.assign((size_t)n_sigma * (2 * L + 1), 0.0);
    double *w = tab.data(), *u = w + (size_t)n_sigma * L, *den = u + (size_t)n_sigma * L;
    for (int32_t s = 0; s < n_sigma; ++s) {
        qc_weight_table(sigmas[s], L, w + (size_t)s * L, u + (size_t)s * L);
        den[s] = 2.0 * (sigmas[s] * sigmas[s]);
    }
}

bool qc_potential_tables_inline(int32_t n_sigma, int32_t L) {
    return (size_t)n_sigma * (2 * L + 1) <= (size_t)INLINE_DOUBLES;
}

qc_status qc_potential_launch(qc_ctx *ctx, int32_t n, const int32_t *hist, int32_t Dmax, const int32_t *D_dev,
                              int32_t n_sigma, const std::vector<double> &tab, const double *dtab, double *V,
                              cudaStream_t stream) {
    const int32_t L = Dmax + 1;
    dim3 grid(qc_ceil_div(n, 256) < 2 * ctx->num_sms ? qc_ceil_div(n, 256) : 2 * ctx->num_sms, n_sigma);
    if (qc_potential_tables_inline(n_sigma, L)) {
        InlineTables it;
        std::copy(tab.begin(), tab.end(), it.t);
        potential_kernel_inline<<<grid, 256, 0, stream>>>(n, Dmax, D_dev, n_sigma, hist, it, V);
    } else {
        potential_kernel<<<grid, 256, 0, stream>>>(n, Dmax, D_dev, hist, dtab, dtab + (size_t)n_sigma * L,
                                                   dtab + 2 * (size_t)n_sigma * L, V);
    }
    QC_LAUNCHED(ctx);
    return QC_OK;
}

qc_status qc_potential_from_hist(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V,
                                 cudaStream_t stream) {
    qc_range range("qc.potential");
    qc_ctx *ctx = g->ctx;
    // while the BFS is still queued ahead, D is known on the device only: the
    // tables cover every histogram row and the kernel stops at the recorded D
    const int32_t Dmax = g->bfs_queued ? g->hist_rows - 1 : g->D;
    const int32_t *D_dev = g->bfs_queued ? g->bfs_out.as<int32_t>() + 1 : nullptr;
    const int32_t L = Dmax + 1;
    std::vector<double> tab;
    qc_potential_tables(sigmas, n_sigma, L, tab);
    if (qc_potential_tables_inline(n_sigma, L))
        return qc_potential_launch(ctx, g->n, g->hist.as<int32_t>(), Dmax, D_dev, n_sigma, tab, nullptr, V, stream);
    qc_buffer dtab;
    QC_TRY(dtab.allocate(ctx, sizeof(double) * tab.size(), stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(dtab.ptr, tab.data(), dtab.bytes, cudaMemcpyHostToDevice, stream));
    // the host table must outlive the asynchronous copy
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    return qc_potential_launch(ctx, g->n, g->hist.as<int32_t>(), Dmax, D_dev, n_sigma, tab, dtab.as<double>(), V,
                               stream);
}
