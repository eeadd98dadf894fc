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

// The largest distance: D, or (when the BFS that fills hist is still queued ahead
// on the stream) the one the BFS recorded, D_dev[0] - 1, at most D.
__device__ __forceinline__ int32_t distance_bound(int32_t D, const int32_t *D_dev) {
    return D_dev ? max(0, min(D, *D_dev - 1)) : D;
}

// c as a double, built on the integer pipe (exact: c < 2^31 has at most 31
// significant bits), so that GB300's narrow binary64 pipe only multiplies and adds.
__device__ __forceinline__ double count_to_double(int c) {
    if (c <= 0) return (double)c;                    // not in a valid histogram
    const unsigned uc = (unsigned)c;
    const int lz = __clz(uc);                        // c > 0: top bit at 31 - lz
    const unsigned long long e = 1023ull + 31ull - (unsigned long long)lz;
    const unsigned long long m = ((unsigned long long)uc << (21 + lz)) & ((1ull << 52) - 1ull);
    return __longlong_as_double((long long)((e << 52) | m));
}

// The descent's order-preserving key of a potential (IEEE order, -0 equal to +0).
__device__ __forceinline__ long long potential_key(double x) {
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

// V of one (sigma, node).  hist is level-major, so a warp reads 32 consecutive
// counts per level.  Distance 0 (the node itself, h = 1 in every histogram) needs
// no binary64 work: 1 * x = x and 0 + x = x exactly, so the sums start at
// (u[0], w[0]); any other count there takes the general step.
__device__ __forceinline__ double potential_of(int32_t n, int v, int32_t D, const int32_t *__restrict__ hist,
                                              const double *us, const double *ws, double den) {
    double sum1 = 0.0, sum2 = 0.0;
    int d = 0;
    if (hist[v] == 1) {
        sum1 = us[0];
        sum2 = ws[0];
        d = 1;
    }
    for (; d <= D; ++d) {
        const int c = hist[(size_t)d * n + v];
        if (c == 0) continue;          // adds +0.0 to non-negative sums: no change
        const double h = count_to_double(c);
        sum1 = __dadd_rn(sum1, __dmul_rn(h, us[d]));
        sum2 = __dadd_rn(sum2, __dmul_rn(h, ws[d]));
    }
    return __ddiv_rn(__ddiv_rn(sum1, sum2), den);
}

// One thread per (sigma, node).  tables: w[s][d], u[s][d] for d = 0..D, den[s] = 2 sigma^2.
// K (optional): the keys of the descent, node-major K[v * S + s].
__global__ void potential_kernel(int32_t n, int32_t Dmax, const int32_t *D_dev, int32_t S,
                                 const int32_t *__restrict__ hist, const double *__restrict__ w,
                                 const double *__restrict__ u, const double *__restrict__ den,
                                 double *__restrict__ V, long long *__restrict__ K) {
    const int s = blockIdx.y;
    const double *ws = w + (size_t)s * (Dmax + 1);
    const double *us = u + (size_t)s * (Dmax + 1);
    const int32_t D = distance_bound(Dmax, D_dev);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double x = potential_of(n, v, D, hist, us, ws, den[s]);
        V[(size_t)s * n + v] = x;
        if (K) K[(size_t)v * S + s] = potential_key(x);
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
                                        const __grid_constant__ InlineTables tab, double *__restrict__ V,
                                        long long *__restrict__ K) {
    const int s = blockIdx.y;
    const int L = Dmax + 1;
    const double *ws = tab.t + s * L;
    const double *us = tab.t + S * L + s * L;
    const double den = tab.t[2 * S * L + s];
    const int32_t D = distance_bound(Dmax, D_dev);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double x = potential_of(n, v, D, hist, us, ws, den);
        V[(size_t)s * n + v] = x;
        if (K) K[(size_t)v * S + s] = potential_key(x);
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
                              long long *keys, cudaStream_t stream) {
    const int32_t L = Dmax + 1;
    dim3 grid(qc_ceil_div(n, 256) < 2 * ctx->num_sms ? qc_ceil_div(n, 256) : 2 * ctx->num_sms, n_sigma);
    if (qc_potential_tables_inline(n_sigma, L)) {
        InlineTables it;
        std::copy(tab.begin(), tab.end(), it.t);
        potential_kernel_inline<<<grid, 256, 0, stream>>>(n, Dmax, D_dev, n_sigma, hist, it, V, keys);
    } else {
        potential_kernel<<<grid, 256, 0, stream>>>(n, Dmax, D_dev, n_sigma, hist, dtab, dtab + (size_t)n_sigma * L,
                                                   dtab + 2 * (size_t)n_sigma * L, V, keys);
    }
    QC_LAUNCHED(ctx);
    return QC_OK;
}

qc_status qc_potential_from_hist(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V,
                                 cudaStream_t stream, long long *keys) {
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
        return qc_potential_launch(ctx, g->n, g->hist.as<int32_t>(), Dmax, D_dev, n_sigma, tab, nullptr, V, keys,
                                   stream);
    qc_buffer dtab;
    QC_TRY(dtab.allocate(ctx, sizeof(double) * tab.size(), stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(dtab.ptr, tab.data(), dtab.bytes, cudaMemcpyHostToDevice, stream));
    // the host table must outlive the asynchronous copy
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    return qc_potential_launch(ctx, g->n, g->hist.as<int32_t>(), Dmax, D_dev, n_sigma, tab, dtab.as<double>(), V,
                               keys, stream);
}
