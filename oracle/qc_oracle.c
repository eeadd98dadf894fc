/*
 * Plain CPU oracle for graph Quantum Clustering (arXiv 2305.14641).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package's smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  The CUDA library never
 * links, loads or calls this file, and this file shares no code with it.
 *
 * What it computes, for one unweighted graph in CSR form (undirected, or
 * directed with row i holding the arcs i -> j; every step follows the rows),
 * and, in part 7, for a graph with positive edge weights:
 *   1. hop distances from a source by a FIFO-queue BFS (Section 3.1: the
 *      distance between nodes, read as the number of edges on a shortest
 *      path; an unreachable pair has infinite distance);
 *   2. the per-node distance histogram h_i(d) = #{j : dist(i, j) = d},
 *      j running over every node including i itself (Algorithm 1 sums over
 *      all n nodes);
 *   3. the potential of Eq. 7 (last line) as Algorithm 1 computes it,
 *      v(i) = (sum1 / sum2) / (2 sigma^2) with sum1 = sum_j d^2 exp(-d^2/2sigma^2)
 *      and sum2 = sum_j exp(-d^2/2sigma^2); the terms are grouped by distance
 *      (canonical form: ascending d, one exp per distance) and, separately,
 *      summed pair by pair (literal form, one exp per pair);
 *   4. Graph Gradient Descent (Algorithm 2 and the prose after Algorithm 4):
 *      each node points at its lowest-potential neighbour (first one in
 *      ascending index on ties) when that potential is strictly lower than
 *      its own, else at itself;
 *   5. cluster centers (Algorithm 3): the root each node's parent chain
 *      reaches, found iteratively with path compression.
 *
 * Readings of the paper taken here, where it is silent or garbled: an
 * unreachable pair contributes nothing (its distance is infinite); the self
 * term has d = 0 (Algorithm 1 sums over all n nodes); a node moves only to a
 * strictly lower neighbour (the prose after Algorithm 4; equal potentials on a
 * bridge must not merge two cliques); among equal minima the lowest index wins;
 * the label is the root's id (Algorithm 3 returns the root).
 *
 * Floating point: IEEE binary64 throughout; compile with -ffp-contract=off so
 * that no multiply-add is fused.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- 1. hop distances (Section 3.1, hop reading) ------------------------- */

/* dist[j] = hops from src to j, or -1 when j is unreachable.  queue: n ints of
 * scratch.  Returns the largest finite distance (the eccentricity of src). */
int32_t qco_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                int32_t src, int32_t *dist, int32_t *queue)
{
    for (int32_t j = 0; j < n; ++j) dist[j] = -1;
    int32_t head = 0, tail = 0, ecc = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t x = col_idx[e];
            if (dist[x] < 0) {
                dist[x] = dist[u] + 1;
                if (dist[x] > ecc) ecc = dist[x];
                queue[tail++] = x;
            }
        }
    }
    return ecc;
}

/* ---- 2. per-node distance histograms (Algorithm 1's sum over j) ---------- */

typedef struct {
    int32_t n;
    const int32_t *row_ptr, *col_idx;
    const int32_t *nodes;
    int64_t first, last;       /* rows [first, last) of the node list */
    int32_t cap;
    int32_t *hist;             /* [n_nodes][cap] */
    int32_t *ecc;              /* [n_nodes] */
    int status;
} qco_hist_job;

static void *qco_hist_worker(void *arg)
{
    qco_hist_job *job = (qco_hist_job *)arg;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)job->n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)job->n);
    if (!dist || !queue) {
        job->status = -2;
        free(dist);
        free(queue);
        return NULL;
    }
    for (int64_t k = job->first; k < job->last; ++k) {
        int32_t *h = job->hist + k * (int64_t)job->cap;
        memset(h, 0, sizeof(int32_t) * (size_t)job->cap);
        int32_t e = qco_bfs(job->n, job->row_ptr, job->col_idx, job->nodes[k], dist, queue);
        job->ecc[k] = e;
        if (e >= job->cap) {
            job->status = -1;
            continue;
        }
        for (int32_t j = 0; j < job->n; ++j)
            if (dist[j] >= 0) h[dist[j]] += 1;
    }
    free(dist);
    free(queue);
    return NULL;
}

/* hist[k][d] = #{j : dist(nodes[k], j) = d} for d < cap; ecc[k] = largest finite
 * distance from nodes[k].  The node list is split into `threads` contiguous parts,
 * one pthread each.  Returns 0, -1 if some distance is >= cap (that row is then
 * incomplete; call again with a larger cap), -2 on allocation failure. */
int qco_histograms(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                   int64_t n_nodes, const int32_t *nodes, int32_t cap,
                   int32_t *hist, int32_t *ecc, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > n_nodes) threads = (int)(n_nodes > 0 ? n_nodes : 1);
    qco_hist_job *jobs = (qco_hist_job *)calloc((size_t)threads, sizeof(qco_hist_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return -2;
    }
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (qco_hist_job){n, row_ptr, col_idx, nodes,
                                 n_nodes * t / threads, n_nodes * (t + 1) / threads,
                                 cap, hist, ecc, 0};
    }
    for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, qco_hist_worker, &jobs[t]);
    qco_hist_worker(&jobs[0]);
    for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    int status = 0;
    for (int t = 0; t < threads; ++t)
        if (jobs[t].status < status) status = jobs[t].status;
    free(jobs);
    free(tid);
    return status;
}

/* ---- 3. the potential (Eq. 7, Algorithm 1) -------------------------------- */

/* Per-distance factors for one sigma: w[d] = exp(-d^2 / (2 sigma^2)) and
 * u[d] = d^2 w[d], d = 0..len-1 (the two summands of Algorithm 1 for a node
 * at distance d). */
void qco_weights(double sigma, int32_t len, double *w, double *u)
{
    for (int32_t d = 0; d < len; ++d) {
        double d2 = (double)((int64_t)d * d);
        w[d] = exp(-d2 / (2.0 * (sigma * sigma)));
        u[d] = d2 * w[d];
    }
}

/* Canonical form: for each row k of hist ([rows][cap]),
 *   sum1 = sum_{d=0..cap-1} h(d) u[d],  sum2 = sum_{d=0..cap-1} h(d) w[d]
 * accumulated from 0.0 in ascending d, V[k] = (sum1 / sum2) / (2 sigma^2). */
void qco_potential_hist(const int32_t *hist, int64_t rows, int32_t cap, double sigma,
                        double *V)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)cap);
    double *u = (double *)malloc(sizeof(double) * (size_t)cap);
    qco_weights(sigma, cap, w, u);
    for (int64_t k = 0; k < rows; ++k) {
        const int32_t *h = hist + k * (int64_t)cap;
        double sum1 = 0.0, sum2 = 0.0;
        for (int32_t d = 0; d < cap; ++d) {
            sum1 = sum1 + (double)h[d] * u[d];
            sum2 = sum2 + (double)h[d] * w[d];
        }
        V[k] = (sum1 / sum2) / (2.0 * (sigma * sigma));
    }
    free(w);
    free(u);
}

/* Literal form: Algorithm 1 as written, one term per node j with dist = hop
 * distance from i (dist[j] < 0: unreachable, no term). */
double qco_potential_literal(const int32_t *dist, int32_t n, double sigma)
{
    double sum1 = 0.0, sum2 = 0.0;
    for (int32_t j = 0; j < n; ++j) {
        if (dist[j] < 0) continue;
        double d = (double)dist[j];
        double e = exp(-(d * d) / (2.0 * sigma * sigma));
        sum1 = sum1 + d * d * e;
        sum2 = sum2 + e;
    }
    return (1.0 / (2.0 * sigma * sigma)) * (sum1 / sum2);
}

/* ---- 4. Graph Gradient Descent (Algorithm 2, prose after Algorithm 4) ------ */

/* parent[i] = the first neighbour (ascending index) holding the smallest V among
 * i's neighbours, if that V is strictly below V[i]; otherwise i.  Returns the
 * number of nodes whose minimal neighbours tie (two or more share the minimum and
 * it is below V[i]): the only places where node numbering decides the result. */
int64_t qco_ggd_parent(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *V, int32_t *parent)
{
    int64_t ties = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t best = -1;
        int32_t count = 0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (best < 0 || V[j] < V[best]) {
                best = j;
                count = 1;
            } else if (V[j] == V[best]) {
                count += 1;
            }
        }
        if (best >= 0 && V[best] < V[i]) {
            parent[i] = best;
            if (count > 1) ties += 1;
        } else {
            parent[i] = i;
        }
    }
    return ties;
}

/* ---- 5. cluster centers (Algorithm 3) --------------------------------------- */

/* label[i] = root of i's parent chain.  Iterative find with path compression on a
 * private copy of parent.  Returns the number of roots (clusters). */
int32_t qco_find_centers(int32_t n, const int32_t *parent, int32_t *label)
{
    int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    memcpy(p, parent, sizeof(int32_t) * (size_t)n);
    int32_t roots = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t r = i;
        while (p[r] != r) r = p[r];
        int32_t x = i;
        while (p[x] != r) {
            int32_t next = p[x];
            p[x] = r;
            x = next;
        }
        label[i] = r;
        if (r == i) roots += 1;
    }
    free(p);
    return roots;
}

/* ---- paper-literal distance (Section 3.1 as written) ----------------------- */

/* Distance read straight from the adjacency matrix: 0 from a node to itself,
 * the edge weight (1 in an unweighted graph) to a neighbour, and M, a value
 * above every weight, to every other node.  Node i then has one term at
 * distance 0, deg(i) terms at distance 1 and n - 1 - deg(i) terms at distance M;
 * V is summed in that ascending order like the canonical form above. */
void qco_potential_adjacency(int32_t n, const int32_t *row_ptr, double M, double sigma, double *V)
{
    const double dist[3] = {0.0, 1.0, M};
    double w[3], u[3];
    for (int k = 0; k < 3; ++k) {
        double d2 = dist[k] * dist[k];
        w[k] = exp(-d2 / (2.0 * (sigma * sigma)));
        u[k] = d2 * w[k];
    }
    for (int32_t i = 0; i < n; ++i) {
        int32_t deg = row_ptr[i + 1] - row_ptr[i];
        double h[3] = {1.0, (double)deg, (double)(n - 1 - deg)};
        double sum1 = 0.0, sum2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            sum1 = sum1 + h[k] * u[k];
            sum2 = sum2 + h[k] * w[k];
        }
        V[i] = (sum1 / sum2) / (2.0 * (sigma * sigma));
    }
}

/* ---- 7. weighted graphs (Section 3.1: an edge's distance is its weight) --- */

/* Shortest-path lengths from src over positive edge weights by Dijkstra's
 * algorithm with a binary heap.  A path's length is accumulated hop by hop in
 * path order, dist[v] = dist[u] + w(u, v) in binary64, and the smallest such
 * value is kept; unreachable nodes get +inf.  Returns 0, or -2 if scratch
 * could not be allocated. */
int qco_dijkstra(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *w,
                 int32_t src, double *dist)
{
    /* heap of (key, node) with lazy deletion: at most nnz + 1 entries */
    int64_t cap = (int64_t)row_ptr[n] + 1;
    double *hk = malloc(sizeof(double) * (size_t)cap);
    int32_t *hv = malloc(sizeof(int32_t) * (size_t)cap);
    char *done = calloc((size_t)n, 1);
    if (!hk || !hv || !done) {
        free(hk); free(hv); free(done);
        return -2;
    }
    for (int32_t v = 0; v < n; ++v) dist[v] = INFINITY;
    int64_t size = 0;
    dist[src] = 0.0;
    hk[0] = 0.0; hv[0] = src; size = 1;
    while (size > 0) {
        double k = hk[0];
        int32_t u = hv[0];
        /* pop: move the last entry to the top and sift it down */
        --size;
        if (size > 0) {
            double lk = hk[size];
            int32_t lv = hv[size];
            int64_t i = 0;
            for (;;) {
                int64_t c = 2 * i + 1;
                if (c >= size) break;
                if (c + 1 < size && hk[c + 1] < hk[c]) ++c;
                if (!(hk[c] < lk)) break;
                hk[i] = hk[c]; hv[i] = hv[c];
                i = c;
            }
            hk[i] = lk; hv[i] = lv;
        }
        if (done[u] || k > dist[u]) continue;
        done[u] = 1;
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col_idx[e];
            double nd = dist[u] + w[e];
            if (nd < dist[v]) {
                dist[v] = nd;
                /* push and sift up */
                int64_t i = size++;
                while (i > 0) {
                    int64_t p = (i - 1) / 2;
                    if (!(nd < hk[p])) break;
                    hk[i] = hk[p]; hv[i] = hv[p];
                    i = p;
                }
                hk[i] = nd; hv[i] = v;
            }
        }
    }
    free(hk); free(hv); free(done);
    return 0;
}

/* Algorithm 1 with weighted shortest-path distances: for node i and each
 * sigma, sum1 = sum_j d^2 exp(-d^2 / (2 sigma^2)) and sum2 = sum_j exp(...) over
 * every j in ascending order (unreachable j contribute nothing, j = i adds 1 to
 * sum2), then V = (sum1 / sum2) / (2 sigma^2).  V is [n_sigma][n]. */
struct qco_wpot_job {
    int32_t n;
    const int32_t *row_ptr, *col_idx;
    const double *w, *sigmas;
    int32_t n_sigma;
    double *V;
    int32_t first, step;
    int status;
};

static void *qco_wpot_worker(void *arg)
{
    struct qco_wpot_job *job = arg;
    double *dist = malloc(sizeof(double) * (size_t)job->n);
    if (!dist) { job->status = -2; return NULL; }
    for (int32_t i = job->first; i < job->n; i += job->step) {
        if (qco_dijkstra(job->n, job->row_ptr, job->col_idx, job->w, i, dist) != 0) {
            job->status = -2;
            break;
        }
        for (int32_t s = 0; s < job->n_sigma; ++s) {
            double sigma = job->sigmas[s];
            double sum1 = 0.0, sum2 = 0.0;
            for (int32_t j = 0; j < job->n; ++j) {
                double d = dist[j];
                if (!isfinite(d)) continue;
                double d2 = d * d;
                double e = exp(-d2 / (2.0 * (sigma * sigma)));
                sum1 = sum1 + d2 * e;
                sum2 = sum2 + e;
            }
            job->V[(size_t)s * job->n + i] = (sum1 / sum2) / (2.0 * (sigma * sigma));
        }
    }
    free(dist);
    return NULL;
}

int qco_potential_weighted(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *w,
                           const double *sigmas, int32_t n_sigma, double *V, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    struct qco_wpot_job job[256];
    int started[256];
    int status = 0;
    for (int t = 0; t < threads; ++t) {
        job[t] = (struct qco_wpot_job){n, row_ptr, col_idx, w, sigmas, n_sigma, V, t, threads, 0};
        started[t] = threads > 1 && pthread_create(&tid[t], NULL, qco_wpot_worker, &job[t]) == 0;
        if (!started[t]) qco_wpot_worker(&job[t]);   /* no thread: run the share here */
    }
    for (int t = 0; t < threads; ++t) {
        if (started[t]) pthread_join(tid[t], NULL);
        if (job[t].status) status = job[t].status;
    }
    return status;
}
