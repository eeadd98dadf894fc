// Serving loop: graph-clustering requests of any size, admitted against a
// device-memory budget and batched as they arrive.
//
// Threads:
//   scheduler  admits queued requests in FIFO order while their byte estimate
//              fits the budget and fewer than max_active are on the GPU; groups
//              the admitted requests that fit a CTA (n <= 2048) into one launch
//              of the batched graph-per-CTA kernel on a free stream slot (up to
//              `streams` launches in flight, so newly arrived requests start
//              while earlier ones are still running: continuous batching); a
//              host callback on the stream wakes it when a launch has finished,
//              and it hands the results out;
//   large      worker threads (four by default) run the single-graph path for
//              larger requests (and for any request whose BFS needed more
//              histogram rows than the batched kernel keeps), one request at a
//              time each, on low-priority streams; their persistent kernels
//              fill only a share of the SMs (40% each by default) so that batched
//              launches of small requests, on high-priority streams, keep
//              running beside a large request instead of waiting for it.
// Every request gets its own device copy of its CSR and its own label buffer,
// and every kernel that touches it reads only that request's data, so a result
// does not depend on which other requests shared the launch or the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum class RState { Queued, Active, Done, Failed, Cancelled };

struct Req {
    uint64_t id = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    std::vector<int32_t> rp, ci;
    double sigma = 1.0;
    size_t bytes = 0;
    bool large = false;
    RState state = RState::Queued;
    qc_status status = QC_OK;
    bool cancel = false;
    Clock::time_point t_submit, t_admit, t_start, t_done;
    int32_t batch_size = 0;
    qc_graph *g = nullptr;
    bool borrowed = false;       // g is the caller's resident graph (never destroyed here)
    qc_buffer labels_dev;
    std::vector<int32_t> labels;
    int32_t n_clusters = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    bool busy = false;
    volatile bool finished = false;
    std::vector<Req *> reqs;
    qc_cta_launch *launch = nullptr;
    int32_t *pinned = nullptr;     // labels of every request, then counts, then flags
    size_t pinned_ints = 0;
    std::vector<size_t> offs;
};

qc_status validate_host_csr(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci) {
    if (rp[0] != 0 || rp[n] != nnz) return QC_ERR_INVALID_GRAPH;
    for (int32_t v = 0; v < n; ++v) {
        if (rp[v + 1] < rp[v]) return QC_ERR_INVALID_GRAPH;
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t u = ci[e];
            if (u < 0 || u >= n || u == v) return QC_ERR_INVALID_GRAPH;
            if (e > rp[v] && ci[e - 1] >= u) return QC_ERR_INVALID_GRAPH;
            int32_t lo = rp[u], hi = rp[u + 1] - 1;
            bool found = false;
            while (lo <= hi) {
                const int32_t mid = (lo + hi) / 2;
                if (ci[mid] == v) { found = true; break; }
                if (ci[mid] < v) lo = mid + 1; else hi = mid - 1;
            }
            if (!found) return QC_ERR_INVALID_GRAPH;
        }
    }
    return QC_OK;
}

}  // namespace

struct qc_server {
    qc_ctx *ctx = nullptr;
    size_t budget = 0;
    int32_t max_active = 256;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;        // scheduler wake-ups
    std::condition_variable cv_done;   // a request finished
    std::condition_variable cv_large;  // large-graph worker wake-ups
    std::deque<Req *> queue;
    std::deque<Req *> large_queue;
    std::vector<Req *> pending;        // admitted, waiting for a launch slot
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    size_t resident = 0;
    int32_t active = 0;
    int32_t in_flight = 0;
    qc_server_stats st{};
    std::thread sched;
    std::vector<std::thread> large;
    std::vector<cudaStream_t> large_streams;
    int prio_high = 0, prio_low = 0;   // priorities of the slot and worker streams (the context's)
    float saved_share = 1.0f;          // the context's SM share before the server set its own
    float large_share = 0.4f;          // SM share of the large-request path
    bool divide_share = false;         // split large_share among the large requests running
    int32_t large_running = 0;         // large requests on the GPU right now

    size_t estimate(int32_t n, int64_t nnz, bool is_large) const {
        const size_t csr = 4 * ((size_t)n + 1) + 4 * (size_t)nnz;
        if (!is_large) return csr + 4 * (size_t)n + qc_cta_bytes_per_node() * (size_t)n + 256;
        const size_t wc = (size_t)qc_bfs_chunk_words(ctx, n);
        const size_t R = (wc + 1) / 2, T = R >= 32 ? (R + 31) / 32 : 1;
        return csr + 32 * (size_t)n * R            // two bitset buffers
               + 12 * (size_t)n * T + 16 * ((size_t)n + 2)
               + 4 * (size_t)n * 64                // histogram (grows past 64 levels on demand)
               + 40 * (size_t)n;                   // prep, potential, keys, parents, labels
    }

    void finish(Req *r, RState s, qc_status status) {   // mu held
        r->state = s;
        r->status = status;
        r->t_done = Clock::now();
        if (r->g && !r->borrowed) qc_graph_destroy(r->g);
        r->g = nullptr;
        r->labels_dev.release();
        resident -= r->bytes;
        active -= 1;
        if (s == RState::Done) st.completed++;
        else if (s == RState::Cancelled) st.cancelled++;
        else st.failed++;
        cv_done.notify_all();
        cv.notify_all();
    }

    static void CUDART_CB on_step_done(void *p) {
        auto *pr = static_cast<std::pair<qc_server *, Slot *> *>(p);
        {
            std::lock_guard<std::mutex> lk(pr->first->mu);
            pr->second->finished = true;
        }
        pr->first->cv.notify_all();
        delete pr;
    }

    // Launch the pending small requests on slot `s` (mu not held).
    qc_status launch(Slot &s, std::vector<Req *> &rs) {
        std::vector<qc_graph *> graphs;
        std::vector<double> sig;
        std::vector<int32_t *> lab;
        size_t total = 0;
        s.offs.clear();
        for (Req *r : rs) {
            if (!r->borrowed)
                QC_TRY(qc_graph_create(ctx, r->n, r->nnz, r->rp.data(), r->nnz ? r->ci.data() : nullptr, 0,
                                       s.stream, &r->g));
            QC_TRY(r->labels_dev.allocate(ctx, sizeof(int32_t) * (size_t)r->n, s.stream));
            graphs.push_back(r->g);
            sig.push_back(r->sigma);
            lab.push_back(r->labels_dev.as<int32_t>());
            s.offs.push_back(total);
            total += (size_t)r->n;
        }
        const size_t need = total + 2 * rs.size() + 1;
        if (need > s.pinned_ints) {
            if (s.pinned) cudaFreeHost(s.pinned);
            s.pinned = nullptr;
            s.pinned_ints = 0;
            QC_CUDA_TRY(ctx, cudaMallocHost(&s.pinned, sizeof(int32_t) * need * 2));
            s.pinned_ints = need * 2;
        }
        // the SMs the large requests' persistent kernels leave free, split among the slots
        const int spare = ctx->num_sms - qc_coop_sms(ctx);
        const int max_sms = spare > 0 ? std::max(1, spare / (int)slots.size()) : 0;
        QC_TRY(qc_cta_launch_async(ctx, (int32_t)rs.size(), graphs.data(), sig.data(), lab.data(), max_sms,
                                   s.stream, &s.launch));
        for (size_t i = 0; i < rs.size(); ++i)
            QC_CUDA_TRY(ctx, cudaMemcpyAsync(s.pinned + s.offs[i], lab[i], sizeof(int32_t) * rs[i]->n,
                                             cudaMemcpyDeviceToHost, s.stream));
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(s.pinned + total, qc_cta_counts(s.launch), sizeof(int32_t) * rs.size(),
                                         cudaMemcpyDeviceToHost, s.stream));
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(s.pinned + total + rs.size(), qc_cta_flags(s.launch),
                                         sizeof(int32_t) * (rs.size() + 1), cudaMemcpyDeviceToHost, s.stream));
        auto *pr = new std::pair<qc_server *, Slot *>(this, &s);
        cudaError_t e = cudaLaunchHostFunc(s.stream, on_step_done, pr);
        if (e != cudaSuccess) {
            delete pr;
            QC_CUDA_TRY(ctx, e);
        }
        return QC_OK;
    }

    // Hand out the results of a finished slot (mu held).
    void complete(Slot &s) {
        // debug build: a failed bounds check in the launch fails its requests
        const qc_status dbg = qc_debug_take(ctx);
        size_t total = 0;
        for (Req *r : s.reqs) total += (size_t)r->n;
        const int32_t *counts = s.pinned + total;
        const int32_t *flags = counts + s.reqs.size();
        for (size_t i = 0; i < s.reqs.size(); ++i) {
            Req *r = s.reqs[i];
            if (r->cancel) {
                finish(r, RState::Cancelled, QC_ERR_CANCELLED);
                continue;
            }
            if (dbg != QC_OK) {
                finish(r, RState::Failed, dbg);
                continue;
            }
            if (flags[i]) {          // deeper than the batched kernel keeps: single-graph path
                r->large = true;
                large_queue.push_back(r);
                cv_large.notify_all();
                continue;
            }
            r->labels.assign(s.pinned + s.offs[i], s.pinned + s.offs[i] + r->n);
            r->n_clusters = counts[i];
            finish(r, RState::Done, QC_OK);
        }
        qc_cta_launch_free(s.launch);
        s.launch = nullptr;
        s.reqs.clear();
        s.busy = false;
        s.finished = false;
        in_flight -= 1;
    }

    void scheduler() {
        cudaSetDevice(ctx->device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            for (Slot &s : slots)
                if (s.busy && s.finished) complete(s);
            // admission, FIFO
            while (!queue.empty() && active < max_active) {
                Req *r = queue.front();
                if (r->cancel) {
                    queue.pop_front();
                    r->state = RState::Cancelled;
                    r->status = QC_ERR_CANCELLED;
                    r->t_done = Clock::now();
                    st.cancelled++;
                    cv_done.notify_all();
                    continue;
                }
                if (resident + r->bytes > budget) break;
                queue.pop_front();
                resident += r->bytes;
                if (resident > st.peak_bytes_resident) st.peak_bytes_resident = resident;
                active += 1;
                r->state = RState::Active;
                r->t_admit = Clock::now();
                if (r->large) {
                    large_queue.push_back(r);
                    cv_large.notify_all();
                } else {
                    pending.push_back(r);
                }
            }
            Slot *free_slot = nullptr;
            for (Slot &s : slots)
                if (!s.busy) { free_slot = &s; break; }
            if (!pending.empty() && free_slot) {
                std::vector<Req *> rs;
                rs.swap(pending);
                const Clock::time_point t_launch = Clock::now();
                for (Req *r : rs) {
                    r->batch_size = (int32_t)rs.size();
                    r->t_start = t_launch;
                }
                free_slot->busy = true;
                free_slot->finished = false;
                free_slot->reqs = rs;
                in_flight += 1;
                if (in_flight > st.peak_in_flight) st.peak_in_flight = in_flight;
                st.steps++;
                lk.unlock();
                const qc_status status = launch(*free_slot, rs);
                lk.lock();
                if (status != QC_OK) {
                    if (free_slot->launch) {
                        cudaStreamSynchronize(free_slot->stream);
                        qc_cta_launch_free(free_slot->launch);
                        free_slot->launch = nullptr;
                    }
                    for (Req *r : rs) finish(r, RState::Failed, status);
                    free_slot->reqs.clear();
                    free_slot->busy = false;
                    in_flight -= 1;
                }
                continue;
            }
            if (stop && queue.empty() && pending.empty() && in_flight == 0) break;
            cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }

    void large_worker(int idx) {
        cudaStream_t large_stream = large_streams[idx];
        cudaSetDevice(ctx->device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            if (large_queue.empty()) {
                if (stop && queue.empty() && pending.empty() && in_flight == 0) break;
                cv_large.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
            Req *r = large_queue.front();
            large_queue.pop_front();
            if (r->cancel) {
                finish(r, RState::Cancelled, QC_ERR_CANCELLED);
                continue;
            }
            r->t_start = Clock::now();
            large_running += 1;
            // this request's persistent kernels fill large_share of the SMs, or that share
            // split among the large requests running now
            qc_thread_sm_share = divide_share ? large_share / (float)large_running : large_share;
            lk.unlock();
            qc_status status = QC_OK;
            if (!r->borrowed) {
                if (r->g) {
                    qc_graph_destroy(r->g);
                    r->g = nullptr;
                }
                // large requests are validated here, on the device (see qc_server_submit)
                status = qc_graph_create(ctx, r->n, r->nnz, r->rp.data(), r->nnz ? r->ci.data() : nullptr,
                                         QC_VALIDATE, large_stream, &r->g);
            }
            if (status == QC_OK && !r->labels_dev.ptr)
                status = r->labels_dev.allocate(ctx, sizeof(int32_t) * (size_t)r->n, large_stream);
            int32_t nc = 0;
            if (status == QC_OK) {
                // a resident graph may carry several requests: one solve on it at a time
                // (its cached histogram serves every sigma after the first)
                std::lock_guard<std::mutex> glk(r->g->use_mu);
                status = qc_solve(r->g, &r->sigma, 1, nullptr, r->labels_dev.as<int32_t>(), &nc, large_stream);
            }
            std::vector<int32_t> host;
            if (status == QC_OK) {
                host.resize(r->n);
                if (cudaMemcpy(host.data(), r->labels_dev.ptr, sizeof(int32_t) * r->n, cudaMemcpyDeviceToHost) !=
                    cudaSuccess)
                    status = QC_ERR_CUDA;
            }
            lk.lock();
            large_running -= 1;
            st.large_solved++;
            if (status == QC_OK) {
                r->labels.swap(host);
                r->n_clusters = nc;
                r->batch_size = 0;
                finish(r, r->cancel ? RState::Cancelled : RState::Done, r->cancel ? QC_ERR_CANCELLED : QC_OK);
            } else {
                finish(r, RState::Failed, status);
            }
        }
    }

    void fill(Req *r, int32_t *labels_out, int32_t *n_clusters, qc_request_info *info) {
        if (labels_out && r->state == RState::Done) memcpy(labels_out, r->labels.data(), sizeof(int32_t) * r->n);
        if (n_clusters) *n_clusters = r->n_clusters;
        if (info) {
            info->admit_ms = r->state == RState::Cancelled && r->t_admit.time_since_epoch().count() == 0
                                 ? -1.0
                                 : std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
            info->start_ms = r->t_start.time_since_epoch().count() == 0
                                 ? -1.0
                                 : std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
            info->done_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
            info->n = r->n;
            info->nnz = r->nnz;
            info->batch_size = r->batch_size;
        }
    }
};

extern "C" {

qc_status qc_server_create(qc_ctx *ctx, const qc_server_config *cfg, qc_server **out) {
    if (!ctx || !out) return QC_ERR_INVALID_ARG;
    *out = nullptr;
    auto s = std::make_unique<qc_server>();
    s->ctx = ctx;
    s->budget = (cfg && cfg->mem_budget_bytes) ? cfg->mem_budget_bytes
                                               : (ctx->budget ? ctx->budget : (size_t)100 << 30);
    s->max_active = (cfg && cfg->max_active > 0) ? cfg->max_active : 256;
    const int ns = (cfg && cfg->streams > 0) ? cfg->streams : 4;
    // defaults from measurement on the Poisson mix of 64..65536-node graphs: four
    // workers at 40% of the SMs each beat one worker on the whole GPU (a large
    // request is bound by its per-level steps, not by SMs)
    const int nl = (cfg && cfg->large_workers > 0) ? cfg->large_workers : 4;
    const float share = (cfg && cfg->large_sm_share > 0.f && cfg->large_sm_share <= 1.f) ? cfg->large_sm_share
                                                                                          : 0.4f;
    s->saved_share = ctx->coop_sm_share.load();
    ctx->coop_sm_share = share;
    s->large_share = share;
    s->divide_share = cfg && cfg->divide_share;
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    // batched launches of small requests first: highest stream priority
    int prio_low = 0, prio_high = 0;
    QC_CUDA_TRY(ctx, cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    s->prio_low = prio_low;
    s->prio_high = prio_high;
    s->slots.resize(ns);
    for (Slot &sl : s->slots) QC_CUDA_TRY(ctx, qc_stream_acquire(ctx, prio_high, &sl.stream));
    s->large_streams.resize(nl);
    for (cudaStream_t &ls : s->large_streams) QC_CUDA_TRY(ctx, qc_stream_acquire(ctx, prio_low, &ls));
    qc_server *raw = s.get();
    s->sched = std::thread([raw] { raw->scheduler(); });
    for (int i = 0; i < (int)s->large_streams.size(); ++i)
        s->large.emplace_back([raw, i] { raw->large_worker(i); });
    *out = s.release();
    return QC_OK;
}

qc_status qc_server_submit(qc_server *s, int32_t n, int64_t nnz, const int32_t *row_ptr,
                           const int32_t *col_idx, double sigma, uint64_t *req_id) {
    if (!s || !req_id || n < 1 || nnz < 0 || nnz >= (int64_t(1) << 31) || !row_ptr || (nnz > 0 && !col_idx) ||
        !qc_sigma_ok(sigma))
        return QC_ERR_INVALID_ARG;
    // row_ptr on the host always; the whole CSR on the host for requests the
    // batched kernel takes, on the device (by the worker) for the others
    if (row_ptr[0] != 0 || row_ptr[n] != nnz) return QC_ERR_INVALID_GRAPH;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return QC_ERR_INVALID_GRAPH;
    if (n <= qc_cta_max_nodes()) QC_TRY(validate_host_csr(n, nnz, row_ptr, col_idx));
    auto r = std::make_unique<Req>();
    r->n = n;
    r->nnz = nnz;
    r->rp.assign(row_ptr, row_ptr + n + 1);
    r->ci.assign(col_idx, col_idx + nnz);
    r->sigma = sigma;
    r->large = n > qc_cta_max_nodes();
    r->bytes = s->estimate(n, nnz, r->large);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->bytes > s->budget || s->stop) {
        qc_set_error(s->ctx, "request of %zu estimated bytes exceeds the serving budget of %zu", r->bytes,
                     s->budget);
        return QC_ERR_BUDGET;
    }
    r->id = s->next_id++;
    *req_id = r->id;
    s->queue.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
    s->st.submitted++;
    s->cv.notify_all();
    return QC_OK;
}

qc_status qc_server_submit_graph(qc_server *s, qc_graph *g, double sigma, uint64_t *req_id) {
    if (!s || !g || !req_id || !qc_sigma_ok(sigma)) return QC_ERR_INVALID_ARG;
    if (g->ctx != s->ctx) {
        qc_set_error(s->ctx, "qc_server_submit_graph: the graph belongs to another context");
        return QC_ERR_INVALID_ARG;
    }
    auto r = std::make_unique<Req>();
    r->n = g->n;
    r->nnz = g->nnz;
    r->g = g;
    r->borrowed = true;
    r->sigma = sigma;
    r->large = g->n > qc_cta_max_nodes();
    // the CSR is resident already: only the request's scratch counts
    r->bytes = s->estimate(g->n, g->nnz, r->large) - (4 * ((size_t)g->n + 1) + 4 * (size_t)g->nnz);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->bytes > s->budget || s->stop) {
        qc_set_error(s->ctx, "request of %zu estimated bytes exceeds the serving budget of %zu", r->bytes,
                     s->budget);
        return QC_ERR_BUDGET;
    }
    r->id = s->next_id++;
    *req_id = r->id;
    s->queue.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
    s->st.submitted++;
    s->cv.notify_all();
    return QC_OK;
}

qc_status qc_server_poll(qc_server *s, uint64_t req_id, int32_t *labels_out, int32_t *n_clusters,
                         qc_request_info *info, int *done) {
    if (!s || !done) return QC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return QC_ERR_INVALID_ARG;
    Req *r = it->second.get();
    if (r->state == RState::Queued || r->state == RState::Active) {
        *done = 0;
        return QC_OK;
    }
    *done = 1;
    s->fill(r, labels_out, n_clusters, info);
    const qc_status status = r->status;
    s->reqs.erase(it);
    return status;
}

qc_status qc_server_wait(qc_server *s, uint64_t req_id, int64_t timeout_ms, int32_t *labels_out,
                         int32_t *n_clusters, qc_request_info *info) {
    if (!s) return QC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return QC_ERR_INVALID_ARG;
    Req *r = it->second.get();
    auto ready = [&] { return r->state != RState::Queued && r->state != RState::Active; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return QC_ERR_NOT_READY;
    s->fill(r, labels_out, n_clusters, info);
    const qc_status status = r->status;
    s->reqs.erase(r->id);
    return status;
}

qc_status qc_server_cancel(qc_server *s, uint64_t req_id) {
    if (!s) return QC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return QC_ERR_INVALID_ARG;
    it->second->cancel = true;
    s->cv.notify_all();
    return QC_OK;
}

qc_status qc_server_get_stats(qc_server *s, qc_server_stats *out) {
    if (!s || !out) return QC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->bytes_resident = s->resident;
    out->active = s->active;
    out->queued = (int32_t)s->queue.size();
    return QC_OK;
}

void qc_server_destroy(qc_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Req *r : s->queue) r->cancel = true;
        s->cv.notify_all();
        s->cv_large.notify_all();
    }
    if (s->sched.joinable()) s->sched.join();
    for (std::thread &t : s->large)
        if (t.joinable()) t.join();
    // requests' memory is given back on the streams it was allocated on; those stay
    // with the context, which also keeps them for graphs the caller lent
    for (Slot &sl : s->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (cudaStream_t ls : s->large_streams)
        if (ls) cudaStreamSynchronize(ls);
    for (auto &kv : s->reqs) {
        Req *r = kv.second.get();
        if (r->g && !r->borrowed) qc_graph_destroy(r->g);
        r->g = nullptr;
        r->labels_dev.release();
    }
    for (Slot &sl : s->slots) {
        if (sl.launch) qc_cta_launch_free(sl.launch);
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            qc_stream_release(s->ctx, sl.stream, s->prio_high);
        }
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    for (cudaStream_t ls : s->large_streams)
        if (ls) {
            cudaStreamSynchronize(ls);
            qc_stream_release(s->ctx, ls, s->prio_low);
        }
    s->ctx->coop_sm_share = s->saved_share;
    delete s;
}

}  // extern "C"
