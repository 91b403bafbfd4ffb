// Serving loop for k-clique queries on resident graphs (include/kcl.h,
// kcl_server_*).  The paper has no serving layer; this is the library's
// request loop:
//   - graphs stay resident on the device (the caller's loaded handles);
//   - `slots` worker threads each own a CUDA stream, a view (their own
//     scratch on whatever graph a query names) and a batch context, so the
//     work of concurrently admitted queries overlaps on the GPU;
//   - a query is admitted when its scratch estimate fits in the remaining
//     budget (a query larger than the whole budget runs alone);
//   - continuous batching: when a worker frees up it takes the oldest query;
//     queries on small graphs are gathered with the other queued small-graph
//     queries into one batched pass (disjoint union, kcl_count_batch), and
//     queued duplicates of the query it picks share its result.
// Results are exact and identical to the same query run alone.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "kcl_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t ticket;
    kcl_graph *g;  // resolved under the lock at submission; the graph table may grow later
    uint32_t graph, k;
    kcl_ordering ord;
    int list;
    uint64_t scratch;
    double submit_s;
};

struct Slot {
    kcl_graph *view = nullptr;   // retargeted to the graph of each single query
    kcl_batch *batch = nullptr;
    cudaStream_t stream = nullptr;
    std::thread thread;
};

}  // namespace

struct kcl_server {
    int device = 0;
    int num_sms = 0;
    uint64_t budget = 0, in_use = 0;
    uint64_t small_nnz = 0;       // graphs with at most this many CSR entries are batched
    uint32_t max_batch = 64;
    std::atomic<uint64_t> time_limit_ms{0};  // per pass (kcl_server_set_time_limit; 0 = none)
    std::vector<kcl_graph *> graphs;
    std::vector<Slot> slots;
    std::deque<Job> queue;
    std::vector<kcl_server_result> results;  // by ticket
    std::vector<uint8_t> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint32_t running = 0;
    Clock::time_point t0;
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Device scratch a query may need: the per-call workspace (about 70 bytes
// per vertex and 2 per CSR entry) plus the listing kernels' arena bound.
uint64_t scratch_estimate(const kcl_server *s, const kcl_graph *g, uint32_t k) {
    uint64_t ws = 72ull * ((uint64_t)g->n + 1) + 2ull * g->nnz + (1u << 20);
    uint64_t arena = 4ull * std::max(kcl::bitcol_arena_words(k, s->num_sms, g->max_deg),
                                     kcl::sdegree_arena_words(k, s->num_sms, g->max_deg));
    return ws + arena;
}

void finish(kcl_server *s, const Job &j, kcl_status st, uint64_t count, uint64_t cks, double start,
            double end, uint32_t batch) {
    kcl_server_result &r = s->results[j.ticket];
    r.status = st;
    r.count = count;
    r.checksum = j.list ? cks : 0;
    r.submit_s = j.submit_s;
    r.start_s = start;
    r.done_s = end;
    r.batch = batch;
    s->done[j.ticket] = 1;
}

void worker(kcl_server *s, Slot *slot) {
    cudaSetDevice(s->device);
    std::vector<Job> group;
    std::vector<kcl_graph *> gs;
    std::vector<uint32_t> ks;
    std::vector<kcl_ordering> ords;
    std::vector<uint64_t> counts, cks;
    for (;;) {
        group.clear();
        uint64_t scratch = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stop && s->queue.empty()) return;
                if (!s->queue.empty()) {
                    const Job &head = s->queue.front();
                    bool fits = s->in_use + head.scratch <= s->budget || s->running == 0;
                    if (fits) break;
                }
                s->cv_work.wait(lk);
            }
            Job head = s->queue.front();
            s->queue.pop_front();
            group.push_back(head);
            scratch = head.scratch;
            const bool small = head.g->nnz <= s->small_nnz;
            // gather: other small-graph queries (batch), or duplicates of head
            for (auto it = s->queue.begin(); it != s->queue.end() && group.size() < s->max_batch;) {
                bool dup = it->graph == head.graph && it->k == head.k && it->ord == head.ord &&
                           it->list == head.list;
                bool take = dup || (small && it->g->nnz <= s->small_nnz &&
                                    s->in_use + scratch + it->scratch <= s->budget);
                if (take) {
                    if (!dup) scratch += it->scratch;
                    group.push_back(*it);
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
            s->in_use += scratch;
            s->running++;
        }
        const double start = s->now();
        const Job &head = group[0];
        bool all_dups = true;
        for (const Job &j : group)
            all_dups = all_dups && j.graph == head.graph && j.k == head.k && j.ord == head.ord &&
                       j.list == head.list;
        std::vector<kcl_status> sts(group.size(), KCL_OK);
        counts.assign(group.size(), 0);
        cks.assign(group.size(), 0);
        const uint64_t limit = s->time_limit_ms.load();
        if (all_dups) {
            // one single call answers every copy
            kcl_graph *g = head.g;
            kcl_graph *v = slot->view;
            v->n = g->n;
            v->nnz = g->nnz;
            v->rp = g->rp;
            v->col = g->col;
            v->max_deg = g->max_deg;
            v->time_limit_ms = limit;
            uint64_t c = 0, h = 0, w = 0;
            kcl_status st = head.list ? kcl_list(v, head.k, head.ord, nullptr, &c, &h, &w)
                                      : kcl_count(v, head.k, head.ord, &c);
            for (size_t i = 0; i < group.size(); i++) { sts[i] = st; counts[i] = c; cks[i] = h; }
        } else {
            gs.clear(); ks.clear(); ords.clear();
            bool any_list = false;
            for (const Job &j : group) {
                gs.push_back(j.g);
                ks.push_back(j.k);
                ords.push_back(j.ord);
                any_list = any_list || j.list;
            }
            // a batched pass answers group.size() queries: each keeps its own share
            kcl_batch_set_time_limit(slot->batch, limit * group.size());
            kcl_status st = kcl_count_batch(slot->batch, gs.data(), ks.data(), ords.data(),
                                            (uint32_t)gs.size(), counts.data(),
                                            any_list ? cks.data() : nullptr);
            for (size_t i = 0; i < group.size(); i++) sts[i] = st;
        }
        const double end = s->now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < group.size(); i++)
                finish(s, group[i], sts[i], counts[i], cks[i], start, end, (uint32_t)group.size());
            s->in_use -= scratch;
            s->running--;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

kcl_status kcl_server_create(uint32_t slots, uint64_t scratch_budget_bytes, uint64_t small_nnz,
                             kcl_server **out) {
    if (!out || slots == 0 || slots > 256) return KCL_EINVAL;
    *out = nullptr;
    kcl_server *s = new (std::nothrow) kcl_server();
    if (!s) return KCL_ENOMEM;
    s->budget = scratch_budget_bytes;
    s->small_nnz = small_nnz;
    s->t0 = Clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete s;
        return KCL_ECUDA;
    }
    s->slots.resize(slots);
    for (Slot &sl : s->slots) {
        kcl_status st = KCL_OK;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) st = KCL_ECUDA;
        if (st == KCL_OK) {
            sl.view = new (std::nothrow) kcl_graph();
            if (!sl.view) st = KCL_ENOMEM;
        }
        if (st == KCL_OK) {
            sl.view->device = s->device;
            sl.view->num_sms = s->num_sms;
            sl.view->stream = sl.stream;
            sl.view->owns_csr = false;
            st = kcl_batch_create(sl.stream, &sl.batch);
        }
        if (st != KCL_OK) {
            (void)cudaGetLastError();
            kcl_server_destroy(s);
            return st;
        }
    }
    for (Slot &sl : s->slots) sl.thread = std::thread(worker, s, &sl);
    *out = s;
    return KCL_OK;
}

kcl_status kcl_server_add_graph(kcl_server *s, kcl_graph *g, uint32_t *id) {
    if (!s || !g || !id || g->device != s->device) return KCL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *id = (uint32_t)s->graphs.size();
    s->graphs.push_back(g);
    return KCL_OK;
}

kcl_status kcl_server_submit(kcl_server *s, uint32_t graph, uint32_t k, kcl_ordering ord, int list,
                             uint64_t *ticket) {
    if (!s || !ticket) return KCL_EINVAL;
    if (k < 3 || k > KCL_MAX_K || (ord != KCL_ORDER_DEGREE && ord != KCL_ORDER_COLOR)) return KCL_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (graph >= s->graphs.size() || s->stop) return KCL_EINVAL;
        Job j;
        j.ticket = s->results.size();
        j.g = s->graphs[graph];
        j.graph = graph;
        j.k = k;
        j.ord = ord;
        j.list = list ? 1 : 0;
        j.scratch = scratch_estimate(s, s->graphs[graph], k);
        j.submit_s = s->now();
        s->results.push_back(kcl_server_result());
        s->done.push_back(0);
        s->queue.push_back(j);
        *ticket = j.ticket;
    }
    s->cv_work.notify_one();
    return KCL_OK;
}

kcl_status kcl_server_poll(kcl_server *s, uint64_t ticket, int *done, kcl_server_result *out) {
    if (!s || !done) return KCL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket >= s->results.size()) return KCL_EINVAL;
    *done = s->done[ticket];
    if (*done && out) *out = s->results[ticket];
    return KCL_OK;
}

kcl_status kcl_server_wait(kcl_server *s, uint64_t ticket, kcl_server_result *out) {
    if (!s) return KCL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket >= s->results.size()) return KCL_EINVAL;
    s->cv_done.wait(lk, [&] { return s->done[ticket] != 0; });
    if (out) *out = s->results[ticket];
    return KCL_OK;
}

double kcl_server_clock(const kcl_server *s) { return s ? s->now() : 0.0; }

kcl_status kcl_server_set_time_limit(kcl_server *s, uint64_t ms) {
    if (!s) return KCL_EINVAL;
    s->time_limit_ms.store(ms);
    return KCL_OK;
}

void kcl_server_destroy(kcl_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (Slot &sl : s->slots)
        if (sl.thread.joinable()) sl.thread.join();
    for (Slot &sl : s->slots) {
        if (sl.batch) kcl_batch_free(sl.batch);
        if (sl.view) kcl_free_graph(sl.view);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    (void)cudaGetLastError();
    delete s;
}

}  // extern "C"
