// Serving: a request loop over a resident data graph with continuous
// batching.
//
// Requests enter a FIFO queue.  Each of a few group workers, with its own
// CUDA stream and its own batch (fixed device buffers and a captured matcher
// launch, batch.cu), repeatedly takes every request at the head of the queue
// whose projected device bytes still fit in what the budget has left
// (admission), up to a group cap, and runs them as one batch: their CSTs
// (Alg. 1) and partitions (Alg. 2) are built together and one matcher launch
// enumerates all of their chunks, warps stealing work across the requests.
// Requests that arrive while a group is on the GPU form the next group and
// are admitted as soon as a worker and memory free up; with two or more
// workers one group's build overlaps another's matcher on the device.  At
// low load a group is a single request, which then has the whole GPU; under
// load the groups grow and the loop reaches the batched throughput.  Every
// result carries its arrival, admission and finish times on one steady
// clock, from which the caller reads latency.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

using namespace fast;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id = 0;
    std::vector<int32_t> labels, edges;
    uint64_t t_arrive = 0;
    uint64_t projected = 0;
};

}  // namespace

struct fast_server {
    const fast_graph* g = nullptr;
    fast_config cfg;
    uint64_t budget = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> pending;
    std::vector<fast_result> done;
    uint64_t next_id = 1;
    uint64_t in_use = 0;
    int running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::vector<fast_batch*> batches;    // one per worker: a group's buffers and captured launch
    int group_cap = 1024;                // requests per group
    uint64_t groups = 0, grouped = 0;    // groups formed, requests in them
    std::vector<double> label_deg;       // mean degree of the vertices of each label
};

namespace {

// Projected device bytes of a query's CST: for every query vertex, its label
// bucket (candidate ids, two bitmaps with ranks over V(G)); for every query
// edge, the neighbour lists of the bucket of one end (the top-down and
// non-tree lists are at most that), and the matcher's fixed scratch.  The
// query is not validated yet (its build does that and reports a malformed
// query in the result's status), so labels outside G's range count as empty
// buckets and edges with an endpoint outside the query are skipped.
uint64_t projected_bytes(const fast_server* S, const Req& r) {
    const fast_graph* g = S->g;
    const int k = (int)r.labels.size();
    double b = 16.0 * 1024 * 1024;               // matcher counters, queue, chunk lists
    auto known = [&](int32_t l) { return l >= 0 && l < g->num_labels; };
    auto bucket = [&](int32_t l) -> double {
        return known(l) ? (double)(g->lab_ptr_host[l + 1] - g->lab_ptr_host[l]) : 0.0;
    };
    auto lists = [&](int32_t l) -> double { return known(l) ? S->label_deg[l] * bucket(l) : 0.0; };
    for (int u = 0; u < k; u++) b += 4.0 * bucket(r.labels[u]) + 2.0 * (double)g->n / 8.0 + 8.0 * bucket(r.labels[u]);
    for (size_t e = 0; e + 1 < r.edges.size(); e += 2) {
        int32_t a = r.edges[e], c = r.edges[e + 1];
        if (a < 0 || a >= k || c < 0 || c >= k) continue;
        int32_t la = r.labels[a], lb = r.labels[c];
        b += 4.0 * std::max(lists(la), lists(lb)) + 12.0 * (bucket(la) + bucket(lb));
    }
    return (uint64_t)b;
}

constexpr int kSmallGroup = 4;           // requests: at most this many run on one CTA per SM

// One group worker: take the admissible head of the queue, run it as one
// batch, report every request of it.
void worker_main(fast_server* S, int w) {
    cudaSetDevice(S->device);
    cudaStream_t st = S->streams[w];
    fast_batch* b = S->batches[w];
    std::vector<Req> grp;
    std::vector<fast_query_desc> qd;
    std::vector<uint64_t> counts;
    std::vector<int32_t> status;
    for (;;) {
        grp.clear();
        uint64_t t_start = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] {
                if (S->stop) return true;
                if (S->pending.empty()) return false;
                const Req& h = S->pending.front();
                return S->running == 0 || h.projected <= S->budget - std::min(S->budget, S->in_use) ||
                       h.projected > S->budget;
            });
            if (S->stop) return;                 // requests not yet started are dropped
            t_start = now_ns();
            // the admissible head of the queue, in order: a request beyond the
            // whole budget is answered at once; the group stops at the first
            // request that does not fit in what is left (FIFO), or at the cap
            while (!S->pending.empty() && (int)grp.size() < S->group_cap) {
                Req& h = S->pending.front();
                if (h.projected > S->budget) {
                    fast_result res;
                    memset(&res, 0, sizeof(res));
                    res.id = h.id; res.status = FAST_ERR_OOM;
                    res.t_arrive_ns = h.t_arrive; res.t_start_ns = res.t_done_ns = now_ns();
                    S->done.push_back(res);
                    S->pending.pop_front();
                    continue;
                }
                const bool idle = S->running == 0 && grp.empty();
                if (!idle && h.projected > S->budget - std::min(S->budget, S->in_use)) break;
                S->in_use += h.projected;
                S->running++;
                grp.push_back(std::move(h));
                S->pending.pop_front();
            }
            if (!grp.empty()) { S->groups++; S->grouped += grp.size(); }
        }
        S->cv.notify_all();
        if (grp.empty()) continue;
        const int n = (int)grp.size();
        qd.resize(n);
        counts.assign(n, 0);
        status.assign(n, FAST_OK);
        for (int i = 0; i < n; i++) {
            qd[i].n = (int32_t)grp[i].labels.size();
            qd[i].m = (int32_t)(grp[i].edges.size() / 2);
            qd[i].labels = grp[i].labels.data();
            qd[i].edges = grp[i].edges.data();
        }
        // a small group's matcher launch takes one CTA per SM, leaving room on
        // every SM for the other workers' kernels; a large group takes the
        // configured shape
        {
            fast_config lc;
            fast_batch_config(b, 4, &lc, nullptr);
            const int32_t bps = n <= kSmallGroup ? 1 : S->cfg.blocks_per_sm;
            if (lc.blocks_per_sm != bps) {
                lc.blocks_per_sm = bps;
                fast_batch_config(b, 4, nullptr, &lc);
            }
        }
        int rc = fast_batch_run(b, n, qd.data(), counts.data(), status.data(), st);
        const uint64_t t_done = now_ns();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (int i = 0; i < n; i++) {
                fast_result res;
                memset(&res, 0, sizeof(res));
                res.id = grp[i].id;
                res.t_arrive_ns = grp[i].t_arrive;
                res.t_start_ns = t_start;
                res.t_done_ns = t_done;
                res.count = rc == FAST_OK ? counts[i] : 0;
                res.status = rc == FAST_OK ? status[i] : rc;
                S->in_use -= grp[i].projected;
                S->running--;
                S->done.push_back(res);
            }
        }
        S->cv.notify_all();
    }
}

__global__ void k_label_degree(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ label, int64_t n,
                               unsigned long long* __restrict__ sum) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) atomicAdd(&sum[label[v]], (unsigned long long)(row_ptr[v + 1] - row_ptr[v]));
}

}  // namespace

extern "C" uint64_t fast_now_ns(void) { return now_ns(); }

extern "C" int fast_server_create(const fast_graph* g, const fast_config* cfg, uint64_t budget_bytes, int32_t workers,
                                  fast_server** out) {
    if (!out) return set_error(FAST_ERR_INVALID, "fast_server_create: out is NULL");
    *out = nullptr;
    if (!g || budget_bytes == 0) return set_error(FAST_ERR_INVALID, "fast_server_create: bad graph or budget");
    fast_server* S = new fast_server();
    S->g = g;
    if (cfg) S->cfg = *cfg; else fast_config_default(&S->cfg);
    S->budget = budget_bytes;
    cudaGetDevice(&S->device);
    int W = workers > 0 ? workers : 4;
    // mean degree per label, for the admission estimate
    unsigned long long* sum = nullptr;
    cudaStream_t s0 = nullptr;
    int rc = dalloc(&sum, g->num_labels, s0);
    if (rc == FAST_OK) {
        cudaMemsetAsync(sum, 0, g->num_labels * sizeof(unsigned long long), s0);
        k_label_degree<<<(unsigned)ceil_div(g->n, 256), 256, 0, s0>>>(g->row_ptr, g->label, g->n, sum);
        note_launch();
        std::vector<unsigned long long> h(g->num_labels);
        cudaMemcpyAsync(h.data(), sum, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s0);
        cudaError_t e = cudaStreamSynchronize(s0);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_server_create", __FILE__, __LINE__);
        S->label_deg.resize(g->num_labels);
        for (int l = 0; l < g->num_labels; l++) {
            double cnt = (double)(g->lab_ptr_host[l + 1] - g->lab_ptr_host[l]);
            S->label_deg[l] = cnt > 0 ? (double)h[l] / cnt : 0.0;
        }
    }
    dfree(sum, s0);
    cudaStreamSynchronize(s0);
    if (rc != FAST_OK) { delete S; return rc; }
    S->streams.assign(W, nullptr);
    S->batches.assign(W, nullptr);
    for (int w = 0; w < W && rc == FAST_OK; w++) {
        if (cudaStreamCreateWithFlags(&S->streams[w], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(FAST_ERR_CUDA, "fast_server_create: stream");
            break;
        }
        rc = fast_batch_create(g, &S->cfg, S->group_cap, 0, &S->batches[w]);
    }
    if (rc != FAST_OK) {
        for (auto x : S->batches) if (x) fast_free_batch(x);
        for (auto x : S->streams) if (x) cudaStreamDestroy(x);
        delete S;
        return rc;
    }
    for (int w = 0; w < W; w++) S->workers.emplace_back(worker_main, S, w);
    *out = S;
    return FAST_OK;
}

extern "C" int fast_server_submit(fast_server* S, const fast_query_desc* q, uint64_t* id_out) {
    if (!S || !q || q->n < 1 || q->n > FAST_MAX_QUERY || !q->labels || (q->m > 0 && !q->edges) || q->m < 0)
        return set_error(FAST_ERR_INVALID, "fast_server_submit: bad query");
    Req r;
    r.labels.assign(q->labels, q->labels + q->n);
    r.edges.assign(q->edges, q->edges + 2 * q->m);
    r.t_arrive = now_ns();
    r.projected = projected_bytes(S, r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r.id = S->next_id++;
        if (id_out) *id_out = r.id;
        S->pending.push_back(std::move(r));
    }
    S->cv.notify_all();
    return FAST_OK;
}

extern "C" int fast_server_poll(fast_server* S, int32_t max_results, fast_result* out, int32_t* n_out,
                                int32_t wait_ms) {
    if (!S || !n_out || max_results < 0 || (max_results > 0 && !out))
        return set_error(FAST_ERR_INVALID, "fast_server_poll: bad arguments");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
    int n = std::min<int>(max_results, (int)S->done.size());
    for (int i = 0; i < n; i++) out[i] = S->done[i];
    S->done.erase(S->done.begin(), S->done.begin() + n);
    *n_out = n;
    return FAST_OK;
}

extern "C" int fast_server_stats(fast_server* S, int64_t* pending, int64_t* running, uint64_t* in_use_bytes) {
    if (!S) return set_error(FAST_ERR_INVALID, "fast_server_stats: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (pending) *pending = (int64_t)S->pending.size();
    if (running) *running = S->running;
    if (in_use_bytes) *in_use_bytes = S->in_use;
    return FAST_OK;
}

extern "C" int fast_server_groups(fast_server* S, uint64_t* groups, uint64_t* requests) {
    if (!S) return set_error(FAST_ERR_INVALID, "fast_server_groups: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (groups) *groups = S->groups;
    if (requests) *requests = S->grouped;
    return FAST_OK;
}

extern "C" void fast_server_destroy(fast_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto b : S->batches) fast_free_batch(b);
    for (auto st : S->streams) cudaStreamDestroy(st);
    delete S;
}
