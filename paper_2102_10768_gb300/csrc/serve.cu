// Serving: a request loop over a resident data graph with continuous
// batching.
//
// Requests enter a FIFO queue.  Worker threads, each with its own CUDA
// stream, take the head request as soon as they are free and the request's
// projected device bytes fit in what the budget has left (admission); they
// build its CST (Alg. 1), partition it (Alg. 2) and launch the matcher on
// their own stream.  Requests that arrive while others run are admitted as
// workers and memory free up, and their kernels overlap on the device with
// the ones already running (each matcher launch takes a share of the SMs, so
// several run at once).  Every result carries its arrival, start and finish
// times on one steady clock, from which the caller reads latency.
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

void worker_main(fast_server* S, int w) {
    cudaSetDevice(S->device);
    cudaStream_t st = S->streams[w];
    for (;;) {
        Req r;
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
            if (S->pending.empty()) continue;
            r = std::move(S->pending.front());
            S->pending.pop_front();
            if (r.projected > S->budget) {
                fast_result res;
                memset(&res, 0, sizeof(res));
                res.id = r.id; res.status = FAST_ERR_OOM;
                res.t_arrive_ns = r.t_arrive; res.t_start_ns = res.t_done_ns = now_ns();
                S->done.push_back(res);
                S->cv.notify_all();
                continue;
            }
            S->in_use += r.projected;
            S->running++;
        }
        fast_result res;
        memset(&res, 0, sizeof(res));
        res.id = r.id;
        res.t_arrive_ns = r.t_arrive;
        res.t_start_ns = now_ns();
        fast_query_desc q;
        q.n = (int32_t)r.labels.size();
        q.m = (int32_t)(r.edges.size() / 2);
        q.labels = r.labels.data();
        q.edges = r.edges.data();
        fast_cst* c = nullptr;
        fast_chunks* ch = nullptr;
        uint64_t count = 0;
        int rc = fast_build_cst(S->g, &q, &S->cfg, st, &c);
        if (rc == FAST_OK) rc = fast_partition(c, &S->cfg, st, &ch);
        if (rc == FAST_OK) rc = fast_match_ex(c, ch, &S->cfg, 0, nullptr, &count, nullptr, nullptr, st);
        if (ch) fast_free_chunks(ch);
        if (c) fast_free_cst(c);
        res.count = count;
        res.status = rc;
        res.t_done_ns = now_ns();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= r.projected;
            S->running--;
            S->done.push_back(res);
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
    S->streams.resize(W);
    for (auto& st : S->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto x : S->streams) if (x) cudaStreamDestroy(x);
            delete S;
            return set_error(FAST_ERR_CUDA, "fast_server_create: stream");
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

extern "C" void fast_server_destroy(fast_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto st : S->streams) cudaStreamDestroy(st);
    delete S;
}
