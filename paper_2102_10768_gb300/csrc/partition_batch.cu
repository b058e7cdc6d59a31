// Batched CST partition (Sec. IV-B, Algorithm 2): the partitions of many
// queries' CSTs built together, level by level.
//
// The pending parts of all queries are one item array, grouped by query in
// query order (query q owns items qoff[q] .. qoff[q+1]-1); each kernel finds
// an item's query by binary search and applies that query's plan, with the
// same device helpers (part_funcs.cuh) as the per-query partition.  A level
// is one count pass over all items, global exclusive scans, one kernel that
// gathers each query's totals, and one host round trip for the whole batch;
// a second pass runs only when some query's level would pass its
// max_chunks, with that query's split cap (the other queries' counts do not
// change).  Then the finished chunks are written and the parts of the next
// level are summed, still grouped by query.  A query whose level hit its cap
// keeps that level's parts as its last chunks and goes inactive; its items
// stay in place and every later kernel skips them.  At the end one copy
// kernel gathers each query's chunk list, level by level, into its own
// exact-size array -- the same list, in the same order, as fast_partition
// gives.
#include <algorithm>
#include <cstring>
#include <vector>

#include "cst_funcs.cuh"
#include "internal.cuh"
#include "part_funcs.cuh"
#include "seg.cuh"

using namespace fast;

namespace {

// item t -> its query (the last q with qoff[q] <= t)
__device__ __forceinline__ int query_of(const int64_t* __restrict__ qoff, int nq, int64_t t) {
    return seg_of_tile(qoff, nq, t);
}

// per query: split cap of this pass (0: none), |C(root)|, and whether it
// still partitions
struct QState {
    uint64_t kcap;
    uint32_t root_n;
    int32_t active;
};

// one thread per pending item: classify and count the kept parts (as
// k_part_count, with the item's plan)
__global__ void k_part_count_b(const PartPlan* __restrict__ plans, const QState* __restrict__ qs,
                               const int64_t* __restrict__ qoff, int nq, Chunk* __restrict__ items, int64_t nitems,
                               int64_t* __restrict__ nparts, int64_t* __restrict__ nemit,
                               int64_t* __restrict__ nlive) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems) return;
    const int q = query_of(qoff, nq, t);
    if (!qs[q].active) { nparts[t] = 0; nemit[t] = 0; nlive[t] = 0; return; }
    const PartPlan& P = plans[q];
    const uint64_t kcap = qs[q].kcap;
    Chunk c = items[t];
    uint64_t kk = 0;
    int act = classify(P, c, qs[q].root_n, &kk);
    if (kcap && kk > kcap) kk = kcap;
    items[t] = c;
    nlive[t] = act != 0 ? 1 : 0;
    int64_t np = 0;
    if (act == 2) {
        if (!sampled(P)) np = (int64_t)kk;
        else
            for (uint64_t i = 0; i < kk; i++)
                np += keep_part(P, c.j, kk, mix64(c.id + (i + 1) * 0x9E3779B97F4A7C15ull)) ? 1 : 0;
    }
    nparts[t] = np;
    nemit[t] = act == 1 ? 1 : 0;
}

// per query: parts, emitted chunks and live items of its range
__global__ void k_part_totals(const int64_t* __restrict__ part_off, const int64_t* __restrict__ emit_off,
                              const int64_t* __restrict__ live_off, const int64_t* __restrict__ qoff, int nq,
                              int64_t* __restrict__ out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int64_t a = qoff[q], b = qoff[q + 1];
    out[3 * q + 0] = part_off[b] - part_off[a];
    out[3 * q + 1] = emit_off[b] - emit_off[a];
    out[3 * q + 2] = live_off[b] - live_off[a];
}

// one thread per pending item: emitted chunks, and the part records of
// sampled splits (as k_part_write)
__global__ void k_part_write_b(const PartPlan* __restrict__ plans, const QState* __restrict__ qs,
                               const int64_t* __restrict__ qoff, int nq, const Chunk* __restrict__ items,
                               int64_t nitems, const int64_t* __restrict__ part_off,
                               const int64_t* __restrict__ emit_off, PartRec* __restrict__ parts,
                               Chunk* __restrict__ emitted) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems) return;
    const int q = query_of(qoff, nq, t);
    if (!qs[q].active) return;
    const PartPlan& P = plans[q];
    const uint64_t kcap = qs[q].kcap;
    Chunk c = items[t];
    int64_t np = part_off[t + 1] - part_off[t];
    int64_t ne = emit_off[t + 1] - emit_off[t];
    if (ne) emitted[emit_off[t]] = c;
    if (!np || !sampled(P)) return;
    uint32_t n = c.b - c.a;
    uint64_t kk = c.w / P.delta_w + (c.w % P.delta_w != 0);
    if (kk > n) kk = n;
    if (kcap && kk > kcap) kk = kcap;
    uint64_t f = prefix_factor(P, c);
    int64_t o = part_off[t];
    for (uint64_t i = 0; i < kk; i++) {
        uint64_t id = mix64(c.id + (i + 1) * 0x9E3779B97F4A7C15ull);
        if (!keep_part(P, c.j, kk, id)) continue;
        PartRec r;
        r.item = (uint32_t)t;
        r.a = c.a + (uint32_t)((i * (uint64_t)n) / kk);
        r.b = c.a + (uint32_t)(((i + 1) * (uint64_t)n) / kk);
        r.pad = 0;
        r.id = id;
        r.f = f;
        parts[o++] = r;
    }
}

// one warp per part: W' = F * (saturating sum of c over the run), as
// k_part_sum; a part of an unsampled query is derived from its item t (the
// last with part_off[t] <= p) and its index there.
__global__ void k_part_sum_b(const PartPlan* __restrict__ plans, const int64_t* __restrict__ qoff, int nq,
                             const Chunk* __restrict__ items, int64_t nitems, const int64_t* __restrict__ part_off,
                             const PartRec* __restrict__ parts, int64_t nparts, Chunk* __restrict__ next) {
    const int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w; p < nparts; p += nw) {
        int64_t lo = 0, hi = nitems;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (part_off[mid] <= p) lo = mid; else hi = mid;
        }
        const PartPlan& P = plans[query_of(qoff, nq, lo)];
        PartRec r;
        if (parts && sampled(P)) {
            r = parts[p];
        } else {
            const Chunk& c = items[lo];
            uint64_t i = (uint64_t)(p - part_off[lo]);
            uint64_t kk = (uint64_t)(part_off[lo + 1] - part_off[lo]);
            uint64_t n = c.b - c.a;
            r.item = (uint32_t)lo;
            r.a = c.a + (uint32_t)((i * n) / kk);
            r.b = c.a + (uint32_t)(((i + 1) * n) / kk);
            r.pad = 0;
            r.id = mix64(c.id + (i + 1) * 0x9E3779B97F4A7C15ull);
            r.f = prefix_factor(P, c);
        }
        const Chunk& it = items[r.item];
        int j = it.j;
        const uint64_t* cv = P.cval[j];
        uint64_t s = 0;
        if (j == 0) {
            for (uint64_t x = r.a + lane; x < r.b; x += 32) s = sat_add(s, cv[x]);
        } else {
            int64_t base = P.t_off[j][it.prefix[P.par_pos[j]]];
            for (uint64_t x = r.a + lane; x < r.b; x += 32) s = sat_add(s, cv[P.t_idx[j][base + (int64_t)x]]);
        }
        for (int o = 16; o > 0; o >>= 1) s = sat_add(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane < kMaxK) {
            uint32_t* dst = next[p].prefix;
            dst[lane] = lane < j ? it.prefix[lane] : 0u;
        }
        if (lane == 0) {
            next[p].j = j;
            next[p].a = r.a;
            next[p].b = r.b;
            next[p].pad = 0;
            next[p].w = sat_mul(r.f, s);
            next[p].id = r.id;
        }
    }
}

// ------------------------------------------------------------ host side

struct QP {
    const fast_cst* c = nullptr;
    int idx = 0;                               // in the caller's arrays
    fast_config cfg;
    int64_t cap = 0;                           // max_chunks
    int64_t total = 0;                         // chunks so far
    bool active = false;
    bool last = false;                         // this level's parts are its last chunks
    std::vector<std::pair<const Chunk*, int64_t>> pieces;   // its chunk list, in order
};

int fetch_words(const int64_t* d, std::vector<int64_t>& h, size_t words, cudaStream_t s) {
    h.assign(words, 0);
    if (!words) return FAST_OK;
    cudaError_t e = cudaMemcpyAsync(h.data(), d, words * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? FAST_OK : cuda_status(e, "batched partition sizes", __FILE__, __LINE__);
}

template <class T>
int upload_array(const std::vector<T>& h, T** d, std::vector<unsigned char*>& own, cudaStream_t s) {
    FAST_TRY(dalloc(d, std::max<size_t>(h.size(), 1), s));
    own.push_back((unsigned char*)*d);
    if (!h.empty()) FAST_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return FAST_OK;
}

struct Owned {
    explicit Owned(cudaStream_t s) : s_(s) {}
    ~Owned() {
        for (auto p : v) dfree(p, s_);
    }
    std::vector<unsigned char*> v;
    cudaStream_t s_;
};

int partition_all(std::vector<QP>& Q, cudaStream_t s, fast_chunks** outs) {
    const int nq = (int)Q.size();
    Owned keep(s);                              // plans, item and chunk arrays: until the gather
    std::vector<PartPlan> plans(nq);
    std::vector<QState> st(nq);
    std::vector<int64_t> qoff(nq + 1, 0);
    std::vector<Chunk> items0;
    for (int q = 0; q < nq; q++) {
        const fast_cst* c = Q[q].c;
        plans[q] = make_plan(c, &Q[q].cfg);
        const uint32_t root_n = (uint32_t)c->ncand[c->root];
        st[q].kcap = 0;
        st[q].root_n = root_n;
        Q[q].cap = Q[q].cfg.max_chunks > 0 ? Q[q].cfg.max_chunks : (1ll << 16);
        Q[q].active = root_n > 0 && c->W > 0;
        st[q].active = Q[q].active ? 1 : 0;
        if (Q[q].active) {
            Chunk r0;
            memset(&r0, 0, sizeof(r0));
            r0.j = 0; r0.a = 0; r0.b = root_n; r0.w = c->W; r0.id = mix64(Q[q].cfg.sample_seed);
            items0.push_back(r0);
        }
        qoff[q + 1] = qoff[q] + (Q[q].active ? 1 : 0);
    }
    PartPlan* d_plans = nullptr;
    Chunk* items = nullptr;
    FAST_TRY(upload_array(plans, &d_plans, keep.v, s));
    FAST_TRY(upload_array(items0, &items, keep.v, s));
    int64_t nitems = qoff[nq];
    std::vector<int64_t> tot;
    while (nitems > 0) {
        bool any_active = false;
        for (auto& q : Q) any_active = any_active || q.active;
        if (!any_active) break;
        Owned lvl(s);
        for (int q = 0; q < nq; q++) { st[q].kcap = 0; st[q].active = Q[q].active ? 1 : 0; }
        QState* d_st = nullptr;
        int64_t* d_qoff = nullptr;
        FAST_TRY(upload_array(st, &d_st, lvl.v, s));
        FAST_TRY(upload_array(qoff, &d_qoff, lvl.v, s));
        int64_t* cnt = nullptr;
        int64_t* d_tot = nullptr;
        FAST_TRY(dalloc(&cnt, 3 * (nitems + 1), s));
        lvl.v.push_back((unsigned char*)cnt);
        FAST_TRY(dalloc(&d_tot, 3 * (size_t)nq, s));
        lvl.v.push_back((unsigned char*)d_tot);
        int64_t* part_off = cnt;
        int64_t* emit_off = cnt + nitems + 1;
        int64_t* live_off = cnt + 2 * (nitems + 1);
        for (int pass = 0; pass < 2; pass++) {
            k_part_count_b<<<(unsigned)ceil_div(nitems, 128), 128, 0, s>>>(d_plans, d_st, d_qoff, nq, items, nitems,
                                                                            part_off, emit_off, live_off);
            note_launch();
            FAST_TRY(scan_exclusive<int64_t>(part_off, part_off, nitems, part_off + nitems, s));
            FAST_TRY(scan_exclusive<int64_t>(emit_off, emit_off, nitems, emit_off + nitems, s));
            FAST_TRY(scan_exclusive<int64_t>(live_off, live_off, nitems, live_off + nitems, s));
            k_part_totals<<<(unsigned)ceil_div(nq, 128), 128, 0, s>>>(part_off, emit_off, live_off, d_qoff, nq, d_tot);
            note_launch();
            if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched partition launch");
            FAST_TRY(fetch_words(d_tot, tot, 3 * (size_t)nq, s));
            if (pass == 1) break;
            // a level that would pass a query's max_chunks caps every split of
            // that query at an even share of its room left; the capped parts
            // are its last chunks
            bool capped = false;
            for (int q = 0; q < nq; q++) {
                if (!Q[q].active) continue;
                const int64_t np = tot[3 * q], ne = tot[3 * q + 1], nl = tot[3 * q + 2];
                if (Q[q].total + ne + np <= Q[q].cap) continue;
                const int64_t nsplit = nl - ne;
                const int64_t room = Q[q].cap - Q[q].total - ne;
                st[q].kcap = (uint64_t)std::max<int64_t>(1, nsplit > 0 ? room / nsplit : 1);
                Q[q].last = true;
                capped = true;
            }
            if (!capped) break;
            FAST_CUDA(cudaMemcpyAsync(d_st, st.data(), nq * sizeof(QState), cudaMemcpyHostToDevice, s));
        }
        int64_t np_total = 0, ne_total = 0;
        for (int q = 0; q < nq; q++) { np_total += tot[3 * q]; ne_total += tot[3 * q + 1]; }
        Chunk* em = nullptr;
        if (ne_total) {
            FAST_TRY(dalloc(&em, ne_total, s));
            keep.v.push_back((unsigned char*)em);
        }
        bool smp = false;
        for (int q = 0; q < nq; q++)
            if (Q[q].active && (Q[q].cfg.sample_root > 0.0 || Q[q].cfg.sample_deep > 0.0)) smp = true;
        PartRec* parts = nullptr;
        if (smp) {
            FAST_TRY(dalloc(&parts, std::max<int64_t>(np_total, 1), s));
            lvl.v.push_back((unsigned char*)parts);
        }
        if (ne_total || smp) {
            k_part_write_b<<<(unsigned)ceil_div(nitems, 128), 128, 0, s>>>(d_plans, d_st, d_qoff, nq, items, nitems,
                                                                            part_off, emit_off, parts, em);
            note_launch();
        }
        Chunk* next = nullptr;
        FAST_TRY(dalloc(&next, std::max<int64_t>(np_total, 1), s));
        keep.v.push_back((unsigned char*)next);
        if (np_total) {
            int64_t blocks = std::min<int64_t>(ceil_div(np_total, 8), (int64_t)num_sms() * 32);
            k_part_sum_b<<<(unsigned)blocks, 256, 0, s>>>(d_plans, d_qoff, nq, items, nitems, part_off, parts, np_total,
                                                          next);
            note_launch();
        }
        if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched partition launch");
        // this level's chunks and the next level's ranges (grouped by query)
        int64_t eo = 0, po = 0;
        for (int q = 0; q < nq; q++) {
            const int64_t np = tot[3 * q], ne = tot[3 * q + 1];
            if (ne) { Q[q].pieces.push_back({em + eo, ne}); Q[q].total += ne; }
            if (Q[q].active && Q[q].last) {
                if (np) { Q[q].pieces.push_back({next + po, np}); Q[q].total += np; }
                Q[q].active = false;
            } else if (Q[q].active && np == 0) {
                Q[q].active = false;
            }
            qoff[q + 1] = qoff[q] + np;
            eo += ne;
            po += np;
        }
        items = next;
        nitems = np_total;
    }
    // every query's chunk list, level by level, into its own array
    std::vector<CopyDesc> cd;
    uint64_t pieces = 0;
    for (int q = 0; q < nq; q++) {
        fast_chunks* ch = new fast_chunks();
        ch->c = Q[q].c;
        ch->n = Q[q].total;
        ch->stream = s;
        outs[Q[q].idx] = ch;
        FAST_TRY(dalloc_direct(&ch->d, Q[q].total, s));                 // outlives the call
        int64_t o = 0;
        for (auto& pc : Q[q].pieces) {
            const uint64_t bytes = (uint64_t)pc.second * sizeof(Chunk);
            cd.push_back({(const unsigned char*)pc.first, (unsigned char*)(ch->d + o), bytes, pieces});
            pieces += (bytes + kPiece - 1) / kPiece;
            o += pc.second;
        }
    }
    if (!cd.empty()) {
        CopyDesc* d = nullptr;
        FAST_TRY(upload_array(cd, &d, keep.v, s));
        const unsigned grid = (unsigned)std::min<uint64_t>(pieces, (uint64_t)num_sms() * 8);
        k_copy_many<<<grid, 256, 0, s>>>(d, (int)cd.size(), pieces);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched partition gather");
    }
    return FAST_OK;
}

}  // namespace

namespace fast {

int partition_batch(const fast_cst* const* csts, int32_t nq, const fast_config* const* cfgs, cudaStream_t s,
                    fast_chunks** outs, int32_t* status) {
    std::vector<QP> Q;
    for (int i = 0; i < nq; i++) {
        outs[i] = nullptr;
        if (!csts[i]) {
            status[i] = set_error(FAST_ERR_INVALID, "fast_partition_batch: cst %d is NULL", i);
            continue;
        }
        status[i] = FAST_OK;
        QP q;
        q.c = csts[i];
        q.idx = i;
        q.cfg = cfgs[i] ? *cfgs[i] : csts[i]->cfg;
        Q.push_back(std::move(q));
    }
    int rc = Q.empty() ? FAST_OK : partition_all(Q, s, outs);
    if (rc != FAST_OK) {
        for (int i = 0; i < nq; i++) {
            if (outs[i]) { dfree_direct(outs[i]->d, s); delete outs[i]; outs[i] = nullptr; }
        }
    }
    return rc;
}

}  // namespace fast

extern "C" int fast_partition_batch(const fast_cst* const* csts, int32_t nq, const fast_config* cfg, void* stream,
                                    fast_chunks** outs, int32_t* status) {
    if (nq < 0 || (nq > 0 && (!csts || !outs || !status)))
        return set_error(FAST_ERR_INVALID, "fast_partition_batch: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    PoolScope scratch(s);
    std::vector<const fast_config*> cfgs(nq, cfg);
    return partition_batch(csts, nq, cfgs.data(), s, outs, status);
}
