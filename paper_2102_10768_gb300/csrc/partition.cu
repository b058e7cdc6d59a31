// CST partition (Sec. IV-B, Algorithm 2) driven by the workload estimate of
// Sec. IV-C, level-synchronous on the device.
//
// A pending part is a Chunk: positions 0..j-1 fixed (prefix), position j
// restricted to the run [a, b) of its list L_j.  Its estimate is
//   W' = F(prefix) * sum_{x in L_j[a..b)} c_{u_j}(x),
//   F(prefix) = prod over prefix positions p, over children c of p placed
//               after j, of the per-row child sum s_{p->c}(prefix[p]),
// which equals the workload DP evaluated on the partitioned tree: restricting
// a candidate set to the part leaves c unchanged for every candidate still
// reachable, and every position after j hangs below a prefix position.
// One level = decide and count parts, write the chunks that are done (and
// the parts of sampled splits), then one warp per part sums its estimate
// (an unsampled part is derived from its item and index); the host reads the
// level's sizes.
#include <vector>

#include "internal.cuh"
#include "prims.cuh"
#include "part_funcs.cuh"

using namespace fast;

namespace {

// one thread per pending item: classify and count the kept parts
__global__ void k_part_count(const PartPlan P, Chunk* __restrict__ items, int64_t nitems, uint32_t root_n,
                             uint64_t kcap, int64_t* __restrict__ nparts, int64_t* __restrict__ nemit,
                             int64_t* __restrict__ nlive) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems) return;
    Chunk c = items[t];
    uint64_t kk = 0;
    int act = classify(P, c, root_n, &kk);
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

// one thread per pending item: write emitted chunks, and the part records
// of sampled splits (without sampling, k_part_sum derives every part from
// its item and its index there)
__global__ void k_part_write(const PartPlan P, const Chunk* __restrict__ items, int64_t nitems, uint64_t kcap,
                             const int64_t* __restrict__ part_off, const int64_t* __restrict__ emit_off,
                             PartRec* __restrict__ parts, Chunk* __restrict__ emitted) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems) return;
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

// Part p of an unsampled level: its item t (the last with part_off[t] <= p)
// and run i = p - part_off[t] of the item's kk = part_off[t+1] - part_off[t]
// even runs (the split factor after the cap).
__device__ PartRec part_of(const PartPlan& P, const Chunk* __restrict__ items, int64_t nitems,
                           const int64_t* __restrict__ part_off, int64_t p) {
    int64_t lo = 0, hi = nitems;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (part_off[mid] <= p) lo = mid; else hi = mid;
    }
    const Chunk& c = items[lo];
    uint64_t i = (uint64_t)(p - part_off[lo]);
    uint64_t kk = (uint64_t)(part_off[lo + 1] - part_off[lo]);
    uint64_t n = c.b - c.a;
    PartRec r;
    r.item = (uint32_t)lo;
    r.a = c.a + (uint32_t)((i * n) / kk);
    r.b = c.a + (uint32_t)(((i + 1) * n) / kk);
    r.pad = 0;
    r.id = mix64(c.id + (i + 1) * 0x9E3779B97F4A7C15ull);
    r.f = prefix_factor(P, c);
    return r;
}

// one warp per part: W' = F * (saturating sum of c over the run).  parts ==
// nullptr: the level is unsampled and part_of() gives each part.
__global__ void k_part_sum(const PartPlan P, const Chunk* __restrict__ items, int64_t nitems,
                           const int64_t* __restrict__ part_off, const PartRec* __restrict__ parts,
                           int64_t nparts, Chunk* __restrict__ next) {
    const int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w; p < nparts; p += nw) {
        PartRec r = parts ? parts[p] : part_of(P, items, nitems, part_off, p);
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

int partition(const fast_cst* c, const fast_config* cfg_in, cudaStream_t s, fast_chunks** out) {
    if (!out) return set_error(FAST_ERR_INVALID, "fast_partition: out is NULL");
    *out = nullptr;
    if (!c) return set_error(FAST_ERR_INVALID, "fast_partition: cst is NULL");
    fast_config cfg;
    if (cfg_in) cfg = *cfg_in; else cfg = c->cfg;
    PartPlan P = make_plan(c, &cfg);
    uint32_t root_n = (uint32_t)c->ncand[c->root];
    std::vector<std::pair<Chunk*, int64_t>> levels;
    int64_t total = 0;
    Chunk* items = nullptr;
    int64_t nitems = 0;
    int rc = FAST_OK;
    int64_t* cnt = nullptr;
    PartRec* parts = nullptr;
    Chunk* next = nullptr;
    const int64_t cap = cfg.max_chunks > 0 ? cfg.max_chunks : (1ll << 16);

    if (root_n > 0 && c->W > 0) {
        Chunk r0;
        memset(&r0, 0, sizeof(r0));
        r0.j = 0; r0.a = 0; r0.b = root_n; r0.w = c->W; r0.id = mix64(cfg.sample_seed);
        rc = dalloc(&items, 1, s);
        if (rc == FAST_OK) {
            cudaError_t e = cudaMemcpyAsync(items, &r0, sizeof(Chunk), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) rc = cuda_status(e, "partition seed", __FILE__, __LINE__);
            nitems = 1;
        }
    }
    bool last = false;                          // this level's parts are final chunks
    while (rc == FAST_OK && nitems > 0) {
        // per item: [0, n] part offsets, [n+1, 2n+1] emit offsets, [2n+2, 3n+2] live offsets
        rc = dalloc(&cnt, 3 * (nitems + 1), s); if (rc) break;
        int64_t* part_off = cnt;
        int64_t* emit_off = cnt + nitems + 1;
        int64_t* live_off = cnt + 2 * (nitems + 1);
        uint64_t kcap = 0;
        int64_t np = 0, ne = 0, nl = 0;
        for (int pass = 0; pass < 2; pass++) {
            k_part_count<<<(unsigned)ceil_div(nitems, 128), 128, 0, s>>>(P, items, nitems, root_n, kcap, part_off,
                                                                          emit_off, live_off);
            note_launch();
            rc = scan_exclusive<int64_t>(part_off, part_off, nitems, part_off + nitems, s); if (rc) break;
            rc = scan_exclusive<int64_t>(emit_off, emit_off, nitems, emit_off + nitems, s); if (rc) break;
            rc = scan_exclusive<int64_t>(live_off, live_off, nitems, live_off + nitems, s); if (rc) break;
            cudaError_t e = cudaMemcpyAsync(&np, part_off + nitems, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&ne, emit_off + nitems, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&nl, live_off + nitems, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { rc = cuda_status(e, "partition level sizes", __FILE__, __LINE__); break; }
            if (pass == 1 || total + ne + np <= cap) break;
            // the level would pass max_chunks: cap every split at an even share of the
            // room left; the capped parts are the last chunks
            int64_t nsplit = nl - ne;
            int64_t room = cap - total - ne;
            kcap = (uint64_t)std::max<int64_t>(1, nsplit > 0 ? room / nsplit : 1);
            last = true;
        }
        if (rc) break;
        Chunk* em = nullptr;
        if (ne) { rc = dalloc(&em, ne, s); if (rc) break; levels.push_back({em, ne}); total += ne; }
        const bool smp = cfg.sample_root > 0.0 || cfg.sample_deep > 0.0;
        if (smp) { rc = dalloc(&parts, np, s); if (rc) break; }
        if (ne || smp) {
            k_part_write<<<(unsigned)ceil_div(nitems, 128), 128, 0, s>>>(P, items, nitems, kcap, part_off, emit_off, parts, em);
            note_launch();
        }
        rc = dalloc(&next, np, s); if (rc) break;
        if (np) {
            int64_t blocks = std::min<int64_t>(ceil_div(np, 8), (int64_t)num_sms() * 32);
            k_part_sum<<<(unsigned)blocks, 256, 0, s>>>(P, items, nitems, part_off, smp ? parts : nullptr, np, next);
            note_launch();
        }
        if (cudaGetLastError() != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "partition kernel launch"); break; }
        dfree(cnt, s); dfree(parts, s); dfree(items, s);
        items = next; next = nullptr;
        nitems = np;
        if (last) {
            // every part is a chunk as it is (W' = 0 parts hold nothing and are dropped later by the matcher)
            if (nitems) { levels.push_back({items, nitems}); total += nitems; items = nullptr; }
            nitems = 0;
        }
    }
    dfree(cnt, s); dfree(parts, s); dfree(next, s); dfree(items, s);
    fast_chunks* ch = nullptr;
    if (rc == FAST_OK) {
        ch = new fast_chunks();
        ch->c = c; ch->n = total; ch->stream = s;
        rc = dalloc_direct(&ch->d, total, s);            // outlives the call
        int64_t o = 0;
        for (auto& lv : levels) {
            if (rc != FAST_OK) break;
            cudaError_t e = cudaMemcpyAsync(ch->d + o, lv.first, lv.second * sizeof(Chunk), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) rc = cuda_status(e, "partition gather", __FILE__, __LINE__);
            o += lv.second;
        }
    }
    for (auto& lv : levels) dfree(lv.first, s);
    if (rc != FAST_OK) {
        if (ch) { dfree_direct(ch->d, s); delete ch; }
        return rc;
    }
    *out = ch;
    return FAST_OK;
}

}  // namespace

extern "C" int fast_partition(const fast_cst* c, const fast_config* cfg, void* stream, fast_chunks** out) {
    PoolScope scratch((cudaStream_t)stream);
    return partition(c, cfg, (cudaStream_t)stream, out);
}

extern "C" int fast_chunks_info(const fast_chunks* ch, int64_t* count, uint64_t* w_sum) {
    if (!ch) return set_error(FAST_ERR_INVALID, "fast_chunks_info: NULL chunks");
    if (count) *count = ch->n;
    if (w_sum) {
        // summed on request from the descriptors (the partition itself
        // does not read them back)
        cudaStream_t s = ch->stream;
        std::vector<Chunk> h(ch->n);
        if (ch->n) FAST_CUDA(cudaMemcpyAsync(h.data(), ch->d, ch->n * sizeof(Chunk), cudaMemcpyDeviceToHost, s));
        FAST_CUDA(cudaStreamSynchronize(s));
        uint64_t ws = 0;
        for (auto& x : h) ws = sat_add(ws, x.w);
        *w_sum = ws;
    }
    return FAST_OK;
}

extern "C" int fast_chunks_copy(const fast_chunks* ch, int32_t* j, int32_t* prefix, int64_t* a, int64_t* b,
                                uint64_t* w, uint64_t* id, void* stream) {
    if (!ch) return set_error(FAST_ERR_INVALID, "fast_chunks_copy: NULL chunks");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Chunk> h(ch->n);
    if (ch->n) FAST_CUDA(cudaMemcpyAsync(h.data(), ch->d, ch->n * sizeof(Chunk), cudaMemcpyDeviceToHost, s));
    FAST_CUDA(cudaStreamSynchronize(s));
    int k = ch->c->k;
    for (int64_t i = 0; i < ch->n; i++) {
        if (j) j[i] = h[i].j;
        if (prefix) for (int t = 0; t < k; t++) prefix[i * k + t] = t < h[i].j ? (int32_t)h[i].prefix[t] : -1;
        if (a) a[i] = h[i].a;
        if (b) b[i] = h[i].b;
        if (w) w[i] = h[i].w;
        if (id) id[i] = h[i].id;
    }
    return FAST_OK;
}

__global__ void k_gather_chunks(const Chunk* __restrict__ src, const int64_t* __restrict__ idx, int64_t n,
                                Chunk* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

extern "C" int fast_chunks_select(const fast_chunks* ch, const int64_t* idx, int64_t n, void* stream,
                                  fast_chunks** out) {
    if (!out) return set_error(FAST_ERR_INVALID, "fast_chunks_select: out is NULL");
    *out = nullptr;
    if (!ch || n < 0 || (n > 0 && !idx)) return set_error(FAST_ERR_INVALID, "fast_chunks_select: bad arguments");
    for (int64_t i = 0; i < n; i++)
        if (idx[i] < 0 || idx[i] >= ch->n)
            return set_error(FAST_ERR_INVALID, "fast_chunks_select: index %lld of %lld chunks", (long long)idx[i],
                             (long long)ch->n);
    cudaStream_t s = (cudaStream_t)stream;
    PoolScope scratch(s);
    fast_chunks* sel = new fast_chunks();
    sel->c = ch->c; sel->n = n; sel->stream = s;
    int64_t* d_idx = nullptr;
    int rc = dalloc_direct(&sel->d, n, s);                       // outlives the call
    if (rc == FAST_OK && n > 0) rc = dalloc(&d_idx, n, s);
    if (rc == FAST_OK && n > 0) {
        cudaError_t e = cudaMemcpyAsync(d_idx, idx, n * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_chunks_select", __FILE__, __LINE__);
    }
    if (rc == FAST_OK && n > 0) {
        k_gather_chunks<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4096), 256, 0, s>>>(ch->d, d_idx, n, sel->d);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_chunks_select", __FILE__, __LINE__);
    }
    dfree(d_idx, s);
    if (rc != FAST_OK) {
        dfree_direct(sel->d, s);
        delete sel;
        return rc;
    }
    *out = sel;
    return FAST_OK;
}

namespace fast {
void chunks_release_nosync(fast_chunks* ch) {
    if (!ch) return;
    dfree_direct(ch->d, ch->stream);
    delete ch;
}
}  // namespace fast

extern "C" void fast_free_chunks(fast_chunks* ch) {
    if (!ch) return;
    cudaStream_t s = ch->stream;
    dfree_direct(ch->d, s);
    delete ch;
    cudaStreamSynchronize(s);
}
