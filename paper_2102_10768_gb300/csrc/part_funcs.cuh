// The partition's plan and device helpers (Sec. IV-B, Algorithm 2, with the
// workload estimate of Sec. IV-C), shared by the per-query partition
// (partition.cu) and the batched one (partition_batch.cu): a CST's arrays
// by matching-order position, the Generator-side candidate checks of a
// fixed prefix, and the classification of a pending part.
#pragma once

#include <cstring>

#include "internal.cuh"
#include "prims.cuh"

namespace fast {

struct PartPlan {
    int k;
    int par_pos[kMaxK];            // position -> parent position (-1 at 0)
    uint32_t child_mask[kMaxK];    // position -> bitmask of child positions
    uint32_t same_lab[kMaxK];      // earlier positions with the same label
    const int32_t* cand[kMaxK];    // by position
    const int64_t* t_off[kMaxK];   // by position (tree edge into it)
    const uint32_t* t_idx[kMaxK];
    const uint64_t* cval[kMaxK];   // by position
    const uint64_t* ssum[kMaxK];   // by position: per row of C(parent position)
    int nt_begin[kMaxK + 1];       // non-tree edges into position i
    int nt_from[kMaxNT];
    const int64_t* n_off[kMaxNT];
    const uint32_t* n_idx[kMaxNT];
    uint64_t delta_w;
    double c_root, c_deep;
};

static __device__ __forceinline__ bool in_list(const uint32_t* a, int64_t lo, int64_t hi, uint32_t x) {
    int64_t end = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < end && a[lo] == x;
}

// may candidate v (index into C of position j) join the fixed prefix?
static __device__ bool prefix_ok(const PartPlan& P, const Chunk& c, uint32_t v) {
    int j = c.j;
    int32_t g = P.cand[j][v];
    uint32_t sl = P.same_lab[j];
    while (sl) {
        int p = __ffs(sl) - 1;
        sl &= sl - 1;
        if (P.cand[p][c.prefix[p]] == g) return false;
    }
    for (int e = P.nt_begin[j]; e < P.nt_begin[j + 1]; e++) {
        uint32_t mf = c.prefix[P.nt_from[e]];
        if (!in_list(P.n_idx[e], P.n_off[e][mf], P.n_off[e][mf + 1], v)) return false;
    }
    return true;
}

struct PartRec {
    uint32_t item;
    uint32_t a, b;
    uint32_t pad;
    uint64_t id;
    uint64_t f;                    // F(prefix)
};

static __device__ __forceinline__ uint32_t list_at(const PartPlan& P, const Chunk& c, uint64_t x) {
    if (c.j == 0) return (uint32_t)x;
    int64_t base = P.t_off[c.j][c.prefix[P.par_pos[c.j]]];
    return P.t_idx[c.j][base + (int64_t)x];
}

static __device__ __forceinline__ uint32_t list_len(const PartPlan& P, const Chunk& c, uint32_t root_n) {
    if (c.j == 0) return root_n;
    uint32_t m = c.prefix[P.par_pos[c.j]];
    return (uint32_t)(P.t_off[c.j][m + 1] - P.t_off[c.j][m]);
}

static __device__ __forceinline__ bool sampled(const PartPlan& P) { return P.c_root > 0.0 || P.c_deep > 0.0; }

static __device__ __forceinline__ bool keep_part(const PartPlan& P, int j, uint64_t kk, uint64_t id) {
    double cs = j == 0 ? P.c_root : P.c_deep;
    if (cs <= 0.0) return true;
    double tau = cs / (double)kk;
    if (!(tau < 1.0)) return true;
    return (double)(id >> 11) * (1.0 / 9007199254740992.0) < tau;
}

// Advance single-candidate runs to the next position (same estimate), then
// classify: 0 drop, 1 emit as a chunk, 2 split.  Writes the advanced item
// back.  Returns the split factor in *kk_out.
static __device__ int classify(const PartPlan& P, Chunk& c, uint32_t root_n, uint64_t* kk_out) {
    for (;;) {
        if (c.w == 0) return 0;
        if (c.w <= P.delta_w) return 1;
        uint32_t n = c.b - c.a;
        if (n == 1) {
            if (c.j + 1 >= P.k) return 1;
            uint32_t v = list_at(P, c, c.a);
            if (!prefix_ok(P, c, v)) return 0;
            c.prefix[c.j] = v;
            c.j += 1;
            c.a = 0;
            c.b = list_len(P, c, root_n);
            continue;
        }
        uint64_t kk = c.w / P.delta_w + (c.w % P.delta_w != 0);
        if (kk > n) kk = n;
        *kk_out = kk;
        return 2;
    }
}

static __device__ uint64_t prefix_factor(const PartPlan& P, const Chunk& c) {
    uint64_t f = 1;
    for (int p = 0; p < c.j; p++) {
        uint32_t m = P.child_mask[p];
        while (m) {
            int ch = __ffs(m) - 1;
            m &= m - 1;
            if (ch > c.j) f = sat_mul(f, P.ssum[ch][c.prefix[p]]);
        }
    }
    return f;
}

static PartPlan make_plan(const fast_cst* c, const fast_config* cfg) {
    PartPlan P;
    memset(&P, 0, sizeof(P));
    P.k = c->k;
    for (int i = 0; i < c->k; i++) {
        int u = c->order[i];
        P.par_pos[i] = c->parent[u] < 0 ? -1 : c->pos[c->parent[u]];
        P.t_off[i] = c->t_off[u];
        P.t_idx[i] = c->t_idx[u];
        P.cval[i] = c->cval[u];
        P.ssum[i] = c->ssum[u];
        P.cand[i] = c->cand[u];
        P.child_mask[i] = 0;
        P.same_lab[i] = 0;
        for (int p = 0; p < i; p++)
            if (c->qlabel[c->order[p]] == c->qlabel[u]) P.same_lab[i] |= 1u << p;
    }
    for (int i = 1; i < c->k; i++) P.child_mask[P.par_pos[i]] |= 1u << i;
    int e = 0;
    for (int i = 0; i < c->k; i++) {
        P.nt_begin[i] = e;
        for (int t = 0; t < c->nnt; t++) {
            if (c->pos[c->nt_to[t]] != i) continue;
            P.nt_from[e] = c->pos[c->nt_from[t]];
            P.n_off[e] = c->n_off[t];
            P.n_idx[e] = c->n_idx[t];
            e++;
        }
    }
    P.nt_begin[c->k] = e;
    P.delta_w = cfg->delta_w ? cfg->delta_w : 1;
    P.c_root = cfg->sample_root;
    P.c_deep = cfg->sample_deep;
    return P;
}

}  // namespace fast
