/*
 * fast.h -- C ABI of a GB300 (sm_103a) implementation of candidate-search-tree
 * subgraph matching, after "FAST: FPGA-based Subgraph Matching on Massive
 * Graphs" (Jin, Yang, Lin, Yang, Qin, Peng; arXiv 2102.10768).
 *
 * Problem (Sec. II-A, Definition 1 and the problem statement): given a
 * labelled query graph q and a labelled data graph G, both undirected and
 * simple, enumerate every embedding -- every injective map M: V(q) -> V(G)
 * with l_q(u) = l_G(M(u)) for every u and (M(u), M(u')) in E(G) for every
 * query edge (u, u').  Embeddings are maps, not subgraphs: a copy of q in G is
 * reached once per automorphism of q.
 *
 * Pipeline (each step is CUDA on the device; the host only sequences them):
 *   fast_load_graph  -- CSR of G plus a label index (the data model of
 *                       Sec. II-A).
 *   fast_build_cst   -- the candidate search tree CST of Sec. IV-A
 *                       (Algorithm 1): candidate filter, top-down
 *                       construction over a BFS tree t_q of q, bottom-up
 *                       refinement, non-tree candidate edges, and the
 *                       workload estimate of Sec. IV-C.
 *   fast_partition   -- the CST partition of Sec. IV-B (Algorithm 2) into
 *                       chunks whose workload estimate is bounded.
 *   fast_match       -- enumeration over the CST (the semantics of
 *                       Algorithms 4-8, Sec. V-A): a uint64 count and,
 *                       optionally, the first k embeddings found.
 *
 * Conventions for every entry point:
 *   - Return value: FAST_OK (0) or one of the FAST_ERR_* codes below; the
 *     thread-local fast_last_error() then describes the failure.  Outputs
 *     are undefined after an error unless stated otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL: the legacy default
 *     stream).  Work is enqueued on it; calls that must report sizes or
 *     counts to the host synchronise it before returning.
 *   - Handles (fast_graph, fast_cst, fast_chunks) are opaque, owned by the
 *     library and released with their fast_free_* function.  Input arrays
 *     are copied; the caller keeps ownership of everything it passes in.
 *   - Device memory is on the current CUDA device.  Graphs and chunk lists
 *     are allocated stream-ordered (cudaMallocAsync); a CST holds one
 *     exact-size stream-ordered block; the temporaries of a call come from
 *     a scratch pool of cached device blocks (one per calling thread, and
 *     one per batch or server worker), kept until that thread, batch or
 *     server ends.  fast_match_noalloc allocates nothing.
 */
#ifndef FAST_GB300_H
#define FAST_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define FAST_OK 0
#define FAST_ERR_INVALID 1   /* bad argument: ids out of range, q.n > 32, disconnected q, ... */
#define FAST_ERR_OOM 2       /* a device allocation failed */
#define FAST_ERR_TIMEOUT 3   /* fast_match ran past config.time_budget_s; the count is partial */
#define FAST_ERR_OVERFLOW 4  /* the embedding count reached 2^64 - 1 (saturated) */
#define FAST_ERR_CUDA 5      /* a CUDA call or kernel launch failed */
#define FAST_ERR_LIMIT 6     /* reserved */

#define FAST_MAX_QUERY 32    /* query vertices per query (one warp lane each) */

/* flags for fast_load_graph */
#define FAST_PTR_DEVICE 1    /* edges and labels are device pointers */

typedef struct fast_graph fast_graph;
typedef struct fast_cst fast_cst;
typedef struct fast_chunks fast_chunks;

/* A query graph q (Sec. II-A).  Host arrays; vertices are 0..n-1. */
typedef struct {
    int32_t n;               /* |V(q)|, 1..FAST_MAX_QUERY */
    int32_t m;               /* number of entries in edges */
    const int32_t* labels;   /* [n] vertex labels, >= 0 */
    const int32_t* edges;    /* [m][2] undirected edges; repeats are ignored, loops rejected */
} fast_query_desc;

/* Tunables.  fast_config_default() fills documented defaults. */
typedef struct {
    /* Partition (Sec. IV-B, Algorithm 2): a chunk holds a workload estimate
     * W' <= delta_w (Sec. IV-C).  The split factor of a part is
     * k = min(ceil(W'/delta_w), |C'(u)|). */
    uint64_t delta_w;
    /* Optional seeded sampling of the partition: a part produced by a split
     * into k parts is kept iff u01(id) < min(1, c/k), c = sample_root for a
     * split of the root's candidates and sample_deep deeper (c <= 0 keeps
     * every part, i.e. the chunks cover the whole search space). */
    double sample_root;
    double sample_deep;
    uint64_t sample_seed;
    int64_t max_chunks;      /* chunks of one partition at most: a level that would pass it caps its splits (fast_partition) */
    /* Matcher launch shape: warps per CTA and CTAs per SM (persistent). */
    int32_t warps_per_block;
    int32_t blocks_per_sm;
    /* Wall-clock budget for one fast_match call, seconds (<= 0: none). */
    double time_budget_s;
    /* Enumeration limit: fast_match stops once `limit` embeddings are found
     * and reports min(total, limit), exactly (0: enumerate everything). */
    uint64_t limit;
    /* Cells of the matcher's ring of donated runs (work given away to idle
     * warps); a full ring only means a busy warp keeps its work.  0: the
     * default, 65536 (4096 for fast_match_noalloc); larger values are
     * clamped to the default.  Results never depend on it. */
    int64_t queue_cells;
    /* Matching order O of fast_build_cst.  0: the paper's path-based order
     * (Sec. IV-B): a depth-first walk of t_q, children by increasing
     * (|C(u)|, u).  1: greedy: after the root, repeatedly the vertex whose
     * t_q parent is placed with the most query edges to placed vertices
     * (ties: smaller |C(u)|, then smaller u).  2: the BFS order of t_q.
     * 3: after the root, repeatedly the vertex whose t_q parent is placed
     * with the fewest candidates (ties: smaller u).  The paper's method
     * takes any connected order (Sec. IV-B, and its order study of
     * Sec. VI); every rule places a vertex after its t_q parent, and
     * embeddings and counts never depend on the rule. */
    int32_t order_rule;
    /* Candidate filter of fast_build_cst (Sec. IV-A, local features).  0:
     * label and degree, C0(u) = { v : l(v) = l_q(u), d(v) >= d_q(u) }.  1:
     * also neighbour label frequencies: for every label, v has at least as
     * many neighbours with it as u has (smaller CSTs; the same embeddings). */
    int32_t filter_rule;
    /* How fast_batch_run and fast_match_batch build the CSTs and partitions
     * of a batch.  0: each query's fast_build_cst and fast_partition on a
     * pool of host threads.  1: the CSTs together (fast_build_cst_batch),
     * the partitions on the threads.  2: both together (also
     * fast_partition_batch).  The CSTs and chunk lists, and so every
     * result, are the same either way; fast_batch_create rejects other
     * values. */
    int32_t build_rule;
    /* Bottom-up refinement of the CST (Sec. IV-A).  0: the paper's single
     * pass.  2: the same pass where a candidate v of u must also have, for
     * every query neighbour w of u joined by a non-tree edge, a neighbour in
     * C(w) as it stands when u is reached (refined for vertices later in the
     * BFS order, top-down for earlier ones): smaller CSTs, the same
     * embeddings.  Rule 2 is built by fast_build_cst_batch only (the batch
     * with build_rule >= 1); fast_build_cst and build_rule 0 reject it. */
    int32_t refine_rule;
    /* The matcher kernel (Sec. V-A semantics either way).  0: fused -- every
     * warp runs the whole search.  1: warp-specialised (the task-generator
     * separation of Sec. V-D): in every CTA `validators` warps take, from a
     * ring in shared memory, the last-position extensions that the other
     * warps (the expanders) hand them, and count those positions' embeddings.
     * Rule 1 applies to counting launches (no per-chunk counts, no embeddings
     * written, no counting pass); the others run the fused kernel.  Results
     * never depend on it. */
    int32_t matcher_rule;
    int32_t validators;      /* rule 1: validator warps per CTA (0: half of warps_per_block) */
} fast_config;

/* Default tunables: delta_w = 2^20, no sampling, max_chunks = 2^16,
 * 8 warps per CTA, 4 CTAs per SM, no time budget, no limit, every rule 0. */
void fast_config_default(fast_config* cfg);

/* Thread-local message for the last failing call ("" if none). */
const char* fast_last_error(void);

/* ----------------------------------------------------------- data graph */

/*
 * Build the device-resident data graph G (Sec. II-A: undirected, labelled,
 * simple).  edges: [m][2] vertex ids in 0..n-1; both directions are stored,
 * self loops and repeated edges are dropped.  labels: [n], >= 0 and below
 * 2^23.  Host pointers unless flags has FAST_PTR_DEVICE.  n <= 2^31 - 1 and
 * 2m < 2^32.  Layout on the device: int64 row offsets [n+1], int32 neighbour
 * ids, int32 labels, and a label index (vertices grouped by label, ascending
 * id within a label).  Each neighbour list is sorted by (label of the
 * neighbour, id) -- with a directory of its label runs, so that the CST
 * build (Alg. 1) reads only the neighbours with the label it keeps -- when
 * 2 * bits(n - 1) + bits(labels - 1) <= 64; otherwise by id alone.
 * Errors: FAST_ERR_INVALID for ids or labels out of range.
 */
int fast_load_graph(int64_t n, int64_t m, const int32_t* edges, const int32_t* labels, int flags,
                    void* stream, fast_graph** out);

/* n, number of stored (directed) adjacency entries = 2|E(G)|, label count
 * (max label + 1) and maximum degree D_G. */
int fast_graph_info(const fast_graph* g, int64_t* n, int64_t* nadj, int32_t* num_labels, int64_t* max_degree);

/* Copy the CSR to host arrays row_ptr[n+1] and col[nadj], rows in the
 * layout above (a test aid). */
int fast_graph_copy_csr(const fast_graph* g, int64_t* row_ptr, int32_t* col, void* stream);

/* Free G.  Device memory the library frees stays pooled in this process
 * (the stream-ordered allocator's default pool, kept from one batched step
 * to the next); freeing a graph also hands the pooled memory back. */
void fast_free_graph(fast_graph* g);

/* ----------------------------------------------------------------- CST */

/*
 * Build the candidate search tree of q over G (Sec. IV-A, Algorithm 1) and
 * its workload estimate (Sec. IV-C), entirely on the device:
 *   filter:    C0(u) = { v : l(v) = l_q(u), d_G(v) >= d_q(u) }.
 *   root:      argmin_u |C0(u)| / d_q(u), ties to the smaller id; t_q is the
 *              BFS tree from it (neighbours in increasing id).
 *   top-down:  in BFS order, C(u) = vertices of C0(u) adjacent to some
 *              candidate of the parent, and N^{u_p}_u(v_p) = N_G(v_p) n C(u).
 *   bottom-up: in reverse BFS order, child lists are cut to the refined
 *              child sets and v leaves C(u) when one of them is empty.
 *   order:     the matching order O is the depth-first preorder of t_q with
 *              children taken by increasing (|C|, id) -- whole root-to-leaf
 *              paths in turn.
 *   non-tree:  for each query edge outside t_q, from its earlier endpoint
 *              u_j to its later endpoint u_i in O: N^{u_j}_{u_i}(v) =
 *              N_G(v) n C(u_i), for v in C(u_j).
 *   workload:  c_u(v) = 1 at leaves, c_u(v) = prod over children u' of
 *              sum_{v' in N^u_{u'}(v)} c_{u'}(v'), W = sum over C(root); in
 *              saturating uint64 and in float64.
 * Lists are stored as sorted candidate-local indices.  The call synchronises
 * `stream` a few times (candidate counts decide the root and the order).
 * An empty candidate set is not an error: the CST then has no embeddings.
 * Errors: FAST_ERR_INVALID for a bad or disconnected query.
 */
int fast_build_cst(const fast_graph* g, const fast_query_desc* q, const fast_config* cfg, void* stream,
                   fast_cst** out);

/*
 * The CSTs of nq queries built together (Sec. IV-A, Algorithm 1, and the
 * workload estimate of Sec. IV-C, as fast_build_cst): the steps go over BFS
 * positions, and each step is one launch for the vertex at that position of
 * every query, with one or two host round trips per position for the whole
 * batch instead of a few per query.  outs[i] receives query i's CST, which
 * is the same, array for array, as fast_build_cst gives; the caller frees
 * each with fast_free_cst.  status[i] is FAST_OK, or FAST_ERR_INVALID for a
 * bad query (outs[i] is then NULL).  Queries are built in groups of up to
 * 1024.  qs, outs and status are host arrays of nq entries.
 * Returns FAST_ERR_INVALID for bad arguments, FAST_ERR_OOM or FAST_ERR_CUDA
 * when a group fails (every outs[i] is then NULL), else FAST_OK.
 */
int fast_build_cst_batch(const fast_graph* g, int32_t nq, const fast_query_desc* qs, const fast_config* cfg,
                         void* stream, fast_cst** outs, int32_t* status);

/*
 * Shape of a CST: k = |V(q)|; root; order[k] (position -> query vertex);
 * parent[k] (query vertex -> parent in t_q, -1 for the root); cand[k]
 * (query vertex -> |C(u)|); W as saturating uint64 and float64.  Any output
 * pointer may be NULL.
 */
int fast_cst_info(const fast_cst* c, int32_t* k, int32_t* root, int32_t* order, int32_t* parent,
                  int64_t* cand, uint64_t* w_u64, double* w_f64);

/* Copy C(u) (sorted data-vertex ids, |C(u)| entries) to host memory. */
int fast_cst_candidates(const fast_cst* c, int32_t u, int32_t* out, void* stream);

/* Number of list entries of the tree edge into u (0 for the root). */
int fast_cst_tree_size(const fast_cst* c, int32_t u, int64_t* entries);

/* Copy the tree lists into u: off[|C(parent(u))|+1] and idx[entries]
 * (candidate-local indices into C(u)); row i belongs to C(parent(u))[i]. */
int fast_cst_tree_lists(const fast_cst* c, int32_t u, int64_t* off, uint32_t* idx, void* stream);

/* Number of non-tree CST edges, and the endpoints (query vertices, earlier
 * then later in O) and list size of edge e. */
int fast_cst_nontree_count(const fast_cst* c, int32_t* count);
int fast_cst_nontree_edge(const fast_cst* c, int32_t e, int32_t* from_u, int32_t* to_u, int64_t* entries);

/* Copy the lists of non-tree edge e: off[|C(from)|+1], idx[entries]. */
int fast_cst_nontree_lists(const fast_cst* c, int32_t e, int64_t* off, uint32_t* idx, void* stream);

/* Copy c_u(v) for u's candidates (saturating uint64, |C(u)| entries). */
int fast_cst_workload(const fast_cst* c, int32_t u, uint64_t* out, void* stream);

void fast_free_cst(fast_cst* c);

/* ------------------------------------------------------------ partition */

/*
 * Partition the CST (Sec. IV-B, Algorithm 2).  Since every position before
 * the split position is then a single candidate, a chunk is
 * (j, the candidates of positions 0..j-1, a run [a, b) of the list L_j),
 * where L_j is C(root) when j = 0 and otherwise the tree list, towards
 * position j, of the candidate at position j's parent position.  Runs are
 * even contiguous slices; a run with W' <= delta_w is a chunk (W' = 0 runs
 * hold no embedding and are dropped); a run of one candidate joins the fixed
 * prefix and moves on to the next position -- unless it repeats a fixed
 * candidate or lacks a CST edge to a fixed non-tree neighbour, in which case
 * it holds no embedding and is dropped; longer runs split again.  Runs are
 * processed level by level; if a level would bring the chunk count above
 * cfg->max_chunks, each of its splits is capped at
 * max(1, (max_chunks - chunks so far - runs finishing) / runs splitting)
 * parts and those parts are the last chunks (their W' may exceed delta_w).
 * With sampling off the chunks are disjoint and cover every embedding.  The
 * host reads a few sizes per level.
 */
int fast_partition(const fast_cst* c, const fast_config* cfg, void* stream, fast_chunks** out);

/*
 * The partitions of nq CSTs built together (Sec. IV-B, Algorithm 2, as
 * fast_partition): the pending parts of all CSTs are processed level by
 * level in one set of launches, with one host round trip per level for the
 * whole batch (two when some CST's level hits its max_chunks).  outs[i]
 * receives CST i's chunk list, the same list in the same order as
 * fast_partition gives with cfg (NULL: each CST's own configuration); free
 * each with fast_free_chunks.  status[i] is FAST_OK, or FAST_ERR_INVALID for
 * a NULL CST (outs[i] is then NULL).  csts, outs and status are host arrays
 * of nq entries.  Returns FAST_ERR_INVALID for bad arguments, FAST_ERR_OOM or
 * FAST_ERR_CUDA when the batch fails (every outs[i] is then NULL), else
 * FAST_OK.
 */
int fast_partition_batch(const fast_cst* const* csts, int32_t nq, const fast_config* cfg, void* stream,
                         fast_chunks** outs, int32_t* status);

/* Number of chunks, and their summed workload estimate (saturating; summed
 * on request: asking for it reads the descriptors back on the partition's
 * stream and synchronises it). */
int fast_chunks_info(const fast_chunks* ch, int64_t* count, uint64_t* w_sum);

/*
 * A new chunk list holding chunks idx[0..n) of ch (host indices, in that
 * order; each in 0..count-1, else FAST_ERR_INVALID), for the same CST: a
 * rank's share when the chunks of one query are split over several GPUs
 * (partitions are disjoint, complete search spaces, Sec. IV-B, so the
 * counts of the shares add up to the query's).  Free with fast_free_chunks.
 * Synchronises `stream`.
 */
int fast_chunks_select(const fast_chunks* ch, const int64_t* idx, int64_t n, void* stream, fast_chunks** out);

/*
 * Copy the chunk descriptors to host arrays of `count` entries: j[i],
 * prefix[i][k] (candidate-local indices of positions 0..j-1; -1 beyond),
 * a[i], b[i], w[i] (W', saturating uint64), id[i] (sampling id).
 */
int fast_chunks_copy(const fast_chunks* ch, int32_t* j, int32_t* prefix, int64_t* a, int64_t* b,
                     uint64_t* w, uint64_t* id, void* stream);

void fast_free_chunks(fast_chunks* ch);

/* ---------------------------------------------------------------- match */

/*
 * Enumerate the embeddings in `chunks` (NULL: the whole CST as one chunk)
 * -- the semantics of Algorithms 4-8 (Sec. V-A): every partial result is
 * extended by the candidates of the next position in the tree list of its
 * parent's image (Generator), kept only if the new vertex is not already
 * used (VisitedValidator) and is adjacent to the images of its earlier
 * non-tree neighbours in the CST (EdgeValidator), and reported once complete
 * (Synchronizer).  The Generator may scan whichever of those lists is
 * shortest (their intersection is the same set).
 *   k:           embeddings to write (0: count only).
 *   emb_out:     k rows x |V(q)| uint32 data-vertex ids, column u = M(u)
 *                (query vertex id order); any k embeddings of the
 *                enumerated set, each once.  NULL iff k == 0.  Device (or
 *                managed) memory is written by the kernel directly; any
 *                other pointer is taken as host memory: the rows go to a
 *                library-owned device buffer of min(k, limit) rows first
 *                and are copied to emb_out before the call returns.
 *   count_out:   host; total number of embeddings in the chunks.
 *   written_out: host; rows written = min(k, count).
 *   chunk_counts: optional device buffer of one uint64 per chunk (with
 *                chunks NULL, one: the count of the whole CST).  Given, it
 *                keeps every run on the warp that took it (no donation).
 * The call synchronises `stream`.  FAST_ERR_TIMEOUT (time budget spent)
 * and FAST_ERR_OVERFLOW leave a partial or saturated count in *count_out.
 */
int fast_match(const fast_cst* c, const fast_chunks* chunks, uint64_t k, uint32_t* emb_out,
               uint64_t* count_out, uint64_t* written_out, void* stream);

/* fast_match with an explicit launch configuration and per-chunk counts. */
int fast_match_ex(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg, uint64_t k,
                  uint32_t* emb_out, uint64_t* count_out, uint64_t* written_out, uint64_t* chunk_counts,
                  void* stream);

/*
 * Counting pass over the same search: out[0] = bytes the search requested
 * (as fast_last_match_bytes), out[1 + d] for d < k = partial results with
 * d+1 positions mapped that pass every check.  out has k + 1 entries; host
 * memory.
 */
int fast_match_stats(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg, uint64_t* out,
                     void* stream);

/* --------------------------------------------------------------- batch */

typedef struct fast_batch fast_batch;

/*
 * A reusable context for matching many queries in one matcher launch (the
 * data-parallel use of independent CSTs the paper notes in its multi-FPGA
 * discussion, Sec. VI, on one device).  Owns fixed device buffers for up to
 * max_queries queries, `threads` host worker threads' CUDA streams (<= 0:
 * 8), and, once run, a CUDA graph of the matcher launch that later runs
 * replay.  cfg (NULL: defaults) seeds every query-size class's configuration
 * (classes: |V(q)| <= 4, 8, 16, 24, 32); cfg->limit, time_budget_s and
 * build_rule apply to every query of a run.  FAST_ERR_INVALID for a
 * build_rule outside 0..2, or a refine_rule other than 0 (or 2 with
 * build_rule >= 1).  Uses the current CUDA device.  One call at a
 * time per fast_batch (its buffers, graph and per-worker scratch pools are
 * shared by its runs); separate fast_batch objects may run concurrently.
 */
int fast_batch_create(const fast_graph* g, const fast_config* cfg, int32_t max_queries, int32_t threads,
                      fast_batch** out);

/*
 * Match nq queries (nq <= max_queries): the worker threads build each
 * query's CST and partition concurrently on their own streams (cfg's
 * build_rule 1: the CSTs of all queries are built together first, 2: the
 * partitions too); then one graph-replayed matcher launch enumerates all
 * chunks of all queries, warps sharing work across queries.  counts_out[i] (host) = number of embeddings
 * of query i (min(total, limit) when cfg->limit > 0); status_out[i] (host) =
 * FAST_OK, the error of that query's CST build or partition (the others
 * still run), or FAST_ERR_TIMEOUT when the time budget ended the launch
 * before the query was done.  Synchronises `stream`.
 */
int fast_batch_run(fast_batch* b, int32_t nq, const fast_query_desc* queries, uint64_t* counts_out,
                   int32_t* status_out, void* stream);

/* Last run: wall time of the CST/partition phase, event time of the matcher
 * launch, bytes the matcher requested, and chunks matched. */
int fast_batch_timing(const fast_batch* b, double* build_ms, double* match_ms, uint64_t* match_bytes, int64_t* chunks);

/* Last run's matcher launch: bytes requested (as fast_last_match_bytes) and
 * their floor (as fast_last_match_floor_bytes), over all its queries. */
int fast_batch_bytes(const fast_batch* b, uint64_t* requested, uint64_t* floor);

/* Read (get != NULL) and/or replace (set != NULL) the configuration of the
 * size class that a query of size_class_k vertices falls into. */
int fast_batch_config(fast_batch* b, int32_t size_class_k, fast_config* get, const fast_config* set);

/*
 * Autotune on sample queries: per size class present in the sample, the
 * partition's delta_w and max_chunks (how deep the level-synchronous
 * partition goes before the depth-first matcher takes over), then the
 * matcher's launch shape (warps per CTA, CTAs per SM), each choice by the
 * wall time of batch runs over the sample (the better of two runs per
 * choice).  *best_ms (nullable) receives
 * the best full-sample time.  Results stay in the batch's configuration.
 */
int fast_batch_autotune(fast_batch* b, int32_t nq, const fast_query_desc* sample, double* best_ms, void* stream);

void fast_free_batch(fast_batch* b);

/* One-shot: create a batch for nq queries, run it, free it. */
int fast_match_batch(const fast_graph* g, int32_t nq, const fast_query_desc* queries, const fast_config* cfg,
                     uint64_t* counts_out, int32_t* status_out, void* stream);

/* ------------------------------------------------------------- serving */

typedef struct fast_server fast_server;

/* One finished request. Times are fast_now_ns() readings. */
typedef struct {
    uint64_t id;
    uint64_t count;          /* embeddings (min(total, limit) when cfg->limit > 0) */
    int32_t status;          /* FAST_OK, a CST/partition/match error, or FAST_ERR_OOM when the
                                request's projected bytes exceed the whole budget */
    int32_t pad;
    uint64_t t_arrive_ns;    /* submitted */
    uint64_t t_start_ns;     /* admitted into a group */
    uint64_t t_done_ns;      /* count known */
} fast_result;

/*
 * A request loop over the resident data graph g (the host/accelerator task
 * flow of Sec. IV, kept on one GPU) with continuous batching: requests wait
 * in a FIFO queue; each of `workers` group workers (<= 0: 4), with its own
 * CUDA stream and its own batch (as fast_batch_create with cfg, up to 1024
 * requests), takes every request at the head of the queue whose projected
 * device bytes -- label buckets and neighbour lists its CST can hold, plus
 * the matcher's scratch -- fit in what budget_bytes leaves (the head
 * request is always admitted when nothing runs) and runs them as one batch:
 * their CSTs and partitions are built together (cfg->build_rule) and one
 * matcher launch enumerates all of them (cfg->warps_per_block warps per
 * CTA; cfg->blocks_per_sm CTAs per SM, or one for a group of at most four
 * requests, so that the launches of several small groups share the SMs).  Requests arriving while a group is on the GPU
 * form the next group; with two or more workers one group's build overlaps
 * another's matcher on the device.  cfg NULL: defaults.  Errors as
 * fast_batch_create.
 */
int fast_server_create(const fast_graph* g, const fast_config* cfg, uint64_t budget_bytes, int32_t workers,
                       fast_server** out);

/* Queue one query (its arrays are copied); *id_out (nullable) gets its id.
 * FAST_ERR_INVALID here only for a NULL server or query, a vertex count
 * outside 1..32, NULL arrays or a negative edge count; any other malformed
 * query (an edge endpoint out of range, a loop, a negative label, a
 * disconnected graph) is queued and comes back with status FAST_ERR_INVALID
 * in its result. */
int fast_server_submit(fast_server* s, const fast_query_desc* q, uint64_t* id_out);

/* Move up to max_results (>= 0) finished requests into out (any order),
 * waiting up to wait_ms for the first one when none is ready; *n_out = how
 * many. */
int fast_server_poll(fast_server* s, int32_t max_results, fast_result* out, int32_t* n_out, int32_t wait_ms);

/* Requests queued, requests running, projected bytes admitted. */
int fast_server_stats(fast_server* s, int64_t* pending, int64_t* running, uint64_t* in_use_bytes);

/* Groups formed so far and the requests they held (their mean size). */
int fast_server_groups(fast_server* s, uint64_t* groups, uint64_t* requests);

/* Stop: requests still queued are dropped, running ones finish. */
void fast_server_destroy(fast_server* s);

/* The steady clock of the result timestamps, in nanoseconds. */
uint64_t fast_now_ns(void);

/*
 * fast_match_noalloc -- fast_match for callers that must not allocate device
 * memory.  This entry point has no counterpart in the paper; it exists for
 * embedders whose device memory is already owned by another allocator (a
 * framework's caching pool that holds the whole GPU), for serving loops that
 * forbid allocator calls once they are running so that latency and memory
 * stay fixed, and for code on threads or callbacks where the CUDA allocator
 * must not be entered.  Every other entry point allocates stream-ordered
 * scratch; this one allocates nothing -- no cudaMalloc, cudaMallocAsync or
 * cudaFree, no host staging buffer.
 *
 * Scratch: one file-scope device array of fast_match_noalloc_scratch_bytes()
 * bytes (about 5.9 MB: the counter block, a ring of 4096 donated runs and
 * up to 32768 root-run descriptors) that every GPU loading the library keeps
 * until the process exits.  The first call on a device looks up its address
 * (cudaGetSymbolAddress, with that device current).  All calls share the
 * array and leave the last call's contents in it; each call clears what
 * must start at zero.  Calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * the shared array and must be serialised by the caller.
 *
 * Arguments as fast_match_ex (no per-chunk counts), except: emb_out must be
 * device (or managed) memory when k > 0 -- a host buffer would need staging
 * -- and, with chunks == NULL, the launch shape may ask for at most 32768
 * root runs (4 per warp).  Either violation returns FAST_ERR_INVALID with a
 * message; nothing runs.  The call synchronises `stream`.
 */
int fast_match_noalloc(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg, uint64_t k,
                       uint32_t* emb_out, uint64_t* count_out, uint64_t* written_out, void* stream);

/* Size in bytes of the static scratch array fast_match_noalloc uses. */
uint64_t fast_match_noalloc_scratch_bytes(void);

/* ---------------------------------------------------------- measurement */

/* Testing hook (failure injection on the host): the next `after` device
 * allocations of the library succeed and the one after them fails with
 * FAST_ERR_OOM, once; after < 0 turns it off (the default).  It drives every
 * allocation error path without touching the GPU.  Returns the countdown it
 * replaces: >= 0 while the failure is still to come, -1 once it has happened
 * (or when it was off). */
int64_t fast_inject_alloc_failure(int64_t after);

/* Duration in milliseconds of the last matcher kernel launched by this host
 * thread, measured with CUDA events recorded on the launching stream around
 * the kernel (0 if none ran). */
double fast_last_match_ms(void);

/* Bytes the last fast_match on this host thread requested from memory:
 * 16 B of offsets per list opened (a tree list per extended partial result,
 * a non-tree list per earlier non-tree neighbour), 4 B per generator-list
 * entry scanned, 4 B per list entry the membership checks read (merge tiles,
 * gallops, the prefix checks' binary searches), 4 B per data-vertex id
 * gathered, and 4|V(q)| B per embedding written.  Counted by every lane of
 * the search itself, whichever level of the memory hierarchy serves it. */
uint64_t fast_last_match_bytes(void);

/* The floor of fast_last_match_bytes for the same launch: what any search
 * over the CST that scans the shortest list into each position must read.
 * Per extension of a partial result to position d: the new image (4 B),
 * 16 B of offsets for the tree list and for each earlier non-tree
 * neighbour's list into d, and 4 B per entry of the shortest of those lists;
 * per candidate in all of them while an earlier position has its label, its
 * data vertex (4 B); per embedding written, 4|V(q)| B.  A chunk of a
 * partition that starts at position j > 0 counts its run as one such
 * extension.  Without a partition the count is independent of how the
 * work is spread over warps, and equals the oracle's floor for the same CST
 * and order. */
uint64_t fast_last_match_floor_bytes(void);

/* Kernels launched by the library since the process started (all threads). */
uint64_t fast_kernel_launches(void);

/* Host round trips (device-to-host size reads the host waited for) of the
 * calling thread's last batched CST build (fast_build_cst_batch, or a batch
 * run with build_rule 2).  A batch of at most 8 queries whose bounded
 * top-down arrays fit in 2 GB builds its top-down pass with none: its
 * arrays are sized by host-known bounds (|C0| of the parent, the graph's
 * count of adjacency entries between the two labels) and the kernels read
 * the real sizes on the device. */
uint64_t fast_last_build_round_trips(void);

#ifdef __cplusplus
}
#endif

#endif /* FAST_GB300_H */
