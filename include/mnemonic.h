/*
 * mnemonic.h -- C ABI of a B300-native incremental subgraph matcher for
 * streaming multigraphs (Mnemonic, arXiv 2206.09983).
 *
 * Problem (Sec. II-B, "Problem Definition"): given a data graph G, a query
 * graph G_Q and a batch dG of edge insertions (or deletions), report the
 * embeddings dS that appear (or disappear), so that S(G + dG) = S(G) + dS.
 * The driver loop of Alg. 1 applies each snapshot's insertions first and its
 * deletions second; one call of mn_insert_batch is one such snapshot for a
 * count window (window_edges > 0): insert the batch, then expire the oldest
 * edges beyond the window.
 *
 * Data edges keep their own identity (Sec. I, Sec. II-A: every edge has an
 * id, so parallel edges with distinct timestamps are distinct).  Here the id
 * of an edge is its arrival sequence number `seq` (0, 1, 2, ... over the life
 * of the graph).  Timestamps must be strictly increasing in arrival order.
 *
 * Embedding (Sec. II-B): a vertex map f and an edge map g with
 * src(g(e)) = f(s(e)), dst(g(e)) = f(t(e)); query vertex label mask a subset
 * of the data vertex's mask (0 = any); query edge label -1 (any) or equal;
 * edge attribute and timestamp inside the query edge's half-open ranges;
 * MN_ISO requires f injective, MN_HOMO does not (Sec. III); temporal
 * constraints require ts(g(a)) < ts(g(b)) for precedence pairs (Sec. VII-C).
 *
 * Result records (one per embedding) are, per query, nv uint32 vertex ids
 * (f(u_0) ... f(u_{nv-1})), zero padding to an 8-byte boundary, then ne
 * uint64 edge seqs (seq(g(e_0)) ... seq(g(e_{ne-1}))); mn_record_layout
 * gives the size.  Records come in no particular order.
 *
 * Errors: every call returns MN_OK (0) or a negative mn_status; the message
 * of the last failing call on a graph is in mn_last_error.  On a validation
 * error nothing is applied.  Handles are not thread-safe: one thread per
 * graph handle; distinct handles are independent.
 *
 * Ownership: every input pointer is read before the call returns; the
 * library copies what it keeps.  Count arrays in mn_batch_result are owned by
 * the library and stay valid until the next call on the same graph.
 * Embedding lists stay on the device until the next insert/delete call.
 */
#ifndef MNEMONIC_H
#define MNEMONIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mn_status;

#define MN_OK                    0
#define MN_ERR_INVALID_ARG      -1  /* bad pointer, size, flag or query */
#define MN_ERR_INVALID_VERTEX   -2  /* vertex id >= num_vertices or label >= num_edge_labels */
#define MN_ERR_TS_ORDER         -3  /* timestamps not strictly increasing */
#define MN_ERR_OOM              -4  /* device allocation failed or over mem_budget_bytes */
#define MN_ERR_ADMISSION        -5  /* batch larger than max_batch or the ring is full */
#define MN_ERR_OUTPUT_OVERFLOW  -6  /* result lists beyond mem_budget_bytes; counts exact */
#define MN_ERR_TIMEOUT          -7  /* a bounded device wait gave up */
#define MN_ERR_DEVICE           -8  /* a CUDA call failed */
#define MN_ERR_STATE            -9  /* call not valid in the graph's current state */

#define MN_MAX_QV 16           /* query vertices */
#define MN_MAX_QE 16           /* query edges */
#define MN_LABEL_ANY (-1)

#define MN_ISO  0
#define MN_HOMO 1

#define MN_TEMPORAL_NONE  0    /* no ordering */
#define MN_TEMPORAL_CHAIN 1    /* ts(g(e_0)) < ts(g(e_1)) < ... in declaration order */
#define MN_TEMPORAL_PAIRS 2    /* ts(g(a)) < ts(g(b)) for each listed pair (a, b) */

/* insert/delete flags */
#define MN_DEVICE_PTR 0x1u     /* the edge (or seq) array is device memory */
#define MN_COUNT_ONLY 0x2u     /* count embeddings, keep no lists */
#define MN_ASYNC      0x4u     /* mn_insert_batch only queues the batch; mn_batch_wait completes it */

/* fetch destination flags */
#define MN_DST_HOST   0x0u
#define MN_DST_DEVICE 0x1u
#define MN_FETCH_SORTED 0x2u   /* records in ascending (vertex tuple, edge-seq tuple) order */

typedef struct mn_graph mn_graph;

/* One data edge as the caller hands it in (24 bytes, ts 8-byte aligned). */
typedef struct {
    uint32_t src, dst;      /* vertex ids < num_vertices */
    uint32_t label;         /* edge label < num_edge_labels */
    int32_t  attr;          /* edge attribute */
    int64_t  ts;            /* timestamp, strictly increasing over the stream */
} mn_edge;

typedef struct {
    uint32_t num_vertices;
    uint32_t num_edge_labels;            /* 1..256 */
    const uint32_t *vertex_label_mask;   /* host, num_vertices entries, copied; NULL = all 0 */
    uint64_t window_edges;               /* count window W; 0 = insert-only */
    uint64_t max_batch;                  /* largest insert or delete batch */
    uint64_t edge_capacity;              /* insert-only: most edges ever held; ignored with a window */
    uint64_t out_capacity;               /* initial records per (query, sign) list; 0 = 1M */
    uint64_t mem_budget_bytes;           /* cap on device memory the graph may hold; 0 = none */
    uint32_t max_queries;                /* 1..64 */
    int32_t  device;                     /* CUDA device ordinal */
    void    *cuda_stream;                /* cudaStream_t to run on; NULL = the graph makes one */
} mn_graph_config;

typedef struct {
    uint32_t src, dst;                   /* query vertex ids < nv; src != dst */
    int32_t  label;                      /* edge label or MN_LABEL_ANY */
    int32_t  attr_lo, attr_hi;           /* attr in [attr_lo, attr_hi) */
    int32_t  pad_;
    int64_t  ts_lo, ts_hi;               /* ts in [ts_lo, ts_hi) */
} mn_qedge;

typedef struct {
    uint32_t nv, ne;                     /* 2..MN_MAX_QV vertices, 1..MN_MAX_QE edges, connected */
    const uint32_t *vlabel_mask;         /* nv entries; NULL = all 0 (any) */
    const mn_qedge *edges;               /* ne entries; no two with the same (src, dst) */
    uint32_t semantics;                  /* MN_ISO or MN_HOMO */
    uint32_t temporal;                   /* MN_TEMPORAL_* */
    uint32_t n_prec;                     /* MN_TEMPORAL_PAIRS: number of pairs */
    const uint32_t *prec;                /* 2 * n_prec query-edge indices (a, b) */
} mn_query_desc;

typedef struct {
    uint64_t batch_id;                   /* 1, 2, ... per insert/delete call */
    uint64_t seq_lo, seq_hi;             /* seqs given to the inserted edges */
    uint64_t expired_lo, expired_hi;     /* seqs that left the window in this call */
    uint32_t num_queries;
    const uint64_t *count_pos;           /* per query |dS+| (library-owned) */
    const uint64_t *count_neg;           /* per query |dS-| (library-owned) */
} mn_batch_result;

/* Create an empty graph on `device` (Sec. III, InitializeStream: window size
 * and batch size are the snapshot generator's parameters).  Allocates the
 * edge ring, the label-partitioned adjacency and its delta buffers on the
 * device.  *out is NULL on error. */
mn_status mn_create_graph(const mn_graph_config *cfg, mn_graph **out);

/* Free every device and host resource of the graph; NULL is ignored. */
void mn_destroy_graph(mn_graph *g);

/* Register a query (Sec. III, InitializeIndex: root, query tree and one
 * matching order per starting query edge, Sec. VI "Matching order
 * computation"; masks of Table I) and build its DEBI words over the live
 * edges (Sec. IV-A).  No embeddings are reported for edges already live.
 * *query_id receives 0, 1, ... in registration order. */
mn_status mn_register_query(mn_graph *g, const mn_query_desc *q, uint32_t *query_id);

/* One snapshot (Alg. 1; Alg. 2 batchInserts then batchDeletes): append n
 * edges (host array, or device array with MN_DEVICE_PTR), report dS+ for
 * every query, then, with a window, expire the oldest edges beyond
 * window_edges and report dS- computed before their removal.  n may be 0.
 * `out` may be NULL.  With MN_ASYNC the call only queues the batch (see
 * mn_batch_wait). */
mn_status mn_insert_batch(mn_graph *g, const mn_edge *edges, uint64_t n, uint32_t flags,
                          mn_batch_result *out);

/* Complete the batch that mn_insert_batch queued with MN_ASYNC (Sec. V-A:
 * one snapshot's work runs on the GPU while the host prepares the next).
 * With MN_ASYNC, mn_insert_batch returns once every kernel of the snapshot is
 * queued on the graph's stream; its `out` gets the batch id, seq ranges and
 * count arrays whose values are valid only after mn_batch_wait returns.  The
 * host edge array must stay valid until then.  mn_batch_wait waits for the
 * enumeration, grows and re-runs result lists that overflowed, commits the
 * batch (or, on a validation error such as MN_ERR_TS_ORDER, applies nothing)
 * and fills `out` (may be NULL) as a synchronous insert would; it returns
 * what that insert would have returned.  While a batch is pending, the calls
 * that read or change the graph (insert, delete, fetch, register, static
 * counts, DEBI and adjacency reads, training) return MN_ERR_STATE.  A
 * batch_id that was already completed gives MN_OK; an unknown one
 * MN_ERR_INVALID_ARG. */
mn_status mn_batch_wait(mn_graph *g, uint64_t batch_id, mn_batch_result *out);

/* Explicit deletion of live edges by seq (Alg. 2 batchDeletes): report dS-
 * on the graph before removal, then remove them.  Every seq must be live and
 * listed once. */
mn_status mn_delete_batch(mn_graph *g, const uint64_t *seqs, uint64_t n, uint32_t flags,
                          mn_batch_result *out);

/* Copy records [offset, offset + max_records) of the last batch's list for
 * (query_id, sign: +1 new, -1 removed) to dst (host, or device with
 * MN_DST_DEVICE).  *n_written gets the number copied.  batch_id must be the
 * last batch's id.  Records come in no particular order unless
 * MN_FETCH_SORTED is set: the list is then sorted on the device (the first
 * sorted fetch of a batch sorts it in place, with scratch of 8 B plus one
 * record per record, allocated for the sort and freed; later fetches of the
 * batch, sorted or not, return sorted records), ascending by the vertex ids
 * f(u_0), ..., f(u_{nv-1}) and then the edge seqs; MN_ERR_INVALID_ARG for a
 * list above 2^32 records, MN_ERR_OOM if the scratch cannot be allocated. */
mn_status mn_fetch_embeddings(mn_graph *g, uint64_t batch_id, uint32_t query_id, int32_t sign,
                              uint64_t offset, uint64_t max_records, void *dst,
                              uint32_t dst_flags, uint64_t *n_written);

/* Record layout of a query's results: vertex count, edge count, bytes. */
mn_status mn_record_layout(const mn_graph *g, uint32_t query_id, uint32_t *nv, uint32_t *ne,
                           uint32_t *record_bytes);

/* |S(G)| for a query over the live window (Sec. II-B), by seeding every live
 * edge at query edge 0. */
mn_status mn_count_static(mn_graph *g, uint32_t query_id, uint64_t *count);

/* Matching-order policies (mn_set_order_policy).  Every candidate order is
 * a connected order of the query, so the policy changes the work, never the
 * result.  Candidate 0 is the paper's order (Sec. III preprocessing: most
 * selective root, BFS tree; Sec. VI: per-seed order, path to the root first);
 * candidates 1-3 are greedy alternatives (most-connected vertex next,
 * query edge nearest in declaration order next, highest query degree next). */
#define MN_ORDER_PAPER   0   /* always candidate 0 (default) */
#define MN_ORDER_EXPLORE 1   /* a pseudo-random candidate per seed; per-seed SM cycles are logged for training */
#define MN_ORDER_LEARNED 2   /* the candidate with the smallest predicted cost, if it beats the
                                paper's order by at least the query's margin
                                (mn_set_order_margin; default 2x); otherwise the
                                paper's order */

#define MN_MLP_FEATURES 16
/* FP32 parameter block of the work model, in this order: W1[16][128],
 * b1[128], W2[128][128], b2[128], w3[128], b3 (row-major, input-major). */
#define MN_MLP_PARAMS 18817

mn_status mn_set_order_policy(mn_graph *g, uint32_t policy);

/* Train the work model on the samples logged under MN_ORDER_EXPLORE: full
 * batch Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error
 * of log2(1 + cycles) (the SM cycles the enumerator spent per seed), `epochs`
 * steps, each gradient on the tensor cores (see mn_mlp_gradient); the loss
 * before the first and after the last step go to *loss_first / *loss_last
 * (either may be NULL).  MN_ERR_STATE if nothing has been logged,
 * MN_ERR_TIMEOUT if an MMA completion was not seen within the wait bound. */
mn_status mn_train_order_model(mn_graph *g, uint32_t epochs, float lr, float *loss_first,
                               float *loss_last);

/* Copy the model's MN_MLP_PARAMS parameters to host `get` (if not NULL),
 * then replace them with host `set` (if not NULL). */
mn_status mn_order_model_params(mn_graph *g, float *get, const float *set);

/* Test hooks of the model's kernels, host pointers, on `device`: the
 * tensor-core (tcgen05) forward pass over n rows of 16 BF16 features (x holds
 * raw BF16 bit patterns) into y[n], and the tensor-core gradient of the mean
 * squared error against targets t[n] into grad[MN_MLP_PARAMS] with the loss
 * in *loss.  Both use BF16 weights and BF16 layer-1 activations with FP32
 * accumulation; the gradient also rounds dZ2 and dZ1 to BF16 as MMA
 * operands.  MN_ERR_TIMEOUT if an MMA completion was not seen within the
 * kernels' wait bound. */
mn_status mn_mlp_forward(int32_t device, const float *params, const uint16_t *x, uint64_t n,
                         float *y);
mn_status mn_mlp_gradient(int32_t device, const float *params, const uint16_t *x, const float *t,
                          uint64_t n, float *grad, float *loss);

/* Dual simulation of a registered query over the live window (Sec. III
 * names it among the matching variants the index serves; Sec. VII-C runs it
 * per snapshot): the largest relation S between query vertices u and data
 * vertices v such that v carries u's vertex labels and, for every query edge
 * e leaving (entering) u, some live data edge leaving (entering) v matches e
 * (the edgeMatcher, i.e. its DEBI bit e) and leads to (comes from) a data
 * vertex related to e's other endpoint.  If some query vertex is related to
 * no data vertex the query does not match and S is empty.  Temporal
 * precedence is ignored (it constrains edge instances, not vertices).
 * sim (host, or device with MN_DST_DEVICE; may be NULL) receives
 * num_vertices words, bit u of word v set iff (u, v) is in S; *pairs (may be
 * NULL) gets |S|.  The relation is recomputed from the index on every call;
 * the first call allocates num_vertices words of device scratch (kept until
 * mn_destroy_graph; MN_ERR_OOM beyond mem_budget_bytes).  The passes run
 * in groups of 8 per host check; mn_stats.dualsim_passes counts them.  MN_ERR_INVALID_ARG
 * for an unknown query_id, MN_ERR_STATE while a queued batch is pending. */
mn_status mn_dual_simulation(mn_graph *g, uint32_t query_id, uint32_t *sim, uint32_t dst_flags,
                             uint64_t *pairs);

/* Device memory the graph holds now (*used), the most it has held (*peak)
 * and its budget (mem_budget_bytes, 0 = none), in bytes (Sec. VII-D measures
 * the index's memory over a stream).  Any pointer may be NULL; the only error
 * is a NULL graph (MN_ERR_INVALID_ARG). */
mn_status mn_memory_info(const mn_graph *g, uint64_t *used, uint64_t *peak, uint64_t *budget);

/* Periodic reset (Sec. VII-D: the cumulative index can be discarded at any
 * snapshot and rebuilt from it): every registered query's DEBI words are
 * cleared and recomputed by the edgeMatcher over the live window.  The words
 * here are a function of each edge alone, so the rebuilt index equals the old
 * one and later results are unchanged; the call restores that state after
 * anything that disturbed it.  MN_ERR_STATE while a queued batch is
 * pending. */
mn_status mn_reset_index(mn_graph *g);

/* Time-window snapshots instead of a count window (Sec. VII-D: the LANL
 * stream runs with a 24-hour window): after each insert batch whose newest
 * timestamp is T, the live edges with ts <= T - window expire, with their dS-
 * reported as for a count window (computed before their removal; they can
 * include edges of the batch itself).  Only for graphs created without a
 * count window (window_edges = 0); edge_capacity must hold the live window
 * plus a batch, else the insert returns MN_ERR_ADMISSION.  window = 0 turns
 * it off.  Each insert then reads the cut back from the device once (one
 * extra host synchronisation). */
mn_status mn_set_time_window(mn_graph *g, int64_t window);

/* Seed sharding of one stream over `count` graphs, one per GPU.  The work
 * units of Sec. VI "Work decomposition" are the seeds, and any partition of
 * them gives the same union.  This graph enumerates only the seeds (seq,
 * query, query edge) whose hash modulo count is `index`.  Every shard ingests
 * the whole stream (a search reaches any part of the window); counts and
 * lists are then this shard's part: disjoint across shards, summing (and
 * concatenating) to the unsharded result.  Applies to inserts, deletes and
 * static counts.  Default: index 0 of 1 (no sharding).  MN_ERR_INVALID_ARG
 * unless index < count; MN_ERR_STATE while a queued batch is pending. */
mn_status mn_set_shard(mn_graph *g, uint32_t index, uint32_t count);

/* Launch parameters of the enumerator (none changes any result): resident
 * blocks of 4 warps per SM in its persistent grid (0 = the occupancy limit, 5 on B300),
 * the smallest candidate range a busy warp hands to an idle one (0 = 40; at
 * least 33), the deepest search depth that may be split (0 = any), and the
 * preferred shared-memory carve-out in percent of the SM's unified L1/shared
 * storage (-1 = the driver's choice; less shared memory leaves more L1 for
 * the adjacency and DEBI reads).  mn_get_tuning reads them back with the
 * occupancy limit. */
mn_status mn_set_tuning(mn_graph *g, uint32_t blocks_per_sm, uint32_t split_min, uint32_t split_depth,
                        int32_t smem_carveout);
mn_status mn_get_tuning(const mn_graph *g, uint32_t *blocks_per_sm, uint32_t *max_blocks_per_sm,
                        uint32_t *split_min, uint32_t *split_depth, int32_t *smem_carveout);

/* Learned work splits (the learned counterpart of the paper's pull-based
 * distribution of work units, Sec. VI): under MN_ORDER_LEARNED, a seed whose
 * predicted work under its chosen order is at least 2^log2_cycles SM cycles
 * has the candidate range of its first search depth handed to the
 * work-splitting queue in up to 16 pieces as soon as a warp takes it, instead
 * of waiting for idle warps to ask.  log2_cycles <= 0 turns it off (the
 * default); NaN is MN_ERR_INVALID_ARG.  Results are unaffected.
 * mn_get_presplit reads the threshold back (0 = off). */
mn_status mn_set_presplit(mn_graph *g, float log2_cycles);
mn_status mn_get_presplit(const mn_graph *g, float *log2_cycles);

/* Shared-memory staging of adjacency slices in the enumerator (Sec. III
 * enumerator, its candidate scans): a candidate range of the last two search
 * depths -- swept 32 entries at a time with no descent in between -- that
 * holds at least min_entries entries is read through two shared-memory
 * windows of 128 entries per warp, each filled by bulk asynchronous copies
 * (the TMA unit) of the range's neighbour and seq slices, the next window
 * fetched while the current ones are tested.  min_entries = 0 turns it off
 * (the default); 1..31 is MN_ERR_INVALID_ARG.  Results are unaffected;
 * mn_stats.entries_staged counts the entries read this way.
 * mn_get_slice_staging reads the setting back. */
mn_status mn_set_slice_staging(mn_graph *g, uint32_t min_entries);
mn_status mn_get_slice_staging(const mn_graph *g, uint32_t *min_entries);

/* Online autotuning of the launch parameters above (under MN_ORDER_LEARNED
 * after the margin trial of mn_set_order_margin, below): each of the next
 * insert batches that enumerates runs under one candidate configuration,
 * `batches_per_config` batches each; then the configuration with the least
 * enumeration time per unit of work (adjacency entries tested + candidates
 * bound) is kept.  Results are unaffected.  The candidates (listed by
 * mn_autotune_candidates) are: resident blocks per SM at the occupancy limit
 * x split threshold {40, 64, 128} x split depth {3, any} x pre-split
 * threshold {off, 2^20, 2^22 cycles}, all without slice staging, plus split
 * threshold 40 at any depth with staging of ranges of at least {256, 1024}
 * entries (mn_set_slice_staging).  Then the DEBI filtering (mn_set_filtering)
 * is tried on 8 live inserting batches: it is turned on (its full pass to
 * build the sets is not timed) and kept up to date on all of them, while the
 * batches alternate between enumerating without it (timed over the
 * enumeration; their filter pass runs afterwards, untimed) and with it (timed
 * from the filter pass to the end of the enumeration), so that differences
 * between stretches of the stream fall on both arms alike; the filtering is
 * kept when it is at least 3% faster per inserted edge (it removes seeds and
 * candidates but costs a pass per batch, so which wins depends on the
 * queries).  mn_autotune_state reports whether tuning is
 * still running and how many of its batches are left; mn_autotune_filter_result
 * gives the trial's times (ms per 1,000 inserted edges) and choice
 * (MN_ERR_STATE before a trial has finished). */
mn_status mn_autotune(mn_graph *g, uint32_t batches_per_config);
mn_status mn_autotune_state(const mn_graph *g, int32_t *active, uint32_t *batches_left);
mn_status mn_autotune_filter_result(const mn_graph *g, double *ms_per_kedge_off, double *ms_per_kedge_on,
                                    int32_t *filtering_kept);

/* The learned order's margin, in log2 units of predicted cost (SM cycles):
 * under MN_ORDER_LEARNED a seed leaves the paper's order (Sec. III
 * preprocessing, the fallback) only for a candidate whose predicted cost is
 * at least 2^margin times smaller.  Each query has its own margin; the
 * default for every query is 1 (2x).  0 trusts the model outright; a large
 * margin keeps the paper's order.  Results are unaffected; only the work
 * changes.  mn_set_order_margin sets every query's margin (also of queries
 * registered later), mn_set_query_margin one registered query's
 * (MN_ERR_INVALID_ARG for another id); both refuse a negative, infinite or
 * NaN margin (MN_ERR_INVALID_ARG).  mn_get_order_margin reads a registered
 * query's margin, or with query_id = MN_DEFAULT_MARGIN the one queries
 * registered later get.
 *
 * How far the model's ranking can be trusted depends on the query, so when
 * mn_autotune starts under MN_ORDER_LEARNED it first runs a margin trial on 6
 * live inserting batches.  Only a seed whose model pick beats the paper's
 * order by a predicted gain in (0, 6) log2 units can be decided differently
 * by the candidate margins {0, 0.5, 1, 2, 3, 6}; such a seed takes the paper's
 * order or the pick with equal odds (drawn pseudo-randomly per seed), and
 * the enumerator logs the SM cycles of its work units per (query, gain
 * interval between two candidates, arm).  Since a margin picks the model's
 * order exactly for the intervals at or above it, each candidate's cycles
 * follow from the two arms' means per interval; each registered query keeps
 * the margin of the fewest estimated cycles (both arms run on random halves
 * of the same batches' seeds, so batch-to-batch differences cancel), and the
 * margin of the fewest cycles over all queries becomes the default for later
 * queries; the launch candidates and the filtering trial follow.  (Switching
 * the policy away from learned before the trial ends skips it.)
 * mn_autotune_margin_result gives, for candidate k < *n (= 6): margins[k],
 * cycles_per_seed[k] (the estimated SM cycles per trial seed under margin k,
 * over all queries) and, for registered query q, query_cycles_per_seed[q *
 * cap + k] (0 for a query none of whose seeds depended on the margin: it
 * keeps the default); any of the three may be NULL, and MN_ERR_INVALID_ARG if
 * cap is below *n.  *kept (may be NULL) gets the default margin chosen.
 * MN_ERR_STATE before a margin trial has finished. */
#define MN_DEFAULT_MARGIN 0xffffffffu
mn_status mn_set_order_margin(mn_graph *g, float log2_margin);
mn_status mn_set_query_margin(mn_graph *g, uint32_t query_id, float log2_margin);
mn_status mn_get_order_margin(const mn_graph *g, uint32_t query_id, float *log2_margin);
mn_status mn_autotune_margin_result(const mn_graph *g, uint32_t cap, float *margins, double *cycles_per_seed,
                                    double *query_cycles_per_seed, uint32_t *n, float *kept);

/* One candidate of the autotuner (presplit_log2 = 0: pre-splitting off;
 * slice_min = 0: no shared-memory staging, mn_set_slice_staging). */
typedef struct {
    uint32_t blocks_per_sm, split_min, split_depth;
    float presplit_log2;
    uint32_t slice_min;
} mn_tune_config;

/* Copy the autotuner's candidates to out[0..cap) (out may be NULL to ask for
 * the count); *n gets the count; MN_ERR_INVALID_ARG if out is too small. */
mn_status mn_autotune_candidates(mn_graph *g, uint32_t cap, mn_tune_config *out, uint32_t *n);

/* What the last mn_autotune measured per candidate: enumeration time (ms,
 * CUDA events on the graph's stream) and work (adjacency entries tested +
 * candidates bound) summed over its batches; zeros for candidates not yet
 * run.  *n gets the count; out (NULL: count only) must hold it. */
typedef struct {
    mn_tune_config config;
    double enumerate_ms;
    double work;
} mn_tune_result;
mn_status mn_autotune_results(const mn_graph *g, uint32_t cap, mn_tune_result *out, uint32_t *n);

/* Largest live window mn_count_static_noalloc accepts: its seed scratch
 * holds one 8-byte work unit per live edge. */
#define MN_NOALLOC_MAX_SEEDS (1u << 22)

/* The same count as mn_count_static, for callers that must not allocate
 * device memory during the call: code that runs while a memory pool is fully
 * reserved by another framework, real-time or serving loops that cannot
 * afford an allocation's latency or failure, and code whose allocations are
 * audited.  mn_count_static grows its seed buffer with cudaMalloc when the
 * window grows; this variant never calls cudaMalloc, cudaFree or any
 * allocating routine.  Its scratch is one fixed array in the library's
 * device memory (32 MiB plus 3 KiB; every GPU that loads the library holds it
 * until the process exits).  The paper has no counterpart.
 *   - The first call on a device looks up the array's device address with
 *     that device current and caches it; make that first call before any
 *     stream capture.
 *   - All calls share the array and it keeps the last call's contents; the
 *     call clears what must start at zero.  Calls that overlap on the GPU
 *     (two threads, two graphs, or two streams at once) race on it: run them
 *     one after another.
 *   - A live window larger than MN_NOALLOC_MAX_SEEDS edges is rejected with
 *     MN_ERR_INVALID_ARG before any work is queued. */
mn_status mn_count_static_noalloc(mn_graph *g, uint32_t query_id, uint64_t *count);

/* DEBI neighbourhood filtering (Sec. V-A "Batch Processing", Sec. IV-A):
 * on each query's tree (root = the most selective query vertex: fewest data
 * vertices carrying its labels per unit of query degree, ties to the smaller
 * id; BFS tree, neighbours in ascending (vertex, edge) order), the top-down
 * sets TD(u) (f1: reached from a root candidate along matching tree edges;
 * f2/f3 under isomorphism: at least as many live edges and distinct
 * neighbours per edge label and direction as u has query edges) and the
 * bottom-up sets BU(u) (f4: the subtree of u has matching edges into BU of
 * every child), one pass each, on the live graph.  The filtered DEBI bit of
 * a tree edge is its edgeMatcher bit with the parent side in TD and the child
 * side in BU; the enumerator binds query vertex u only to vertices of BU(u).
 * Results are unchanged (every embedding lies in the sets).  Enabling builds
 * the sets of every registered query (and of each one registered later);
 * afterwards they are maintained from the endpoints of the inserted, expired
 * and deleted edges (the unified frontier), before each enumeration.  The
 * state costs, per query, 3 bitmaps and one frontier list of num_vertices
 * entries per query vertex.  0 turns it off.  MN_ERR_STATE while a queued
 * batch is pending. */
mn_status mn_set_filtering(mn_graph *g, int32_t enable);

/* Test hook of the filtering: the query tree (root, parent[u] and the tree
 * edge into u, -1 at the root; nv entries each) and, with filtering on, the
 * bitmaps TD and BU (host arrays of nv * ceil(num_vertices / 32) words; bit
 * v of word u * ceil(V / 32) + v / 32).  Any pointer may be NULL; asking for
 * bitmaps with filtering off is MN_ERR_STATE. */
mn_status mn_read_filter(mn_graph *g, uint32_t query_id, uint32_t *td, uint32_t *bu, int32_t *root,
                         int32_t *parent, int32_t *tree_edge);

/* Copy the DEBI words (Sec. IV-A; bit e = the edge matches query edge e) of
 * the edges with seq in [seq_lo, seq_hi) to host memory `words` (uint32
 * each); edges not live read 0.  With filtering on, tree-edge bits are the
 * filtered ones (mn_set_filtering). */
mn_status mn_read_debi(mn_graph *g, uint32_t query_id, uint64_t seq_lo, uint64_t seq_hi,
                       uint32_t *words);

/* Copy the adjacency of direction dir (0 = out, 1 = in) to host memory:
 * entry i is (key[i] = v * num_edge_labels + label, nbr[i], seq[i]), sorted
 * by (key, nbr, seq), live edges only.  *n gets the entry count; arrays must
 * hold `cap` entries (MN_ERR_INVALID_ARG with *n set when they do not). */
mn_status mn_read_adjacency(mn_graph *g, uint32_t dir, uint64_t cap, uint32_t *key,
                            uint32_t *nbr, uint64_t *seq, uint64_t *n);

/* Live window [lo, hi) of seqs and the number of registered queries. */
mn_status mn_graph_info(const mn_graph *g, uint64_t *seq_lo, uint64_t *seq_hi,
                        uint32_t *num_queries);

/* Host spill of expired edges (Sec. IV-A, external memory support: edges
 * leaving the in-memory window are written out together with their index
 * entries, oldest out first).  Every edge that expires from the window (count
 * or time window) is copied, before its ring slot can be reused, into a
 * pinned host FIFO of capacity_edges edges: its mn_edge record, its seq and
 * the DEBI word of every registered query as it was when the edge left the
 * window.  The copies run asynchronously on the graph's stream.  The FIFO
 * holds the most recent capacity_edges expired seqs; older ones are
 * overwritten.  It costs capacity_edges * (32 + 4 * max_queries) bytes of
 * pinned host memory and max_batch * (32 + 4 * max_queries) bytes of device
 * staging.  Set once per graph (MN_ERR_STATE afterwards); MN_ERR_OOM if the
 * host memory cannot be pinned. */
mn_status mn_set_spill(mn_graph *g, uint64_t capacity_edges);

/* Read spilled edges with seqs in [seq_lo, seq_hi): edges[k] (may be NULL)
 * and words[q * (seq_hi - seq_lo) + k] (may be NULL) for the k-th seq.
 * *held_lo / *held_hi (may be NULL) get the seq range the FIFO holds; a
 * range outside it is MN_ERR_INVALID_ARG (the held range is still reported).
 * Waits for the graph's stream first. */
mn_status mn_read_spill(mn_graph *g, uint64_t seq_lo, uint64_t seq_hi, mn_edge *edges, uint32_t *words,
                        uint64_t *held_lo, uint64_t *held_hi);

/* Record each insert batch's kernel chain (ingest, adjacency update,
 * filtering, work units, order choice, enumeration of dS- and dS+) as one
 * CUDA graph and launch it as a whole: one launch instead of a few dozen.
 * The graph is captured per batch and updated in place (cudaGraphExecUpdate),
 * so batch sizes and positions may change; a change of the chain's shape
 * (e.g. another number of merge passes) instantiates it again.  Buffers the
 * chain could grow are sized before recording.  Batches with a time window
 * (a host wait inside the chain), with edges in pageable host memory, or
 * run under autotuning are launched kernel by kernel as before.  Results are
 * unchanged.  0 turns it off (the default); MN_ERR_STATE while a queued batch
 * is pending. */
mn_status mn_set_graph_capture(mn_graph *g, int32_t enable);

/* Bound the enumerator's work: each device warp gives up after max_iters
 * backtracking steps, sets a status word and returns (no spin, no trap).  The
 * batch is still applied to the graph, its counts are partial and the call
 * returns MN_ERR_TIMEOUT; later calls work normally.  0 = no limit (the
 * default).  Lets tests drive the bounded-wait path without faulting. */
mn_status mn_set_work_budget(mn_graph *g, uint64_t max_iters);

/* Bound of the enumerator's only device-side wait.  When a warp runs out of
 * work units (Sec. VI: work units are pulled), it takes a ticket of the
 * work-splitting queue and polls its slot (backing off to ~2 us per poll)
 * until a busy warp hands it a subtree there.  It gives the slot up -- the
 * normal exit, which never loses work: a warp that later publishes into an
 * abandoned slot keeps its task -- once no warp is busy, or after max_polls
 * polls even while warps are busy (0 = the default, 65,536 polls, ~0.13 s).
 * A slot that a publishing warp has reserved but not published within
 * another 4,096 polls (~8 ms; publishing takes microseconds) is given up
 * with a device status: the batch is applied, its counts may be partial and
 * the call returns MN_ERR_TIMEOUT; the graph stays usable.  max_polls above
 * 2^30 is MN_ERR_INVALID_ARG.  Flags: MN_WAIT_HOLD (a test hook) makes every
 * waiting warp neither take a task nor give up its slot, so each such wait
 * runs to its bound and reports MN_ERR_TIMEOUT: the timeout path can be
 * tested without faulting or hanging the GPU. */
#define MN_WAIT_HOLD 0x1u
mn_status mn_set_wait_limit(mn_graph *g, uint32_t max_polls, uint32_t flags);

/* Counters of one graph since creation (or the last mn_reset_stats).  Stage
 * times are device time measured with CUDA events on the graph's stream
 * around each stage when timing is enabled (mn_set_timing), else 0.  The
 * enumerator counters are summed on the device: seeds taken, adjacency
 * entries tested, candidates bound (search-tree nodes) and embeddings
 * emitted (Sec. VII-A counts traversed edges per update the same way). */
typedef struct {
    uint64_t kernel_launches;      /* kernels launched by the library */
    uint64_t batches;              /* insert/delete calls */
    uint64_t enumerate_launches;   /* launches of the enumerator */
    double   ms_ingest;            /* ingest + edgeMatcher */
    double   ms_adjacency;         /* delta sort, compaction, merge, offsets */
    double   ms_seeds;             /* work-unit compaction */
    double   ms_enumerate;         /* backtracking enumerator */
    double   ms_expire;            /* DEBI clear of expired edges */
    uint64_t seeds;
    uint64_t entries_scanned;
    uint64_t binds;
    uint64_t records;
    uint64_t busy_cycles;          /* SM cycles enumerator warps spent inside work units */
    uint64_t tasks_split;          /* subtrees handed from busy to idle warps */
    uint64_t h2d_bytes;            /* bytes the library copied host -> device */
    uint64_t d2h_bytes;            /* bytes copied device -> host (counts, status) */
    uint64_t rerun_launches;       /* enumerator launches that re-ran the seeds of overflowed lists */
    uint64_t dualsim_passes;       /* refinement passes run by mn_dual_simulation */
    double   ms_filter;            /* DEBI filtering passes (mn_set_filtering) */
    uint64_t seeds_filtered;       /* seeds skipped because an endpoint is outside the filtered sets */
    uint64_t filter_changes;       /* vertex-set memberships the filtering passes changed */
    uint64_t graph_launches;       /* insert batches launched as one CUDA graph (mn_set_graph_capture) */
    uint64_t graph_instantiations; /* graph instantiations (the rest were updated in place) */
    uint64_t spill_bytes;          /* bytes copied to the host spill (mn_set_spill) */
    uint64_t entries_staged;       /* adjacency entries read through staged windows */
    double   ms_model;             /* tensor-core forward of the work model (order choice) */
    uint64_t model_launches;       /* its launches */
    double   ms_train;             /* mn_train_order_model on the device (gradients + Adam) */
    uint64_t train_rows;           /* rows through the gradient kernel (samples x passes) */
} mn_stats;

/* Turn per-stage event timing on (1) or off (0, the default). */
mn_status mn_set_timing(mn_graph *g, int enable);

/* Copy the counters to *out. */
mn_status mn_get_stats(const mn_graph *g, mn_stats *out);

/* Zero the counters. */
mn_status mn_reset_stats(mn_graph *g);

/* Message of the last failing call on g (or of the last failing create when
 * g is NULL); never NULL. */
const char *mn_last_error(const mn_graph *g);

#ifdef __cplusplus
}
#endif

#endif /* MNEMONIC_H */
