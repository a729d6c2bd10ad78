// mn_graph.cu -- host runtime and C ABI (include/mnemonic.h) of the
// incremental subgraph matcher (Mnemonic, arXiv 2206.09983) on one B300.
//
// One graph handle owns, on its device:
//   an edge ring of capacity C (a power of two >= window + max batch) holding
//     src, dst, label, attr, ts per edge at slot = seq mod C; slots of
//     expired edges are reused (memory recycling, Sec. IV-A);
//   a label-partitioned adjacency per direction: entries (key = v*L + label,
//     nbr, seq32) sorted by (key, nbr, seq), double-buffered, rebuilt per
//     batch by merging the sorted batch delta into the live base entries,
//     plus offsets of every (vertex, label) segment;
//   per query a DEBI word per slot (Sec. IV-A) and result lists per sign.
// Every batch runs as one chain of kernels on the graph's stream with a
// single host synchronisation at the end (to return the counts).
#include <algorithm>
#include <cmath>
#include <climits>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mn_device.cuh"
#include "mn_learned.cuh"
#include "mn_dualsim.cuh"
#include "mn_filter.cuh"

using namespace mn;

namespace {

thread_local std::string g_create_error;

struct DirArrays {
    uint32_t *key = nullptr, *nbr = nullptr, *s32 = nullptr;
};

struct Ctrl {
    uint32_t status;
    uint32_t nseeds[3];
    uint32_t next_seed[3];
    uint32_t pad_;
    long long last_ts;
    unsigned long long work[8];
    unsigned long long counts[64 * 3];
    unsigned long long time_cut;        // edges a time window expires after this batch
};

enum Stage { S_INGEST = 0, S_ADJ, S_SEEDS, S_ENUM, S_EXPIRE, S_FILTER, S_MODEL, S_COUNT };

struct QueryHost {
    uint32_t nv = 0, ne = 0, iso = 0, temporal = 0;
    uint32_t rec_bytes = 0, goff = 0;
    std::vector<uint32_t> vmask;
    std::vector<mn_qedge> edges;
    std::vector<std::pair<uint32_t, uint32_t>> prec;
    Plan plans[MN_MAX_QE][NCAND];   // [seed edge][candidate order]
    QueryDev dev;
    FilterQuery fq;                 // query tree and degree needs of the DEBI filtering
    // filtering state (mn_set_filtering): TD / BU / queued bitmaps [nv][W32],
    // frontier lists [nv][V], their lengths and snapshots
    uint32_t *td = nullptr, *bu = nullptr, *queued = nullptr, *front = nullptr;
    uint32_t *nfront = nullptr, *nsnap = nullptr;
    uint32_t *debi = nullptr;
    uint8_t *out[2] = {nullptr, nullptr};
    unsigned long long out_cap[2] = {0, 0};
    unsigned long long max_seen[2] = {0, 0};     // the most records one batch put in each list
    uint64_t sorted_batch[2] = {0, 0};   // batch whose list is sorted in place (MN_FETCH_SORTED)
};

uint64_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

uint32_t cdiv(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

}  // namespace

// One enumeration phase: seeds of d_seeds[phase] on adjacency buffer `buf`
// whose lowest seq is `base`; visible seqs [g->lo, vis_hi); query edges before
// the seed edge may use seqs [av_lo, av_hi) only (the batch's complement), or,
// with flags, any visible seq whose slot is not flagged.
struct Phase {
    int phase, buf;
    uint64_t base, vis_hi, av_lo, av_hi;
    bool flags;
};

// A batch queued by mn_insert_batch with MN_ASYNC: what its completion needs.
// the autotuner's candidate margins of the learned order (log2 units)
constexpr uint32_t MT_N = 6, MT_BATCHES = 6;
constexpr float MT_CANDS[MT_N] = {0.f, 0.5f, 1.f, 2.f, 3.f, 6.f};
static_assert(MT_N <= MARGIN_SLOTS / 2, "two trial slots per margin interval");

struct PendingBatch {
    bool active = false;
    uint64_t id = 0, n = 0, x = 0, hi_new = 0;
    bool count_only = false, tune_now = false, trial_now = false, margin_now = false;
    bool trial_off = false;             // a filtering-trial batch enumerated without the filter
    int nph = 0;
    Phase ph[2] = {};
};

struct mn_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t V = 0, L = 0;
    uint64_t W = 0, max_batch = 0, C = 0;
    uint32_t cap_mask = 0;
    uint64_t mem_budget = 0, mem_used = 0, mem_peak = 0;
    uint32_t max_queries = 0;
    uint64_t default_out_cap = 0;
    std::vector<uint32_t> vmask_host;
    std::map<uint32_t, uint64_t> vmask_hist;

    uint64_t lo = 0, hi = 0, merged_lo = 0, batch_id = 0;
    long long last_ts = 0;
    bool have_ts = false;

    uint32_t *d_vmask = nullptr;
    // DEBI filtering (mn_set_filtering): dirty vertices since the last pass
    bool filter = false, filter_dirty = false;
    uint32_t W32 = 0;
    uint32_t *d_dmap = nullptr, *d_dirty = nullptr, *d_ndirty = nullptr;
    FilterQuery *d_fq = nullptr;
    uint32_t **d_bu_ptrs = nullptr;  // per query: its BU bitmaps (the enumerator's vertex test)
    unsigned long long *d_fchanges = nullptr, fchanges_base = 0;
    FilterParams *d_fparams = nullptr;   // per query, copied before each pass
    uint32_t *d_fitems = nullptr;        // (query << 8 | query vertex) items of every level
    unsigned char *h_fstage = nullptr;   // pinned staging of both (reused: every batch ends with a sync)
    uint32_t *r_src = nullptr, *r_dst = nullptr;
    uint8_t *r_label = nullptr, *r_dead = nullptr, *batch_flag = nullptr;
    int32_t *r_attr = nullptr;
    int64_t *r_ts = nullptr;

    // adjacency problems: 0 out / 1 in by neighbour, 2 out / 3 in by arrival
    DirArrays base[2][NPROB];   // [buffer][problem]
    int cur = 0;
    DirArrays delta[NPROB];
    uint32_t *cnt[2] = {nullptr, nullptr}, *offs[2] = {nullptr, nullptr};
    unsigned long long *dkA[NPROB] = {}, *dkB[NPROB] = {};
    uint32_t *dvA[NPROB] = {}, *dvB[NPROB] = {};
    uint32_t *blk[NPROB] = {};
    uint32_t nblk_cap = 0;
    Sched *d_sched = nullptr;   // one scheduler block per enumeration phase
    Task *d_tasks = nullptr;
    uint32_t task_cap = 0, epoch = 0;

    mn_edge *d_edges = nullptr;
    unsigned long long *d_seqs = nullptr;

    std::vector<QueryHost> queries;
    QueryDev *d_queries = nullptr;
    Plan *d_plans = nullptr;
    uint32_t **d_debi_ptrs = nullptr;
    uint8_t **d_out_ptrs = nullptr;
    unsigned long long *d_out_cap = nullptr;

    unsigned long long *d_seeds[3] = {nullptr, nullptr, nullptr};
    uint64_t seed_cap[3] = {0, 0, 0};

    Ctrl *d_ctrl = nullptr, *h_ctrl = nullptr;
    std::vector<uint64_t> count_pos, count_neg;
    PendingBatch pending;       // MN_ASYNC batch not yet completed by mn_batch_wait
    uint32_t shard_idx = 0, shard_cnt = 1;   // seed sharding of the stream (mn_set_shard)
    int64_t time_window = 0;    // > 0: expire by timestamp (mn_set_time_window)
    uint32_t *d_sim = nullptr;  // dual simulation: [V] words
    unsigned long long *d_simctl = nullptr;   // its two flag words, then the pair count
    unsigned long long max_iters = ~0ull;
    uint32_t wait_polls = WAIT_POLLS, wait_hold = 0;   // idle wait of the enumerator (mn_set_wait_limit)
    // per (query, sign): decayed maximum of records per inserted (sign 0) or
    // expired (sign 1) edge, used to size the lists before a launch
    std::vector<double> rec_rate[2];
    int enum_grid = 0;          // persistent grid: SMs x resident blocks per SM
    int nsm = 0, enum_max_per_sm = 0;
    uint32_t split_min = SPLIT_MIN, split_depth = MN_MAX_QE;
    float presplit_log2 = INFINITY;   // learned pre-splitting threshold (log2 predicted cycles); inf = off
    int smem_carveout = -1;     // preferred shared-memory carve-out of the enumerator (%), -1 = driver
    uint32_t slice_min = 0;     // staged windows for last-depth ranges this long (0 = off)
    // online autotuner: candidate launch configurations tried on live batches
    struct TuneCfg { uint32_t bps, split_min, split_depth; float presplit_log2; uint32_t slice_min; };
    bool tuning = false;
    std::vector<TuneCfg> tune_cfgs;
    std::vector<double> tune_ms, tune_work;
    uint32_t tune_per = 1, tune_idx = 0, tune_in = 0;
    cudaEvent_t tune_e0 = nullptr, tune_e1 = nullptr;
    // the autotuner's filtering trial: the filtering is kept up to date over
    // 2 x ft_per live inserting batches that alternate between enumerating
    // without it (off, even ft_idx) and with it (on, odd); the faster per
    // inserted edge is kept
    int ftrial = 0;
    uint32_t ft_idx = 0, ft_per = 4;
    bool ft_off_now = false;            // the pending batch enumerates without the filter
    double ft_ms[2] = {0.0, 0.0}, ft_edges[2] = {0.0, 0.0};
    int ft_choice = -1;                 // -1: no trial has finished
    // the learned order's margins (log2 units of predicted cost by which the
    // best candidate must beat the paper's order): per query (q_margin,
    // mirrored in d_qmargin), pick_margin for queries registered later.  The
    // autotuner's margin trial, run first under MN_ORDER_LEARNED on MT_BATCHES
    // live inserting batches (qcyc_on): each seed whose choice depends on the
    // margin takes the paper's order or the model's pick at random (k_pick),
    // and the SM cycles of its units and the seeds are logged per (query,
    // interval of predicted gain, arm) (d_qcyc, d_qseeds)
    float pick_margin = 1.0f;
    std::vector<float> q_margin;
    float *d_qmargin = nullptr;
    unsigned long long *d_qcyc = nullptr;   // [q][MARGIN_SLOTS]
    uint32_t *d_qseeds = nullptr;           // [q][MARGIN_SLOTS]
    bool qcyc_on = false;
    int mtrial = 0;
    uint32_t mt_idx = 0;
    std::vector<double> mt_qcyc, mt_qseeds;   // [query][MARGIN_SLOTS]: SM cycles, seeds
    int mt_choice = -1;                 // -1: no margin trial has finished
    mn_stats stats{};
    bool timing = false;
    // learned matching order
    uint32_t policy = 0;                 // MN_ORDER_*
    float *d_P = nullptr, *d_G = nullptr, *d_M1 = nullptr, *d_M2 = nullptr, *d_loss = nullptr;
    __nv_bfloat16 *d_w1t = nullptr, *d_w2t = nullptr;
    uint32_t *d_train_status = nullptr;   // training kernels' wait status (ST_TIMEOUT)
    uint64_t adam_step = 0;
    bool packed = false;
    __nv_bfloat16 *d_X = nullptr;        // features, seed_cap x NCAND rows
    float *d_y = nullptr;
    unsigned long long *d_seed_work = nullptr;
    unsigned long long *d_picked = nullptr;  // picked seed words before the heaviest-first scatter
    uint8_t *d_bucket = nullptr;             // their cost buckets
    uint32_t *d_pick_hist = nullptr;         // PICK_BUCKETS sizes, then PICK_BUCKETS cursors
    uint64_t learn_rows = 0;             // capacity of d_X / d_y / d_seed_work (rows)
    __nv_bfloat16 *d_SX = nullptr;       // training ring
    float *d_ST = nullptr;
    uint32_t ring = 1u << 20;
    uint64_t n_samples = 0, explore_round = 0;
    uint32_t *d_temporal = nullptr;
    unsigned long long *d_nsamples = nullptr;   // samples ever logged (ring position)
    // host spill of expired edges (mn_set_spill): a pinned FIFO of records and
    // of the DEBI words of every query at expiry; [spill_lo, spill_hi) held
    SpillRec *h_spill = nullptr;
    uint32_t *h_spill_words = nullptr;   // [max_queries][spill_cap]
    uint64_t spill_cap = 0, spill_lo = 0, spill_hi = 0;
    SpillRec *d_spill = nullptr;         // device staging: max_batch records + words
    uint32_t *d_spill_words = nullptr;
    bool use_graph = false;              // record each eligible insert batch as a CUDA graph
    cudaGraphExec_t gexec = nullptr;     // updated in place batch after batch
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    cudaEvent_t ev_open = nullptr;
    std::string err;
    std::vector<void *> allocs;
};

namespace {

mn_status fail(mn_graph *g, mn_status st, const std::string &msg)
{
    if (g) g->err = msg;
    else g_create_error = msg;
    return st;
}

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(g, MN_ERR_DEVICE, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL()                                                                         \
    do {                                                                              \
        g->stats.kernel_launches++;                                                   \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess)                                                        \
            return fail(g, MN_ERR_DEVICE, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
mn_status dalloc(mn_graph *g, T **p, uint64_t count, bool zero = true)
{
    const uint64_t bytes = std::max<uint64_t>(count, 1) * sizeof(T);
    if (g->mem_budget && g->mem_used + bytes > g->mem_budget)
        return fail(g, MN_ERR_OOM, "device memory budget exceeded");
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(g, MN_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    if (zero) {
        e = cudaMemsetAsync(q, 0, bytes, g->stream);
        if (e != cudaSuccess) return fail(g, MN_ERR_DEVICE, cudaGetErrorString(e));
    }
    g->mem_used += bytes;
    g->mem_peak = std::max(g->mem_peak, g->mem_used);
    g->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return MN_OK;
}

void dfree(mn_graph *g, void *p, uint64_t bytes)
{
    if (!p) return;
    cudaFree(p);
    g->mem_used -= std::min(g->mem_used, bytes);
    g->allocs.erase(std::remove(g->allocs.begin(), g->allocs.end(), p), g->allocs.end());
}

#define TRY(x)                        \
    do {                              \
        mn_status s_ = (x);           \
        if (s_ != MN_OK) return s_;   \
    } while (0)

// Copy the per-query margins of the learned order to the device (between
// batches: nothing of the graph's is queued on the stream then).
mn_status upload_margins(mn_graph *g)
{
    CK(cudaMemcpyAsync(g->d_qmargin, g->q_margin.data(), g->max_queries * sizeof(float), cudaMemcpyHostToDevice,
                       g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return MN_OK;
}

mn_status map_status(mn_graph *g, uint32_t st)
{
    if (st & ST_BAD_VERTEX) return fail(g, MN_ERR_INVALID_VERTEX, "vertex id or edge label out of range");
    if (st & ST_TS_ORDER) return fail(g, MN_ERR_TS_ORDER, "timestamps must be strictly increasing");
    if (st & ST_BAD_DELETE) return fail(g, MN_ERR_INVALID_ARG, "deleted seq not live, already deleted or repeated");
    if (st & ST_TIMEOUT) return fail(g, MN_ERR_TIMEOUT, "enumeration work budget exhausted");
    return MN_OK;
}

// ---------------------------------------------------------------- stage timing

cudaEvent_t take_event(mn_graph *g)
{
    if (!g->ev_pool.empty()) {
        cudaEvent_t e = g->ev_pool.back();
        g->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Mark the start of a stage on the graph's stream (timing on only).
void stage_begin(mn_graph *g)
{
    if (!g->timing) return;
    g->ev_open = take_event(g);
    cudaEventRecord(g->ev_open, g->stream);
}

void stage_end(mn_graph *g, int stage)
{
    if (!g->timing || !g->ev_open) return;
    cudaEvent_t e = take_event(g);
    cudaEventRecord(e, g->stream);
    g->ev_pending.push_back({stage, {g->ev_open, e}});
    g->ev_open = nullptr;
}

// Accumulate the stage times whose end events have completed.
void collect_timing(mn_graph *g)
{
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> keep;
    for (auto &p : g->ev_pending) {
        if (cudaEventQuery(p.second.second) != cudaSuccess) {
            cudaGetLastError();
            keep.push_back(p);
            continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.second.first, p.second.second);
        double *dst[S_COUNT] = {&g->stats.ms_ingest, &g->stats.ms_adjacency, &g->stats.ms_seeds,
                                &g->stats.ms_enumerate, &g->stats.ms_expire, &g->stats.ms_filter,
                                &g->stats.ms_model};
        *dst[p.first] += ms;
        g->ev_pool.push_back(p.second.first);
        g->ev_pool.push_back(p.second.second);
    }
    g->ev_pending.swap(keep);
}

void collect_work(mn_graph *g)
{
    g->stats.seeds += g->h_ctrl->work[0];
    g->stats.entries_scanned += g->h_ctrl->work[1];
    g->stats.binds += g->h_ctrl->work[2];
    g->stats.records += g->h_ctrl->work[3];
    g->stats.busy_cycles += g->h_ctrl->work[4];
    g->stats.tasks_split += g->h_ctrl->work[5];
    g->stats.seeds_filtered += g->h_ctrl->work[6];
    g->stats.entries_staged += g->h_ctrl->work[7];
    collect_timing(g);
}

// ---------------------------------------------------------------- query compiler

// Root = the most selective query vertex (Sec. III preprocessing): fewest data
// vertices whose labels contain the query vertex's labels, per unit of query
// degree; ties to the smaller id.  Query tree = BFS tree from the root with
// neighbours in ascending id.  Per starting query edge, the matching order of
// Sec. VI: for a tree edge (u_p, u) the path from u to the root, then the other
// tree edges in BFS order; for a non-tree edge (u_x, u_y) the tree edges into
// u_y and u_x, then the path from u_x to the root, then BFS order.  Query edges
// whose endpoints are both bound are verified right away (verifyNte).
mn_status compile_query(mn_graph *g, QueryHost &Q)
{
    const uint32_t nv = Q.nv, ne = Q.ne;
    std::vector<uint64_t> cand(nv, 0);
    for (uint32_t u = 0; u < nv; u++)
        for (auto &kv : g->vmask_hist)
            if ((kv.first & Q.vmask[u]) == Q.vmask[u]) cand[u] += kv.second;
    std::vector<uint64_t> deg(nv, 0);
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> adj(nv);   // (nbr, edge)
    for (uint32_t e = 0; e < ne; e++) {
        deg[Q.edges[e].src]++;
        deg[Q.edges[e].dst]++;
        adj[Q.edges[e].src].push_back({Q.edges[e].dst, e});
        adj[Q.edges[e].dst].push_back({Q.edges[e].src, e});
    }
    for (auto &a : adj) std::sort(a.begin(), a.end());
    uint32_t root = 0;
    for (uint32_t u = 1; u < nv; u++)
        if (cand[u] * deg[root] < cand[root] * deg[u]) root = u;   // cand/deg smaller, exactly
    std::vector<int> parent(nv, -1), tedge(nv, -1), bfs;
    std::vector<char> seen(nv, 0);
    bfs.push_back((int)root);
    seen[root] = 1;
    for (size_t h = 0; h < bfs.size(); h++) {
        uint32_t u = (uint32_t)bfs[h];
        for (auto &ne_ : adj[u])
            if (!seen[ne_.first]) {
                seen[ne_.first] = 1;
                parent[ne_.first] = (int)u;
                tedge[ne_.first] = (int)ne_.second;
                bfs.push_back((int)ne_.first);
            }
    }
    if (bfs.size() != nv) return fail(g, MN_ERR_INVALID_ARG, "query graph is not connected");
    {   // the filtering's view of the tree (Sec. V-A): BFS order, parents, tree edges, degree needs
        FilterQuery &F = Q.fq;
        memset(&F, 0, sizeof(F));
        F.nv = nv;
        F.root = root;
        F.iso = Q.iso;
        F.root_qmask = Q.vmask[root];
        for (uint32_t u = 0; u < nv; u++) F.qmask[u] = Q.vmask[u];
        uint32_t nlev = 0;
        for (size_t h = 0; h < bfs.size(); h++) {
            const uint32_t u = (uint32_t)bfs[h];
            F.order[h] = (uint8_t)u;
            F.parent[u] = (int8_t)parent[u];
            F.tedge[u] = (int8_t)tedge[u];
            F.depth[u] = h == 0 ? 0 : (uint8_t)(F.depth[parent[u]] + 1);
            nlev = std::max<uint32_t>(nlev, F.depth[u] + 1u);
            if (parent[u] >= 0) {
                const mn_qedge &te = Q.edges[tedge[u]];
                F.p_is_src[u] = te.src == (uint32_t)parent[u] ? 1 : 0;
                F.tlabel[u] = (int16_t)te.label;
                F.children[parent[u]] |= 1u << u;
            } else {
                F.tlabel[u] = -1;
            }
        }
        F.nlev = nlev;
        for (uint32_t e = 0; e < ne; e++) {
            const mn_qedge &x = Q.edges[e];
            F.need_out[x.src]++;
            F.need_in[x.dst]++;
            if (x.label < 0) continue;
            for (int side = 0; side < 2; side++) {
                const uint32_t u = side ? x.dst : x.src;
                uint32_t k = 0;
                while (k < F.nl[u] && F.lab[u][k] != x.label) k++;
                if (k == F.nl[u]) {
                    if (k == FQ_MAXL) continue;      // more labels than kept: a weaker (still sound) check
                    F.lab[u][k] = (int16_t)x.label;
                    F.nl[u]++;
                }
                if (side) F.lin[u][k]++; else F.lout[u][k]++;
            }
        }
    }
    std::vector<char> is_tree(ne, 0);
    std::vector<int> bfs_edges;
    for (size_t h = 1; h < bfs.size(); h++) {
        is_tree[tedge[bfs[h]]] = 1;
        bfs_edges.push_back(tedge[bfs[h]]);
    }
    // candidate edge sequences per seed edge j; k = 0 is the paper's order
    auto paper_order = [&](uint32_t j) {
        std::vector<int> order;
        const uint32_t a = Q.edges[j].src, b = Q.edges[j].dst;
        auto path_up = [&](int x) {
            while (x != (int)root) { order.push_back(tedge[x]); x = parent[x]; }
        };
        if (is_tree[j]) {
            int child = parent[b] == (int)a && tedge[b] == (int)j ? (int)b : (int)a;
            path_up(child);
        } else {
            if (b != root) order.push_back(tedge[b]);
            if (a != root) { order.push_back(tedge[a]); path_up(parent[a]); }
        }
        for (int e : bfs_edges) order.push_back(e);
        return order;
    };
    // greedy vertex orders: score(u) over unbound u adjacent to the bound set
    auto greedy_order = [&](uint32_t j, int mode) {
        std::vector<int> order;
        std::vector<char> bnd(nv, 0);
        bnd[Q.edges[j].src] = bnd[Q.edges[j].dst] = 1;
        for (uint32_t step = 2; step < nv; step++) {
            int best = -1, best_e = -1;
            long best_score = 0;
            for (uint32_t u = 0; u < nv; u++) {
                if (bnd[u]) continue;
                int links = 0, first_e = -1, near = 1 << 20;
                for (uint32_t e = 0; e < ne; e++) {
                    const uint32_t x = Q.edges[e].src, y = Q.edges[e].dst;
                    if ((x == u && bnd[y]) || (y == u && bnd[x])) {
                        links++;
                        if (first_e < 0) first_e = (int)e;
                        near = std::min(near, std::abs((int)e - (int)j));
                    }
                }
                if (!links) continue;
                long score = mode == 1 ? links * 64 - (long)u            // most connected
                           : mode == 2 ? -(long)near * 64 - (long)u      // temporally nearest
                                       : (long)deg[u] * 64 - (long)u;    // highest query degree
                if (best < 0 || score > best_score) { best = (int)u; best_score = score; best_e = first_e; }
            }
            bnd[best] = 1;
            order.push_back(best_e);
        }
        return order;
    };
    for (uint32_t j = 0; j < ne; j++) {
      for (uint32_t kc = 0; kc < NCAND; kc++) {
        const std::vector<int> order = kc == 0 ? paper_order(j) : greedy_order(j, (int)kc);
        const uint32_t a = Q.edges[j].src, b = Q.edges[j].dst;
        Plan &P = Q.plans[j][kc];
        memset(&P, 0, sizeof(P));
        std::vector<char> placed(ne, 0), bound(nv, 0);
        uint32_t bound_mask = 0;
        int ns = 0;
        auto add_step = [&](uint32_t e, uint8_t kind, uint32_t from, uint32_t to, uint8_t dir) {
            Step &s = P.step[ns++];
            s.qe = (uint8_t)e; s.kind = kind; s.from = (uint8_t)from; s.to = (uint8_t)to;
            s.dir = dir; s.avoid = e < j ? 1 : 0; s.label = (int16_t)Q.edges[e].label;
            s.bound_v = (uint16_t)bound_mask;
            uint16_t pred = 0, succ = 0;
            for (auto &pr : Q.prec) {
                if (pr.second == e && placed[pr.first]) pred |= (uint16_t)(1u << pr.first);
                if (pr.first == e && placed[pr.second]) succ |= (uint16_t)(1u << pr.second);
            }
            s.pred = pred; s.succ = succ;
            placed[e] = 1;
        };
        auto close_all = [&]() {
            for (uint32_t e = 0; e < ne; e++)
                if (!placed[e] && bound[Q.edges[e].src] && bound[Q.edges[e].dst])
                    add_step(e, K_CLOSE, Q.edges[e].src, Q.edges[e].dst, 0);
        };
        add_step(j, K_EXTEND, a, b, 0);   // the seed
        bound[a] = bound[b] = 1;
        bound_mask = (1u << a) | (1u << b);
        close_all();
        for (size_t k = 0; k < order.size(); k++) {
            const uint32_t e = (uint32_t)order[k];
            if (placed[e]) continue;
            const uint32_t s = Q.edges[e].src, d = Q.edges[e].dst;
            if (bound[s] && !bound[d]) {
                add_step(e, K_EXTEND, s, d, 0);
                bound[d] = 1; bound_mask |= 1u << d;
            } else if (bound[d] && !bound[s]) {
                add_step(e, K_EXTEND, d, s, 1);
                bound[s] = 1; bound_mask |= 1u << s;
            } else if (!bound[s] && !bound[d]) {
                return fail(g, MN_ERR_STATE, "matching order reached an unbound edge");
            }
            close_all();
        }
        if (ns != (int)ne) return fail(g, MN_ERR_STATE, "matching order does not cover the query");
        P.nsteps = (uint8_t)ne; P.nv = (uint8_t)nv; P.ne = (uint8_t)ne; P.iso = (uint8_t)Q.iso;
        P.seed_src = (uint8_t)a; P.seed_dst = (uint8_t)b;
        P.rec_bytes = Q.rec_bytes; P.goff = Q.goff;
      }
    }
    memset(&Q.dev, 0, sizeof(Q.dev));
    Q.dev.ne = ne;
    for (uint32_t e = 0; e < ne; e++) {
        QPred &p = Q.dev.e[e];
        p.label = Q.edges[e].label;
        p.vmask_src = Q.vmask[Q.edges[e].src];
        p.vmask_dst = Q.vmask[Q.edges[e].dst];
        p.attr_lo = Q.edges[e].attr_lo; p.attr_hi = Q.edges[e].attr_hi;
        p.ts_lo = Q.edges[e].ts_lo; p.ts_hi = Q.edges[e].ts_hi;
    }
    return MN_OK;
}

// ---------------------------------------------------------------- learned order

// He-uniform initial weights from a fixed splitmix64 stream, zero biases.
void init_params(std::vector<float> &P)
{
    P.assign(P_COUNT, 0.f);
    uint64_t z = 0x4D4E4C4541524EULL;
    auto uni = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return (float)((x >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
    };
    const float a1 = std::sqrt(6.f / NF), a2 = std::sqrt(6.f / NH), a3 = std::sqrt(6.f / NH);
    for (int i = 0; i < NF * NH; i++) P[P_W1 + i] = a1 * uni();
    for (int i = 0; i < NH * NH; i++) P[P_W2 + i] = a2 * uni();
    for (int i = 0; i < NH; i++) P[P_W3 + i] = 0.1f * a3 * uni();
}

mn_status ensure_model(mn_graph *g)
{
    if (g->d_P) return MN_OK;
    TRY(dalloc(g, &g->d_P, P_COUNT, false));
    TRY(dalloc(g, &g->d_G, P_COUNT));
    TRY(dalloc(g, &g->d_M1, P_COUNT));
    TRY(dalloc(g, &g->d_M2, P_COUNT));
    TRY(dalloc(g, &g->d_loss, 1));
    TRY(dalloc(g, &g->d_w1t, NF * NH, false));
    TRY(dalloc(g, &g->d_w2t, NH * NH, false));
    TRY(dalloc(g, &g->d_SX, (uint64_t)g->ring * NF, false));
    TRY(dalloc(g, &g->d_ST, g->ring, false));
    TRY(dalloc(g, &g->d_nsamples, 1));
    TRY(dalloc(g, &g->d_train_status, 1));
    std::vector<float> P;
    init_params(P);
    CK(cudaMemcpyAsync(g->d_P, P.data(), sizeof(float) * P_COUNT, cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->packed = false;
    return MN_OK;
}

mn_status pack_model(mn_graph *g)
{
    if (g->packed) return MN_OK;
    k_mlp_pack<<<cdiv(NH * NH, 256), 256, 0, g->stream>>>(g->d_P, g->d_w1t, g->d_w2t);
    CKL();
    g->packed = true;
    return MN_OK;
}

mn_status ensure_learn_rows(mn_graph *g, uint64_t seeds)
{
    const uint64_t rows = seeds * NCAND;
    if (rows <= g->learn_rows) return MN_OK;
    const uint64_t old = g->learn_rows;
    dfree(g, g->d_X, old * NF * sizeof(__nv_bfloat16));
    dfree(g, g->d_y, old * sizeof(float));
    dfree(g, g->d_seed_work, 2 * (old / NCAND) * sizeof(unsigned long long));
    dfree(g, g->d_picked, (old / NCAND) * sizeof(unsigned long long));
    dfree(g, g->d_bucket, old / NCAND);
    g->d_X = nullptr; g->d_y = nullptr; g->d_seed_work = nullptr; g->learn_rows = 0;
    g->d_picked = nullptr; g->d_bucket = nullptr;
    const uint64_t cap = next_pow2(rows);
    TRY(dalloc(g, &g->d_X, cap * NF, false));
    TRY(dalloc(g, &g->d_y, cap, false));
    TRY(dalloc(g, &g->d_seed_work, 2 * (cap / NCAND), false));     // one half per phase
    TRY(dalloc(g, &g->d_picked, cap / NCAND, false));
    TRY(dalloc(g, &g->d_bucket, cap / NCAND, false));
    if (!g->d_pick_hist) TRY(dalloc(g, &g->d_pick_hist, 2 * PICK_BUCKETS, false));
    g->learn_rows = cap;
    return MN_OK;
}

FeatParams feat_params(mn_graph *g, int phase, bool all)
{
    FeatParams f;
    memset(&f, 0, sizeof(f));
    f.seeds = g->d_seeds[phase];
    f.nseeds = &g->d_ctrl->nseeds[phase];
    f.seed_cap = (uint32_t)std::min<uint64_t>(g->seed_cap[phase], 0xffffffffull);
    f.all_candidates = all ? 1u : 0u;
    f.ring_src = g->r_src;
    f.ring_dst = g->r_dst;
    f.r_label = g->r_label;
    f.offs[0] = g->offs[0];
    f.offs[1] = g->offs[1];
    f.L = g->L;
    f.cap_mask = g->cap_mask;
    f.debi = g->d_debi_ptrs;
    f.plans = g->d_plans;
    f.temporal = g->d_temporal;
    f.X = g->d_X;
    return f;
}

// Per-seed work log of `phase` under exploration (dS+ and dS- of one batch
// are enumerated in one launch, so each has its own half).
unsigned long long *seed_work_of(mn_graph *g, int phase)
{
    return g->d_seed_work + (phase == 1 ? g->learn_rows / NCAND : 0);
}

// Estimated SM cycles of each registered query's trial seeds under each
// candidate margin j, [q][MT_N]: the seeds of gain interval i take the
// model's pick under margin j iff i >= j, so cost(j) = sum over i < j of
// S_i x (mean cycles of its paper-order arm) + sum over i >= j of S_i x
// (mean cycles of its pick arm), S_i the interval's seeds (an empty arm
// takes the other arm's mean).
std::vector<double> margin_costs(const mn_graph *g)
{
    const size_t nq = g->queries.size();
    std::vector<double> cost(nq * MT_N, 0.0);
    for (size_t q = 0; q < nq; q++) {
        const double *C = &g->mt_qcyc[q * MARGIN_SLOTS], *S = &g->mt_qseeds[q * MARGIN_SLOTS];
        for (uint32_t i = 0; i + 1 < MT_N; i++) {
            const double sp = S[2 * i], sb = S[2 * i + 1], si = sp + sb;
            if (si <= 0.0) continue;
            double mp = sp > 0 ? C[2 * i] / sp : 0.0, mb = sb > 0 ? C[2 * i + 1] / sb : 0.0;
            if (sp <= 0) mp = mb;
            if (sb <= 0) mb = mp;
            for (uint32_t j = 0; j < MT_N; j++) cost[q * MT_N + j] += si * (i >= j ? mb : mp);
        }
    }
    return cost;
}

// k_pick's margin-trial argument: the candidates while a trial batch runs,
// else none.
MarginTrial margin_trial(mn_graph *g)
{
    MarginTrial mt;
    memset(&mt, 0, sizeof(mt));
    if (!g->qcyc_on) return mt;
    for (uint32_t k = 0; k < MT_N; k++) mt.m[k] = MT_CANDS[k];     // ascending, from 0
    mt.n = MT_N;
    mt.round = g->mt_idx + 1;
    mt.q_seeds = g->d_qseeds;
    return mt;
}

// Before enumerating `phase`: pick each seed's matching order by policy.
mn_status choose_orders(mn_graph *g, int phase)
{
    if (g->policy == MN_ORDER_PAPER || g->queries.empty()) return MN_OK;
    TRY(ensure_model(g));
    TRY(ensure_learn_rows(g, g->seed_cap[phase]));
    const uint32_t grid = (uint32_t)g->enum_grid;
    const uint32_t cap = (uint32_t)std::min<uint64_t>(g->seed_cap[phase], 0xffffffffull);
    if (g->policy == MN_ORDER_EXPLORE) {
        k_explore<<<grid, 256, 0, g->stream>>>(g->d_seeds[phase], &g->d_ctrl->nseeds[phase], cap,
                                               ++g->explore_round);
        CKL();
    } else {
        TRY(pack_model(g));
        k_features<<<grid, 256, 0, g->stream>>>(feat_params(g, phase, true));
        CKL();
        CK(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        stage_begin(g);
        k_mlp_forward_tc<<<2 * g->nsm, TC_FWD_THREADS, TC_SMEM, g->stream>>>(g->d_X, &g->d_ctrl->nseeds[phase], NCAND, 0,
                                                               g->d_w1t, g->d_w2t, g->d_P, g->d_y,
                                                               &g->d_ctrl->status);
        CKL();
        stage_end(g, S_MODEL);
        g->stats.model_launches++;
        CK(cudaMemsetAsync(g->d_pick_hist, 0, 2 * PICK_BUCKETS * sizeof(uint32_t), g->stream));
        k_pick<<<grid, 256, 0, g->stream>>>(g->d_seeds[phase], &g->d_ctrl->nseeds[phase], cap, g->d_y,
                                            g->d_qmargin, margin_trial(g),
                                            g->presplit_log2, g->d_picked, g->d_bucket,
                                            g->d_pick_hist);
        CKL();
        k_seed_order<<<grid, 256, 0, g->stream>>>(g->d_picked, g->d_bucket, &g->d_ctrl->nseeds[phase], cap,
                                                  g->d_pick_hist, g->d_pick_hist + PICK_BUCKETS,
                                                  g->d_seeds[phase]);
        CKL();
    }
    if (g->policy == MN_ORDER_EXPLORE)
        CK(cudaMemsetAsync(seed_work_of(g, phase), 0, sizeof(unsigned long long) * cap, g->stream));
    return MN_OK;
}

// After enumerating `phase` under exploration: log features and work.
mn_status log_samples(mn_graph *g, int phase)
{
    if (g->policy != MN_ORDER_EXPLORE || g->queries.empty()) return MN_OK;
    const uint32_t grid = (uint32_t)g->enum_grid;
    const uint32_t cap = (uint32_t)std::min<uint64_t>(g->seed_cap[phase], 0xffffffffull);
    k_features<<<grid, 256, 0, g->stream>>>(feat_params(g, phase, false));
    CKL();
    k_log_samples<<<grid, 256, 0, g->stream>>>(g->d_X, seed_work_of(g, phase), &g->d_ctrl->nseeds[phase], cap,
                                                g->d_SX, g->d_ST, g->d_nsamples, g->ring);
    CKL();
    k_advance<<<1, 1, 0, g->stream>>>(g->d_nsamples, &g->d_ctrl->nseeds[phase], cap);
    CKL();
    return MN_OK;
}

// ---------------------------------------------------------------- batch pieces

mn_status ensure_seed_cap(mn_graph *g, int phase, uint64_t need)
{
    if (need <= g->seed_cap[phase]) return MN_OK;
    dfree(g, g->d_seeds[phase], g->seed_cap[phase] * sizeof(unsigned long long));
    g->d_seeds[phase] = nullptr;
    g->seed_cap[phase] = 0;
    uint64_t cap = next_pow2(need);
    TRY(dalloc(g, &g->d_seeds[phase], cap, false));
    g->seed_cap[phase] = cap;
    return MN_OK;
}

// ---------------------------------------------------------------- host spill

// Copy the expired edges [seq_lo, seq_lo + x) and their DEBI words into the
// host FIFO (asynchronous: the copies complete with the graph's stream, at
// the latest by the next call that waits on it); the oldest spilled edges
// are overwritten when it is full.  Chunks of at most max_batch edges go
// through the device staging buffer.
mn_status spill_expired(mn_graph *g, uint64_t seq_lo, uint64_t x)
{
    if (!g->h_spill || x == 0) return MN_OK;
    const uint32_t nq = (uint32_t)g->queries.size();
    for (uint64_t done = 0; done < x;) {
        const uint64_t m = std::min<uint64_t>(x - done, g->max_batch);
        k_spill_pack<<<cdiv(m, 256), 256, 0, g->stream>>>(seq_lo + done, (uint32_t)m, g->cap_mask, g->r_src,
                                                          g->r_dst, g->r_label, g->r_attr, g->r_ts, nq,
                                                          g->d_debi_ptrs, g->d_spill, g->d_spill_words,
                                                          &g->d_ctrl->status);
        CKL();
        // the FIFO position of seq s is s mod spill_cap: copy in at most two pieces
        for (uint64_t k = 0; k < m;) {
            const uint64_t s0 = seq_lo + done + k;
            const uint64_t pos = s0 % g->spill_cap;
            const uint64_t len = std::min<uint64_t>(m - k, g->spill_cap - pos);
            CK(cudaMemcpyAsync(g->h_spill + pos, g->d_spill + k, len * sizeof(SpillRec), cudaMemcpyDeviceToHost,
                               g->stream));
            for (uint32_t q = 0; q < nq; q++)
                CK(cudaMemcpyAsync(g->h_spill_words + (size_t)q * g->spill_cap + pos,
                                   g->d_spill_words + (size_t)q * m + k, len * sizeof(uint32_t),
                                   cudaMemcpyDeviceToHost, g->stream));
            g->stats.spill_bytes += len * (sizeof(SpillRec) + nq * sizeof(uint32_t));
            k += len;
        }
        done += m;
    }
    // expiries are contiguous from the window start at mn_set_spill on
    g->spill_hi = seq_lo + x;
    if (g->spill_hi - g->spill_lo > g->spill_cap) g->spill_lo = g->spill_hi - g->spill_cap;
    return MN_OK;
}

// ---------------------------------------------------------------- DEBI filtering

mn_status filter_globals(mn_graph *g)
{
    if (g->d_dmap) return MN_OK;
    g->W32 = (g->V + 31) / 32;
    TRY(dalloc(g, &g->d_dmap, g->W32));
    TRY(dalloc(g, &g->d_dirty, g->V, false));
    TRY(dalloc(g, &g->d_ndirty, 1));
    TRY(dalloc(g, &g->d_fq, g->max_queries));
    TRY(dalloc(g, &g->d_bu_ptrs, g->max_queries));
    TRY(dalloc(g, &g->d_fchanges, 1));
    TRY(dalloc(g, &g->d_fparams, g->max_queries));
    TRY(dalloc(g, &g->d_fitems, (uint64_t)g->max_queries * MN_MAX_QV * 2));
    CK(cudaMallocHost((void **)&g->h_fstage, sizeof(FilterParams) * g->max_queries +
                                             sizeof(uint32_t) * g->max_queries * MN_MAX_QV * 2));
    return MN_OK;
}

mn_status filter_alloc(mn_graph *g, size_t q)
{
    QueryHost &Q = g->queries[q];
    if (Q.td) return MN_OK;
    const uint64_t bw = (uint64_t)Q.nv * g->W32;
    TRY(dalloc(g, &Q.td, bw));
    TRY(dalloc(g, &Q.bu, bw));
    TRY(dalloc(g, &Q.queued, bw));
    TRY(dalloc(g, &Q.front, (uint64_t)Q.nv * g->V, false));
    TRY(dalloc(g, &Q.nfront, Q.nv));
    TRY(dalloc(g, &Q.nsnap, Q.nv));
    CK(cudaMemcpyAsync(g->d_fq + q, &Q.fq, sizeof(FilterQuery), cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(g->d_bu_ptrs + q, &Q.bu, sizeof(uint32_t *), cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return MN_OK;
}

FilterParams filter_params(mn_graph *g, size_t q, int buf, uint64_t base, uint64_t vis_hi, bool full)
{
    QueryHost &Q = g->queries[q];
    FilterParams p;
    memset(&p, 0, sizeof(p));
    p.fq = g->d_fq + q;
    p.qi = (uint32_t)q;
    p.V = g->V;
    p.L = g->L;
    p.W32 = g->W32;
    p.cap_mask = g->cap_mask;
    for (int t = 0; t < NPROB; t++) { p.nbr[t] = g->base[buf][t].nbr; p.s32[t] = g->base[buf][t].s32; }
    p.offs[0] = g->offs[0];
    p.offs[1] = g->offs[1];
    p.base32 = (uint32_t)base;
    p.vis_lo = (uint32_t)(g->lo - base);
    p.vis_hi = (uint32_t)(vis_hi - base);
    p.debi = Q.debi;
    p.r_dead = g->r_dead;
    p.vmask = g->d_vmask;
    p.td = Q.td;
    p.bu = Q.bu;
    p.queued = Q.queued;
    p.front = Q.front;
    p.nfront = Q.nfront;
    p.nsnap = Q.nsnap;
    p.dirty = g->d_dirty;
    p.ndirty = g->d_ndirty;
    p.full = full ? 1u : 0u;
    p.changes = g->d_fchanges;
    return p;
}

// Mark both endpoints of the edges at seqs [seq_lo, seq_lo + n) (or of the
// listed seqs) dirty for the next filtering pass.
mn_status filter_mark(mn_graph *g, uint64_t seq_lo, uint64_t n, const unsigned long long *seqs)
{
    if (!g->filter || n == 0) return MN_OK;
    k_filter_dirty<<<cdiv(n, 256), 256, 0, g->stream>>>(seq_lo, (uint32_t)n, seqs, g->cap_mask, g->r_src,
                                                        g->r_dst, g->d_dmap, g->d_dirty, g->d_ndirty, g->V,
                                                        &g->d_ctrl->status);
    CKL();
    g->filter_dirty = true;
    return MN_OK;
}

// One filtering pass (top-down then bottom-up over the query trees' levels)
// for every query, or only query `only`, on adjacency buffer `buf` (lowest
// seq `base`) with visible seqs [lo, vis_hi).  full: every vertex is a
// candidate (building the sets); else the dirty vertices and the frontiers.
// All queries' items of one level run in one launch (blockIdx.y = item).
mn_status filter_pass(mn_graph *g, int buf, uint64_t base, uint64_t vis_hi, bool full, int only = -1)
{
    if (!g->filter || g->queries.empty()) return MN_OK;
    const uint32_t *st = &g->d_ctrl->status;
    std::vector<FilterParams> P;
    std::vector<std::vector<uint32_t>> lev;
    for (size_t q = 0; q < g->queries.size(); q++) {
        if (only >= 0 && (int)q != only) continue;
        const FilterQuery &F = g->queries[q].fq;
        const uint32_t pi = (uint32_t)P.size();
        P.push_back(filter_params(g, q, buf, base, vis_hi, full));
        if (lev.size() < F.nlev) lev.resize(F.nlev);
        for (uint32_t h = 0; h < F.nv; h++) {
            const uint32_t u = F.order[h];
            lev[F.depth[u]].push_back(pi << 8 | u);
        }
    }
    std::vector<uint32_t> flat;
    std::vector<size_t> off;
    for (auto &l : lev) { off.push_back(flat.size()); flat.insert(flat.end(), l.begin(), l.end()); }
    FilterParams *hp = reinterpret_cast<FilterParams *>(g->h_fstage);
    uint32_t *hi_ = reinterpret_cast<uint32_t *>(g->h_fstage + sizeof(FilterParams) * g->max_queries);
    std::copy(P.begin(), P.end(), hp);
    std::copy(flat.begin(), flat.end(), hi_);
    CK(cudaMemcpyAsync(g->d_fparams, hp, P.size() * sizeof(FilterParams), cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(g->d_fitems, hi_, flat.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, g->stream));
    stage_begin(g);
    const uint32_t bx = 64;                       // blocks per item
    auto run_level = [&](size_t d, bool td) -> mn_status {
        const uint32_t n = (uint32_t)lev[d].size();
        if (!n) return MN_OK;
        FilterItems it{g->d_fparams, g->d_fitems + off[d]};
        k_filter_snap<<<1, 256, 0, g->stream>>>(it, n);
        CKL();
        if (td) k_filter_td<<<dim3(bx, n), 256, 0, g->stream>>>(it, st);
        else    k_filter_bu<<<dim3(bx, n), 256, 0, g->stream>>>(it, st);
        CKL();
        return MN_OK;
    };
    for (size_t d = 0; d < lev.size(); d++) TRY(run_level(d, true));
    for (size_t d = lev.size(); d-- > 0;) TRY(run_level(d, false));
    if (!full) {
        const uint32_t np = (uint32_t)P.size();
        k_filter_reset<<<dim3(bx, np), 256, 0, g->stream>>>(g->d_fparams, st);
        CKL();
        k_filter_zero_fronts<<<np, 32, 0, g->stream>>>(g->d_fparams, st);
        CKL();
        k_filter_dirty_clear<<<(uint32_t)g->nsm * 8, 256, 0, g->stream>>>(g->d_dmap, g->d_dirty, g->d_ndirty, g->V, st);
        CKL();
        k_filter_zero<<<1, 32, 0, g->stream>>>(g->d_ndirty, 1, st);
        CKL();
        g->filter_dirty = false;
    }
    stage_end(g, S_FILTER);
    return MN_OK;
}

// Bring the sets up to date with the current graph before an enumeration
// outside an insert (deletes, static counts): only when edges changed.
mn_status filter_refresh(mn_graph *g)
{
    if (!g->filter || !g->filter_dirty) return MN_OK;
    return filter_pass(g, g->cur, g->merged_lo, g->hi, false);
}

// One enumerator launch over the seeds of one or two phases (dS+ and dS- of
// one batch share the adjacency buffer and visibility; a single launch has
// one tail instead of two).  The first phase's seeds are taken first.
mn_status launch_enumerate(mn_graph *g, const Phase *ph, int nph, bool count_only,
                           const unsigned long long *qrun = nullptr)
{
    const Phase &a = ph[0];
    EnumParams p;
    memset(&p, 0, sizeof(p));
    for (int t = 0; t < NPROB; t++) {
        p.nbr[t] = g->base[a.buf][t].nbr;
        p.s32[t] = g->base[a.buf][t].s32;
    }
    for (int d = 0; d < 2; d++) p.offs[d] = g->offs[d];
    p.L = g->L;
    p.cap_mask = g->cap_mask;
    p.ring_src = g->r_src;
    p.ring_dst = g->r_dst;
    p.debi = g->d_debi_ptrs;
    p.plans = g->d_plans;
    p.seeds = g->d_seeds[a.phase];
    p.nseeds = &g->d_ctrl->nseeds[a.phase];
    p.seed_cap = (uint32_t)std::min<uint64_t>(g->seed_cap[a.phase], 0xffffffffull);
    p.sched = g->d_sched + a.phase;
    p.tasks = g->d_tasks;
    p.task_cap = g->task_cap;
    p.task_log2 = (uint32_t)__builtin_ctz(g->task_cap);
    g->epoch = (g->epoch + 1) & 0x7fffffffu;              // 31 bits: bit 31 marks abandoned slots
    if (g->epoch == 0) g->epoch = 1;                       // 0 is the zeroed slots' state
    p.epoch = g->epoch;
    p.base32 = (uint32_t)a.base;
    p.base = a.base;
    p.vis_lo = (uint32_t)(g->lo - a.base);
    p.vis_hi = (uint32_t)(a.vis_hi - a.base);
    p.av_lo = (uint32_t)(a.av_lo - a.base);
    p.av_hi = (uint32_t)(a.av_hi - a.base);
    p.batch_flag = a.flags ? g->batch_flag : nullptr;
    p.sign = (uint32_t)a.phase;
    p.counts = g->d_ctrl->counts;
    p.out = g->d_out_ptrs;
    p.out_cap = g->d_out_cap;
    p.count_only = count_only ? 1u : 0u;
    p.max_iters = g->max_iters;
    p.status = &g->d_ctrl->status;
    p.work = g->d_ctrl->work;
    // a re-run (qrun given) logs no work: its seeds were logged by the first run
    const bool explore = g->policy == MN_ORDER_EXPLORE && !qrun;
    p.seed_work = explore && a.phase < 2 ? seed_work_of(g, a.phase) : nullptr;
    p.q_cycles = g->qcyc_on ? g->d_qcyc : nullptr;
    p.qrun[0] = qrun ? qrun[0] : ~0ull;
    p.qrun[1] = qrun ? qrun[1] : ~0ull;
    p.wait_polls = g->wait_polls;
    p.wait_hold = g->wait_hold;
    p.bu = g->filter && !g->ft_off_now ? g->d_bu_ptrs : nullptr;
    p.W32 = g->W32;
    if (nph > 1) {
        const Phase &b = ph[1];
        if (b.buf != a.buf || b.base != a.base || b.vis_hi != a.vis_hi || b.flags != a.flags)
            return fail(g, MN_ERR_STATE, "phases of one launch must share the adjacency view");
        p.seeds1 = g->d_seeds[b.phase];
        p.nseeds1 = &g->d_ctrl->nseeds[b.phase];
        p.seed_cap1 = (uint32_t)std::min<uint64_t>(g->seed_cap[b.phase], 0xffffffffull);
        p.av_lo1 = (uint32_t)(b.av_lo - b.base);
        p.av_hi1 = (uint32_t)(b.av_hi - b.base);
        p.sign1 = (uint32_t)b.phase;
        p.seed_work1 = explore && b.phase < 2 ? seed_work_of(g, b.phase) : nullptr;
    }
    p.split_min = g->split_min;
    p.split_depth = g->split_depth;
    CK(cudaMemsetAsync(g->d_sched + a.phase, 0, sizeof(Sched), g->stream));
    p.stage_min = g->slice_min;
    p.adj_cap = (uint32_t)std::min<uint64_t>(g->C, 0xfffffffcull);
    void (*kern)(EnumParams) = p.bu ? (g->slice_min ? k_enumerate<true, true> : k_enumerate<true, false>)
                                    : (g->slice_min ? k_enumerate<false, true> : k_enumerate<false, false>);
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, g->smem_carveout));
    stage_begin(g);
    kern<<<g->enum_grid, ENUM_WARPS * 32, 0, g->stream>>>(p);
    CKL();
    stage_end(g, S_ENUM);
    g->stats.enumerate_launches++;
    return MN_OK;
}

// Seeds of the edges with seq in [s_lo, s_lo + n) into phase's list.
mn_status launch_seeds_range(mn_graph *g, int phase, uint64_t s_lo, uint64_t n, uint32_t qsel,
                             uint32_t jmask)
{
    const uint32_t nql = qsel == 0xffffffffu ? (uint32_t)g->queries.size() : 1u;
    uint64_t total_ne = 0;
    if (qsel == 0xffffffffu) for (auto &Q : g->queries) total_ne += Q.ne;
    else total_ne = __builtin_popcount(jmask & ((1u << g->queries[qsel].ne) - 1u));
    TRY(ensure_seed_cap(g, phase, std::max<uint64_t>(1, n * total_ne)));
    CK(cudaMemsetAsync(&g->d_ctrl->nseeds[phase], 0, sizeof(uint32_t), g->stream));
    if (n == 0 || nql == 0) return MN_OK;
    const uint64_t threads = n * nql;
    stage_begin(g);
    k_seeds_range<<<cdiv(threads, 256), 256, 0, g->stream>>>(
        s_lo, (uint32_t)n, g->cap_mask, (uint32_t)g->queries.size(), g->d_debi_ptrs, qsel, jmask,
        g->d_seeds[phase], &g->d_ctrl->nseeds[phase], (uint32_t)g->seed_cap[phase],
        g->shard_idx, g->shard_cnt, &g->d_ctrl->status);
    CKL();
    stage_end(g, S_SEEDS);
    return MN_OK;
}

// Rebuild the adjacency into buffer 1-cur: live base entries merged with the
// batch delta (n entries per problem); offsets from the degree counters.
mn_status launch_adjacency_update(mn_graph *g, uint64_t n, const mn_edge *d_edges, uint64_t seq0)
{
    const uint32_t *st = &g->d_ctrl->status;
    const uint32_t n_pad = cdiv(n, SORT_TILE) * SORT_TILE;
    SortSet A, Bs;
    for (int t = 0; t < NPROB; t++) {
        A.k[t] = g->dkA[t]; A.v[t] = g->dvA[t];
        Bs.k[t] = g->dkB[t]; Bs.v[t] = g->dvB[t];
    }
    // sort the delta (all four problems at once)
    k_sort_tiles<<<dim3(n_pad / SORT_TILE, NPROB), 1024, 0, g->stream>>>(A, st);
    CKL();
    for (uint64_t R = SORT_TILE; R < n; R *= 2) {
        const uint32_t threads = cdiv(n, MERGE_ITEMS);
        k_merge_pass<<<dim3(cdiv(threads, 256), NPROB), 256, 0, g->stream>>>(A, Bs, (uint32_t)n,
                                                                             (uint32_t)R, st);
        CKL();
        std::swap(A, Bs);
    }
    auto adj4 = [](DirArrays *d) {
        Adj4 a;
        for (int t = 0; t < NPROB; t++) { a.key[t] = d[t].key; a.nbr[t] = d[t].nbr; a.s32[t] = d[t].s32; }
        return a;
    };
    Adj4 D = adj4(g->delta);
    k_delta_finalize<<<dim3(cdiv(n, 256), NPROB), 256, 0, g->stream>>>(A, D, d_edges, g->cnt[0],
                                                                       g->cnt[1], (uint32_t)n, seq0, st);
    CKL();
    Adj4 blk;
    for (int t = 0; t < NPROB; t++) { blk.key[t] = g->blk[t]; blk.nbr[t] = nullptr; blk.s32[t] = nullptr; }
    // merge the live base entries with the delta into the other base
    // buffer: live counts per tile and their scan, the delta entries'
    // anchors in the base, then one pass over the base tiles
    const uint64_t n_base = g->hi - g->merged_lo;
    const uint32_t lo32 = (uint32_t)g->lo;
    const uint32_t span = (uint32_t)(g->hi - g->lo);
    Adj4 Bse = adj4(g->base[g->cur]);
    Adj4 O = adj4(g->base[1 - g->cur]);
    Adj4 anc;                       // the sort values are free once the delta is final
    for (int t = 0; t < NPROB; t++) { anc.key[t] = g->dvA[t]; anc.nbr[t] = nullptr; anc.s32[t] = nullptr; }
    const uint32_t nb = cdiv(n_base, CTILE);
    if (n_base) {
        k_live_count<<<dim3(nb, NPROB), CBLK, 0, g->stream>>>(Bse, (uint32_t)n_base, lo32, span, blk, st);
        CKL();
        k_scan_blocks<<<NPROB, 1024, 0, g->stream>>>(blk, nb, st);
        CKL();
    }
    k_delta_anchor<<<dim3(cdiv(n, 256), NPROB), 256, 0, g->stream>>>(Bse, D, (uint32_t)n_base, (uint32_t)n,
                                                                      anc, st);
    CKL();
    k_merge_live<<<dim3(std::max(nb, 1u), NPROB), CBLK, 0, g->stream>>>(Bse, D, O, (uint32_t)n_base, (uint32_t)n,
                                                                         lo32, span, blk, anc, st);
    CKL();
    // offsets of the (vertex, label) segments (shared by both orders)
    const uint64_t nvl = (uint64_t)g->V * g->L;
    const uint32_t nbo = cdiv(nvl, CTILE);
    k_scan_reduce<<<dim3(nbo, 2), CBLK, 0, g->stream>>>(g->cnt[0], g->cnt[1], (uint32_t)nvl, g->blk[0],
                                                         g->blk[1], st);
    CKL();
    k_scan_blocks<<<2, 1024, 0, g->stream>>>(blk, nbo, st);
    CKL();
    k_scan_apply<<<dim3(nbo, 2), CBLK, 0, g->stream>>>(g->cnt[0], g->cnt[1], (uint32_t)nvl, g->blk[0],
                                                        g->blk[1], g->offs[0], g->offs[1], st);
    CKL();
    return MN_OK;
}

mn_status read_ctrl(mn_graph *g)
{
    CK(cudaMemcpyAsync(g->h_ctrl, g->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->stats.d2h_bytes += sizeof(Ctrl);
    collect_work(g);
    CK(cudaMemsetAsync(g->d_ctrl->work, 0, sizeof(g->h_ctrl->work), g->stream));
    return MN_OK;
}

// Make the list of (query q, phase) hold at least `need` records (grown to
// a power of two with a quarter of headroom), within the memory budget.
// *grown tells whether it was reallocated; the device pointer table is
// refreshed by sync_out_table.
mn_status ensure_out_cap(mn_graph *g, size_t q, int phase, uint64_t need, bool *grown, bool *over_budget)
{
    *grown = false;
    QueryHost &Q = g->queries[q];
    if (need <= Q.out_cap[phase]) return MN_OK;
    const uint64_t cap = next_pow2(need + need / 4);
    const uint64_t bytes = cap * Q.rec_bytes;
    const uint64_t old = Q.out_cap[phase] * Q.rec_bytes;
    if (g->mem_budget && g->mem_used - old + bytes > g->mem_budget) {
        *over_budget = true;
        return MN_OK;
    }
    dfree(g, Q.out[phase], old);
    Q.out[phase] = nullptr;
    Q.out_cap[phase] = 0;
    TRY(dalloc(g, &Q.out[phase], bytes, false));
    Q.out_cap[phase] = cap;
    *grown = true;
    return MN_OK;
}

mn_status sync_out_table(mn_graph *g)
{
    std::vector<uint8_t *> ptrs(g->max_queries * 2, nullptr);
    std::vector<unsigned long long> caps(g->max_queries * 2, 0);
    for (size_t q = 0; q < g->queries.size(); q++)
        for (int s = 0; s < 2; s++) {
            ptrs[q * 2 + s] = g->queries[q].out[s];
            caps[q * 2 + s] = g->queries[q].out_cap[s];
        }
    CK(cudaMemcpyAsync(g->d_out_ptrs, ptrs.data(), ptrs.size() * sizeof(uint8_t *),
                       cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(g->d_out_cap, caps.data(), caps.size() * sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, g->stream));
    // the host arrays are freed on return: the copies must have read them
    CK(cudaStreamSynchronize(g->stream));
    return MN_OK;
}

// Grow the result lists of `phase` to the exact counts (within the memory
// budget).  Sets bit q of *rerun for every list that was too small.
mn_status grow_outputs(mn_graph *g, int phase, unsigned long long *rerun, bool *over_budget)
{
    *rerun = 0;
    bool any = false;
    for (size_t q = 0; q < g->queries.size(); q++) {
        const unsigned long long c = g->h_ctrl->counts[q * 3 + phase];
        if (c <= g->queries[q].out_cap[phase]) continue;
        bool grown = false;
        TRY(ensure_out_cap(g, q, phase, c, &grown, over_budget));
        if (grown) { *rerun |= 1ull << q; any = true; }
    }
    if (any) TRY(sync_out_table(g));
    return MN_OK;
}

// Before a launch: lists of queries whose recent batches produced more
// records per edge than this batch's lists hold are grown now, so that the
// batch is not enumerated twice.
constexpr uint64_t PRESIZE_MAX_BYTES = 16ull << 30;  // per result list

mn_status presize_outputs(mn_graph *g, uint64_t n_new, uint64_t n_expired)
{
    bool any = false, over = false;
    for (int s = 0; s < 2; s++) {
        const uint64_t edges = s == 0 ? n_new : n_expired;
        if (!edges) continue;
        for (size_t q = 0; q < g->queries.size() && q < g->rec_rate[s].size(); q++) {
            // three times the decayed maximum: a batch that brings a hub
            // into play multiplies one query's output, and a second launch
            // costs more than the memory (lists are grown within the budget);
            // but at most four times the most records one batch has put in
            // the list, and never past PRESIZE_MAX_BYTES, so that one small
            // batch's rate times a large batch cannot claim the device (a
            // list that overflows is grown to its exact count)
            const double est = std::min({3.0 * g->rec_rate[s][q] * (double)edges,
                                         4.0 * (double)g->queries[q].max_seen[s] + 65536.0,
                                         (double)(PRESIZE_MAX_BYTES / g->queries[q].rec_bytes)});
            if (est <= (double)g->queries[q].out_cap[s]) continue;
            bool grown = false;
            TRY(ensure_out_cap(g, q, s, (uint64_t)est, &grown, &over));
            any = any || grown;
        }
    }
    if (any) TRY(sync_out_table(g));
    return MN_OK;
}

// After a batch: update the records-per-edge estimates (a decayed maximum).
void note_rates(mn_graph *g, uint64_t n_new, uint64_t n_expired)
{
    for (int s = 0; s < 2; s++) {
        const uint64_t edges = s == 0 ? n_new : n_expired;
        g->rec_rate[s].resize(g->queries.size(), 0.0);
        if (!edges) continue;
        for (size_t q = 0; q < g->queries.size(); q++) {
            const double r = (double)g->h_ctrl->counts[q * 3 + s] / (double)edges;
            g->rec_rate[s][q] = std::max(0.9 * g->rec_rate[s][q], r);
            g->queries[q].max_seen[s] = std::max(g->queries[q].max_seen[s], g->h_ctrl->counts[q * 3 + s]);
        }
    }
}

void fill_result(mn_graph *g, mn_batch_result *out, uint64_t seq_lo, uint64_t seq_hi,
                 uint64_t ex_lo, uint64_t ex_hi)
{
    const size_t nq = g->queries.size();
    g->count_pos.assign(nq, 0);
    g->count_neg.assign(nq, 0);
    for (size_t q = 0; q < nq; q++) {
        g->count_pos[q] = g->h_ctrl->counts[q * 3 + 0];
        g->count_neg[q] = g->h_ctrl->counts[q * 3 + 1];
    }
    if (!out) return;
    out->batch_id = g->batch_id;
    out->seq_lo = seq_lo;
    out->seq_hi = seq_hi;
    out->expired_lo = ex_lo;
    out->expired_hi = ex_hi;
    out->num_queries = (uint32_t)nq;
    out->count_pos = g->count_pos.data();
    out->count_neg = g->count_neg.data();
}

// Check the status of the launched phases.  Counts are exact even when a
// list overflowed (records past a list's end are counted, not written); the
// lists that overflowed are grown to the exact count and only their
// (query, phase) seeds are enumerated again, in one launch.
mn_status enumerate_phases(mn_graph *g, const Phase *ph, int nph, bool count_only, bool *over_budget)
{
    TRY(read_ctrl(g));
    if (g->h_ctrl->status) return map_status(g, g->h_ctrl->status);
    if (count_only) return MN_OK;
    for (int round = 0; round < 2; round++) {
        unsigned long long rerun[2] = {0, 0};   // per launch seed set
        for (int k = 0; k < nph; k++) TRY(grow_outputs(g, ph[k].phase, &rerun[k], over_budget));
        if (!rerun[0] && !rerun[1]) break;
        for (int k = 0; k < nph; k++)
            for (size_t q = 0; q < g->queries.size(); q++)
                if ((rerun[k] >> q) & 1ull)
                    CK(cudaMemsetAsync(&g->d_ctrl->counts[q * 3 + ph[k].phase], 0, sizeof(unsigned long long),
                                       g->stream));
        TRY(launch_enumerate(g, ph, nph, false, rerun));
        g->stats.rerun_launches++;
        TRY(read_ctrl(g));
        if (g->h_ctrl->status) return map_status(g, g->h_ctrl->status);
    }
    return MN_OK;
}

// The autotuner's candidate launch configurations, at the occupancy limit of
// resident blocks per SM (the kernel is latency-bound): split threshold x
// split depth x learned pre-split threshold (off, or seeds predicted above
// 2^20 / 2^22 SM cycles; it acts only under MN_ORDER_LEARNED).
void build_tune_candidates(mn_graph *g)
{
    g->tune_cfgs.clear();
    const uint32_t b = (uint32_t)g->enum_max_per_sm;
    for (uint32_t sm : {40u, 64u, 128u})
        for (uint32_t sd : {3u, (uint32_t)MN_MAX_QE})
            for (float th : {INFINITY, 20.f, 22.f}) g->tune_cfgs.push_back({b, sm, sd, th, 0u});
    // shared-memory staging of long last-depth ranges, at the default split
    for (uint32_t sl : {256u, 1024u}) g->tune_cfgs.push_back({b, 40u, (uint32_t)MN_MAX_QE, INFINITY, sl});
}

// Turn the DEBI filtering on: per-query sets built by one full pass over the
// current graph (nothing may be pending).
mn_status filter_enable(mn_graph *g)
{
    if (g->filter) return MN_OK;
    TRY(filter_globals(g));
    for (size_t q = 0; q < g->queries.size(); q++) TRY(filter_alloc(g, q));
    g->filter = true;
    // build every query's sets on the current graph; nothing is pending then
    CK(cudaMemsetAsync(&g->d_ctrl->status, 0, sizeof(uint32_t), g->stream));
    TRY(filter_pass(g, g->cur, g->merged_lo, g->hi, true));
    CK(cudaMemsetAsync(g->d_dmap, 0, sizeof(uint32_t) * g->W32, g->stream));
    CK(cudaMemsetAsync(g->d_ndirty, 0, sizeof(uint32_t), g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->filter_dirty = false;
    return MN_OK;
}

}  // namespace

// Complete the queued batch g->pending: wait for its enumeration, grow and
// re-run overflowed lists, then commit (or, on a validation error, apply
// nothing) and report.
static mn_status insert_finish(mn_graph *g, mn_batch_result *out)
{
    const PendingBatch pd = g->pending;
    g->pending.active = false;
    const uint64_t n = pd.n, x = pd.x, hi_new = pd.hi_new;
    const bool count_only = pd.count_only, tune_now = pd.tune_now, trial_now = pd.trial_now;
    const bool margin_now = pd.margin_now;
    const int nph = pd.nph;
    const Phase *ph = pd.ph;
    bool over_budget = false;
    const mn_status est = enumerate_phases(g, ph, nph, count_only, &over_budget);
    g->ft_off_now = false;                   // every launch of the batch has run
    int ft_switch = 0;                       // after the commit: 1 turn the filtering on, -1 off
    if (tune_now && est == MN_OK) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g->tune_e0, g->tune_e1));
        g->tune_ms[g->tune_idx] += ms;
        g->tune_work[g->tune_idx] += (double)(g->h_ctrl->work[1] + g->h_ctrl->work[2]) + 1.0;
        if (++g->tune_in >= g->tune_per) {
            g->tune_in = 0;
            if (++g->tune_idx == g->tune_cfgs.size()) {       // keep the fastest per unit of work
                size_t best = 0;
                for (size_t k = 1; k < g->tune_cfgs.size(); k++)
                    if (g->tune_ms[k] / g->tune_work[k] < g->tune_ms[best] / g->tune_work[best]) best = k;
                const auto &c = g->tune_cfgs[best];
                g->enum_grid = g->nsm * (int)c.bps;
                g->split_min = c.split_min;
                g->split_depth = c.split_depth;
                g->presplit_log2 = c.presplit_log2;
                g->slice_min = c.slice_min;
                g->tuning = false;
                // then the filtering trial, with the filtering turned on (and
                // its sets built, untimed) after this batch's commit
                g->ftrial = 1;
                g->ft_idx = 0;
                g->ft_ms[0] = g->ft_ms[1] = g->ft_edges[0] = g->ft_edges[1] = 0.0;
                ft_switch = 1;
            }
        }
    }
    g->qcyc_on = false;
    if (margin_now && est == MN_OK) {
        const size_t nq = g->queries.size(), ns = nq * MARGIN_SLOTS;
        std::vector<unsigned long long> qc(ns);
        std::vector<uint32_t> qs(ns);
        CK(cudaMemcpyAsync(qc.data(), g->d_qcyc, ns * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           g->stream));
        CK(cudaMemcpyAsync(qs.data(), g->d_qseeds, ns * sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        for (size_t i = 0; i < ns; i++) {
            g->mt_qcyc[i] += (double)qc[i];
            g->mt_qseeds[i] += (double)qs[i];
        }
        if (++g->mt_idx >= MT_BATCHES) {
            // each query keeps the margin of the least estimated cycles
            // (margin_costs); queries registered later take the margin of the
            // least cycles summed over all queries
            const std::vector<double> cost = margin_costs(g);
            double tot[MT_N] = {};
            for (size_t q = 0; q < nq; q++)
                for (uint32_t j = 0; j < MT_N; j++) tot[j] += cost[q * MT_N + j];
            uint32_t best = 0;
            for (uint32_t j = 1; j < MT_N; j++)
                if (tot[j] < tot[best]) best = j;
            g->pick_margin = MT_CANDS[best];
            g->mt_choice = (int)best;
            for (size_t q = 0; q < g->max_queries; q++) g->q_margin[q] = g->pick_margin;
            for (size_t q = 0; q < nq; q++) {
                uint32_t bq = 0;
                double any = 0.0;
                for (uint32_t j = 0; j < MT_N; j++) any += cost[q * MT_N + j];
                if (any <= 0.0) continue;                  // no seed of q depended on the margin
                for (uint32_t j = 1; j < MT_N; j++)
                    if (cost[q * MT_N + j] < cost[q * MT_N + bq]) bq = j;
                g->q_margin[q] = MT_CANDS[bq];
            }
            TRY(upload_margins(g));
            g->mtrial = 0;
            g->tuning = true;                      // then the launch parameters
        }
    }
    if (trial_now && est == MN_OK) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g->tune_e0, g->tune_e1));
        const int arm = pd.trial_off ? 0 : 1;
        g->ft_ms[arm] += ms;
        g->ft_edges[arm] += (double)n;
        if (++g->ft_idx >= 2 * g->ft_per) {
            // kept only when clearly faster: the dirty-vertex marking at
            // insertion and expiry is outside the timed span
            const bool on = g->ft_ms[1] / g->ft_edges[1] < 0.97 * (g->ft_ms[0] / g->ft_edges[0]);
            g->ft_choice = on ? 1 : 0;
            g->ftrial = 0;
            if (!on) ft_switch = -1;
        }
    }
    if (est != MN_OK && est != MN_ERR_TIMEOUT) return est;   // validation: nothing applied
    // commit (also after a timeout: the adjacency update ran; counts are partial)
    const std::string timeout_msg = g->err;
    if (g->policy == MN_ORDER_EXPLORE)
        for (int k = 0; k < nph; k++) g->n_samples += g->h_ctrl->nseeds[ph[k].phase];
    CK(cudaMemsetAsync(&g->d_ctrl->status, 0, sizeof(uint32_t), g->stream));
    const uint64_t seq_lo = g->hi;
    if (n) {
        g->cur = 1 - g->cur;
        g->merged_lo = g->lo;
        g->last_ts = g->h_ctrl->last_ts;
        g->have_ts = true;
    }
    g->hi = hi_new;
    const uint64_t ex_lo = g->lo;
    if (x) {
        TRY(filter_mark(g, g->lo, x, nullptr));
        TRY(spill_expired(g, g->lo, x));
        stage_begin(g);
        k_expire<<<cdiv(x, 256), 256, 0, g->stream>>>(g->lo, (uint32_t)x, g->cap_mask, g->L,
                                                      (uint32_t)g->queries.size(), g->d_debi_ptrs,
                                                      g->r_src, g->r_dst, g->r_label, g->cnt[0],
                                                      g->cnt[1], &g->d_ctrl->status);
        CKL();
        stage_end(g, S_EXPIRE);
        g->lo += x;
    }
    g->batch_id++;
    g->stats.batches++;
    if (!count_only && est == MN_OK) note_rates(g, n, x);
    if (ft_switch > 0) TRY(filter_enable(g));
    if (ft_switch < 0) g->filter = false;
    fill_result(g, out, seq_lo, hi_new, ex_lo, ex_lo + x);
    if (est == MN_ERR_TIMEOUT) return fail(g, MN_ERR_TIMEOUT, timeout_msg);
    if (over_budget) return fail(g, MN_ERR_OUTPUT_OVERFLOW, "result lists truncated at mem_budget_bytes");
    return MN_OK;
}

namespace mn {

// Time-window snapshots (the paper's LANL runs use a 24-hour window, Sec.
// VII-D): how many of the seqs [lo, hi) have a timestamp at most
// newest - window.  They are a prefix (timestamps increase with seq), found by
// one thread's binary search over the ring.  Nothing when the batch failed
// validation.
__global__ void k_time_cut(uint64_t lo, uint64_t hi, uint32_t cap_mask, const int64_t *r_ts,
                           const long long *newest, long long window, unsigned long long *x_out,
                           const uint32_t *status)
{
    if (*status) { *x_out = 0; return; }
    const long long t = *newest;
    const long long cut = t < LLONG_MIN + window ? LLONG_MIN : t - window;
    uint64_t a = lo, b = hi;                 // first seq with ts > cut
    while (a < b) {
        const uint64_t mid = a + (b - a) / 2;
        if (r_ts[mid & cap_mask] <= cut) a = mid + 1;
        else b = mid;
    }
    *x_out = a - lo;
}

}  // namespace mn

// Entry points that read or change the graph refuse while a batch queued
// with MN_ASYNC is pending (its completion still changes the graph).
static mn_status refuse_if_pending(mn_graph *g)
{
    if (g->pending.active)
        return fail(g, MN_ERR_STATE, "a batch queued with MN_ASYNC is pending: call mn_batch_wait first");
    return MN_OK;
}

// ====================================================================== C ABI

extern "C" {

mn_status mn_create_graph(const mn_graph_config *cfg, mn_graph **out)
{
    mn_graph *g = nullptr;
    if (!out) return fail(nullptr, MN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, MN_ERR_INVALID_ARG, "cfg is NULL");
    if (cfg->num_vertices == 0 || cfg->num_edge_labels == 0 || cfg->num_edge_labels > 256)
        return fail(nullptr, MN_ERR_INVALID_ARG, "num_vertices must be > 0, num_edge_labels in 1..256");
    if ((uint64_t)cfg->num_vertices * cfg->num_edge_labels >= 0xffffffffull)
        return fail(nullptr, MN_ERR_INVALID_ARG, "num_vertices * num_edge_labels must be < 2^32");
    if (cfg->max_batch == 0 || cfg->max_batch > (1ull << 26))
        return fail(nullptr, MN_ERR_INVALID_ARG, "max_batch must be in 1..2^26");
    if (cfg->max_queries == 0 || cfg->max_queries > 64)
        return fail(nullptr, MN_ERR_INVALID_ARG, "max_queries must be in 1..64");
    uint64_t need = cfg->window_edges ? cfg->window_edges + cfg->max_batch : cfg->edge_capacity;
    if (need == 0) return fail(nullptr, MN_ERR_INVALID_ARG, "insert-only graphs need edge_capacity");
    if (cfg->window_edges && cfg->max_batch > cfg->window_edges)
        return fail(nullptr, MN_ERR_INVALID_ARG, "max_batch must not exceed window_edges");
    if (need > (1ull << 30)) return fail(nullptr, MN_ERR_INVALID_ARG, "capacity above 2^30 edges");

    g = new mn_graph();
    g->device = cfg->device;
    g->V = cfg->num_vertices;
    g->L = cfg->num_edge_labels;
    g->W = cfg->window_edges;
    g->max_batch = cfg->max_batch;
    g->C = next_pow2(std::max<uint64_t>(need, 1024));
    g->cap_mask = (uint32_t)(g->C - 1);
    g->mem_budget = cfg->mem_budget_bytes;
    g->max_queries = cfg->max_queries;
    g->default_out_cap = cfg->out_capacity ? cfg->out_capacity : (1ull << 20);
    g->vmask_host.assign(g->V, 0);
    if (cfg->vertex_label_mask)
        memcpy(g->vmask_host.data(), cfg->vertex_label_mask, sizeof(uint32_t) * g->V);
    for (uint32_t v = 0; v < g->V; v++) g->vmask_hist[g->vmask_host[v]]++;

    auto bail = [&](mn_status s) {
        std::string m = g->err;
        mn_destroy_graph(g);
        g_create_error = m;
        return s;
    };
    cudaError_t e = cudaSetDevice(g->device);
    if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MN_ERR_DEVICE); }
    if (cfg->cuda_stream) {
        g->stream = (cudaStream_t)cfg->cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MN_ERR_DEVICE); }
        g->own_stream = true;
    }
    const uint64_t C = g->C;
    const uint64_t nvl = (uint64_t)g->V * g->L;
    mn_status s = MN_OK;
#define A(x) do { s = (x); if (s != MN_OK) return bail(s); } while (0)
    A(dalloc(g, &g->d_vmask, g->V));
    A(dalloc(g, &g->r_src, C, false));
    A(dalloc(g, &g->r_dst, C, false));
    A(dalloc(g, &g->r_label, C, false));
    A(dalloc(g, &g->r_dead, C));
    A(dalloc(g, &g->batch_flag, C));
    A(dalloc(g, &g->r_attr, C, false));
    A(dalloc(g, &g->r_ts, C, false));
    for (int b = 0; b < 2; b++)
        for (int t = 0; t < NPROB; t++) {
            A(dalloc(g, &g->base[b][t].key, C, false));
            A(dalloc(g, &g->base[b][t].nbr, C, false));
            A(dalloc(g, &g->base[b][t].s32, C, false));
        }
    const uint64_t mb_pad = (uint64_t)cdiv(g->max_batch, SORT_TILE) * SORT_TILE;
    for (int t = 0; t < NPROB; t++) {
        A(dalloc(g, &g->delta[t].key, g->max_batch, false));
        A(dalloc(g, &g->delta[t].nbr, g->max_batch, false));
        A(dalloc(g, &g->delta[t].s32, g->max_batch, false));
        A(dalloc(g, &g->dkA[t], mb_pad, false));
        A(dalloc(g, &g->dkB[t], mb_pad, false));
        A(dalloc(g, &g->dvA[t], mb_pad, false));
        A(dalloc(g, &g->dvB[t], mb_pad, false));
    }
    for (int d = 0; d < 2; d++) {
        A(dalloc(g, &g->cnt[d], nvl));
        A(dalloc(g, &g->offs[d], nvl + 1));
    }
    g->nblk_cap = cdiv(std::max<uint64_t>(C, nvl), CTILE) + 1;
    for (int t = 0; t < NPROB; t++) A(dalloc(g, &g->blk[t], g->nblk_cap));
    g->task_cap = 1u << 19;
    A(dalloc(g, &g->d_sched, 3));
    A(dalloc(g, &g->d_tasks, g->task_cap));
    A(dalloc(g, &g->d_edges, g->max_batch, false));
    A(dalloc(g, &g->d_seqs, g->max_batch, false));
    A(dalloc(g, &g->d_queries, g->max_queries));
    A(dalloc(g, &g->d_plans, (uint64_t)g->max_queries * MN_MAX_QE * NCAND));
    A(dalloc(g, &g->d_debi_ptrs, g->max_queries));
    A(dalloc(g, &g->d_out_ptrs, (uint64_t)g->max_queries * 2));
    A(dalloc(g, &g->d_out_cap, (uint64_t)g->max_queries * 2));
    A(dalloc(g, &g->d_ctrl, 1));
    A(dalloc(g, &g->d_temporal, g->max_queries));
    A(dalloc(g, &g->d_qmargin, g->max_queries, false));
    A(dalloc(g, &g->d_qcyc, (uint64_t)g->max_queries * MARGIN_SLOTS));
    A(dalloc(g, &g->d_qseeds, (uint64_t)g->max_queries * MARGIN_SLOTS));
#undef A
    {
        int nsm = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enumerate<false, false>, ENUM_WARPS * 32, 0);
        if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MN_ERR_DEVICE); }
        g->nsm = nsm;
        g->enum_max_per_sm = std::max(per_sm, 1);
        // as many resident blocks as fit (the kernel is latency-bound)
        g->enum_grid = nsm * g->enum_max_per_sm;
    }
    e = cudaMallocHost((void **)&g->h_ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MN_ERR_OOM); }
    memset(g->h_ctrl, 0, sizeof(Ctrl));
    g->q_margin.assign(g->max_queries, g->pick_margin);
    e = cudaMemcpyAsync(g->d_vmask, g->vmask_host.data(), sizeof(uint32_t) * g->V,
                        cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_qmargin, g->q_margin.data(), sizeof(float) * g->max_queries,
                            cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MN_ERR_DEVICE); }
    *out = g;
    return MN_OK;
}

void mn_destroy_graph(mn_graph *g)
{
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *p : g->allocs) cudaFree(p);
    g->allocs.clear();
    for (auto &p : g->ev_pending) { cudaEventDestroy(p.second.first); cudaEventDestroy(p.second.second); }
    for (auto e : g->ev_pool) cudaEventDestroy(e);
    if (g->ev_open) cudaEventDestroy(g->ev_open);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->tune_e0) cudaEventDestroy(g->tune_e0);
    if (g->tune_e1) cudaEventDestroy(g->tune_e1);
    if (g->h_ctrl) cudaFreeHost(g->h_ctrl);
    if (g->h_fstage) cudaFreeHost(g->h_fstage);
    if (g->h_spill) cudaFreeHost(g->h_spill);
    if (g->h_spill_words) cudaFreeHost(g->h_spill_words);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

const char *mn_last_error(const mn_graph *g)
{
    if (!g) return g_create_error.c_str();
    return g->err.c_str();
}

mn_status mn_register_query(mn_graph *g, const mn_query_desc *d, uint32_t *query_id)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (!d || !query_id || !d->edges) return fail(g, MN_ERR_INVALID_ARG, "NULL argument");
    if (g->queries.size() >= g->max_queries) return fail(g, MN_ERR_STATE, "max_queries reached");
    if (d->nv < 2 || d->nv > MN_MAX_QV || d->ne < 1 || d->ne > MN_MAX_QE)
        return fail(g, MN_ERR_INVALID_ARG, "query needs 2..16 vertices and 1..16 edges");
    if (d->semantics != MN_ISO && d->semantics != MN_HOMO)
        return fail(g, MN_ERR_INVALID_ARG, "semantics must be MN_ISO or MN_HOMO");
    QueryHost Q;
    Q.nv = d->nv; Q.ne = d->ne;
    Q.iso = d->semantics == MN_ISO;
    Q.temporal = d->temporal;
    Q.vmask.assign(d->nv, 0);
    if (d->vlabel_mask) memcpy(Q.vmask.data(), d->vlabel_mask, sizeof(uint32_t) * d->nv);
    Q.edges.assign(d->edges, d->edges + d->ne);
    for (uint32_t e = 0; e < d->ne; e++) {
        const mn_qedge &x = Q.edges[e];
        if (x.src >= d->nv || x.dst >= d->nv || x.src == x.dst)
            return fail(g, MN_ERR_INVALID_ARG, "query edge endpoints must be distinct and < nv");
        if (x.label < -1 || x.label >= (int32_t)g->L)
            return fail(g, MN_ERR_INVALID_ARG, "query edge label must be -1 or < num_edge_labels");
        for (uint32_t f = 0; f < e; f++)
            if (Q.edges[f].src == x.src && Q.edges[f].dst == x.dst)
                return fail(g, MN_ERR_INVALID_ARG, "two query edges with the same (src, dst)");
    }
    if (d->temporal == MN_TEMPORAL_CHAIN) {
        for (uint32_t e = 0; e + 1 < d->ne; e++) Q.prec.push_back({e, e + 1});
    } else if (d->temporal == MN_TEMPORAL_PAIRS) {
        if (d->n_prec && !d->prec) return fail(g, MN_ERR_INVALID_ARG, "prec is NULL");
        for (uint32_t k = 0; k < d->n_prec; k++) {
            uint32_t a = d->prec[2 * k], b = d->prec[2 * k + 1];
            if (a >= d->ne || b >= d->ne || a == b)
                return fail(g, MN_ERR_INVALID_ARG, "precedence pair out of range");
            Q.prec.push_back({a, b});
        }
    } else if (d->temporal != MN_TEMPORAL_NONE) {
        return fail(g, MN_ERR_INVALID_ARG, "unknown temporal mode");
    }
    Q.goff = (4 * Q.nv + 7) / 8 * 8;
    Q.rec_bytes = Q.goff + 8 * Q.ne;
    TRY(compile_query(g, Q));

    const uint32_t qid = (uint32_t)g->queries.size();
    TRY(dalloc(g, &Q.debi, g->C));
    for (int s = 0; s < 2; s++) {
        TRY(dalloc(g, &Q.out[s], g->default_out_cap * Q.rec_bytes, false));
        Q.out_cap[s] = g->default_out_cap;
    }
    CK(cudaMemcpyAsync(g->d_queries + qid, &Q.dev, sizeof(QueryDev), cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(g->d_plans + (uint64_t)qid * MN_MAX_QE * NCAND, Q.plans, sizeof(Q.plans),
                       cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(g->d_debi_ptrs + qid, &Q.debi, sizeof(uint32_t *), cudaMemcpyHostToDevice, g->stream));
    const uint32_t tflag = Q.prec.empty() ? 0u : 1u;
    CK(cudaMemcpyAsync(g->d_temporal + qid, &tflag, sizeof(uint32_t), cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(g->d_out_ptrs + 2 * qid, Q.out, 2 * sizeof(uint8_t *), cudaMemcpyHostToDevice,
                       g->stream));
    CK(cudaMemcpyAsync(g->d_out_cap + 2 * qid, Q.out_cap, 2 * sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, g->stream));
    const uint64_t live = g->hi - g->lo;
    if (live) {
        k_match_range<<<cdiv(live, 256), 256, 0, g->stream>>>(
            g->lo, (uint32_t)live, g->cap_mask, g->r_src, g->r_dst, g->r_label, g->r_attr, g->r_ts,
            g->r_dead, g->d_vmask, g->d_queries + qid, Q.debi);
        CKL();
    }
    CK(cudaStreamSynchronize(g->stream));
    g->queries.push_back(Q);
    *query_id = qid;
    if (g->filter) {
        TRY(filter_alloc(g, qid));
        CK(cudaMemsetAsync(&g->d_ctrl->status, 0, sizeof(uint32_t), g->stream));
        TRY(filter_pass(g, g->cur, g->merged_lo, g->hi, true, (int)qid));
        CK(cudaStreamSynchronize(g->stream));
    }
    return MN_OK;
}

// The kernels of one insert batch, queued on the graph's stream: ingest and
// edgeMatcher, adjacency update, time cut, filtering, work units, order
// choice and the enumeration of dS- and dS+.  On return *x, ph and *nph
// describe the queued phases.  With capture the same calls are recorded in a
// CUDA graph (nothing here may then allocate or wait: the callers size every
// buffer first).
static mn_status queue_batch(mn_graph *g, const mn_edge *edges, uint64_t n, uint32_t flags, uint64_t hi_new,
                             uint64_t *x_io, Phase *ph, int *nph_out, bool count_only, bool tune_now,
                             bool trial_now = false)
{
    uint64_t x = *x_io;
    CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(Ctrl), g->stream));
    if (n) {
        const mn_edge *src = edges;
        if (!(flags & MN_DEVICE_PTR)) {
            CK(cudaMemcpyAsync(g->d_edges, edges, n * sizeof(mn_edge), cudaMemcpyHostToDevice, g->stream));
            g->stats.h2d_bytes += n * sizeof(mn_edge);
            src = g->d_edges;
        }
        IngestParams ip;
        memset(&ip, 0, sizeof(ip));
        ip.edges = src;
        ip.n = (uint32_t)n;
        ip.n_pad = cdiv(n, SORT_TILE) * SORT_TILE;
        ip.seq0 = g->hi;
        ip.last_ts = g->have_ts ? g->last_ts : INT64_MIN;
        ip.V = g->V; ip.L = g->L; ip.cap_mask = g->cap_mask;
        ip.r_src = g->r_src; ip.r_dst = g->r_dst; ip.r_label = g->r_label; ip.r_dead = g->r_dead;
        ip.r_attr = g->r_attr; ip.r_ts = g->r_ts;
        ip.vmask = g->d_vmask;
        ip.nq = (uint32_t)g->queries.size();
        ip.queries = g->d_queries;
        ip.debi = g->d_debi_ptrs;
        for (int t = 0; t < NPROB; t++) { ip.sort.k[t] = g->dkA[t]; ip.sort.v[t] = g->dvA[t]; }
        ip.status = &g->d_ctrl->status;
        ip.last_ts_out = &g->d_ctrl->last_ts;
        stage_begin(g);
        k_ingest<<<cdiv(ip.n_pad, 256), 256, 0, g->stream>>>(ip);
        CKL();
        stage_end(g, S_INGEST);
        stage_begin(g);
        TRY(launch_adjacency_update(g, n, src, g->hi));
        stage_end(g, S_ADJ);
        TRY(filter_mark(g, g->hi, n, nullptr));
        if (g->time_window > 0) {
            // time window: the oldest edges up to newest - window expire now
            k_time_cut<<<1, 1, 0, g->stream>>>(g->lo, hi_new, g->cap_mask, g->r_ts, &g->d_ctrl->last_ts,
                                              (long long)g->time_window, &g->d_ctrl->time_cut,
                                              &g->d_ctrl->status);
            CKL();
            CK(cudaMemcpyAsync(&g->h_ctrl->time_cut, &g->d_ctrl->time_cut, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            g->stats.d2h_bytes += sizeof(unsigned long long);
            x = g->h_ctrl->time_cut;
        }
    }
    // the filtering trial times an on batch from its filter pass to the end of
    // the enumeration; an off batch (g->ft_off_now) enumerates without the
    // filter, and its pass runs after the enumeration, untimed, only to keep
    // the sets up to date
    const bool ft_off = trial_now && g->ft_off_now;
    if (trial_now && !ft_off) CK(cudaEventRecord(g->tune_e0, g->stream));
    // DEBI filtering on G1 (the new adjacency, the expiring edges still visible)
    if (n && !ft_off) TRY(filter_pass(g, 1 - g->cur, g->lo, hi_new, false));
    if (tune_now || ft_off) CK(cudaEventRecord(g->tune_e0, g->stream));
    // the adjacency enumerated holds seqs from `base` on: the new buffer was
    // merged at lo; without new edges the current one was merged at merged_lo
    const int nbuf = n ? 1 - g->cur : g->cur;
    const uint64_t nbase = n ? g->lo : g->merged_lo;
    // dS- first: its seeds (the oldest edges) start the longest searches
    int nph = 0;
    if (x && !g->queries.empty()) {
        // dS-: query edges before the seed edge avoid the expiring [lo, lo + x)
        ph[nph++] = Phase{1, nbuf, nbase, hi_new, g->lo + x, hi_new, false};
        TRY(launch_seeds_range(g, 1, g->lo, x, 0xffffffffu, 0xffffu));
    }
    if (n && !g->queries.empty()) {
        // dS+: query edges before the seed edge avoid the batch [hi, hi_new)
        ph[nph++] = Phase{0, nbuf, nbase, hi_new, g->lo, g->hi, false};
        TRY(launch_seeds_range(g, 0, g->hi, n, 0xffffffffu, 0xffffu));
    }
    if (nph && g->policy != MN_ORDER_PAPER)
        TRY(ensure_learn_rows(g, std::max(g->seed_cap[0], g->seed_cap[1])));
    for (int k = 0; k < nph; k++) TRY(choose_orders(g, ph[k].phase));
    if (nph && !count_only) TRY(presize_outputs(g, n, x));
    if (nph) TRY(launch_enumerate(g, ph, nph, count_only));
    for (int k = 0; k < nph; k++) TRY(log_samples(g, ph[k].phase));
    if (tune_now || trial_now) CK(cudaEventRecord(g->tune_e1, g->stream));
    if (n && ft_off) TRY(filter_pass(g, 1 - g->cur, g->lo, hi_new, false));
    *x_io = x;
    *nph_out = nph;
    return MN_OK;
}

// A batch may be recorded as a CUDA graph: no host wait inside its chain (no
// time window), its edges on the device or in pinned host memory, and no
// autotuning in progress.
static bool graph_eligible(mn_graph *g, const mn_edge *edges, uint64_t n, uint32_t flags, bool tune_now)
{
    if (!g->use_graph || g->time_window > 0 || tune_now) return false;
    if (n && !(flags & MN_DEVICE_PTR)) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, edges) != cudaSuccess) { cudaGetLastError(); return false; }
        if (a.type != cudaMemoryTypeHost) return false;          // pageable: not capturable
    }
    return true;
}

mn_status mn_insert_batch(mn_graph *g, const mn_edge *edges, uint64_t n, uint32_t flags,
                          mn_batch_result *out)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (n && !edges) return fail(g, MN_ERR_INVALID_ARG, "edges is NULL");
    if (n > g->max_batch) return fail(g, MN_ERR_ADMISSION, "batch larger than max_batch");
    if (!g->W && g->hi + n - g->lo > g->C) return fail(g, MN_ERR_ADMISSION, "edge ring is full");
    CK(cudaSetDevice(g->device));
    const bool count_only = (flags & MN_COUNT_ONLY) != 0;
    const uint64_t hi_new = g->hi + n;
    uint64_t x = (g->W && hi_new - g->lo > g->W) ? hi_new - g->lo - g->W : 0;
    // autotuning: run this batch's enumeration under the next candidate
    if (g->mtrial && g->policy != MN_ORDER_LEARNED) {   // the margin acts only on learned orders
        g->mtrial = 0;
        g->tuning = true;
    }
    const bool margin_now = g->mtrial && !g->queries.empty() && n;
    g->qcyc_on = margin_now;
    if (margin_now) {
        const size_t ns = g->queries.size() * MARGIN_SLOTS;
        CK(cudaMemsetAsync(g->d_qcyc, 0, ns * sizeof(unsigned long long), g->stream));
        CK(cudaMemsetAsync(g->d_qseeds, 0, ns * sizeof(uint32_t), g->stream));
    }
    const bool tune_now = g->tuning && !g->queries.empty() && (n || x);
    const bool trial_now = !tune_now && g->ftrial && !g->queries.empty() && n;
    // a filtering-trial batch with an even index enumerates without the filter
    const bool trial_off = trial_now && (g->ft_idx & 1u) == 0;
    g->ft_off_now = trial_off;
    if (tune_now) {
        const auto &c = g->tune_cfgs[g->tune_idx];
        g->enum_grid = g->nsm * (int)c.bps;
        g->split_min = c.split_min;
        g->split_depth = c.split_depth;
        g->presplit_log2 = c.presplit_log2;
        g->slice_min = c.slice_min;
    }
    Phase ph[2];
    int nph = 0;
    if (graph_eligible(g, edges, n, flags, tune_now || trial_now || margin_now)) {
        // size everything the chain would grow, then record it
        if (!g->queries.empty()) {
            uint64_t total_ne = 0;
            for (auto &Q : g->queries) total_ne += Q.ne;
            TRY(ensure_seed_cap(g, 1, std::max<uint64_t>(1, x * total_ne)));
            TRY(ensure_seed_cap(g, 0, std::max<uint64_t>(1, n * total_ne)));
            if (g->policy != MN_ORDER_PAPER) {
                TRY(ensure_model(g));
                TRY(ensure_learn_rows(g, std::max(g->seed_cap[0], g->seed_cap[1])));
                if (g->policy == MN_ORDER_LEARNED) TRY(pack_model(g));
            }
            if (!count_only) TRY(presize_outputs(g, n, x));
        }
        const bool timing = g->timing;
        g->timing = false;                         // stage events stay out of the graph
        CK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed));
        const mn_status qs = queue_batch(g, edges, n, flags, hi_new, &x, ph, &nph, count_only, false);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(g->stream, &graph);
        g->timing = timing;
        if (qs != MN_OK) {
            if (graph) cudaGraphDestroy(graph);
            return qs;
        }
        if (ec != cudaSuccess) return fail(g, MN_ERR_DEVICE, std::string("capture: ") + cudaGetErrorString(ec));
        if (g->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(g->gexec, graph, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(g->gexec);
                g->gexec = nullptr;
            }
        }
        if (!g->gexec) {
            const cudaError_t ei = cudaGraphInstantiate(&g->gexec, graph, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(graph);
                g->gexec = nullptr;
                return fail(g, MN_ERR_DEVICE, std::string("graph instantiate: ") + cudaGetErrorString(ei));
            }
            g->stats.graph_instantiations++;
        }
        cudaGraphDestroy(graph);
        CK(cudaGraphLaunch(g->gexec, g->stream));
        g->stats.graph_launches++;
    } else {
        TRY(queue_batch(g, edges, n, flags, hi_new, &x, ph, &nph, count_only, tune_now,
                        trial_now || margin_now));
    }
    PendingBatch &pd = g->pending;
    pd.active = true;
    pd.id = g->batch_id + 1;
    pd.n = n;
    pd.x = x;
    pd.hi_new = hi_new;
    pd.count_only = count_only;
    pd.tune_now = tune_now;
    pd.trial_now = trial_now;
    pd.trial_off = trial_off;
    pd.margin_now = margin_now;
    pd.nph = nph;
    for (int k = 0; k < nph; k++) pd.ph[k] = ph[k];
    if (flags & MN_ASYNC) {
        // queued: the result's counts are filled in by mn_batch_wait
        const size_t nq = g->queries.size();
        g->count_pos.assign(nq, 0);
        g->count_neg.assign(nq, 0);
        if (out) {
            out->batch_id = pd.id;
            out->seq_lo = g->hi;
            out->seq_hi = hi_new;
            out->expired_lo = g->lo;
            out->expired_hi = g->lo + x;
            out->num_queries = (uint32_t)nq;
            out->count_pos = g->count_pos.data();
            out->count_neg = g->count_neg.data();
        }
        return MN_OK;
    }
    return insert_finish(g, out);
}

mn_status mn_batch_wait(mn_graph *g, uint64_t batch_id, mn_batch_result *out)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    if (g->pending.active && g->pending.id == batch_id) {
        CK(cudaSetDevice(g->device));
        return insert_finish(g, out);
    }
    if (!g->pending.active && batch_id <= g->batch_id) return MN_OK;   // completed already
    return fail(g, MN_ERR_INVALID_ARG, "no batch with this id is queued");
}

mn_status mn_delete_batch(mn_graph *g, const uint64_t *seqs, uint64_t n, uint32_t flags,
                          mn_batch_result *out)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (n && !seqs) return fail(g, MN_ERR_INVALID_ARG, "seqs is NULL");
    if (n > g->max_batch) return fail(g, MN_ERR_ADMISSION, "batch larger than max_batch");
    CK(cudaSetDevice(g->device));
    const bool count_only = (flags & MN_COUNT_ONLY) != 0;
    CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(Ctrl), g->stream));
    const unsigned long long *ds = reinterpret_cast<const unsigned long long *>(seqs);
    if (n && !(flags & MN_DEVICE_PTR)) {
        CK(cudaMemcpyAsync(g->d_seqs, seqs, n * sizeof(uint64_t), cudaMemcpyHostToDevice, g->stream));
        g->stats.h2d_bytes += n * sizeof(uint64_t);
        ds = g->d_seqs;
    }
    const uint32_t nq = (uint32_t)g->queries.size();
    if (n) {
        k_delete_mark<<<cdiv(n, 256), 256, 0, g->stream>>>(ds, (uint32_t)n, g->lo, g->hi, g->cap_mask,
                                                           g->r_dead, g->batch_flag, &g->d_ctrl->status);
        CKL();
    }
    TRY(filter_refresh(g));
    Phase ph[1] = {Phase{1, g->cur, g->merged_lo, g->hi, g->lo, g->hi, true}};
    int nph = 0;
    if (n && nq) {
        uint64_t total_ne = 0;
        for (auto &Q : g->queries) total_ne += Q.ne;
        TRY(ensure_seed_cap(g, 1, n * total_ne));
        k_seeds_list<<<cdiv(n * nq, 256), 256, 0, g->stream>>>(ds, (uint32_t)n, g->cap_mask, nq,
                                                                g->d_debi_ptrs, g->d_seeds[1],
                                                                &g->d_ctrl->nseeds[1],
                                                                (uint32_t)g->seed_cap[1], g->shard_idx,
                                                                g->shard_cnt, &g->d_ctrl->status);
        CKL();
        TRY(launch_enumerate(g, ph, 1, count_only));
        nph = 1;
    }
    bool over_budget = false;
    mn_status st = enumerate_phases(g, ph, nph, count_only, &over_budget);
    if (n) {
        k_delete_apply<<<cdiv(n, 256), 256, 0, g->stream>>>(ds, (uint32_t)n, g->cap_mask, nq,
                                                            g->d_debi_ptrs, g->r_dead, g->batch_flag,
                                                            &g->d_ctrl->status);
        CKL();
        TRY(filter_mark(g, 0, n, ds));
        CK(cudaStreamSynchronize(g->stream));
    }
    if (st != MN_OK) return st;
    g->batch_id++;
    g->stats.batches++;
    fill_result(g, out, g->hi, g->hi, 0, 0);
    if (over_budget) return fail(g, MN_ERR_OUTPUT_OVERFLOW, "result lists truncated at mem_budget_bytes");
    return MN_OK;
}

mn_status mn_fetch_embeddings(mn_graph *g, uint64_t batch_id, uint32_t query_id, int32_t sign,
                              uint64_t offset, uint64_t max_records, void *dst, uint32_t dst_flags,
                              uint64_t *n_written)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (!n_written) return fail(g, MN_ERR_INVALID_ARG, "n_written is NULL");
    *n_written = 0;
    if (query_id >= g->queries.size()) return fail(g, MN_ERR_INVALID_ARG, "unknown query id");
    if (sign != 1 && sign != -1) return fail(g, MN_ERR_INVALID_ARG, "sign must be +1 or -1");
    if (batch_id != g->batch_id || batch_id == 0)
        return fail(g, MN_ERR_STATE, "only the last batch's lists are kept");
    if (dst_flags & ~(MN_DST_DEVICE | MN_FETCH_SORTED)) return fail(g, MN_ERR_INVALID_ARG, "unknown fetch flags");
    const int s = sign > 0 ? 0 : 1;
    QueryHost &Q = g->queries[query_id];
    const uint64_t total = s == 0 ? g->count_pos[query_id] : g->count_neg[query_id];
    const uint64_t avail = std::min<uint64_t>(total, Q.out_cap[s]);
    if (offset >= avail || max_records == 0) return MN_OK;
    const uint64_t cnt = std::min<uint64_t>(max_records, avail - offset);
    if (!dst) return fail(g, MN_ERR_INVALID_ARG, "dst is NULL");
    CK(cudaSetDevice(g->device));
    if ((dst_flags & MN_FETCH_SORTED) && avail > 0xffffffffull)
        return fail(g, MN_ERR_INVALID_ARG, "sorted fetch of a list above 2^32 records");
    if ((dst_flags & MN_FETCH_SORTED) && Q.sorted_batch[s] != batch_id && avail > 1) {
        // sort the whole list once for this batch, in place: runs of
        // MERGE_ITEMS sorted per thread, index merge passes, then one gather
        // through a scratch list
        uint32_t *ia = nullptr, *ib = nullptr, *bad = nullptr;
        uint8_t *tmp = nullptr;
        mn_status st = dalloc(g, &ia, avail, false);
        if (st == MN_OK) st = dalloc(g, &ib, avail, false);
        if (st == MN_OK) st = dalloc(g, &tmp, avail * Q.rec_bytes, false);
        if (st == MN_OK) st = dalloc(g, &bad, 1, true);
        uint32_t h_bad = 0;
        if (st == MN_OK) {
            const uint32_t n = (uint32_t)avail;
            const uint32_t blocks = cdiv(cdiv(n, MERGE_ITEMS), 256);
            k_rec_sort_runs<<<blocks, 256, 0, g->stream>>>(Q.out[s], Q.rec_bytes, Q.nv, Q.ne, Q.goff, ia, n);
            for (uint64_t R = MERGE_ITEMS; R < n; R *= 2) {
                k_rec_merge_pass<<<blocks, 256, 0, g->stream>>>(Q.out[s], Q.rec_bytes, Q.nv, Q.ne, Q.goff,
                                                                 ia, ib, n, (uint32_t)R);
                std::swap(ia, ib);
            }
            k_rec_gather<<<(uint32_t)g->nsm * 8, 256, 0, g->stream>>>(Q.out[s], Q.rec_bytes, ia, n, tmp, bad);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e == cudaSuccess && !h_bad)
                e = cudaMemcpyAsync(Q.out[s], tmp, avail * Q.rec_bytes, cudaMemcpyDeviceToDevice, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) st = fail(g, MN_ERR_DEVICE, std::string("sorted fetch: ") + cudaGetErrorString(e));
            else if (h_bad) st = fail(g, MN_ERR_DEVICE, "sorted fetch: index out of range in the permutation");
        }
        if (ia) dfree(g, ia, avail * sizeof(uint32_t));
        if (ib) dfree(g, ib, avail * sizeof(uint32_t));
        if (tmp) dfree(g, tmp, avail * Q.rec_bytes);
        if (bad) dfree(g, bad, sizeof(uint32_t));
        if (st != MN_OK) return st;
        Q.sorted_batch[s] = batch_id;
    }
    CK(cudaMemcpyAsync(dst, Q.out[s] + offset * Q.rec_bytes, cnt * Q.rec_bytes,
                       (dst_flags & MN_DST_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       g->stream));
    CK(cudaStreamSynchronize(g->stream));
    *n_written = cnt;
    return MN_OK;
}

mn_status mn_record_layout(const mn_graph *g, uint32_t query_id, uint32_t *nv, uint32_t *ne,
                           uint32_t *record_bytes)
{
    if (!g || query_id >= g->queries.size()) return MN_ERR_INVALID_ARG;
    const QueryHost &Q = g->queries[query_id];
    if (nv) *nv = Q.nv;
    if (ne) *ne = Q.ne;
    if (record_bytes) *record_bytes = Q.rec_bytes;
    return MN_OK;
}

mn_status mn_count_static(mn_graph *g, uint32_t query_id, uint64_t *count)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (!count || query_id >= g->queries.size()) return fail(g, MN_ERR_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(g->device));
    CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(Ctrl), g->stream));
    TRY(filter_refresh(g));
    const uint64_t live = g->hi - g->lo;
    TRY(launch_seeds_range(g, 2, g->lo, live, query_id, 1u));
    const Phase ps{2, g->cur, g->merged_lo, g->hi, g->lo, g->hi, false};
    TRY(launch_enumerate(g, &ps, 1, true));
    TRY(read_ctrl(g));
    if (g->h_ctrl->status) return map_status(g, g->h_ctrl->status);
    *count = g->h_ctrl->counts[query_id * 3 + 2];
    return MN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation count

namespace {

// Scratch of mn_count_static_noalloc, in 8-byte words: [0, 4) status and seed
// count (u32 each), [4, 11) the enumerator's seven work counters, [16, 208)
// counts (3 per query, 64 queries), [256, 336) scheduler words (one 128-byte
// line each), [384, 384 + MN_NOALLOC_MAX_SEEDS) seeds.
constexpr uint32_t NA_WORK = 4, NA_COUNTS = 16, NA_SCHED = 256, NA_SEEDS = 384;
static_assert(NA_WORK + 8 <= NA_COUNTS, "work counters overlap the counts");
static_assert(NA_COUNTS + 3 * 64 <= NA_SCHED, "counts overlap the scheduler words");
static_assert(NA_SCHED * 8 + sizeof(Sched) <= NA_SEEDS * 8, "scheduler words overlap the seeds");
constexpr uint64_t NA_WORDS = NA_SEEDS + (uint64_t)MN_NOALLOC_MAX_SEEDS;
static __device__ __align__(256) unsigned long long mn_noalloc_scratch[NA_WORDS];

std::mutex na_mutex;
void *na_addr[256];   // device address of the scratch per device ordinal (set-up once)

// Device address of the scratch on g's device (which must be current).  In
// host code the symbol is only a host-side stand-in; the kernel needs this
// address.
mn_status noalloc_scratch(mn_graph *g, unsigned long long **out)
{
    if (g->device < 0 || g->device >= 256) return fail(g, MN_ERR_INVALID_ARG, "device ordinal");
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_addr[g->device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, mn_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(g, MN_ERR_DEVICE, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        na_addr[g->device] = ptr;
    }
    *out = reinterpret_cast<unsigned long long *>(na_addr[g->device]);
    return MN_OK;
}

}  // namespace

extern "C" {

mn_status mn_count_static_noalloc(mn_graph *g, uint32_t query_id, uint64_t *count)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (!count || query_id >= g->queries.size()) return fail(g, MN_ERR_INVALID_ARG, "bad argument");
    const uint64_t live = g->hi - g->lo;
    if (live > MN_NOALLOC_MAX_SEEDS)
        return fail(g, MN_ERR_INVALID_ARG,
                    "live window of " + std::to_string(live) +
                        " edges exceeds the no-allocation scratch (at most 4194304 edges)");
    CK(cudaSetDevice(g->device));
    unsigned long long *base = nullptr;
    TRY(noalloc_scratch(g, &base));
    uint32_t *ctl = reinterpret_cast<uint32_t *>(base);
    unsigned long long *seeds = base + NA_SEEDS;
    CK(cudaMemsetAsync(base, 0, NA_SEEDS * sizeof(unsigned long long), g->stream));
    if (live) {
        k_seeds_range<<<cdiv(live, 256), 256, 0, g->stream>>>(
            g->lo, (uint32_t)live, g->cap_mask, (uint32_t)g->queries.size(), g->d_debi_ptrs,
            query_id, 1u, seeds, &ctl[1], MN_NOALLOC_MAX_SEEDS, g->shard_idx, g->shard_cnt, &ctl[0]);
        CKL();
    }
    EnumParams p;
    memset(&p, 0, sizeof(p));
    for (int t = 0; t < NPROB; t++) {
        p.nbr[t] = g->base[g->cur][t].nbr;
        p.s32[t] = g->base[g->cur][t].s32;
    }
    for (int d = 0; d < 2; d++) p.offs[d] = g->offs[d];
    p.L = g->L;
    p.cap_mask = g->cap_mask;
    p.ring_src = g->r_src;
    p.ring_dst = g->r_dst;
    p.debi = g->d_debi_ptrs;
    p.plans = g->d_plans;
    p.seeds = seeds;
    p.nseeds = &ctl[1];
    p.seed_cap = MN_NOALLOC_MAX_SEEDS;
    p.sched = reinterpret_cast<Sched *>(base + NA_SCHED);   // no task queue: no splitting
    p.base32 = (uint32_t)g->merged_lo;
    p.base = g->merged_lo;
    p.vis_lo = (uint32_t)(g->lo - g->merged_lo);
    p.vis_hi = (uint32_t)(g->hi - g->merged_lo);
    p.av_lo = p.vis_lo;
    p.av_hi = p.vis_hi;
    p.sign = 2;
    p.counts = base + NA_COUNTS;
    p.count_only = 1;
    p.max_iters = g->max_iters;
    p.status = &ctl[0];
    p.work = base + NA_WORK;
    p.wait_polls = g->wait_polls;
    p.qrun[0] = p.qrun[1] = ~0ull;
    CK(cudaFuncSetAttribute(k_enumerate<false, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                            g->smem_carveout));
    k_enumerate<false, false><<<g->enum_grid, ENUM_WARPS * 32, 0, g->stream>>>(p);
    CKL();
    uint32_t st = 0;
    unsigned long long c = 0;
    CK(cudaMemcpyAsync(&st, &ctl[0], sizeof(st), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&c, base + NA_COUNTS + query_id * 3 + 2, sizeof(c), cudaMemcpyDeviceToHost,
                       g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (st) return map_status(g, st);
    *count = c;
    return MN_OK;
}

mn_status mn_read_debi(mn_graph *g, uint32_t query_id, uint64_t seq_lo, uint64_t seq_hi,
                       uint32_t *words)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (query_id >= g->queries.size() || seq_hi < seq_lo || (seq_hi > seq_lo && !words))
        return fail(g, MN_ERR_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(g->device));
    std::vector<uint32_t> all(g->C);
    const uint32_t *src = g->queries[query_id].debi;
    uint32_t *tmp = nullptr;
    if (g->filter && g->hi > g->lo) {          // filtered words of the live window
        TRY(filter_refresh(g));
        CK(cudaMemsetAsync(&g->d_ctrl->status, 0, sizeof(uint32_t), g->stream));
        TRY(dalloc(g, &tmp, g->C));
        const FilterParams fp = filter_params(g, query_id, g->cur, g->merged_lo, g->hi, false);
        const uint64_t live = g->hi - g->lo;
        std::vector<uint32_t> part(live);
        k_filtered_words<<<cdiv(live, 256), 256, 0, g->stream>>>(fp, g->lo, (uint32_t)live, g->r_src, g->r_dst,
                                                                 tmp);
        CKL();
        CK(cudaMemcpyAsync(part.data(), tmp, live * sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        dfree(g, tmp, g->C * sizeof(uint32_t));
        for (uint64_t s = g->lo; s < g->hi; s++) all[s & g->cap_mask] = part[s - g->lo];
        src = nullptr;
    }
    if (src) CK(cudaMemcpyAsync(all.data(), src, g->C * sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    for (uint64_t s = seq_lo; s < seq_hi; s++)
        words[s - seq_lo] = (s >= g->lo && s < g->hi) ? all[s & g->cap_mask] : 0u;
    return MN_OK;
}

mn_status mn_read_adjacency(mn_graph *g, uint32_t dir, uint64_t cap, uint32_t *key, uint32_t *nbr,
                            uint64_t *seq, uint64_t *n)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (dir > 1 || !n) return fail(g, MN_ERR_INVALID_ARG, "bad argument");
    CK(cudaSetDevice(g->device));
    const uint64_t m = g->hi - g->merged_lo;
    std::vector<uint32_t> k(m), b(m), s(m);
    std::vector<uint8_t> dead(g->C);
    const DirArrays &D = g->base[g->cur][dir];
    if (m) {
        CK(cudaMemcpyAsync(k.data(), D.key, m * 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaMemcpyAsync(b.data(), D.nbr, m * 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaMemcpyAsync(s.data(), D.s32, m * 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaMemcpyAsync(dead.data(), g->r_dead, g->C, cudaMemcpyDeviceToHost, g->stream));
    }
    CK(cudaStreamSynchronize(g->stream));
    uint64_t w = 0;
    for (uint64_t i = 0; i < m; i++) {
        const uint64_t full = g->lo + (uint32_t)(s[i] - (uint32_t)g->lo);
        if ((uint32_t)(s[i] - (uint32_t)g->lo) >= (uint32_t)(g->hi - g->lo)) continue;
        if (dead[full & g->cap_mask]) continue;
        if (w < cap) {
            if (key) key[w] = k[i];
            if (nbr) nbr[w] = b[i];
            if (seq) seq[w] = full;
        }
        w++;
    }
    *n = w;
    if (w > cap) return fail(g, MN_ERR_INVALID_ARG, "arrays too small");
    return MN_OK;
}

mn_status mn_set_filtering(mn_graph *g, int32_t enable)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    CK(cudaSetDevice(g->device));
    if (!enable) {
        g->filter = false;
        return MN_OK;
    }
    return filter_enable(g);
}


mn_status mn_read_filter(mn_graph *g, uint32_t query_id, uint32_t *td, uint32_t *bu, int32_t *root,
                         int32_t *parent, int32_t *tree_edge)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (query_id >= g->queries.size()) return fail(g, MN_ERR_INVALID_ARG, "no such query");
    const QueryHost &Q = g->queries[query_id];
    if (root) *root = (int32_t)Q.fq.root;
    for (uint32_t u = 0; u < Q.nv; u++) {
        if (parent) parent[u] = Q.fq.parent[u];
        if (tree_edge) tree_edge[u] = Q.fq.tedge[u];
    }
    if (!td && !bu) return MN_OK;
    if (!g->filter) return fail(g, MN_ERR_STATE, "filtering is off");
    CK(cudaSetDevice(g->device));
    TRY(filter_refresh(g));
    const uint64_t bytes = sizeof(uint32_t) * (uint64_t)Q.nv * g->W32;
    if (td) CK(cudaMemcpyAsync(td, Q.td, bytes, cudaMemcpyDeviceToHost, g->stream));
    if (bu) CK(cudaMemcpyAsync(bu, Q.bu, bytes, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return MN_OK;
}

mn_status mn_graph_info(const mn_graph *g, uint64_t *seq_lo, uint64_t *seq_hi, uint32_t *num_queries)
{
    if (!g) return MN_ERR_INVALID_ARG;
    if (seq_lo) *seq_lo = g->lo;
    if (seq_hi) *seq_hi = g->hi;
    if (num_queries) *num_queries = (uint32_t)g->queries.size();
    return MN_OK;
}

mn_status mn_set_timing(mn_graph *g, int enable)
{
    if (!g) return MN_ERR_INVALID_ARG;
    g->timing = enable != 0;
    return MN_OK;
}

mn_status mn_get_stats(const mn_graph *cg, mn_stats *out)
{
    if (!cg || !out) return MN_ERR_INVALID_ARG;
    mn_graph *g = const_cast<mn_graph *>(cg);
    CK(cudaSetDevice(g->device));
    CK(cudaStreamSynchronize(g->stream));
    collect_timing(g);
    if (g->d_fchanges) {
        unsigned long long c = 0;
        CK(cudaMemcpy(&c, g->d_fchanges, sizeof(c), cudaMemcpyDeviceToHost));
        g->stats.filter_changes = c - g->fchanges_base;
    }
    *out = g->stats;
    return MN_OK;
}

mn_status mn_reset_stats(mn_graph *g)
{
    if (!g) return MN_ERR_INVALID_ARG;
    CK(cudaSetDevice(g->device));
    CK(cudaStreamSynchronize(g->stream));
    collect_timing(g);
    g->stats = mn_stats{};
    if (g->d_fchanges) CK(cudaMemcpy(&g->fchanges_base, g->d_fchanges, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost));
    return MN_OK;
}

mn_status mn_set_order_policy(mn_graph *g, uint32_t policy)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    if (policy > MN_ORDER_LEARNED) return fail(g, MN_ERR_INVALID_ARG, "unknown order policy");
    CK(cudaSetDevice(g->device));
    if (policy != MN_ORDER_PAPER) TRY(ensure_model(g));
    g->policy = policy;
    return MN_OK;
}

mn_status mn_train_order_model(mn_graph *g, uint32_t epochs, float lr, float *loss_first,
                               float *loss_last)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    CK(cudaSetDevice(g->device));
    TRY(ensure_model(g));
    unsigned long long total = 0;
    CK(cudaMemcpyAsync(&total, g->d_nsamples, sizeof(total), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (total == 0) return fail(g, MN_ERR_STATE, "no logged samples: run batches under MN_ORDER_EXPLORE");
    const uint32_t n = (uint32_t)std::min<unsigned long long>(total, g->ring);
    CK(cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM));
    const uint32_t grid = (uint32_t)std::min<uint64_t>(cdiv(n, TC_M), (uint64_t)g->nsm);
    CK(cudaMemsetAsync(g->d_train_status, 0, sizeof(uint32_t), g->stream));
    cudaEvent_t t0 = take_event(g), t1 = take_event(g);
    CK(cudaEventRecord(t0, g->stream));
    float l0 = 0.f, l1 = 0.f;
    for (uint32_t e = 0; e <= epochs; e++) {
        CK(cudaMemsetAsync(g->d_G, 0, sizeof(float) * P_COUNT, g->stream));
        CK(cudaMemsetAsync(g->d_loss, 0, sizeof(float), g->stream));
        k_mlp_grad_tc<<<grid, TG_THREADS, TG_SMEM, g->stream>>>(g->d_SX, g->d_ST, n, g->d_P, g->d_G, g->d_loss,
                                                         g->d_train_status);
        CKL();
        if (e == 0 || e == epochs) {
            float l = 0.f;
            CK(cudaMemcpyAsync(&l, g->d_loss, sizeof(float), cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            if (e == 0) l0 = l; else l1 = l;
        }
        if (e == epochs) break;
        g->adam_step++;
        const float c1 = 1.f - std::pow(0.9f, (float)g->adam_step);
        const float c2 = 1.f - std::pow(0.999f, (float)g->adam_step);
        k_adam<<<cdiv(P_COUNT, 256), 256, 0, g->stream>>>(g->d_P, g->d_G, g->d_M1, g->d_M2, P_COUNT, lr,
                                                          0.9f, 0.999f, 1e-8f, c1, c2);
        CKL();
    }
    g->packed = false;
    CK(cudaEventRecord(t1, g->stream));
    uint32_t tst = 0;
    CK(cudaMemcpyAsync(&tst, g->d_train_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    float tms = 0.f;
    CK(cudaEventElapsedTime(&tms, t0, t1));
    g->ev_pool.push_back(t0);
    g->ev_pool.push_back(t1);
    g->stats.ms_train += tms;
    g->stats.train_rows += (uint64_t)n * (epochs + 1);
    if (tst) return fail(g, MN_ERR_TIMEOUT, "training: MMA completion not seen within the wait bound");
    if (loss_first) *loss_first = l0;
    if (loss_last) *loss_last = l1;
    return MN_OK;
}

mn_status mn_order_model_params(mn_graph *g, float *get, const float *set)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    CK(cudaSetDevice(g->device));
    TRY(ensure_model(g));
    if (get) {
        CK(cudaMemcpyAsync(get, g->d_P, sizeof(float) * P_COUNT, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    if (set) {
        CK(cudaMemcpyAsync(g->d_P, set, sizeof(float) * P_COUNT, cudaMemcpyHostToDevice, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        g->packed = false;
    }
    return MN_OK;
}

mn_status mn_set_shard(mn_graph *g, uint32_t index, uint32_t count)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (count == 0 || index >= count) return fail(g, MN_ERR_INVALID_ARG, "need index < count");
    g->shard_idx = index;
    g->shard_cnt = count;
    return MN_OK;
}

mn_status mn_set_time_window(mn_graph *g, int64_t window)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (window < 0) return fail(g, MN_ERR_INVALID_ARG, "window must be >= 0");
    if (window && g->W) return fail(g, MN_ERR_INVALID_ARG, "this graph already has a count window");
    g->time_window = window;
    return MN_OK;
}

mn_status mn_memory_info(const mn_graph *g, uint64_t *used, uint64_t *peak, uint64_t *budget)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    if (used) *used = g->mem_used;
    if (peak) *peak = g->mem_peak;
    if (budget) *budget = g->mem_budget;
    return MN_OK;
}

mn_status mn_reset_index(mn_graph *g)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    CK(cudaSetDevice(g->device));
    const uint64_t live = g->hi - g->lo;
    for (size_t q = 0; q < g->queries.size(); q++) {
        const QueryHost &Q = g->queries[q];
        CK(cudaMemsetAsync(Q.debi, 0, g->C * sizeof(uint32_t), g->stream));
        if (live) {
            k_match_range<<<cdiv(live, 256), 256, 0, g->stream>>>(
                g->lo, (uint32_t)live, g->cap_mask, g->r_src, g->r_dst, g->r_label, g->r_attr, g->r_ts,
                g->r_dead, g->d_vmask, g->d_queries + q, Q.debi);
            CKL();
        }
    }
    if (g->filter) {                       // the filtered sets follow the rebuilt words
        CK(cudaMemsetAsync(&g->d_ctrl->status, 0, sizeof(uint32_t), g->stream));
        TRY(filter_pass(g, g->cur, g->merged_lo, g->hi, true));
        CK(cudaMemsetAsync(g->d_dmap, 0, sizeof(uint32_t) * g->W32, g->stream));
        CK(cudaMemsetAsync(g->d_ndirty, 0, sizeof(uint32_t), g->stream));
        g->filter_dirty = false;
    }
    CK(cudaStreamSynchronize(g->stream));
    return MN_OK;
}

mn_status mn_dual_simulation(mn_graph *g, uint32_t query_id, uint32_t *sim, uint32_t dst_flags,
                             uint64_t *pairs)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (query_id >= g->queries.size()) return fail(g, MN_ERR_INVALID_ARG, "no such query");
    CK(cudaSetDevice(g->device));
    if (!g->d_sim) TRY(dalloc(g, &g->d_sim, (uint64_t)g->V, false));
    if (!g->d_simctl) TRY(dalloc(g, &g->d_simctl, 2));
    const QueryHost &Q = g->queries[query_id];
    DualSimParams p;
    memset(&p, 0, sizeof(p));
    p.nv = Q.nv;
    p.ne = Q.ne;
    p.V = g->V;
    p.L = g->L;
    p.cap_mask = g->cap_mask;
    p.base32 = (uint32_t)g->merged_lo;
    p.vis_lo = (uint32_t)(g->lo - g->merged_lo);
    p.vis_hi = (uint32_t)(g->hi - g->merged_lo);
    for (uint32_t u = 0; u < Q.nv; u++) p.qmask[u] = Q.vmask[u];
    for (uint32_t e = 0; e < Q.ne; e++) {
        p.esrc[e] = (uint8_t)Q.edges[e].src;
        p.edst[e] = (uint8_t)Q.edges[e].dst;
        p.out_e[Q.edges[e].src] |= 1u << e;
        p.in_e[Q.edges[e].dst] |= 1u << e;
    }
    for (int d = 0; d < 2; d++) {
        p.offs[d] = g->offs[d];
        p.nbr[d] = g->base[g->cur][d].nbr;
        p.s32[d] = g->base[g->cur][d].s32;
    }
    p.debi = Q.debi;
    p.vmask = g->d_vmask;
    p.sim = g->d_sim;
    p.flags = reinterpret_cast<uint32_t *>(g->d_simctl);
    unsigned long long *d_pairs = g->d_simctl + 1;
    const uint32_t grid = cdiv(g->V, 256);
    k_dualsim_init<<<grid, 256, 0, g->stream>>>(p);
    CKL();
    // refine until a pass removes nothing (each pass that changes anything
    // removes a pair, so V * nv + 1 passes bound the loop); DS_PASSES passes
    // per host check: the changed flag is sticky over a group (a pass after
    // the fixpoint changes nothing, so the extra passes are harmless)
    constexpr uint32_t DS_PASSES = 8;
    uint32_t changed = 1;
    uint64_t passes = 0;
    while (changed) {
        if (passes > (uint64_t)g->V * Q.nv + DS_PASSES)
            return fail(g, MN_ERR_DEVICE, "dual simulation did not settle");
        CK(cudaMemsetAsync(p.flags, 0, sizeof(uint32_t), g->stream));
        for (uint32_t k = 0; k < DS_PASSES; k++) {
            k_dualsim_pass<<<grid, 256, 0, g->stream>>>(p);
            CKL();
        }
        passes += DS_PASSES;
        CK(cudaMemcpyAsync(&changed, p.flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    g->stats.dualsim_passes += passes;
    CK(cudaMemsetAsync(g->d_simctl, 0, 2 * sizeof(unsigned long long), g->stream));
    k_dualsim_summary<<<grid, 256, 0, g->stream>>>(p, d_pairs);
    CKL();
    uint32_t present = 0;
    unsigned long long npairs = 0;
    CK(cudaMemcpyAsync(&present, p.flags + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&npairs, d_pairs, sizeof(npairs), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    const bool match = present == (Q.nv >= 32 ? 0xffffffffu : (1u << Q.nv) - 1u);
    if (!match) {                    // some query vertex has no image: no match
        CK(cudaMemsetAsync(g->d_sim, 0, sizeof(uint32_t) * g->V, g->stream));
        npairs = 0;
    }
    if (sim) {
        const cudaMemcpyKind k = (dst_flags & MN_DST_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(sim, g->d_sim, sizeof(uint32_t) * g->V, k, g->stream));
    }
    CK(cudaStreamSynchronize(g->stream));
    if (pairs) *pairs = npairs;
    return MN_OK;
}

mn_status mn_set_tuning(mn_graph *g, uint32_t blocks_per_sm, uint32_t split_min, uint32_t split_depth,
                        int32_t smem_carveout)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    if (smem_carveout < -1 || smem_carveout > 100)
        return fail(g, MN_ERR_INVALID_ARG, "smem_carveout must be -1 or 0..100");
    g->smem_carveout = smem_carveout;
    if (blocks_per_sm > (uint32_t)g->enum_max_per_sm)
        return fail(g, MN_ERR_INVALID_ARG, "blocks_per_sm above the enumerator's occupancy limit");
    g->enum_grid = g->nsm * (int)(blocks_per_sm ? blocks_per_sm : (uint32_t)g->enum_max_per_sm);
    g->split_min = split_min ? std::max<uint32_t>(split_min, 33) : SPLIT_MIN;
    g->split_depth = split_depth ? split_depth : MN_MAX_QE;
    return MN_OK;
}

mn_status mn_autotune(mn_graph *g, uint32_t batches_per_config)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    CK(cudaSetDevice(g->device));
    if (!g->tune_e0) CK(cudaEventCreate(&g->tune_e0));
    if (!g->tune_e1) CK(cudaEventCreate(&g->tune_e1));
    build_tune_candidates(g);
    g->tune_ms.assign(g->tune_cfgs.size(), 0.0);
    g->tune_work.assign(g->tune_cfgs.size(), 0.0);
    g->tune_per = std::max<uint32_t>(batches_per_config, 1);
    g->tune_idx = 0;
    g->tune_in = 0;
    // under learned orders the margin trial comes first, then the launch
    g->mtrial = g->policy == MN_ORDER_LEARNED ? 1 : 0;
    g->mt_idx = 0;
    g->mt_qcyc.assign((size_t)MARGIN_SLOTS * g->max_queries, 0.0);
    g->mt_qseeds.assign((size_t)MARGIN_SLOTS * g->max_queries, 0.0);
    g->mt_choice = -1;
    g->tuning = !g->mtrial;
    return MN_OK;
}

mn_status mn_autotune_candidates(mn_graph *g, uint32_t cap, mn_tune_config *out, uint32_t *n)
{
    if (!g || !n) return fail(g, MN_ERR_INVALID_ARG, "NULL argument");
    build_tune_candidates(g);
    *n = (uint32_t)g->tune_cfgs.size();
    for (uint32_t k = 0; k < *n && k < cap && out; k++) {
        const auto &c = g->tune_cfgs[k];
        out[k].blocks_per_sm = c.bps;
        out[k].split_min = c.split_min;
        out[k].split_depth = c.split_depth;
        out[k].presplit_log2 = std::isinf(c.presplit_log2) ? 0.f : c.presplit_log2;
        out[k].slice_min = c.slice_min;
    }
    if (out && cap < *n) return fail(g, MN_ERR_INVALID_ARG, "array too small");
    return MN_OK;
}

mn_status mn_autotune_results(const mn_graph *g, uint32_t cap, mn_tune_result *out, uint32_t *n)
{
    if (!g || !n) return MN_ERR_INVALID_ARG;
    *n = (uint32_t)std::min(g->tune_cfgs.size(), g->tune_ms.size());
    if (!out) return MN_OK;
    if (cap < *n) return MN_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < *n; k++) {
        const auto &c = g->tune_cfgs[k];
        out[k].config.blocks_per_sm = c.bps;
        out[k].config.split_min = c.split_min;
        out[k].config.split_depth = c.split_depth;
        out[k].config.presplit_log2 = std::isinf(c.presplit_log2) ? 0.f : c.presplit_log2;
        out[k].config.slice_min = c.slice_min;
        out[k].enumerate_ms = g->tune_ms[k];
        out[k].work = g->tune_work[k];
    }
    return MN_OK;
}

mn_status mn_set_presplit(mn_graph *g, float log2_cycles)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    if (std::isnan(log2_cycles)) return fail(g, MN_ERR_INVALID_ARG, "threshold is NaN");
    g->presplit_log2 = log2_cycles > 0.f ? log2_cycles : INFINITY;
    return MN_OK;
}

mn_status mn_set_slice_staging(mn_graph *g, uint32_t min_entries)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    if (min_entries && min_entries < 32) return fail(g, MN_ERR_INVALID_ARG, "min_entries below one chunk (32)");
    g->slice_min = min_entries;
    return MN_OK;
}

mn_status mn_get_slice_staging(const mn_graph *g, uint32_t *min_entries)
{
    if (!g || !min_entries) return MN_ERR_INVALID_ARG;
    *min_entries = g->slice_min;
    return MN_OK;
}

mn_status mn_autotune_state(const mn_graph *g, int32_t *active, uint32_t *batches_left)
{
    if (!g) return MN_ERR_INVALID_ARG;
    if (active) *active = (g->mtrial || g->tuning || g->ftrial) ? 1 : 0;
    if (batches_left) {
        uint64_t left = 0;
        if (g->mtrial)
            left = (uint64_t)(MT_BATCHES - g->mt_idx) + (uint64_t)g->tune_cfgs.size() * g->tune_per +
                   2ull * g->ft_per;
        else if (g->tuning)
            left = (uint64_t)(g->tune_cfgs.size() - g->tune_idx) * g->tune_per - g->tune_in + 2ull * g->ft_per;
        else if (g->ftrial)
            left = 2ull * g->ft_per - g->ft_idx;
        *batches_left = (uint32_t)left;
    }
    return MN_OK;
}

mn_status mn_autotune_filter_result(const mn_graph *g, double *ms_per_kedge_off, double *ms_per_kedge_on,
                                    int32_t *filtering_kept)
{
    if (!g) return MN_ERR_INVALID_ARG;
    if (g->ft_choice < 0) return MN_ERR_STATE;
    if (ms_per_kedge_off) *ms_per_kedge_off = 1e3 * g->ft_ms[0] / std::max(g->ft_edges[0], 1.0);
    if (ms_per_kedge_on) *ms_per_kedge_on = 1e3 * g->ft_ms[1] / std::max(g->ft_edges[1], 1.0);
    if (filtering_kept) *filtering_kept = g->ft_choice;
    return MN_OK;
}

static bool margin_ok(float m) { return m >= 0.f && !std::isinf(m); }   // false for NaN too

mn_status mn_set_order_margin(mn_graph *g, float log2_margin)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (!margin_ok(log2_margin)) return fail(g, MN_ERR_INVALID_ARG, "margin must be finite and >= 0");
    CK(cudaSetDevice(g->device));
    g->pick_margin = log2_margin;
    for (auto &m : g->q_margin) m = log2_margin;
    return upload_margins(g);
}

mn_status mn_set_query_margin(mn_graph *g, uint32_t query_id, float log2_margin)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (query_id >= g->queries.size()) return fail(g, MN_ERR_INVALID_ARG, "no such query");
    if (!margin_ok(log2_margin)) return fail(g, MN_ERR_INVALID_ARG, "margin must be finite and >= 0");
    CK(cudaSetDevice(g->device));
    g->q_margin[query_id] = log2_margin;
    return upload_margins(g);
}

mn_status mn_get_order_margin(const mn_graph *g, uint32_t query_id, float *log2_margin)
{
    if (!g || !log2_margin) return MN_ERR_INVALID_ARG;
    if (query_id == MN_DEFAULT_MARGIN) { *log2_margin = g->pick_margin; return MN_OK; }
    if (query_id >= g->queries.size()) return MN_ERR_INVALID_ARG;
    *log2_margin = g->q_margin[query_id];
    return MN_OK;
}

mn_status mn_autotune_margin_result(const mn_graph *g, uint32_t cap, float *margins, double *cycles_per_seed,
                                    double *query_cycles_per_seed, uint32_t *n, float *kept)
{
    if (!g || !n) return MN_ERR_INVALID_ARG;
    *n = MT_N;
    if (g->mt_choice < 0) return MN_ERR_STATE;
    if ((margins || cycles_per_seed || query_cycles_per_seed) && cap < MT_N) return MN_ERR_INVALID_ARG;
    const size_t nq = g->queries.size();
    const std::vector<double> cost = margin_costs(g);
    double all = 0.0;
    std::vector<double> seeds(nq, 0.0);
    for (size_t q = 0; q < nq; q++) {
        for (uint32_t s = 0; s < 2 * (MT_N - 1); s++)     // the intervals' two arms
            seeds[q] += g->mt_qseeds[q * MARGIN_SLOTS + s];
        all += seeds[q];
    }
    for (uint32_t j = 0; j < MT_N; j++) {
        if (margins) margins[j] = MT_CANDS[j];
        double c = 0.0;
        for (size_t q = 0; q < nq; q++) {
            c += cost[q * MT_N + j];
            if (query_cycles_per_seed)
                query_cycles_per_seed[q * cap + j] = seeds[q] > 0 ? cost[q * MT_N + j] / seeds[q] : 0.0;
        }
        if (cycles_per_seed) cycles_per_seed[j] = all > 0 ? c / all : 0.0;
    }
    if (kept) *kept = MT_CANDS[g->mt_choice];
    return MN_OK;
}

mn_status mn_get_presplit(const mn_graph *g, float *log2_cycles)
{
    if (!g || !log2_cycles) return MN_ERR_INVALID_ARG;
    *log2_cycles = std::isinf(g->presplit_log2) ? 0.f : g->presplit_log2;
    return MN_OK;
}

mn_status mn_get_tuning(const mn_graph *g, uint32_t *blocks_per_sm, uint32_t *max_blocks_per_sm,
                        uint32_t *split_min, uint32_t *split_depth, int32_t *smem_carveout)
{
    if (!g) return MN_ERR_INVALID_ARG;
    if (smem_carveout) *smem_carveout = g->smem_carveout;
    if (blocks_per_sm) *blocks_per_sm = (uint32_t)(g->enum_grid / std::max(g->nsm, 1));
    if (max_blocks_per_sm) *max_blocks_per_sm = (uint32_t)g->enum_max_per_sm;
    if (split_min) *split_min = g->split_min;
    if (split_depth) *split_depth = g->split_depth;
    return MN_OK;
}

// Test hook: per-warp loop budget of the enumerator (0 restores no limit).
// A tiny budget makes a bounded device loop give up and report MN_ERR_TIMEOUT.
mn_status mn_set_spill(mn_graph *g, uint64_t capacity_edges)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (g->h_spill) return fail(g, MN_ERR_STATE, "the spill is set already");
    if (capacity_edges == 0) return fail(g, MN_ERR_INVALID_ARG, "capacity must be > 0");
    CK(cudaSetDevice(g->device));
    if (cudaMallocHost((void **)&g->h_spill, capacity_edges * sizeof(SpillRec)) != cudaSuccess ||
        cudaMallocHost((void **)&g->h_spill_words, capacity_edges * g->max_queries * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        if (g->h_spill) cudaFreeHost(g->h_spill);
        g->h_spill = nullptr;
        return fail(g, MN_ERR_OOM, "pinned host memory for the spill");
    }
    TRY(dalloc(g, &g->d_spill, g->max_batch, false));
    TRY(dalloc(g, &g->d_spill_words, (uint64_t)g->max_batch * g->max_queries, false));
    g->spill_cap = capacity_edges;
    g->spill_lo = g->spill_hi = g->lo;
    return MN_OK;
}

mn_status mn_read_spill(mn_graph *g, uint64_t seq_lo, uint64_t seq_hi, mn_edge *edges, uint32_t *words,
                        uint64_t *held_lo, uint64_t *held_hi)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    if (!g->h_spill) return fail(g, MN_ERR_STATE, "no spill (mn_set_spill)");
    CK(cudaSetDevice(g->device));
    CK(cudaStreamSynchronize(g->stream));      // the copies of the last expiry have landed
    if (held_lo) *held_lo = g->spill_lo;
    if (held_hi) *held_hi = g->spill_hi;
    if (seq_hi <= seq_lo) return MN_OK;
    if (seq_lo < g->spill_lo || seq_hi > g->spill_hi)
        return fail(g, MN_ERR_INVALID_ARG, "seqs outside the spilled range");
    const uint32_t nq = (uint32_t)g->queries.size();
    for (uint64_t s = seq_lo; s < seq_hi; s++) {
        const uint64_t pos = s % g->spill_cap;
        if (edges) edges[s - seq_lo] = g->h_spill[pos].e;
        if (words)
            for (uint32_t q = 0; q < nq; q++)
                words[(size_t)q * (seq_hi - seq_lo) + (s - seq_lo)] = g->h_spill_words[(size_t)q * g->spill_cap + pos];
    }
    return MN_OK;
}

mn_status mn_set_graph_capture(mn_graph *g, int32_t enable)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    TRY(refuse_if_pending(g));
    g->use_graph = enable != 0;
    return MN_OK;
}

mn_status mn_set_work_budget(mn_graph *g, uint64_t max_iters)
{
    if (!g) return MN_ERR_INVALID_ARG;
    g->max_iters = max_iters ? max_iters : ~0ull;
    return MN_OK;
}

mn_status mn_set_wait_limit(mn_graph *g, uint32_t max_polls, uint32_t flags)
{
    if (!g) return fail(nullptr, MN_ERR_INVALID_ARG, "graph is NULL");
    if (flags & ~MN_WAIT_HOLD) return fail(g, MN_ERR_INVALID_ARG, "unknown wait flags");
    if (max_polls > (1u << 30)) return fail(g, MN_ERR_INVALID_ARG, "max_polls above 2^30");
    g->wait_polls = max_polls ? max_polls : WAIT_POLLS;
    g->wait_hold = (flags & MN_WAIT_HOLD) ? 1u : 0u;
    return MN_OK;
}

}  // extern "C"

// ====================================================================== model test hooks

namespace {
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};
}  // namespace

extern "C" {

mn_status mn_mlp_forward(int32_t device, const float *params, const uint16_t *x, uint64_t n, float *y)
{
    mn_graph *g = nullptr;
    if (!params || (n && (!x || !y))) return fail(nullptr, MN_ERR_INVALID_ARG, "NULL argument");
    if (n > (1ull << 28)) return fail(nullptr, MN_ERR_INVALID_ARG, "too many rows");
    CK(cudaSetDevice(device));
    DevBuf P, X, Y, W1, W2, St;
    CK(cudaMalloc(&P.p, sizeof(float) * P_COUNT));
    CK(cudaMalloc(&St.p, sizeof(uint32_t)));
    CK(cudaMemset(St.p, 0, sizeof(uint32_t)));
    CK(cudaMalloc(&X.p, 2 * NF * std::max<uint64_t>(n, 1)));
    CK(cudaMalloc(&Y.p, sizeof(float) * std::max<uint64_t>(n, 1)));
    CK(cudaMalloc(&W1.p, 2 * NF * NH));
    CK(cudaMalloc(&W2.p, 2 * NH * NH));
    CK(cudaMemcpy(P.p, params, sizeof(float) * P_COUNT, cudaMemcpyHostToDevice));
    if (n) CK(cudaMemcpy(X.p, x, 2 * NF * n, cudaMemcpyHostToDevice));
    k_mlp_pack<<<cdiv(NH * NH, 256), 256>>>((float *)P.p, (__nv_bfloat16 *)W1.p, (__nv_bfloat16 *)W2.p);
    CK(cudaGetLastError());
    if (n) {
        int nsm = 0;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
        CK(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        k_mlp_forward_tc<<<(uint32_t)std::min<uint64_t>(cdiv(n, TC_M), 2ull * nsm), TC_FWD_THREADS, TC_SMEM>>>(
            (const __nv_bfloat16 *)X.p, nullptr, 1, (uint32_t)n, (const __nv_bfloat16 *)W1.p,
            (const __nv_bfloat16 *)W2.p, (const float *)P.p, (float *)Y.p, (uint32_t *)St.p);
        CK(cudaGetLastError());
        uint32_t st = 0;
        CK(cudaMemcpy(&st, St.p, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        if (st) return fail(nullptr, MN_ERR_TIMEOUT, "tensor-core forward: MMA completion not seen");
        CK(cudaMemcpy(y, Y.p, sizeof(float) * n, cudaMemcpyDeviceToHost));
    }
    CK(cudaDeviceSynchronize());
    return MN_OK;
}

mn_status mn_mlp_gradient(int32_t device, const float *params, const uint16_t *x, const float *t,
                          uint64_t n, float *grad, float *loss)
{
    mn_graph *g = nullptr;
    if (!params || !grad || !loss || (n && (!x || !t))) return fail(nullptr, MN_ERR_INVALID_ARG, "NULL argument");
    if (n > (1ull << 28)) return fail(nullptr, MN_ERR_INVALID_ARG, "too many rows");
    CK(cudaSetDevice(device));
    CK(cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM));
    DevBuf P, X, T, G, L, St;
    CK(cudaMalloc(&St.p, sizeof(uint32_t)));
    CK(cudaMemset(St.p, 0, sizeof(uint32_t)));
    CK(cudaMalloc(&P.p, sizeof(float) * P_COUNT));
    CK(cudaMalloc(&G.p, sizeof(float) * P_COUNT));
    CK(cudaMalloc(&L.p, sizeof(float)));
    CK(cudaMalloc(&X.p, 2 * NF * std::max<uint64_t>(n, 1)));
    CK(cudaMalloc(&T.p, sizeof(float) * std::max<uint64_t>(n, 1)));
    CK(cudaMemcpy(P.p, params, sizeof(float) * P_COUNT, cudaMemcpyHostToDevice));
    if (n) {
        CK(cudaMemcpy(X.p, x, 2 * NF * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(T.p, t, sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    CK(cudaMemset(G.p, 0, sizeof(float) * P_COUNT));
    CK(cudaMemset(L.p, 0, sizeof(float)));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    if (n) {
        k_mlp_grad_tc<<<(uint32_t)std::min<uint64_t>(cdiv(n, TC_M), (uint64_t)nsm), TG_THREADS, TG_SMEM>>>(
            (const __nv_bfloat16 *)X.p, (const float *)T.p, (uint32_t)n, (const float *)P.p, (float *)G.p,
            (float *)L.p, (uint32_t *)St.p);
        CK(cudaGetLastError());
        uint32_t st = 0;
        CK(cudaMemcpy(&st, St.p, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        if (st) return fail(nullptr, MN_ERR_TIMEOUT, "tensor-core gradient: MMA completion not seen");
    }
    CK(cudaMemcpy(grad, G.p, sizeof(float) * P_COUNT, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(loss, L.p, sizeof(float), cudaMemcpyDeviceToHost));
    return MN_OK;
}

}  // extern "C"
