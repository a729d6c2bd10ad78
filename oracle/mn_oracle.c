/*
 * mn_oracle.c -- plain, slow CPU oracle for incremental subgraph matching
 * on a streaming multigraph (Mnemonic, arXiv 2206.09983).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Sec. II-B, "Problem Definition"):
 *   G is a set of live data edges, each with its own id (here: its arrival
 *   seq), so parallel edges are distinct (Sec. I, Sec. II-A "each edge is
 *   assigned an id").  For a query G_Q an embedding is a pair (f, g):
 *     f : V_Q -> V,   g : E_Q -> live edges,
 *     src(g(e)) = f(s(e)), dst(g(e)) = f(t(e))   (directed, Sec. II-A),
 *     L_Q(u) subset-of L(f(u)) for every query vertex (Sec. II-B; an empty
 *       query label set matches anything, Fig. 1 caption),
 *     query edge label is "any" or equal to the data edge label (Sec. II-B),
 *     edge attribute and timestamp inside the query edge's ranges (Sec. I:
 *       matching on vertex and edge attributes),
 *     isomorphism: f injective (Sec. II-B); homomorphism: no injectivity and
 *       one data edge may serve several query edges (Sec. III),
 *     temporal order: ts(g(a)) < ts(g(b)) for every precedence pair (a, b)
 *       encoded in the query (Sec. VII-C, time-constrained isomorphism).
 *   The incremental result for a batch B is the set of embeddings of the
 *   graph that use at least one edge of B (Sec. II-B: S(G + dG) = S(G) + dS;
 *   new embeddings for insertions, removed ones for deletions, Sec. VII-A).
 *
 * Three tiers, all plain loops:
 *   or_brute_force   every vertex map f in V^{n_q}, then the cartesian
 *                    product of matching parallel edges per query edge;
 *   or_delta         per batch edge x and per query edge e it satisfies,
 *                    a recursive DFS that binds one query edge at a time,
 *                    collecting every (f, g) with g(e) = x, then sort+unique
 *                    (no masking: duplicates are removed by the set);
 *   or_count_static  |S(G)|: the same DFS seeded from every live edge at
 *                    query edge 0 only, counted without storing.
 *   or_delta_count_omp  the first-edge count of dS with the batch edges
 *                    spread over OpenMP threads (timing of the CPU baseline).
 * Every candidate is re-checked against the full definition at the leaf.
 *
 * Records are rows of (n_q + k_q) uint64 values: f(u_0..u_{n_q-1}) followed
 * by seq(g(e_0..e_{k_q-1})), sorted lexicographically.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXV 16
#define OR_MAXE 16
#define OR_MAXP 256

typedef struct {
    int32_t nv, ne;
    uint32_t vmask[OR_MAXV];
    int32_t esrc[OR_MAXE], edst[OR_MAXE], elabel[OR_MAXE];
    int32_t attr_lo[OR_MAXE], attr_hi[OR_MAXE];
    int64_t ts_lo[OR_MAXE], ts_hi[OR_MAXE];
    int32_t iso;
    int32_t nprec;
    int32_t prec_a[OR_MAXP], prec_b[OR_MAXP];
} or_query;

typedef struct {
    uint64_t n, cap;
    int32_t width;
    uint64_t *rows;
} or_result;

/* A data graph as seen by the oracle: parallel arrays over m edges. */
typedef struct {
    uint32_t nV;
    const uint32_t *vmask;
    uint64_t m;
    const uint32_t *src, *dst;
    const uint8_t *label;
    const int32_t *attr;
    const int64_t *ts;
    const uint64_t *seq;
    const uint8_t *alive;     /* NULL: every edge is live */
    const uint8_t *in_batch;  /* NULL: no batch */
} or_graph;

/* ------------------------------------------------------------ results */

static void res_push(or_result *r, const uint64_t *row)
{
    if (r->n == r->cap) {
        r->cap = r->cap ? r->cap * 2 : 1024;
        r->rows = (uint64_t *)realloc(r->rows, r->cap * (uint64_t)r->width * sizeof(uint64_t));
    }
    memcpy(r->rows + r->n * (uint64_t)r->width, row, (size_t)r->width * sizeof(uint64_t));
    r->n++;
}

static int g_sort_width;
static int row_cmp(const void *a, const void *b)
{
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    for (int i = 0; i < g_sort_width; i++) {
        if (x[i] < y[i]) return -1;
        if (x[i] > y[i]) return 1;
    }
    return 0;
}

static void res_sort_unique(or_result *r)
{
    if (r->n == 0) return;
    g_sort_width = r->width;
    qsort(r->rows, r->n, (size_t)r->width * sizeof(uint64_t), row_cmp);
    uint64_t w = 1;
    for (uint64_t i = 1; i < r->n; i++) {
        if (row_cmp(r->rows + (i - 1) * r->width, r->rows + i * r->width) != 0) {
            if (w != i)
                memcpy(r->rows + w * r->width, r->rows + i * r->width,
                       (size_t)r->width * sizeof(uint64_t));
            w++;
        }
    }
    r->n = w;
}

void or_result_free(or_result *r)
{
    if (!r) return;
    free(r->rows);
    free(r);
}

/* ------------------------------------------------------------ predicates */

static int edge_live(const or_graph *G, uint64_t i)
{
    return G->alive == NULL || G->alive[i] != 0;
}

/* The edgeMatcher of Sec. III for query edge e and data edge i: label,
 * endpoint vertex labels (subset test), attribute and timestamp ranges. */
static int edge_match(const or_graph *G, const or_query *q, int e, uint64_t i)
{
    uint32_t ms = q->vmask[q->esrc[e]], md = q->vmask[q->edst[e]];
    if (q->elabel[e] >= 0 && (int32_t)G->label[i] != q->elabel[e]) return 0;
    if ((G->vmask[G->src[i]] & ms) != ms) return 0;
    if ((G->vmask[G->dst[i]] & md) != md) return 0;
    if (G->attr[i] < q->attr_lo[e] || G->attr[i] >= q->attr_hi[e]) return 0;
    if (G->ts[i] < q->ts_lo[e] || G->ts[i] >= q->ts_hi[e]) return 0;
    return 1;
}

/* Full definition check of one candidate (f, g) -- g holds edge indices. */
static int full_check(const or_graph *G, const or_query *q, const uint32_t *f,
                      const uint64_t *g, int need_batch)
{
    for (int u = 0; u < q->nv; u++)
        if ((G->vmask[f[u]] & q->vmask[u]) != q->vmask[u]) return 0;
    if (q->iso)
        for (int a = 0; a < q->nv; a++)
            for (int b = a + 1; b < q->nv; b++)
                if (f[a] == f[b]) return 0;
    int any_batch = 0;
    for (int e = 0; e < q->ne; e++) {
        uint64_t i = g[e];
        if (!edge_live(G, i)) return 0;
        if (G->src[i] != f[q->esrc[e]] || G->dst[i] != f[q->edst[e]]) return 0;
        if (!edge_match(G, q, e, i)) return 0;
        if (G->in_batch && G->in_batch[i]) any_batch = 1;
    }
    for (int p = 0; p < q->nprec; p++)
        if (!(G->ts[g[q->prec_a[p]]] < G->ts[g[q->prec_b[p]]])) return 0;
    if (need_batch && !any_batch) return 0;
    return 1;
}

static void emit(const or_graph *G, const or_query *q, const uint32_t *f,
                 const uint64_t *g, or_result *out)
{
    uint64_t row[OR_MAXV + OR_MAXE];
    for (int u = 0; u < q->nv; u++) row[u] = f[u];
    for (int e = 0; e < q->ne; e++) row[q->nv + e] = G->seq[g[e]];
    res_push(out, row);
}

/* ------------------------------------------------------------ brute force */

or_result *or_brute_force(const or_graph *G, const or_query *q)
{
    or_result *out = (or_result *)calloc(1, sizeof(or_result));
    out->width = q->nv + q->ne;
    uint32_t f[OR_MAXV];
    uint64_t *cand[OR_MAXE];
    uint64_t ncand[OR_MAXE];
    for (int e = 0; e < q->ne; e++) cand[e] = (uint64_t *)malloc((G->m + 1) * sizeof(uint64_t));
    memset(f, 0, sizeof(f));
    for (;;) {
        /* all edges from f(s(e)) to f(t(e)) matching e, per query edge */
        int empty = 0;
        for (int e = 0; e < q->ne && !empty; e++) {
            ncand[e] = 0;
            for (uint64_t i = 0; i < G->m; i++)
                if (edge_live(G, i) && G->src[i] == f[q->esrc[e]] &&
                    G->dst[i] == f[q->edst[e]] && edge_match(G, q, e, i))
                    cand[e][ncand[e]++] = i;
            if (ncand[e] == 0) empty = 1;
        }
        if (!empty) {
            uint64_t pick[OR_MAXE], g[OR_MAXE];
            memset(pick, 0, sizeof(pick));
            for (;;) {
                for (int e = 0; e < q->ne; e++) g[e] = cand[e][pick[e]];
                if (full_check(G, q, f, g, G->in_batch != NULL)) emit(G, q, f, g, out);
                int e = 0;
                while (e < q->ne && ++pick[e] == ncand[e]) pick[e++] = 0;
                if (e == q->ne) break;
            }
        }
        int u = 0;
        while (u < q->nv && ++f[u] == G->nV) f[u++] = 0;
        if (u == q->nv) break;
    }
    for (int e = 0; e < q->ne; e++) free(cand[e]);
    g_sort_width = out->width;
    if (out->n) qsort(out->rows, out->n, (size_t)out->width * sizeof(uint64_t), row_cmp);
    return out;
}

/* ------------------------------------------------------------ seed DFS */

typedef struct {
    const or_graph *G;
    const or_query *q;
    uint64_t *out_start, *out_idx, *in_start, *in_idx;
    int order[OR_MAXE];
    uint32_t f[OR_MAXV];
    int bound[OR_MAXV];
    int ebound[OR_MAXE];
    uint64_t g[OR_MAXE];
    int need_batch;
    or_result *out;
    uint64_t count;
    uint64_t nodes, max_nodes;  /* DFS nodes visited; 0 = no budget */
} dfs_ctx;

static void build_adjacency(dfs_ctx *c)
{
    const or_graph *G = c->G;
    c->out_start = (uint64_t *)calloc((size_t)G->nV + 1, sizeof(uint64_t));
    c->in_start = (uint64_t *)calloc((size_t)G->nV + 1, sizeof(uint64_t));
    c->out_idx = (uint64_t *)malloc((G->m + 1) * sizeof(uint64_t));
    c->in_idx = (uint64_t *)malloc((G->m + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < G->m; i++) {
        if (!edge_live(G, i)) continue;
        c->out_start[G->src[i] + 1]++;
        c->in_start[G->dst[i] + 1]++;
    }
    for (uint32_t v = 0; v < G->nV; v++) {
        c->out_start[v + 1] += c->out_start[v];
        c->in_start[v + 1] += c->in_start[v];
    }
    uint64_t *po = (uint64_t *)malloc(((size_t)G->nV + 1) * sizeof(uint64_t));
    uint64_t *pi = (uint64_t *)malloc(((size_t)G->nV + 1) * sizeof(uint64_t));
    memcpy(po, c->out_start, ((size_t)G->nV + 1) * sizeof(uint64_t));
    memcpy(pi, c->in_start, ((size_t)G->nV + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < G->m; i++) {
        if (!edge_live(G, i)) continue;
        c->out_idx[po[G->src[i]]++] = i;
        c->in_idx[pi[G->dst[i]]++] = i;
    }
    free(po);
    free(pi);
}

static void free_adjacency(dfs_ctx *c)
{
    free(c->out_start); free(c->in_start); free(c->out_idx); free(c->in_idx);
}

/* A connected order of the query edges starting at edge j: repeatedly the
 * lowest-numbered unplaced edge that touches an already bound vertex. */
static int connected_order(const or_query *q, int j, int *order)
{
    int placed[OR_MAXE] = {0}, bnd[OR_MAXV] = {0};
    order[0] = j; placed[j] = 1;
    bnd[q->esrc[j]] = bnd[q->edst[j]] = 1;
    for (int k = 1; k < q->ne; k++) {
        int pick = -1;
        for (int e = 0; e < q->ne && pick < 0; e++)
            if (!placed[e] && (bnd[q->esrc[e]] || bnd[q->edst[e]])) pick = e;
        if (pick < 0) return 0;  /* query not connected */
        order[k] = pick; placed[pick] = 1;
        bnd[q->esrc[pick]] = bnd[q->edst[pick]] = 1;
    }
    return 1;
}

static int used_elsewhere(const dfs_ctx *c, uint32_t v)
{
    for (int u = 0; u < c->q->nv; u++)
        if (c->bound[u] && c->f[u] == v) return 1;
    return 0;
}

static void dfs(dfs_ctx *c, int k);

/* Precedence pairs whose other edge is already bound must already hold for
 * edge e mapped to data edge i (a necessary condition of the leaf check). */
static int temporal_ok(const dfs_ctx *c, int e, uint64_t i)
{
    const or_query *q = c->q;
    const or_graph *G = c->G;
    for (int p = 0; p < q->nprec; p++) {
        int a = q->prec_a[p], b = q->prec_b[p];
        if (a == e && c->ebound[b] && !(G->ts[i] < G->ts[c->g[b]])) return 0;
        if (b == e && c->ebound[a] && !(G->ts[c->g[a]] < G->ts[i])) return 0;
    }
    return 1;
}

static void try_edge(dfs_ctx *c, int k, int e, uint64_t i)
{
    const or_graph *G = c->G;
    const or_query *q = c->q;
    int a = q->esrc[e], b = q->edst[e];
    if (c->max_nodes && c->nodes >= c->max_nodes) return;
    c->nodes++;
    if (!edge_match(G, q, e, i)) return;
    if (!temporal_ok(c, e, i)) return;
    int bind_a = !c->bound[a], bind_b = !c->bound[b];
    if (!bind_a && c->f[a] != G->src[i]) return;
    if (!bind_b && c->f[b] != G->dst[i]) return;
    if (a == b) {                       /* query self-loop */
        if (G->src[i] != G->dst[i]) return;
        bind_b = 0;
    }
    if (q->iso) {
        if (bind_a && used_elsewhere(c, G->src[i])) return;
        if (bind_b && used_elsewhere(c, G->dst[i])) return;
        if (bind_a && bind_b && G->src[i] == G->dst[i]) return;
    }
    if (bind_a) { c->f[a] = G->src[i]; c->bound[a] = 1; }
    if (bind_b) { c->f[b] = G->dst[i]; c->bound[b] = 1; }
    c->g[e] = i;
    c->ebound[e] = 1;
    dfs(c, k + 1);
    c->ebound[e] = 0;
    if (bind_a) c->bound[a] = 0;
    if (bind_b) c->bound[b] = 0;
}

static void dfs(dfs_ctx *c, int k)
{
    const or_graph *G = c->G;
    const or_query *q = c->q;
    if (k == q->ne) {
        if (full_check(G, q, c->f, c->g, c->need_batch)) {
            if (c->out) emit(G, q, c->f, c->g, c->out);
            c->count++;
        }
        return;
    }
    int e = c->order[k];
    int a = q->esrc[e], b = q->edst[e];
    if (c->bound[a]) {
        uint32_t v = c->f[a];
        for (uint64_t p = c->out_start[v]; p < c->out_start[v + 1]; p++)
            try_edge(c, k, e, c->out_idx[p]);
    } else {
        uint32_t v = c->f[b];
        for (uint64_t p = c->in_start[v]; p < c->in_start[v + 1]; p++)
            try_edge(c, k, e, c->in_idx[p]);
    }
}

/* Seed the DFS with data edge x bound to query edge e. */
static void seed(dfs_ctx *c, int e, uint64_t x)
{
    memset(c->bound, 0, sizeof(c->bound));
    memset(c->ebound, 0, sizeof(c->ebound));
    connected_order(c->q, e, c->order);
    try_edge(c, 0, e, x);
}

/* dS for a batch: every embedding of the live graph using >= 1 batch edge. */
or_result *or_delta(const or_graph *G, const or_query *q)
{
    dfs_ctx c;
    memset(&c, 0, sizeof(c));
    c.G = G; c.q = q; c.need_batch = 1;
    c.out = (or_result *)calloc(1, sizeof(or_result));
    c.out->width = q->nv + q->ne;
    int tmp[OR_MAXE];
    if (!connected_order(q, 0, tmp) || G->in_batch == NULL) return c.out;
    build_adjacency(&c);
    for (uint64_t x = 0; x < G->m; x++) {
        if (!G->in_batch[x] || !edge_live(G, x)) continue;
        for (int e = 0; e < q->ne; e++) seed(&c, e, x);
    }
    free_adjacency(&c);
    res_sort_unique(c.out);
    return c.out;
}

/* |dS| only (no lists kept): the same seeds, deduplicated by requiring that
 * the seed's query edge is the first query edge mapped into the batch.  This
 * is a second, independent way to count the set that or_delta lists. */
uint64_t or_delta_count(const or_graph *G, const or_query *q)
{
    dfs_ctx c;
    memset(&c, 0, sizeof(c));
    c.G = G; c.q = q; c.need_batch = 1;
    int tmp[OR_MAXE];
    if (!connected_order(q, 0, tmp) || G->in_batch == NULL) return 0;
    or_result scratch;
    memset(&scratch, 0, sizeof(scratch));
    scratch.width = q->nv + q->ne;
    build_adjacency(&c);
    uint64_t total = 0;
    for (uint64_t x = 0; x < G->m; x++) {
        if (!G->in_batch[x] || !edge_live(G, x)) continue;
        for (int e = 0; e < q->ne; e++) {
            c.out = &scratch;
            scratch.n = 0;
            seed(&c, e, x);
            for (uint64_t r = 0; r < scratch.n; r++) {
                /* keep the row only if no query edge before e maps to a batch edge */
                const uint64_t *row = scratch.rows + r * scratch.width;
                int first = 1;
                for (int i = 0; i < e && first; i++) {
                    uint64_t s = row[q->nv + i];
                    /* seq -> edge index: the graph arrays are in seq order */
                    uint64_t lo = 0, hi = G->m;
                    while (lo < hi) {
                        uint64_t mid = (lo + hi) / 2;
                        if (G->seq[mid] < s) lo = mid + 1; else hi = mid;
                    }
                    if (lo < G->m && G->seq[lo] == s && G->in_batch[lo]) first = 0;
                }
                total += (uint64_t)first;
            }
        }
    }
    free(scratch.rows);
    free_adjacency(&c);
    return total;
}

/* |dS| with a DFS node budget (for sizing workloads): returns 1 and leaves
 * *count partial when the budget runs out, else 0 with the exact count.
 * Embeddings are counted once, at the first query edge mapped to a batch
 * edge (the seed's query edge), as in or_delta_count. */
int or_delta_count_budget(const or_graph *G, const or_query *q, uint64_t max_nodes,
                          uint64_t *count)
{
    dfs_ctx c;
    memset(&c, 0, sizeof(c));
    c.G = G; c.q = q; c.need_batch = 1; c.max_nodes = max_nodes;
    *count = 0;
    int tmp[OR_MAXE];
    if (!connected_order(q, 0, tmp) || G->in_batch == NULL) return 0;
    or_result scratch;
    memset(&scratch, 0, sizeof(scratch));
    scratch.width = q->nv + q->ne;
    build_adjacency(&c);
    for (uint64_t x = 0; x < G->m && !(max_nodes && c.nodes >= max_nodes); x++) {
        if (!G->in_batch[x] || !edge_live(G, x)) continue;
        for (int e = 0; e < q->ne; e++) {
            c.out = &scratch;
            scratch.n = 0;
            seed(&c, e, x);
            for (uint64_t r = 0; r < scratch.n; r++) {
                const uint64_t *row = scratch.rows + r * scratch.width;
                int first = 1;
                for (int i = 0; i < e && first; i++) {
                    uint64_t sq = row[q->nv + i];
                    uint64_t lo = 0, hi = G->m;
                    while (lo < hi) {
                        uint64_t mid = (lo + hi) / 2;
                        if (G->seq[mid] < sq) lo = mid + 1; else hi = mid;
                    }
                    if (lo < G->m && G->seq[lo] == sq && G->in_batch[lo]) first = 0;
                }
                *count += (uint64_t)first;
            }
        }
    }
    free(scratch.rows);
    free_adjacency(&c);
    return (max_nodes && c.nodes >= max_nodes) ? 1 : 0;
}

/* |dS| as or_delta_count computes it, with the batch edges spread over
 * `nthreads` OpenMP threads (0 = all cores): the CPU design point of the
 * paper's system (Sec. VI, OpenMP over work units; Sec. VII, 24 threads),
 * used to time the CPU baseline.  Each thread has its own DFS state and
 * scratch list; the adjacency is built once and only read.  The sum does not
 * depend on the schedule. */
uint64_t or_delta_count_omp(const or_graph *G, const or_query *q, int nthreads)
{
    dfs_ctx c0;
    memset(&c0, 0, sizeof(c0));
    c0.G = G; c0.q = q; c0.need_batch = 1;
    int tmp[OR_MAXE];
    if (!connected_order(q, 0, tmp) || G->in_batch == NULL) return 0;
    build_adjacency(&c0);
    uint64_t total = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel reduction(+ : total)
    {
        dfs_ctx c = c0;
        or_result scratch;
        memset(&scratch, 0, sizeof(scratch));
        scratch.width = q->nv + q->ne;
#pragma omp for schedule(dynamic, 16)
        for (int64_t xi = 0; xi < (int64_t)G->m; xi++) {
            const uint64_t x = (uint64_t)xi;
            if (!G->in_batch[x] || !edge_live(G, x)) continue;
            for (int e = 0; e < q->ne; e++) {
                c.out = &scratch;
                scratch.n = 0;
                seed(&c, e, x);
                for (uint64_t r = 0; r < scratch.n; r++) {
                    const uint64_t *row = scratch.rows + r * scratch.width;
                    int first = 1;
                    for (int i = 0; i < e && first; i++) {
                        uint64_t sq = row[q->nv + i];
                        uint64_t lo = 0, hi = G->m;
                        while (lo < hi) {
                            uint64_t mid = (lo + hi) / 2;
                            if (G->seq[mid] < sq) lo = mid + 1; else hi = mid;
                        }
                        if (lo < G->m && G->seq[lo] == sq && G->in_batch[lo]) first = 0;
                    }
                    total += (uint64_t)first;
                }
            }
        }
        free(scratch.rows);
    }
    free_adjacency(&c0);
    return total;
}

/* Threads or_delta_count_omp runs with when asked for all cores. */
int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* |S(G)|: every embedding has exactly one image of query edge 0. */
uint64_t or_count_static(const or_graph *G, const or_query *q)
{
    dfs_ctx c;
    memset(&c, 0, sizeof(c));
    c.G = G; c.q = q; c.need_batch = 0;
    int tmp[OR_MAXE];
    if (!connected_order(q, 0, tmp)) return 0;
    or_graph H = *G;
    H.in_batch = NULL;
    c.G = &H;
    build_adjacency(&c);
    for (uint64_t x = 0; x < H.m; x++)
        if (edge_live(&H, x)) seed(&c, 0, x);
    free_adjacency(&c);
    return c.count;
}

/* S(G) as a sorted list (small graphs). */
or_result *or_list_static(const or_graph *G, const or_query *q)
{
    dfs_ctx c;
    memset(&c, 0, sizeof(c));
    or_graph H = *G;
    H.in_batch = NULL;
    c.G = &H; c.q = q; c.need_batch = 0;
    c.out = (or_result *)calloc(1, sizeof(or_result));
    c.out->width = q->nv + q->ne;
    int tmp[OR_MAXE];
    if (!connected_order(q, 0, tmp)) return c.out;
    build_adjacency(&c);
    for (uint64_t x = 0; x < H.m; x++)
        if (edge_live(&H, x)) seed(&c, 0, x);
    free_adjacency(&c);
    res_sort_unique(c.out);
    return c.out;
}

/* The DEBI word of Sec. IV-A at match level: bit e is set iff data edge i
 * satisfies the edgeMatcher for query edge e. */
void or_debi_words(const or_graph *G, const or_query *q, uint32_t *out)
{
    for (uint64_t i = 0; i < G->m; i++) {
        uint32_t w = 0;
        if (edge_live(G, i))
            for (int e = 0; e < q->ne; e++)
                if (edge_match(G, q, e, i)) w |= 1u << e;
        out[i] = w;
    }
}
