// mn_filter.cuh -- DEBI neighbourhood filtering (Sec. V-A, "Batch
// Processing"; Sec. IV-A) on the device.
//
// Per query, on its query tree (root = the most selective query vertex, BFS
// tree), two vertex sets per query vertex u, kept as bitmaps over the data
// vertices:
//   TD(u)  top-down (f1 + f2/f3): TD(root) = vertices with root's labels
//          passing f2/f3; TD(u) = vertices v passing f2/f3 for u with a live
//          edge matching the tree edge e(u) (its edgeMatcher bit) from a
//          vertex of TD(parent(u));
//   BU(u)  bottom-up (f4): the v in TD(u) that, for every child c of u, have
//          a live edge matching e(c) to a vertex of BU(c).
// f2 / f3 (isomorphism only): for every edge label l of u's query edges and
// in each direction, v has at least as many live edges with label l, and as
// many distinct neighbours over them, as u has query edges with label l;
// likewise over all labels.  The filtered DEBI bit of a tree edge e(u) at a
// data edge is its edgeMatcher bit and (parent side in TD(parent(u)), child
// side in BU(u)); the enumerator uses the vertex form: every vertex it binds
// to query vertex u must lie in BU(u) (which every embedding satisfies).
//
// One top-down and one bottom-up pass: the sets are a function of the live
// graph.  They are maintained from a unified frontier: the endpoints of every
// edge inserted, expired or deleted since the last pass (the dirty list) are
// re-evaluated for every query vertex, level by level in BFS order for TD and
// in reverse for BU; a vertex whose membership changes puts its tree
// neighbours over matching edges on the frontier of the next level (children
// for TD, the parent for BU).  Re-evaluating a candidate recomputes its
// membership from the current graph and the already final sets of the level
// before, so growth (insertions) and shrinking (expiry, deletion: the
// paper's reverse pass) are the same step.  A full pass (every vertex a
// candidate) builds the sets when filtering starts.
#pragma once
#include "mn_device.cuh"

namespace mn {

constexpr int FQ_MAXL = 8;   // distinct edge labels with a degree need per query vertex

struct FilterQuery {
    uint32_t nv, root, nlev;
    uint32_t iso;
    uint8_t order[MN_MAX_QV];         // BFS order
    uint8_t depth[MN_MAX_QV];
    int8_t parent[MN_MAX_QV];
    int8_t tedge[MN_MAX_QV];          // tree edge into u (-1 at the root)
    uint8_t p_is_src[MN_MAX_QV];      // parent(u) is the source of e(u)
    int16_t tlabel[MN_MAX_QV];        // label of e(u) (-1 = any)
    uint32_t children[MN_MAX_QV];     // bit c: c is a child of u
    uint32_t root_qmask;
    uint32_t qmask[MN_MAX_QV];        // label mask of every query vertex
    // f2 / f3 needs (isomorphism): totals and per label, both directions
    uint8_t need_out[MN_MAX_QV], need_in[MN_MAX_QV];
    uint8_t nl[MN_MAX_QV];
    int16_t lab[MN_MAX_QV][FQ_MAXL];
    uint8_t lout[MN_MAX_QV][FQ_MAXL], lin[MN_MAX_QV][FQ_MAXL];
};

struct FilterParams {
    const FilterQuery *fq;            // this query
    uint32_t qi;                      // query index (DEBI words)
    uint32_t V, L, W32, cap_mask;
    const uint32_t *nbr[NPROB], *s32[NPROB];   // adjacency of the buffer enumerated next
    const uint32_t *offs[2];
    uint32_t base32, vis_lo, vis_hi;  // visible seqs relative to base32
    const uint32_t *debi;             // edgeMatcher words of the query
    const uint8_t *r_dead;
    const uint32_t *vmask;
    uint32_t *td, *bu;                // [nv][W32]
    uint32_t *queued;                 // [nv][W32]: on the frontier of u already
    uint32_t *front;                  // [nv][V] frontier lists
    uint32_t *nfront;                 // [nv] list lengths (appended to during a pass)
    const uint32_t *nsnap;            // [nv] lengths when the current kernel was queued: it reads
                                      // entries below these only (later ones may be unwritten)
    const uint32_t *dirty;            // dirty vertices
    const uint32_t *ndirty;
    uint32_t full;                    // 1: every vertex is a candidate (full pass)
    unsigned long long *changes;      // membership flips (work counter)
};

__device__ __forceinline__ bool bit_of(const uint32_t *bm, uint32_t v)
{
    return (bm[v >> 5] >> (v & 31)) & 1u;
}

__device__ __forceinline__ bool entry_live(const FilterParams &p, uint32_t sv)
{
    const uint32_t rel = sv - p.base32;
    return rel >= p.vis_lo && rel < p.vis_hi && !p.r_dead[sv & p.cap_mask];
}

// The slice of v's adjacency in direction dir (0 out, 1 in) for label l (-1:
// all labels), in the by-neighbour order of that direction.
__device__ __forceinline__ void slice_of(const FilterParams &p, uint32_t v, uint32_t dir, int32_t l,
                                         uint32_t &b, uint32_t &e)
{
    const uint32_t *o = p.offs[dir];
    if (l >= 0) { b = o[v * p.L + l]; e = o[v * p.L + l + 1]; }
    else        { b = o[v * p.L];     e = o[v * p.L + p.L]; }
}

// At least `need` live entries and `need` distinct neighbours among them in
// v's slice (dir, l).  A by-neighbour slice sorts by neighbour within each
// label, so for l >= 0 the distinct count is the number of neighbour runs
// with a live entry; over all labels (l = -1) runs of different labels may
// repeat a neighbour, so up to `need` distinct neighbours are kept.
__device__ bool enough(const FilterParams &p, uint32_t v, uint32_t dir, int32_t l, uint32_t need)
{
    if (need == 0) return true;
    uint32_t b, e;
    slice_of(p, v, dir, l, b, e);
    if (e - b < need) return false;
    const uint32_t *nb = p.nbr[dir], *sq = p.s32[dir];
    uint32_t live = 0, nd = 0;
    uint32_t seen[MN_MAX_QE];
    uint32_t prev = 0xffffffffu;
    bool prev_live = false;
    for (uint32_t i = b; i < e && (live < need || nd < need); i++) {
        const uint32_t w = nb[i];
        if (!entry_live(p, sq[i])) continue;
        live++;
        if (l >= 0) {
            if (!(prev_live && w == prev)) nd++;
            prev = w;
            prev_live = true;
        } else if (nd < need) {
            bool dup = false;
            for (uint32_t k = 0; k < nd; k++) dup = dup || seen[k] == w;
            if (!dup) seen[nd++] = w;
        }
    }
    return live >= need && nd >= need;
}

__device__ bool degree_ok(const FilterParams &p, uint32_t v, uint32_t u)
{
    const FilterQuery &Q = *p.fq;
    if (!Q.iso) return true;
    if (!enough(p, v, 0, -1, Q.need_out[u]) || !enough(p, v, 1, -1, Q.need_in[u])) return false;
    for (uint32_t k = 0; k < Q.nl[u]; k++) {
        if (!enough(p, v, 0, Q.lab[u][k], Q.lout[u][k])) return false;
        if (!enough(p, v, 1, Q.lab[u][k], Q.lin[u][k])) return false;
    }
    return true;
}

// Some live edge in v's slice for tree edge e (v on side `vside_src` of it:
// true = v is e's source) whose edgeMatcher bit e is set and whose other
// endpoint is in bitmap `other`.
__device__ bool has_support(const FilterParams &p, uint32_t v, uint32_t e, bool v_is_src, int32_t l,
                            const uint32_t *other)
{
    const uint32_t dir = v_is_src ? 0u : 1u;
    uint32_t b, en;
    slice_of(p, v, dir, l, b, en);
    const uint32_t *nb = p.nbr[dir], *sq = p.s32[dir];
    for (uint32_t i = b; i < en; i++) {
        const uint32_t sv = sq[i];
        const uint32_t rel = sv - p.base32;
        if (rel < p.vis_lo || rel >= p.vis_hi) continue;
        if (!((p.debi[sv & p.cap_mask] >> e) & 1u)) continue;   // 0 for deleted edges
        if (bit_of(other, nb[i])) return true;
    }
    return false;
}

// Put the other endpoints of v's edges matching tree edge e (live, bit e) on
// the frontier of query vertex w.
__device__ void push_over(const FilterParams &p, uint32_t v, uint32_t e, bool v_is_src, int32_t l, uint32_t w)
{
    const uint32_t dir = v_is_src ? 0u : 1u;
    uint32_t b, en;
    slice_of(p, v, dir, l, b, en);
    const uint32_t *nb = p.nbr[dir], *sq = p.s32[dir];
    uint32_t *qd = p.queued + (size_t)w * p.W32;
    for (uint32_t i = b; i < en; i++) {
        const uint32_t sv = sq[i];
        const uint32_t rel = sv - p.base32;
        if (rel < p.vis_lo || rel >= p.vis_hi) continue;
        if (!((p.debi[sv & p.cap_mask] >> e) & 1u)) continue;
        const uint32_t x = nb[i];
        const uint32_t bit = 1u << (x & 31);
        if (atomicOr(&qd[x >> 5], bit) & bit) continue;          // already queued
        const uint32_t k = atomicAdd(&p.nfront[w], 1u);
        if (k < p.V) p.front[(size_t)w * p.V + k] = x;
    }
}

__device__ __forceinline__ void set_bit(uint32_t *bm, uint32_t v, bool on)
{
    if (on) atomicOr(&bm[v >> 5], 1u << (v & 31));
    else    atomicAnd(&bm[v >> 5], ~(1u << (v & 31)));
}

// Candidate k of query vertex u: the dirty list first, then u's frontier
// (full pass: every vertex).
__device__ __forceinline__ bool candidate(const FilterParams &p, uint32_t u, uint32_t k, uint32_t &v)
{
    if (p.full) { v = k; return k < p.V; }
    const uint32_t nd = *p.ndirty;
    if (k < nd) { v = p.dirty[k]; return true; }
    k -= nd;
    if (k < min(p.nsnap[u], p.V)) { v = p.front[(size_t)u * p.V + k]; return true; }
    return false;
}

// One (query, query vertex) item of a level: blockIdx.y indexes items[],
// each a query index << 8 | query vertex; params[q] is query q's state.
struct FilterItems {
    const FilterParams *params;
    const uint32_t *items;
};

// Top-down re-evaluation of the candidates of every item of one level.
__global__ void k_filter_td(FilterItems it, const uint32_t *status)
{
    if (*status) return;
    const uint32_t item = it.items[blockIdx.y];
    const FilterParams &p = it.params[item >> 8];
    const uint32_t u = item & 0xff;
    const FilterQuery &Q = *p.fq;
    const uint32_t total = p.full ? p.V : *p.ndirty + min(p.nsnap[u], p.V);
    uint32_t *tdu = p.td + (size_t)u * p.W32;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        uint32_t v;
        if (!candidate(p, u, k, v)) continue;
        bool now = (p.vmask[v] & Q.qmask[u]) == Q.qmask[u];       // cheap test first
        if (now) {
            if (u == Q.root) {
                now = degree_ok(p, v, u);
            } else {
                const uint32_t pu = (uint32_t)Q.parent[u], e = (uint32_t)Q.tedge[u];
                now = has_support(p, v, e, !Q.p_is_src[u], Q.tlabel[u], p.td + (size_t)pu * p.W32) &&
                      degree_ok(p, v, u);
            }
        }
        const bool was = bit_of(tdu, v);
        if (now == was) continue;
        set_bit(tdu, v, now);
        atomicAdd(p.changes, 1ull);
        if (p.full) continue;
        // BU of u must be re-evaluated at v; children's TD at v's neighbours
        const uint32_t bit = 1u << (v & 31);
        if (!(atomicOr(&p.queued[(size_t)u * p.W32 + (v >> 5)], bit) & bit)) {
            const uint32_t kk = atomicAdd(&p.nfront[u], 1u);
            if (kk < p.V) p.front[(size_t)u * p.V + kk] = v;
        }
        for (uint32_t cm = Q.children[u]; cm; cm &= cm - 1) {
            const uint32_t c = __ffs(cm) - 1;
            push_over(p, v, (uint32_t)Q.tedge[c], Q.p_is_src[c] != 0, Q.tlabel[c], c);
        }
    }
}

// Bottom-up re-evaluation of the candidates of every item of one level.
__global__ void k_filter_bu(FilterItems it, const uint32_t *status)
{
    if (*status) return;
    const uint32_t item = it.items[blockIdx.y];
    const FilterParams &p = it.params[item >> 8];
    const uint32_t u = item & 0xff;
    const FilterQuery &Q = *p.fq;
    const uint32_t total = p.full ? p.V : *p.ndirty + min(p.nsnap[u], p.V);
    uint32_t *buu = p.bu + (size_t)u * p.W32;
    const uint32_t *tdu = p.td + (size_t)u * p.W32;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        uint32_t v;
        if (!candidate(p, u, k, v)) continue;
        bool now = bit_of(tdu, v);
        for (uint32_t cm = Q.children[u]; cm && now; cm &= cm - 1) {
            const uint32_t c = __ffs(cm) - 1;
            now = has_support(p, v, (uint32_t)Q.tedge[c], Q.p_is_src[c] != 0, Q.tlabel[c],
                              p.bu + (size_t)c * p.W32);
        }
        const bool was = bit_of(buu, v);
        if (now == was) continue;
        set_bit(buu, v, now);
        atomicAdd(p.changes, 1ull);
        if (p.full || u == Q.root) continue;
        const uint32_t pu = (uint32_t)Q.parent[u];
        push_over(p, v, (uint32_t)Q.tedge[u], !Q.p_is_src[u], Q.tlabel[u], pu);
    }
}

// One list per query vertex u serves both passes: TD candidates pushed by
// the parent's flips, then u's own TD flips (BU must look at them), then the
// children's BU flips (BU candidates of u); each vertex enters it at most once
// (the queued bitmap), so a list never exceeds V entries.
//
// After a pass: clear the queued bits of every listed vertex (the counts are
// zeroed by the host).
__global__ void k_filter_reset(const FilterParams *params, const uint32_t *status)
{
    if (*status) return;
    const FilterParams &p = params[blockIdx.y];
    const uint32_t nv = p.fq->nv;
    for (uint32_t u = 0; u < nv; u++) {
        const uint32_t n = min(p.nfront[u], p.V);
        uint32_t *qd = p.queued + (size_t)u * p.W32;
        for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const uint32_t x = p.front[(size_t)u * p.V + k];
            atomicAnd(&qd[x >> 5], ~(1u << (x & 31)));
        }
    }
}

// Zero n counters (after the lists they count were cleared).
__global__ void k_filter_zero(uint32_t *c, uint32_t n, const uint32_t *status)
{
    if (*status) return;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) c[i] = 0;
}

// Zero every query's frontier lengths (blockIdx.x = query).
__global__ void k_filter_zero_fronts(const FilterParams *params, const uint32_t *status)
{
    if (*status) return;
    const FilterParams &p = params[blockIdx.x];
    for (uint32_t i = threadIdx.x; i < p.fq->nv; i += blockDim.x) p.nfront[i] = 0;
}

// nsnap = nfront for every item of the level queued next.
__global__ void k_filter_snap(FilterItems it, uint32_t n)
{
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t item = it.items[i];
        const FilterParams &p = it.params[item >> 8];
        const uint32_t u = item & 0xff;
        const_cast<uint32_t *>(p.nsnap)[u] = p.nfront[u];
    }
}

// Dirty vertices: both endpoints of the edges at ring slots of seqs
// [seq_lo, seq_lo + n) (or of the seqs listed), deduplicated by a bitmap.
__global__ void k_filter_dirty(uint64_t seq_lo, uint32_t n, const unsigned long long *seqs, uint32_t cap_mask,
                               const uint32_t *r_src, const uint32_t *r_dst, uint32_t *dmap,
                               uint32_t *dirty, uint32_t *ndirty, uint32_t cap, const uint32_t *status)
{
    if (*status) return;                     // a rejected batch changes nothing
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t slot = (uint32_t)(seqs ? seqs[i] : seq_lo + i) & cap_mask;
    const uint32_t ends[2] = {r_src[slot], r_dst[slot]};
    for (int t = 0; t < 2; t++) {
        const uint32_t x = ends[t];
        if (x >= cap) continue;              // cap = number of vertices
        const uint32_t bit = 1u << (x & 31);
        if (atomicOr(&dmap[x >> 5], bit) & bit) continue;
        const uint32_t k = atomicAdd(ndirty, 1u);
        if (k < cap) dirty[k] = x;
    }
}

__global__ void k_filter_dirty_clear(uint32_t *dmap, const uint32_t *dirty, const uint32_t *ndirty, uint32_t cap,
                                     const uint32_t *status)
{
    if (*status) return;
    const uint32_t n = min(*ndirty, cap);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t x = dirty[k];
        atomicAnd(&dmap[x >> 5], ~(1u << (x & 31)));
    }
}

// Filtered DEBI words of the seqs [seq_lo, seq_lo + n) (the read API).
__global__ void k_filtered_words(FilterParams p, uint64_t seq_lo, uint32_t n, const uint32_t *r_src,
                                 const uint32_t *r_dst, uint32_t *out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const FilterQuery &Q = *p.fq;
    const uint32_t slot = (uint32_t)(seq_lo + i) & p.cap_mask;
    uint32_t w = p.debi[slot];
    const uint32_t s = r_src[slot], d = r_dst[slot];
    for (uint32_t k = 1; k < Q.nv; k++) {
        const uint32_t u = Q.order[k];
        const uint32_t e = (uint32_t)Q.tedge[u], pu = (uint32_t)Q.parent[u];
        const uint32_t pv = Q.p_is_src[u] ? s : d, uv = Q.p_is_src[u] ? d : s;
        if (!(bit_of(p.td + (size_t)pu * p.W32, pv) && bit_of(p.bu + (size_t)u * p.W32, uv))) w &= ~(1u << e);
    }
    out[i] = w;
}

}  // namespace mn
