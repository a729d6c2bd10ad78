// mn_device.cuh -- device data structures and kernels of the incremental
// matcher (Mnemonic, arXiv 2206.09983) for sm_103a.
//
// Hot path per edge batch (Alg. 2, batchInserts then batchDeletes):
//   k_ingest          validate, append to the edge ring, edgeMatcher -> DEBI
//                     words (Sec. IV-A "Updating"), delta sort keys
//   k_sort_tiles /    sort the batch's adjacency entries by (vertex, label,
//   k_merge_pass      neighbour), ties by arrival
//   k_delta_finalize  delta entries + per-(vertex,label) degree counts
//   k_live_count /    live entries per base tile, the delta entries' anchors
//   k_delta_anchor    in the base
//   k_merge_live      merge base and delta into the new sorted adjacency in
//                     one pass, dropping the entries that left the window
//                     (memory recycling, Sec. IV-A)
//   k_scan_*          offsets of every (vertex, label) segment
//   k_seeds_*         work units: one per (batch edge, query, query edge)
//                     whose DEBI bit is set (Sec. VI "Work decomposition"),
//                     optionally only this graph's shard of them
//   k_enumerate       warp-per-seed backtracking (Sec. III enumerator) with
//                     the masks of Table I and the per-seed matching orders
//                     of Sec. VI; one launch per batch for dS- and dS+
//   k_expire          clear DEBI words of expired edges (Sec. IV-A)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "mnemonic.h"

namespace mn {

constexpr uint32_t FULL = 0xffffffffu;

// device status bits (host maps them to mn_status)
constexpr uint32_t ST_BAD_VERTEX = 1u;
constexpr uint32_t ST_TS_ORDER   = 2u;
constexpr uint32_t ST_BAD_DELETE = 4u;
constexpr uint32_t ST_TIMEOUT    = 8u;

// One query edge's edgeMatcher predicate (Sec. III: labels of the edge and
// both endpoints; Sec. I: vertex and edge attributes).
struct QPred {
    int32_t label;          // -1 = any
    uint32_t vmask_src;     // query vertex label masks (subset test)
    uint32_t vmask_dst;
    int32_t attr_lo, attr_hi;
    int32_t pad_;
    int64_t ts_lo, ts_hi;
};

struct QueryDev {
    uint32_t ne, pad_[3];
    QPred e[MN_MAX_QE];
};

// One step of a per-seed matching order: binds query edge `qe`.
//   EXTEND: `from` is bound, `to` is not; scan the adjacency of f(from) in
//           direction `dir` (0 = out: edge from->to, 1 = in: edge to->from).
//   CLOSE : both bound; find the parallel instances between them.
constexpr uint8_t K_EXTEND = 0, K_CLOSE = 1;
struct Step {
    uint8_t qe, kind, from, to;
    uint8_t dir, avoid;     // avoid: qe precedes the seed edge -> no batch edge (Table I)
    int16_t label;
    uint16_t pred, succ;    // bound query edges that must be older / newer
    uint16_t bound_v, pad_; // query vertices bound before this step
};
static_assert(sizeof(Step) == 16, "Step is 16 bytes");

// Candidate matching orders compiled per (query, seed edge); 0 is the
// paper's order (Sec. VI), the others are greedy alternatives that a learned
// model may pick per seed.
constexpr int NCAND = 4;

// 16-byte aligned: lanes load their step with one 16-byte vector load.
struct alignas(16) Plan {
    Step step[MN_MAX_QE];   // step[0] is the seed edge
    uint8_t nsteps, nv, ne, iso;
    uint8_t seed_src, seed_dst, pad_[2];
    uint32_t rec_bytes, goff;
};
static_assert(sizeof(Plan) % 16 == 0, "Plan rows must keep 16-byte alignment");

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- bulk asynchronous copies (the TMA unit's non-tensor mode) and mbarriers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// order this thread's earlier shared-memory accesses before later
// asynchronous-proxy writes to the same buffer
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16), completion counted in bytes on *bar
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ uint32_t match_word(const QueryDev *q, uint32_t label, int32_t attr,
                                               int64_t ts, uint32_t ms, uint32_t md)
{
    uint32_t w = 0;
    const uint32_t ne = q->ne;
    for (uint32_t e = 0; e < ne; e++) {
        const QPred &P = q->e[e];
        bool ok = (P.label < 0 || (uint32_t)P.label == label) &&
                  ((ms & P.vmask_src) == P.vmask_src) && ((md & P.vmask_dst) == P.vmask_dst) &&
                  attr >= P.attr_lo && attr < P.attr_hi && ts >= P.ts_lo && ts < P.ts_hi;
        w |= (uint32_t)ok << e;
    }
    return w;
}

// Block-wide exclusive scan of one value per thread (blockDim multiple of 32,
// at most 1024).  Returns the exclusive prefix; *total gets the block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, s, d);
            if (lane >= d) s += y;
        }
        warp_sums[lane] = s;   // inclusive over warps
    }
    __syncthreads();
    uint32_t warp_off = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[nw - 1];
    uint32_t r = warp_off + x - v;
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ ingest

// The four adjacency orders kept per graph: 0 = out by neighbour, 1 = in by
// neighbour, 2 = out by arrival, 3 = in by arrival.  Both orders group entries
// by key = v * L + label; within a (vertex, label) segment the neighbour order
// sorts by (nbr, seq) and the arrival order by seq.
constexpr int NPROB = 4;

struct SortSet {
    unsigned long long *k[NPROB];
    uint32_t *v[NPROB];
};

struct Adj4 {
    uint32_t *key[NPROB], *nbr[NPROB], *s32[NPROB];
};

// p[t] of a kernel parameter array for a run-time t (blockIdx.y = problem),
// by selects: indexing the parameter array itself copies it to local memory
template <class T>
__device__ __forceinline__ T sel4(T const (&p)[NPROB], int t)
{
    T r = p[0];
#pragma unroll
    for (int k = 1; k < NPROB; k++)
        if (t == k) r = p[k];
    return r;
}

struct IngestParams {
    const mn_edge *edges;
    uint32_t n, n_pad;
    uint64_t seq0;
    int64_t last_ts;
    uint32_t V, L, cap_mask;
    uint32_t *r_src, *r_dst;
    uint8_t *r_label, *r_dead;
    int32_t *r_attr;
    int64_t *r_ts;
    const uint32_t *vmask;
    uint32_t nq;
    const QueryDev *queries;
    uint32_t *const *debi;
    SortSet sort;
    uint32_t *status;
    long long *last_ts_out;
};

// Append the batch to the ring, compute its DEBI words for every query
// (edgeMatcher, Sec. III / IV-A) and emit the sort keys of its adjacency
// entries in both orders.  Invalid batches are flagged in *status; every
// later kernel of the batch checks the flag, and ring slots written here were
// free.
__global__ void k_ingest(IngestParams p)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_pad) return;
    if (i >= p.n) {
        for (int t = 0; t < NPROB; t++) { p.sort.k[t][i] = ~0ull; p.sort.v[t][i] = ~0u; }
        return;
    }
    const mn_edge e = p.edges[i];
    const int64_t prev = i == 0 ? p.last_ts : p.edges[i - 1].ts;
    uint32_t err = 0;
    if (e.src >= p.V || e.dst >= p.V || e.label >= p.L) err |= ST_BAD_VERTEX;
    if (e.ts <= prev) err |= ST_TS_ORDER;
    if (err) atomicOr(p.status, err);
    if (i == p.n - 1) *p.last_ts_out = e.ts;
    const uint32_t slot = (uint32_t)(p.seq0 + i) & p.cap_mask;
    p.r_src[slot] = e.src;
    p.r_dst[slot] = e.dst;
    p.r_label[slot] = (uint8_t)e.label;
    p.r_attr[slot] = e.attr;
    p.r_ts[slot] = e.ts;
    p.r_dead[slot] = 0;
    const uint32_t ms = err ? 0u : p.vmask[e.src];
    const uint32_t md = err ? 0u : p.vmask[e.dst];
    for (uint32_t q = 0; q < p.nq; q++)
        p.debi[q][slot] = err ? 0u : match_word(&p.queries[q], e.label, e.attr, e.ts, ms, md);
    const uint32_t L = p.L;
    const unsigned long long ks = err ? 0ull : (unsigned long long)(e.src * L + e.label) << 32;
    const unsigned long long kd = err ? 0ull : (unsigned long long)(e.dst * L + e.label) << 32;
    p.sort.k[0][i] = ks | e.dst;
    p.sort.k[1][i] = kd | e.src;
    p.sort.k[2][i] = ks | i;
    p.sort.k[3][i] = kd | i;
    for (int t = 0; t < NPROB; t++) p.sort.v[t][i] = i;
}

// Bulk edgeMatcher over live slots [seq_lo, seq_hi) for one query
// (query registration and periodic reset, Sec. VII-D).
__global__ void k_match_range(uint64_t seq_lo, uint32_t n, uint32_t cap_mask,
                              const uint32_t *r_src, const uint32_t *r_dst, const uint8_t *r_label,
                              const int32_t *r_attr, const int64_t *r_ts, const uint8_t *r_dead,
                              const uint32_t *vmask, const QueryDev *q, uint32_t *debi)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t slot = (uint32_t)(seq_lo + i) & cap_mask;
    uint32_t w = 0;
    if (!r_dead[slot])
        w = match_word(q, r_label[slot], r_attr[slot], r_ts[slot], vmask[r_src[slot]],
                       vmask[r_dst[slot]]);
    debi[slot] = w;
}

// ------------------------------------------------------------------ delta sort

constexpr int SORT_TILE = 2048;

__device__ __forceinline__ bool kv_greater(unsigned long long ka, uint32_t va,
                                           unsigned long long kb, uint32_t vb)
{
    return ka > kb || (ka == kb && va > vb);
}

// Bitonic sort of SORT_TILE (key, index) pairs per block; blockIdx.y = problem.
__global__ void __launch_bounds__(1024) k_sort_tiles(SortSet s, const uint32_t *status)
{
    if (*status) return;
    __shared__ unsigned long long sk[SORT_TILE];
    __shared__ uint32_t sv[SORT_TILE];
    unsigned long long *key = sel4(s.k, blockIdx.y);
    uint32_t *val = sel4(s.v, blockIdx.y);
    const uint32_t base = blockIdx.x * SORT_TILE;
    for (int i = threadIdx.x; i < SORT_TILE; i += blockDim.x) {
        sk[i] = key[base + i];
        sv[i] = val[base + i];
    }
    __syncthreads();
    for (int k = 2; k <= SORT_TILE; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < SORT_TILE; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool asc = (i & k) == 0;
                    bool gt = kv_greater(sk[i], sv[i], sk[ixj], sv[ixj]);
                    if (gt == asc) {
                        unsigned long long tk = sk[i]; sk[i] = sk[ixj]; sk[ixj] = tk;
                        uint32_t tv = sv[i]; sv[i] = sv[ixj]; sv[ixj] = tv;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < SORT_TILE; i += blockDim.x) {
        key[base + i] = sk[i];
        val[base + i] = sv[i];
    }
}

constexpr int MERGE_ITEMS = 8;

// One pass of a bottom-up merge sort: merge neighbouring sorted runs of
// length R into runs of 2R (merge path per thread).  blockIdx.y = problem.
__global__ void k_merge_pass(SortSet src, SortSet dst, uint32_t n, uint32_t R,
                             const uint32_t *status)
{
    if (*status) return;
    const unsigned long long *ks = sel4(src.k, blockIdx.y);
    const uint32_t *vs = sel4(src.v, blockIdx.y);
    unsigned long long *kd = sel4(dst.k, blockIdx.y);
    uint32_t *vd = sel4(dst.v, blockIdx.y);
    const uint32_t o = (blockIdx.x * blockDim.x + threadIdx.x) * MERGE_ITEMS;
    if (o >= n) return;
    const uint32_t pbase = o / (2 * R) * (2 * R);
    const uint32_t nA = min(R, n - pbase);
    const uint32_t nB = min(R, n - pbase - nA);
    const unsigned long long *KA = ks + pbase, *KB = KA + nA;
    const uint32_t *VA = vs + pbase, *VB = VA + nA;
    const uint32_t d = o - pbase;
    uint32_t lo = d > nB ? d - nB : 0, hi = min(d, nA);
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (!kv_greater(KA[mid], VA[mid], KB[d - 1 - mid], VB[d - 1 - mid])) lo = mid + 1;
        else hi = mid;
    }
    uint32_t i = lo, j = d - lo;
    for (int t = 0; t < MERGE_ITEMS && o + t < pbase + nA + nB; t++) {
        bool takeA = j >= nB || (i < nA && !kv_greater(KA[i], VA[i], KB[j], VB[j]));
        if (takeA) { kd[o + t] = KA[i]; vd[o + t] = VA[i]; i++; }
        else       { kd[o + t] = KB[j]; vd[o + t] = VB[j]; j++; }
    }
}

// Sorted (key, index) pairs -> delta adjacency entries of each problem, and
// +1 on the (vertex, label) degree counters (counted once, from the
// neighbour-order problems).  blockIdx.y = problem.
__global__ void k_delta_finalize(SortSet s, Adj4 d, const mn_edge *edges, uint32_t *cnt0,
                                 uint32_t *cnt1, uint32_t n, uint64_t seq0, const uint32_t *status)
{
    if (*status) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = blockIdx.y;
    const unsigned long long k = sel4(s.k, t)[i];
    const uint32_t v = sel4(s.v, t)[i];
    const uint32_t key = (uint32_t)(k >> 32);
    sel4(d.key, t)[i] = key;
    sel4(d.nbr, t)[i] = t < 2 ? (uint32_t)k : ((t & 1) ? edges[v].src : edges[v].dst);
    sel4(d.s32, t)[i] = (uint32_t)(seq0 + v);
    if (t == 0) atomicAdd(&cnt0[key], 1u);
    if (t == 1) atomicAdd(&cnt1[key], 1u);
}

// ------------------------------------------------------------------ base compaction

constexpr int CBLK = 256, CITEMS = 8, CTILE = CBLK * CITEMS;

// Tiles of CTILE items are read striped: item u of thread t sits at tile
// position u * CBLK + t, so that each load and store of a warp covers 128
// contiguous bytes.  Exclusive prefix sums of such a tile in position order:
// v[u] becomes the sum of the items before it; *total gets the tile's sum.
__device__ __forceinline__ void striped_excl_scan(uint32_t (&v)[CITEMS], uint32_t *total)
{
    constexpr int NW = CBLK / 32;
    static_assert(CITEMS * NW == 64, "one warp scans the per-(item, warp) sums two per lane");
    __shared__ uint32_t part[CITEMS * NW];
    __shared__ uint32_t tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl[CITEMS];
#pragma unroll
    for (int u = 0; u < CITEMS; u++) {
        uint32_t x = v[u];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, d);
            if (lane >= d) x += y;
        }
        incl[u] = x;
        if (lane == 31) part[u * NW + w] = x;
    }
    __syncthreads();
    if (w == 0) {
        const uint32_t a = part[2 * lane], b = part[2 * lane + 1];
        uint32_t s = a + b;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, s, d);
            if (lane >= d) s += y;
        }
        part[2 * lane] = s - a - b;
        part[2 * lane + 1] = s - b;
        if (lane == 31) tot = s;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < CITEMS; u++) v[u] = part[u * NW + w] + incl[u] - v[u];
    *total = tot;
    __syncthreads();                      // part and tot are free again
}

// Live entries (seq >= lo) per tile of the base adjacency; blockIdx.y = problem.
__global__ void __launch_bounds__(CBLK) k_live_count(Adj4 a, uint32_t n, uint32_t lo32,
                                                     uint32_t live_span, Adj4 blk,
                                                     const uint32_t *status)
{
    if (*status) return;
    const uint32_t *s = sel4(a.s32, blockIdx.y);
    const uint32_t base = blockIdx.x * CTILE + threadIdx.x;
    uint32_t c = 0;
#pragma unroll
    for (int t = 0; t < CITEMS; t++) {
        uint32_t i = base + t * CBLK;
        c += (i < n && (uint32_t)(s[i] - lo32) < live_span) ? 1u : 0u;
    }
    uint32_t total;
    block_excl_scan(c, &total);
    if (threadIdx.x == 0) sel4(blk.key, blockIdx.y)[blockIdx.x] = total;
}

// In-place exclusive scan of nb values per problem (one block per problem,
// blockIdx.x = problem, arrays in b.key[]).
__global__ void __launch_bounds__(1024) k_scan_blocks(Adj4 b, uint32_t nb, const uint32_t *status)
{
    if (*status) return;
    uint32_t *a = sel4(b.key, blockIdx.x);
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        uint32_t i = base + threadIdx.x;
        uint32_t v = i < nb ? a[i] : 0;
        uint32_t total;
        uint32_t ex = block_excl_scan(v, &total);
        if (i < nb) a[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

// Merge of the base adjacency with the sorted delta, with the entries that
// left the window dropped on the way (memory recycling, Sec. IV-A), in one
// pass over the base.  With a(j) = the number of base entries (live or not)
// ordered before delta entry j -- ties take the base first, so a(j) counts
// base keys <= key(j) -- the merged position of a live base entry i is
// (live entries before i) + #{j : a(j) <= i}, and that of delta entry j is
// (live entries before a(j)) + j.  Neighbour order (problems 0, 1) compares
// (key, nbr); arrival order (2, 3) compares key only.

__device__ __forceinline__ unsigned long long adj_key(const uint32_t *K, const uint32_t *N, bool by_nbr,
                                                      uint32_t i)
{
    return ((unsigned long long)K[i] << 32) | (by_nbr ? N[i] : 0u);
}

// a(j) for every delta entry, by binary search over the whole base
// (nA entries); blockIdx.y = problem.
__global__ void k_delta_anchor(Adj4 A, Adj4 B, uint32_t nA, uint32_t nB, Adj4 anchor,
                               const uint32_t *status)
{
    if (*status) return;
    const int t = blockIdx.y;
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nB) return;
    const bool by_nbr = t < 2;
    const unsigned long long kb = adj_key(sel4(B.key, t), sel4(B.nbr, t), by_nbr, j);
    const uint32_t *AK = sel4(A.key, t), *AN = sel4(A.nbr, t);
    uint32_t lo = 0, hi = nA;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (adj_key(AK, AN, by_nbr, mid) <= kb) lo = mid + 1;
        else hi = mid;
    }
    sel4(anchor.key, t)[j] = lo;
}

// First k in [lo, hi) with a[k] > x (hi if none), a non-decreasing.
__device__ __forceinline__ uint32_t upper_in(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t x)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// First k in [lo, hi) with a[k] >= x (hi if none), a non-decreasing.
__device__ __forceinline__ uint32_t lower_in(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t x)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr uint32_t ANCHOR_SMEM = 2048;   // delta anchors of one base tile held in shared memory

// One base tile of CTILE entries per block (blockIdx.y = problem): its live
// entries and the delta entries anchored in it (a(j) in [i0, i1); the last
// tile also takes a(j) = nA) go to their merged positions.  blk holds the
// exclusive scan of the live counts per tile (k_live_count, k_scan_blocks).
__global__ void __launch_bounds__(CBLK) k_merge_live(Adj4 A, Adj4 B, Adj4 O, uint32_t nA, uint32_t nB,
                                                     uint32_t lo32, uint32_t live_span, Adj4 blk,
                                                     Adj4 anchor, const uint32_t *status)
{
    if (*status) return;
    __shared__ uint32_t rank[CTILE + 1];       // live entries before each tile position
    __shared__ uint32_t sa[ANCHOR_SMEM];
    __shared__ uint32_t jr[2];
    const int t0 = blockIdx.y;
    const uint32_t *K = sel4(A.key, t0), *N = sel4(A.nbr, t0), *S = sel4(A.s32, t0);
    uint32_t *OK = sel4(O.key, t0), *ON = sel4(O.nbr, t0), *OS = sel4(O.s32, t0);
    const uint32_t *an = sel4(anchor.key, t0);
    const uint32_t i0 = blockIdx.x * CTILE;
    const uint32_t i1 = min(i0 + (uint32_t)CTILE, nA);
    const bool last_tile = blockIdx.x + 1 == gridDim.x;
    // delta entries anchored in this tile: [jlo, jhi)
    if (threadIdx.x == 0) jr[0] = lower_in(an, 0, nB, i0);
    if (threadIdx.x == 1) jr[1] = last_tile ? nB : lower_in(an, 0, nB, i1);
    uint32_t sv[CITEMS], kv[CITEMS], nv[CITEMS], r[CITEMS];
#pragma unroll
    for (int u = 0; u < CITEMS; u++) {          // all three arrays in flight at once
        const uint32_t i = i0 + u * CBLK + threadIdx.x;
        sv[u] = i < i1 ? S[i] : 0;
        kv[u] = i < i1 ? K[i] : 0;
        nv[u] = i < i1 ? N[i] : 0;
    }
#pragma unroll
    for (int u = 0; u < CITEMS; u++) {
        const uint32_t i = i0 + u * CBLK + threadIdx.x;
        r[u] = (i < i1 && (uint32_t)(sv[u] - lo32) < live_span) ? 1u : 0u;
    }
    uint32_t total;
    striped_excl_scan(r, &total);               // synchronises: jr visible
    const uint32_t live0 = nA ? sel4(blk.key, t0)[blockIdx.x] : 0u;
#pragma unroll
    for (int u = 0; u < CITEMS; u++) rank[u * CBLK + threadIdx.x] = r[u];
    if (threadIdx.x == 0) rank[CTILE] = total;
    const uint32_t jlo = jr[0], jhi = jr[1];
    const bool in_smem = jhi - jlo <= ANCHOR_SMEM;
    if (in_smem)
        for (uint32_t k = threadIdx.x; k < jhi - jlo; k += blockDim.x) sa[k] = an[jlo + k];
    __syncthreads();
    // live base entries: #{j : a(j) <= i} delta entries precede entry i
#pragma unroll
    for (int u = 0; u < CITEMS; u++) {
        const uint32_t i = i0 + u * CBLK + threadIdx.x;
        if (i < i1 && (uint32_t)(sv[u] - lo32) < live_span) {
            const uint32_t jp = in_smem ? jlo + upper_in(sa, 0, jhi - jlo, i) : upper_in(an, jlo, jhi, i);
            const uint32_t o = live0 + r[u] + jp;
            OK[o] = kv[u];
            ON[o] = nv[u];
            OS[o] = sv[u];
        }
    }
    // delta entries anchored here
    for (uint32_t j = jlo + threadIdx.x; j < jhi; j += blockDim.x) {
        const uint32_t a = in_smem ? sa[j - jlo] : an[j];
        const uint32_t o = live0 + rank[min(a - i0, (uint32_t)CTILE)] + j;
        OK[o] = sel4(B.key, t0)[j];
        ON[o] = sel4(B.nbr, t0)[j];
        OS[o] = sel4(B.s32, t0)[j];
    }
}

// ------------------------------------------------------------------ offsets scan

// Block sums of the (vertex, label) degree counters.
__global__ void __launch_bounds__(CBLK) k_scan_reduce(const uint32_t *c0, const uint32_t *c1,
                                                      uint32_t n, uint32_t *bs0, uint32_t *bs1,
                                                      const uint32_t *status)
{
    if (*status) return;
    const uint32_t *c = blockIdx.y ? c1 : c0;
    const uint32_t base = blockIdx.x * CTILE + threadIdx.x;
    uint32_t s = 0;
#pragma unroll
    for (int t = 0; t < CITEMS; t++) s += base + t * CBLK < n ? c[base + t * CBLK] : 0u;
    uint32_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) (blockIdx.y ? bs1 : bs0)[blockIdx.x] = total;
}

// offs[i] = sum of counts before i; offs[n] = total (written by the last block).
__global__ void __launch_bounds__(CBLK) k_scan_apply(const uint32_t *c0, const uint32_t *c1,
                                                     uint32_t n, const uint32_t *bs0,
                                                     const uint32_t *bs1, uint32_t *o0,
                                                     uint32_t *o1, const uint32_t *status)
{
    if (*status) return;
    const bool d1 = blockIdx.y != 0;
    const uint32_t *c = d1 ? c1 : c0;
    uint32_t *o = d1 ? o1 : o0;
    const uint32_t base = blockIdx.x * CTILE + threadIdx.x;
    uint32_t v[CITEMS], cnt[CITEMS];
#pragma unroll
    for (int t = 0; t < CITEMS; t++) {
        cnt[t] = base + t * CBLK < n ? c[base + t * CBLK] : 0u;
        v[t] = cnt[t];
    }
    uint32_t total;
    striped_excl_scan(v, &total);
    const uint32_t off = (d1 ? bs1 : bs0)[blockIdx.x];
#pragma unroll
    for (int t = 0; t < CITEMS; t++) {
        const uint32_t i = base + t * CBLK;
        if (i < n) o[i] = off + v[t];
        if (i + 1 == n) o[n] = off + v[t] + cnt[t];   // the thread holding item n-1
    }
}

// ------------------------------------------------------------------ seeds

// Work units (Sec. VI "Work decomposition"): one seed per (edge, query,
// query edge) with the DEBI bit set, for edges with seq in [seq_lo, seq_lo+n).
// Packed as (seq32 << 32) | (query << 8) | query edge.
// Seed sharding: the seeds of one stream split over `count` graphs (one per
// GPU), each enumerating only the seeds (seq, q, j) it owns; the shards'
// results are disjoint and their union is the unsharded result (each
// embedding is reported once, by the seed edge the masks of Table I pick).
// Owner: the splitmix64 finaliser of the seed's key, modulo count.
__device__ __forceinline__ uint32_t seed_shard(uint64_t seq, uint32_t q, uint32_t j, uint32_t count)
{
    unsigned long long z = (seq << 14) ^ ((unsigned long long)q << 6) ^ j;
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z % count);
}

// The bits of seed word w (seed edges of query q at seq) that shard `idx` of
// `count` owns.
__device__ __forceinline__ uint32_t shard_bits(uint32_t w, uint64_t seq, uint32_t q, uint32_t idx,
                                               uint32_t count)
{
    if (count <= 1) return w;
    uint32_t keep = 0;
    for (uint32_t m = w; m; m &= m - 1) {
        const uint32_t j = __ffs(m) - 1;
        if (seed_shard(seq, q, j, count) == idx) keep |= 1u << j;
    }
    return keep;
}

__global__ void k_seeds_range(uint64_t seq_lo, uint32_t n, uint32_t cap_mask, uint32_t nq,
                              uint32_t *const *debi, uint32_t qsel, uint32_t jmask,
                              unsigned long long *seeds, uint32_t *nseeds, uint32_t seed_cap,
                              uint32_t shard_idx, uint32_t shard_cnt, const uint32_t *status)
{
    if (*status) return;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nql = qsel == 0xffffffffu ? nq : 1u;
    const uint32_t i = t / nql;
    const uint32_t q = qsel == 0xffffffffu ? t % nql : qsel;
    uint32_t w = 0;
    uint32_t s32 = 0;
    if (i < n) {
        s32 = (uint32_t)(seq_lo + i);
        w = shard_bits(debi[q][s32 & cap_mask] & jmask, seq_lo + i, q, shard_idx, shard_cnt);
    }
    const uint32_t c = __popc(w);
    const int lane = threadIdx.x & 31;
    uint32_t x = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    uint32_t tot = __shfl_sync(FULL, x, 31);
    uint32_t base = 0;
    if (lane == 31 && tot) base = atomicAdd(nseeds, tot);
    base = __shfl_sync(FULL, base, 31);
    uint32_t pos = base + x - c;
    while (w) {
        uint32_t j = __ffs(w) - 1;
        w &= w - 1;
        if (pos < seed_cap)
            seeds[pos] = ((unsigned long long)s32 << 32) | ((unsigned long long)q << 8) | j;
        pos++;
    }
}

// Seeds for an explicit deletion list (seqs given as u64).
__global__ void k_seeds_list(const unsigned long long *seqs, uint32_t n, uint32_t cap_mask,
                             uint32_t nq, uint32_t *const *debi, unsigned long long *seeds,
                             uint32_t *nseeds, uint32_t seed_cap, uint32_t shard_idx,
                             uint32_t shard_cnt, const uint32_t *status)
{
    if (*status) return;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t i = t / nq, q = t % nq;
    uint32_t w = 0, s32 = 0;
    if (i < n) {
        s32 = (uint32_t)seqs[i];
        w = shard_bits(debi[q][s32 & cap_mask], seqs[i], q, shard_idx, shard_cnt);
    }
    const uint32_t c = __popc(w);
    const int lane = threadIdx.x & 31;
    uint32_t x = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    uint32_t tot = __shfl_sync(FULL, x, 31);
    uint32_t base = 0;
    if (lane == 31 && tot) base = atomicAdd(nseeds, tot);
    base = __shfl_sync(FULL, base, 31);
    uint32_t pos = base + x - c;
    while (w) {
        uint32_t j = __ffs(w) - 1;
        w &= w - 1;
        if (pos < seed_cap)
            seeds[pos] = ((unsigned long long)s32 << 32) | ((unsigned long long)q << 8) | j;
        pos++;
    }
}

// ------------------------------------------------------------------ enumerator

// A split-off subtree: the partial embedding bound above depth `lvl` (f, g)
// and the adjacency index range [beg, end) still to explore at depth `lvl`.
struct alignas(16) Task {
    uint32_t qj_lvl;            // query | seed edge << 16 | depth << 24
    uint32_t beg, end;
    uint32_t kc;                // candidate matching order of the seed
    unsigned long long state;   // slot state (slot_key)
    uint32_t sid, set;          // seed index (work log), seed set
    uint32_t f[MN_MAX_QV];      // data vertex per query vertex
    uint32_t g[MN_MAX_QE];      // seq (relative to the adjacency base) per query edge
};
static_assert(sizeof(Task) == 160, "Task is 160 bytes");

// Scheduler words of one enumerator launch (zeroed before the launch), each
// on its own 128-byte line: the idle count is read by every busy warp and
// must not share a line with the counters that take atomics.
struct alignas(128) SchedWord {
    uint32_t v;
    uint32_t pad_[31];
};
struct Sched {
    SchedWord next_seed;        // seed cursor
    SchedWord q_head, q_tail;   // task queue: tickets drawn by waiters / slots used by publishers
    SchedWord idle;             // warps waiting for work
    SchedWord busy;             // warps running a seed or a task
};

constexpr int ENUM_WARPS = 4;              // warps per block
// Resident blocks per SM the enumerator is compiled for (registers capped at
// 96 per thread): 20 warps per SM hide more of the dependent-load latency than
// 16 warps at 122 registers (the few spilled bytes stay in L1).
constexpr int ENUM_MIN_BLOCKS = 5;
constexpr int STAGE_BYTES = 4096;          // per-warp output staging buffer
constexpr uint32_t SLICE_WIN = 128;        // adjacency entries per staged window (two per warp)
constexpr uint32_t SLICE_WAIT_POLLS = 1u << 20;   // bound on one window's wait
// Idle wait of a ticket holder (polls of its task-ring slot, backing off to
// 2 us per poll): it gives its slot up after wait_polls polls (default
// WAIT_POLLS, ~0.13 s) even while other warps are busy, and reports
// ST_TIMEOUT when a slot that a publisher reserved stays unpublished for
// RESERVE_POLLS more polls (~8 ms; publishing takes microseconds).
constexpr uint32_t WAIT_POLLS = 1u << 16;
constexpr uint32_t RESERVE_POLLS = 1u << 12;
constexpr uint32_t SPLIT_MIN = 40;         // default: split a depth's range only above this many entries
// Seed word flag (set by k_pick): the seed's predicted work is above the
// pre-split threshold.  Seed words: seq32 << 32 | flags and candidate order
// << 24 | query << 8 | query edge; during the autotuner's margin trial bits
// 26-29 hold the seed's trial slot (MARGIN_SLOTS - 1: not in the trial).
constexpr unsigned long long SEED_PRESPLIT = 1ull << 31;
constexpr uint32_t SEED_MARGIN_SHIFT = 26, MARGIN_SLOTS = 16;
constexpr int PRESPLIT_PIECES = 16;

struct EnumParams {
    const uint32_t *nbr[NPROB];         // 0,1: by neighbour (out, in); 2,3: by arrival
    const uint32_t *s32[NPROB];
    const uint32_t *offs[2];
    uint32_t L, cap_mask;
    const uint32_t *ring_src, *ring_dst;
    uint32_t *const *debi;              // [query] -> word per slot
    const Plan *plans;                  // [query * MN_MAX_QE + seed edge]
    const unsigned long long *seeds;
    const uint32_t *nseeds;
    uint32_t seed_cap;
    Sched *sched;
    Task *tasks;                        // NULL: no splitting
    uint32_t task_cap, task_log2, epoch;   // task ring: slots (a power of two), log2
    uint32_t base32;                    // lowest seq held by the adjacency (low 32 bits)
    unsigned long long base;
    uint32_t vis_lo, vis_hi;            // visible seqs, relative to base
    uint32_t av_lo, av_hi;              // seqs allowed on query edges before the seed edge
    const uint8_t *batch_flag;          // optional per-slot batch flags (explicit deletes)
    uint32_t sign;                      // 0 new, 1 removed, 2 static count
    unsigned long long *counts;         // [query * 3 + sign]
    uint8_t *const *out;                // [query * 2 + sign]
    const unsigned long long *out_cap;  // [query * 2 + sign]
    uint32_t count_only;
    unsigned long long max_iters;       // per-warp loop budget (ST_TIMEOUT beyond)
    uint32_t *status;
    unsigned long long *work;           // [seeds, entries tested, binds, records, busy cycles, tasks,
                                        //  seeds whose endpoints the filtering excludes,
                                        //  entries read from staged windows]
    unsigned long long *seed_work;      // optional: SM cycles spent per seed (all its units)
    unsigned long long *q_cycles;       // optional: SM cycles per (query, trial slot of the seed
                                        // word), [q][MARGIN_SLOTS], all units of the seed
    // optional second seed set, enumerated in the same launch after the first
    // (the other phase of the same batch): its seeds, avoid interval, sign and
    // work log; seeds1 == NULL: one set
    const unsigned long long *seeds1;
    const uint32_t *nseeds1;
    uint32_t seed_cap1;
    uint32_t av_lo1, av_hi1, sign1;
    unsigned long long *seed_work1;
    uint32_t split_min;                 // smallest range handed to an idle warp
    uint32_t split_depth;               // deepest search depth that may be split
    uint32_t *const *bu;                // DEBI filtering on: per query its BU bitmaps [nv][W32]
    uint32_t W32;
    uint32_t wait_polls;                // idle wait bound (WAIT_POLLS)
    uint32_t wait_hold;                 // test: holders neither take nor give up their slot
    unsigned long long qrun[2];         // per seed set: bit q set = enumerate query q's seeds
    uint32_t stage_min;                 // STAGE: ranges at the last two depths at least this long
                                        // are read through shared-memory windows
    uint32_t adj_cap;                   // entries allocated per adjacency array (a multiple of 4)
};

__device__ __forceinline__ uint32_t vload(const uint32_t *p)
{
    return *reinterpret_cast<const volatile uint32_t *>(p);
}

__device__ __forceinline__ unsigned long long vload64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// The task queue is a ring of task_cap slots.  Ticket (and slot number) t
// uses slot t mod task_cap in lap t / task_cap.  A slot's 64-bit state only
// grows: slot_key(epoch, lap) + phase, with phase RESERVED (a publisher is
// writing the task), PUBLISHED, ABANDONED (the ticket holder left first) or
// CONSUMED.  States of earlier launches are smaller than any of this launch.
constexpr uint32_t SLOT_RESERVED = 0, SLOT_PUBLISHED = 1, SLOT_ABANDONED = 2, SLOT_CONSUMED = 3;

__device__ __forceinline__ unsigned long long slot_key(uint32_t epoch, uint32_t lap)
{
    return ((unsigned long long)epoch << 32) | ((unsigned long long)lap << 2);
}

// A slot holds no live task: it was abandoned or consumed, or it was last
// used by an earlier launch.
__device__ __forceinline__ bool slot_free(unsigned long long st, uint32_t epoch)
{
    return (uint32_t)(st >> 32) != epoch || (st & 3) >= SLOT_ABANDONED;
}

// First i in [lo, hi) with key(i) >= t (hi if none) for a key that is
// non-decreasing over [lo, hi); 32 lanes probe 32 positions per round.
template <class KeyFn>
__device__ __forceinline__ uint32_t warp_lower_bound_by(KeyFn key, uint32_t lo, uint32_t hi,
                                                        uint32_t t, int lane)
{
    while (hi - lo > 32) {
        uint32_t stride = (hi - lo + 31) >> 5;
        uint32_t pos = lo + (uint32_t)lane * stride;
        bool less = pos < hi && key(pos) < t;
        uint32_t k = __popc(__ballot_sync(FULL, less));
        if (k == 0) return lo;
        uint32_t nlo = lo + (k - 1) * stride + 1;
        uint32_t nhi = lo + k * stride;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    uint32_t pos = lo + (uint32_t)lane;
    bool less = pos < hi && key(pos) < t;
    return lo + __popc(__ballot_sync(FULL, less));
}

// One lane's [r1, r2) = [first i with key(i) >= t1, first i with key(i) >= t2)
// in [lo, hi) for t1 <= t2 and a non-decreasing key: both binary searches in
// lock step, so each step has two independent loads in flight; each search
// also narrows the other (r1 <= r2).  With ENDS, the first and last keys are
// read first (one round of two loads): an interval entirely before or after
// the keys, or a bound at an end, needs no search.
template <bool ENDS, class KeyFn>
__device__ __forceinline__ void lane_bounds2(KeyFn key, uint32_t lo, uint32_t hi, uint32_t t1,
                                             uint32_t t2, uint32_t &r1, uint32_t &r2)
{
    uint32_t l1 = lo, h1 = hi, l2 = lo, h2 = hi;
    if (ENDS && lo < hi) {
        const uint32_t kf = key(lo), kl = key(hi - 1);
        if (kf >= t1) h1 = lo; else l1 = lo + 1;          // key(lo) decides bound 1 or drops lo
        if (kf >= t2) h2 = lo; else l2 = lo + 1;
        if (kl < t1) l1 = hi; else h1 = min(h1, hi - 1);  // key(hi - 1) likewise at the top
        if (kl < t2) l2 = hi; else h2 = min(h2, hi - 1);
    }
    while (l1 < h1 || l2 < h2) {
        const bool a = l1 < h1, b = l2 < h2;
        const uint32_t m1 = (l1 + h1) >> 1, m2 = (l2 + h2) >> 1;
        const uint32_t k1 = a ? key(m1) : 0u, k2 = b ? key(m2) : 0u;
        if (a) { if (k1 < t1) l1 = m1 + 1; else h1 = m1; }
        if (b) { if (k2 < t2) l2 = m2 + 1; else h2 = m2; }
        l2 = max(l2, l1);
        h1 = min(h1, h2);
    }
    r1 = l1;
    r2 = l2;
}

// [r1, r2) = [first i with key(i) >= t1, first i with key(i) >= t2) in
// [lo, hi) for t1 <= t2 and a non-decreasing key; ranges of at most 32 entries
// take one probe round for both bounds.
template <class KeyFn>
__device__ __forceinline__ void warp_bounds(KeyFn key, uint32_t lo, uint32_t hi, uint32_t t1,
                                            uint32_t t2, int lane, uint32_t &r1, uint32_t &r2)
{
    if (hi - lo <= 32) {
        const uint32_t pos = lo + (uint32_t)lane;
        uint32_t kv = 0;
        const bool in = pos < hi;
        if (in) kv = key(pos);
        r1 = lo + __popc(__ballot_sync(FULL, in && kv < t1));
        r2 = t1 < t2 ? lo + __popc(__ballot_sync(FULL, in && kv < t2)) : r1;
        return;
    }
    r1 = warp_lower_bound_by(key, lo, hi, t1, lane);
    r2 = t1 < t2 ? warp_lower_bound_by(key, r1, hi, t2, lane) : r1;
}

// Warp-per-unit backtracking enumerator (Sec. III enumerator, Sec. VI work
// units, matching orders and masks).  Persistent: warps take seeds from a
// cursor (one or two seed sets: dS- then dS+ of a batch), then split-off
// subtrees from the task ring (pull-based distribution of work units).  Lane
// s holds the state of depth s; the candidates of a depth are tested 32 at a
// time, one per lane, and the last two depths are fused (each candidate of
// depth last-1 computes its last-depth range in its own lane).  A depth's
// candidate range is the (vertex, label) slice of the adjacency narrowed by
// binary search to the seqs allowed by the temporal bounds, the window and
// the batch mask; what remains is tested against the DEBI bit and
// injectivity.  When other warps are idle, a warp hands them work: half of a
// large range, the pending candidates of a chunk, or whole last-depth
// ranges.  Embeddings are staged per warp in shared memory and written out in
// contiguous blocks.
// FILTER: the DEBI filtering is on (p.bu set); a separate instantiation, so
// that the unfiltered kernel carries none of its code.
// STAGE: a contiguous candidate range of the last two depths (swept chunk
// after chunk with no descent in between) of at least p.stage_min entries is
// read through two shared-memory windows per warp, each filled by bulk
// asynchronous copies of its nbr and seq slices: window k + 2 is fetched while
// windows k and k + 1 are tested.
template <bool FILTER, bool STAGE>
__global__ void __launch_bounds__(ENUM_WARPS * 32, ENUM_MIN_BLOCKS) k_enumerate(EnumParams p)
{
    __shared__ __align__(16) unsigned char stage_all[ENUM_WARPS][STAGE_BYTES];
    __shared__ __align__(16) uint32_t win_all[STAGE ? ENUM_WARPS : 1][2][2][SLICE_WIN];
    __shared__ __align__(8) unsigned long long wbar_all[STAGE ? ENUM_WARPS : 1][2];
    if (*p.status) return;
    const int lane = threadIdx.x & 31;
    unsigned char *stage = stage_all[threadIdx.x >> 5];
    // staged windows: buffer b holds window k (k & 1 == b) of the range that
    // starts at sg_ws0; sg_bits: 1 << b copy pending on buffer b, 4 << b the
    // parity of buffer b's next phase, 16 a staged range is open
    uint32_t (*win)[2][SLICE_WIN] = win_all[STAGE ? (threadIdx.x >> 5) : 0];
    unsigned long long *wbar = wbar_all[STAGE ? (threadIdx.x >> 5) : 0];
    uint32_t sg_ws0 = 0, sg_wlo = 0, sg_bits = 0;
    if (STAGE) {
        if (lane == 0) {
            mbar_init(&wbar[0], 1);
            mbar_init(&wbar[1], 1);
            mbar_init_fence();
        }
        __syncwarp();
    }
    const uint32_t nseeds0 = min(*p.nseeds, p.seed_cap);
    const uint32_t nseeds = nseeds0 + (p.seeds1 ? min(*p.nseeds1, p.seed_cap1) : 0u);
    Sched *sc = p.sched;
    unsigned long long iters = 0;
    uint32_t poll = 0;                       // chunk counter: check for idle warps every 8th
    // lane 0: the idle-warp count read at the previous check; each check uses
    // it and issues the next read, so the read's latency is not waited on
    uint32_t idle_seen = 0;
    uint32_t poll_mask = 7;                  // check every 8th chunk; every 2nd while many warps idle
    const uint32_t many_idle = gridDim.x * ENUM_WARPS / 4;
    bool seeds_left = true;                  // lane 0: the seed cursor may still have seeds
    unsigned long long w_seeds = 0, w_scanned = 0, w_binds = 0, w_records = 0, w_busy = 0;
    unsigned long long w_tasks = 0, w_pruned = 0, w_staged = 0;
    uint32_t st_n = 0, st_q = 0xffffffffu, st_rb = 0, st_sign = 0;

    // write the staged records of query st_q to its list
    auto flush = [&]() {
        if (st_n == 0) return;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&p.counts[st_q * 3 + st_sign], (unsigned long long)st_n);
        base = __shfl_sync(FULL, base, 0);
        const unsigned long long cap = p.out_cap[st_q * 2 + st_sign];
        const unsigned long long nw = base >= cap ? 0ull : min((unsigned long long)st_n, cap - base);
        unsigned long long *dst =
            reinterpret_cast<unsigned long long *>(p.out[st_q * 2 + st_sign] + base * st_rb);
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(stage);
        const uint32_t words = (uint32_t)(nw * st_rb / 8);
        for (uint32_t w = lane; w < words; w += 32) dst[w] = src[w];
        st_n = 0;
        __syncwarp();
    };

    for (;;) {
        // ---------------------------------------------------------- take a unit
        // Seeds first.  Then a ticket of the task queue: the warp waits on
        // its own slot until a busy warp publishes a task there; when no warp
        // has been busy for a few polls it abandons the slot (a CAS that the
        // publisher loses, keeping its work) and leaves.
        uint32_t kind = 0, unit = 0;
        if (lane == 0) {
            const uint32_t s0 = seeds_left ? atomicAdd(&sc->next_seed.v, 1u) : nseeds;
            if (s0 < nseeds) {
                kind = 1;
                unit = s0;
            } else if (p.tasks) {
                // Ticket holder of slot t in lap L: take the task once it is
                // published; a later lap found on the slot means the ticket
                // was skipped (draw again); when no warp is busy for a few
                // polls, mark a free slot abandoned and leave.
                seeds_left = false;
                atomicAdd(&sc->idle.v, 1u);
                for (uint32_t draws = 0; draws < 64 && !kind; draws++) {
                    const uint32_t t = atomicAdd(&sc->q_head.v, 1u);
                    unsigned long long *st = &p.tasks[t & (p.task_cap - 1)].state;
                    const unsigned long long key = slot_key(p.epoch, t >> p.task_log2);
                    uint32_t nap = 64, quiet = 0;
                    bool leave = false;
                    for (uint32_t it = 0;; it++) {
                        const unsigned long long v = vload64(st);
                        if (!p.wait_hold) {
                            if (v == key + SLOT_PUBLISHED) { kind = 2; unit = t; break; }
                            if (v >= key + 4) break;    // skipped by a later lap
                            if (v != key + SLOT_RESERVED && slot_free(v, p.epoch) &&
                                (it >= p.wait_polls || quiet >= 4)) {
                                if (atomicCAS(st, v, key + SLOT_ABANDONED) == v) { leave = true; break; }
                                continue;               // state moved on: look again
                            }
                        }
                        if (it >= p.wait_polls + RESERVE_POLLS) {   // a reserved slot never published
                            atomicOr(p.status, ST_TIMEOUT);
                            leave = true;
                            break;
                        }
                        if (vload(&sc->busy.v) == 0) quiet++;
                        else quiet = 0;
                        __nanosleep(nap);
                        nap = min(nap * 2, 2048u);
                    }
                    if (leave) break;
                }
                atomicSub(&sc->idle.v, 1u);
            }
            if (kind) atomicAdd(&sc->busy.v, 1u);
        }
        kind = __shfl_sync(FULL, kind, 0);
        unit = __shfl_sync(FULL, unit, 0);
        if (!kind) break;

        // ---------------------------------------------------------- set up the unit
        uint32_t q, j, kc = 0, sid = 0, set = 0, root, f = 0, g = 0, tbeg = 0, tend = 0;
        bool skip = false, presplit = false;
        if (kind == 1) {
            w_seeds++;
            set = unit >= nseeds0 ? 1u : 0u;
            if (set) unit -= nseeds0;
            const unsigned long long sd = (set ? p.seeds1 : p.seeds)[unit];
            const uint32_t seed32 = (uint32_t)(sd >> 32);
            q = (uint32_t)(sd >> 8) & 0xffffu;
            j = (uint32_t)sd & 0xffu;
            kc = (uint32_t)(sd >> 24) & (NCAND - 1);
            presplit = (sd & SEED_PRESPLIT) != 0;
            sid = unit;
            const Plan *pl = &p.plans[(q * MN_MAX_QE + j) * NCAND + kc];
            const uint32_t slot0 = seed32 & p.cap_mask;
            const uint32_t vs = p.ring_src[slot0], vd = p.ring_dst[slot0];
            if (pl->iso && vs == vd) skip = true;
            const unsigned long long qr = set ? p.qrun[1] : p.qrun[0];
            if (!((qr >> (q & 63)) & 1ull)) skip = true;   // this query's seeds are not run
            if (FILTER && !skip) {                         // filtering: both endpoints in BU
                const uint32_t *bq = p.bu[q];
                const uint32_t ss = pl->seed_src, sd = pl->seed_dst;
                if (!((bq[ss * p.W32 + (vs >> 5)] >> (vs & 31)) & 1u) ||
                    !((bq[sd * p.W32 + (vd >> 5)] >> (vd & 31)) & 1u)) {
                    skip = true;
                    w_pruned++;
                }
            }
            if (lane == (int)pl->seed_src) f = vs;
            if (lane == (int)pl->seed_dst) f = vd;
            if (lane == (int)j) g = seed32 - p.base32;
            root = 1;
        } else {
            Task *T = &p.tasks[unit & (p.task_cap - 1)];
            __threadfence();                       // the slot was seen published
            __syncwarp();
            const uint32_t h = __ldcg(&T->qj_lvl);
            q = h & 0xffffu;
            j = (h >> 16) & 0xffu;
            root = h >> 24;
            tbeg = __ldcg(&T->beg);
            tend = __ldcg(&T->end);
            kc = __ldcg(&T->kc);
            sid = __ldcg(&T->sid);
            set = __ldcg(&T->set);
            f = __ldcg(&T->f[lane & 15]);
            g = __ldcg(&T->g[lane & 15]);
            __syncwarp();                          // every lane has read the task
            if (lane == 0) {
                __threadfence();
                atomicExch(&T->state, slot_key(p.epoch, unit >> p.task_log2) + SLOT_CONSUMED);
            }
        }
        const Plan *pl = &p.plans[(q * MN_MAX_QE + j) * NCAND + kc];
        const uint32_t nsteps = pl->nsteps, nv = pl->nv, ne = pl->ne, iso = pl->iso;
        long long t_unit = 0;
        if (lane == 0) t_unit = clock64();
        const uint32_t rec_bytes = pl->rec_bytes, goff = pl->goff;
        uint4 sw = make_uint4(0, 0, 0, 0);
        if (lane < MN_MAX_QE) sw = reinterpret_cast<const uint4 *>(pl->step)[lane];
        const uint32_t *__restrict__ debi = p.debi[q];
        const uint32_t *__restrict__ buq = FILTER ? p.bu[q] : nullptr;   // filtering: BU bitmaps
        const uint32_t sign = set ? p.sign1 : p.sign;       // this unit's output lists
        const uint32_t av_lo = set ? p.av_lo1 : p.av_lo, av_hi = set ? p.av_hi1 : p.av_hi;
        unsigned long long warp_count = 0;
        const bool direct = rec_bytes * 32 > STAGE_BYTES;

        // emit the embeddings completed by the valid lanes of one chunk
        // per-lane overrides: vertex to_new -> nb and edge qe_new -> rel (this
        // lane's candidate); optionally also vertex to2 -> nb2, edge qe2 -> rel2
        auto emit = [&](bool ok, uint32_t to_new, uint32_t nb, uint32_t qe_new, uint32_t rel,
                        uint32_t to2 = 0xffu, uint32_t nb2 = 0, uint32_t qe2 = 0xffu,
                        uint32_t rel2 = 0) {
            const uint32_t m = __ballot_sync(FULL, ok);
            if (!m) return;
            const uint32_t cnt = __popc(m);
            w_records += cnt;
            if (p.count_only) { warp_count += cnt; return; }
            const uint32_t rank = __popc(m & lanemask_lt());
            unsigned char *rec;
            unsigned long long gbase = 0;
            bool wr = ok;
            if (direct) {
                if (lane == 0) gbase = atomicAdd(&p.counts[q * 3 + sign], (unsigned long long)cnt);
                gbase = __shfl_sync(FULL, gbase, 0) + rank;
                wr = ok && gbase < p.out_cap[q * 2 + sign];
                rec = p.out[q * 2 + sign] + gbase * rec_bytes;
            } else {
                if (st_q != q || st_sign != sign || (st_n + cnt) * rec_bytes > STAGE_BYTES) {
                    flush();
                    st_q = q;
                    st_sign = sign;
                    st_rb = rec_bytes;
                }
                rec = stage + (st_n + rank) * rec_bytes;
            }
            for (uint32_t u = 0; u < nv; u++) {
                uint32_t fu = __shfl_sync(FULL, f, u);
                if (u == to2) fu = nb2;
                if (u == to_new) fu = nb;
                if (wr) reinterpret_cast<uint32_t *>(rec)[u] = fu;
            }
            if ((nv & 1) && wr) reinterpret_cast<uint32_t *>(rec)[nv] = 0;
            for (uint32_t e = 0; e < ne; e++) {
                uint32_t ge = __shfl_sync(FULL, g, e);
                if (e == qe2) ge = rel2;
                if (e == qe_new) ge = rel;
                if (wr) reinterpret_cast<unsigned long long *>(rec + goff)[e] = p.base + ge;
            }
            if (!direct) st_n += cnt;
            __syncwarp();
        };

        if (!skip && root >= nsteps) {
            emit(lane == 0, 0xffu, 0, 0xffu, 0);   // one-edge query: the seed is the embedding
            skip = true;
        }
        if (!skip) {
            // per-depth state, lane-distributed (lane s holds depth s)
            uint32_t Lend = 0, Lcur = 0, Lmask = 0, Llo = 0, Lhi = 0, Ltgt = 0, Ldsel = 0;
            uint32_t lvl = root;
            uint32_t qe, kind_s, from, to, dir, avoid, bound_v;
            int32_t label;
            uint32_t end, cur, mask, tlo, thi, tgt, dsel;
            const uint32_t last = nsteps - 1;

            auto decode = [&](uint32_t s) {
                uint32_t w0 = __shfl_sync(FULL, sw.x, s);
                uint32_t w1 = __shfl_sync(FULL, sw.y, s);
                uint32_t w3 = __shfl_sync(FULL, sw.w, s);
                qe = w0 & 0xff; kind_s = (w0 >> 8) & 0xff; from = (w0 >> 16) & 0xff; to = w0 >> 24;
                dir = w1 & 0xff; avoid = (w1 >> 8) & 0xff; label = (int32_t)(int16_t)(w1 >> 16);
                bound_v = w3 & 0xffff;
            };
            auto open = [&](uint32_t s, bool from_task) {
                decode(s);
                const uint32_t w2 = __shfl_sync(FULL, sw.z, s);
                const uint32_t pred = w2 & 0xffff, succ = w2 >> 16;
                const uint32_t pe = (pred >> lane) & 1u, se = (succ >> lane) & 1u;
                tlo = __reduce_max_sync(FULL, pe ? g + 1 : 0u);
                thi = __reduce_min_sync(FULL, se ? g : 0xffffffffu);
                tlo = max(tlo, avoid ? av_lo : p.vis_lo);
                thi = min(thi, avoid ? av_hi : p.vis_hi);
                const uint32_t fv = __shfl_sync(FULL, f, from);
                const uint32_t L = p.L;
                uint32_t beg;
                if (kind_s == K_EXTEND) {
                    dsel = dir + 2;                          // arrival order
                    const uint32_t *o = p.offs[dir];
                    if (label >= 0) { beg = o[fv * L + label]; end = o[fv * L + label + 1]; }
                    else            { beg = o[fv * L];         end = o[fv * L + L]; }
                    tgt = 0;
                    if (label >= 0 && !from_task && beg < end) {
                        const uint32_t *sq = p.s32[dsel];
                        const uint32_t b32 = p.base32;
                        auto key = [&](uint32_t i) { return sq[i] - b32; };
                        uint32_t r1, r2;
                        warp_bounds(key, beg, end, tlo, thi, lane, r1, r2);
                        beg = r1;
                        end = r2;
                    }
                } else {
                    const uint32_t tv = __shfl_sync(FULL, f, to);
                    const uint32_t *oa = p.offs[dir], *ob = p.offs[dir ^ 1u];
                    uint32_t a0, a1, b0, b1;
                    if (label >= 0) {
                        a0 = oa[fv * L + label]; a1 = oa[fv * L + label + 1];
                        b0 = ob[tv * L + label]; b1 = ob[tv * L + label + 1];
                    } else {
                        a0 = oa[fv * L]; a1 = oa[fv * L + L];
                        b0 = ob[tv * L]; b1 = ob[tv * L + L];
                    }
                    if (a1 - a0 <= b1 - b0) { dsel = dir; tgt = tv; beg = a0; end = a1; }
                    else                    { dsel = dir ^ 1u; tgt = fv; beg = b0; end = b1; }
                    if (label >= 0 && !from_task && beg < end) {
                        const uint32_t *nbv = p.nbr[dsel];
                        auto keyn = [&](uint32_t i) { return nbv[i]; };
                        uint32_t lb, ub;
                        warp_bounds(keyn, beg, end, tgt, tgt + 1, lane, lb, ub);
                        if (lb < ub) {
                            const uint32_t *sq = p.s32[dsel];
                            const uint32_t b32 = p.base32;
                            auto key = [&](uint32_t i) { return sq[i] - b32; };
                            warp_bounds(key, lb, ub, tlo, thi, lane, lb, ub);
                        }
                        beg = lb; end = ub;
                    }
                }
                if (from_task) { beg = tbeg; end = tend; }
                cur = beg; mask = 0;
                if (lane == (int)s) { Lend = end; Llo = tlo; Lhi = thi; Ltgt = tgt; Ldsel = dsel; }
            };
            auto restore = [&](uint32_t s) {
                decode(s);
                end = __shfl_sync(FULL, Lend, s);
                cur = __shfl_sync(FULL, Lcur, s);
                mask = __shfl_sync(FULL, Lmask, s);
                tlo = __shfl_sync(FULL, Llo, s);
                thi = __shfl_sync(FULL, Lhi, s);
                tgt = __shfl_sync(FULL, Ltgt, s);
                dsel = __shfl_sync(FULL, Ldsel, s);
            };
            // staged windows (STAGE): wait for buffer b's pending copy (all
            // lanes observe the phase, so all see the data), fetch window k
            // of the open range into buffer k & 1, drain both buffers
            auto sg_wait = [&](uint32_t b) {
                if (!((sg_bits >> b) & 1u)) return;
                const uint32_t par = (sg_bits >> (2 + b)) & 1u;
                for (uint32_t it = 0; !mbar_try_wait(&wbar[b], par); it++) {
                    if (it == SLICE_WAIT_POLLS && lane == 0) atomicOr(p.status, ST_TIMEOUT);
                    if (it >= 2 * SLICE_WAIT_POLLS) break;
                }
                sg_bits &= ~(1u << b);
                sg_bits ^= 4u << b;
            };
            auto sg_issue = [&](uint32_t k) {
                const uint32_t start = sg_ws0 + k * SLICE_WIN;
                if (start >= end) return;
                const uint32_t endr = min((end + 3u) & ~3u, p.adj_cap);
                const uint32_t n = min(SLICE_WIN, endr - start);
                const uint32_t b = k & 1u;
                __syncwarp();                        // every lane is done with the buffer
                if (lane == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&wbar[b], 8u * n);
                    bulk_load(win[b][0], p.nbr[dsel] + start, 4u * n, &wbar[b]);
                    bulk_load(win[b][1], p.s32[dsel] + start, 4u * n, &wbar[b]);
                }
                sg_bits |= 1u << b;
            };
            auto sg_drain = [&]() {
                if (!(sg_bits & 16u)) return;
                sg_wait(0);
                sg_wait(1);
                sg_bits &= ~16u;
            };
            // hand [mid, e) of depth l to the queue, optionally with vertex
            // fo_lane bound to fo_val and edge go_lane to go_val; false if the
            // queue is full
            auto push = [&](uint32_t l, uint32_t mid, uint32_t e, uint32_t fo_lane = 0xffu,
                            uint32_t fo_val = 0, uint32_t go_lane = 0xffu, uint32_t go_val = 0) -> bool {
                // Publish into the next slot: reserve it (it must hold no
                // live task), write, publish.  false: the work stays here.
                uint32_t ok = 0, slot = 0;
                if (lane == 0 && (int32_t)(vload(&sc->q_tail.v) - vload(&sc->q_head.v)) <
                                     (int32_t)(p.task_cap >> 1)) {
                    slot = atomicAdd(&sc->q_tail.v, 1u);          // slots in ticket order
                    unsigned long long *st = &p.tasks[slot & (p.task_cap - 1)].state;
                    const unsigned long long key = slot_key(p.epoch, slot >> p.task_log2);
                    unsigned long long v = vload64(st);
                    for (int i = 0; i < 8 && v < key && slot_free(v, p.epoch); i++) {
                        const unsigned long long prev = atomicCAS(st, v, key + SLOT_RESERVED);
                        if (prev == v) { ok = 1; break; }
                        v = prev;
                    }
                }
                ok = __shfl_sync(FULL, ok, 0);
                if (!ok) return false;
                slot = __shfl_sync(FULL, slot, 0);
                Task *T = &p.tasks[slot & (p.task_cap - 1)];
                uint32_t gg = __shfl_sync(FULL, g, lane & 15);
                if ((uint32_t)(lane & 15) == go_lane) gg = go_val;
                const uint32_t fl = (uint32_t)lane == fo_lane ? fo_val : f;
                reinterpret_cast<uint32_t *>(T)[8 + lane] = lane < 16 ? fl : gg;
                if (lane == 0) {
                    T->qj_lvl = q | (j << 16) | (l << 24);
                    T->beg = mid;
                    T->end = e;
                    T->kc = kc;
                    T->sid = sid;
                    T->set = set;
                }
                __threadfence();
                __syncwarp();
                if (lane == 0)                     // only the reserver moves a reserved slot on
                    atomicExch(&T->state, slot_key(p.epoch, slot >> p.task_log2) + SLOT_PUBLISHED);
                w_tasks++;
                return true;
            };

            // The last two depths fused: every valid candidate of a chunk at
            // depth last-1 computes its own last-depth range (lane-local
            // searches, all candidates at once); the warp then sweeps the
            // concatenated ranges 32 entries at a time, each entry tested with
            // its owner candidate's binding (owner found by a search over the
            // lanes' prefix sums) and emitted with both bindings.
            auto expand_last = [&](bool okc, uint32_t nb_c, uint32_t rel_c) {
                const uint32_t qe_p = qe, to_p = kind_s == K_EXTEND ? to : 0xffu;
                const uint32_t w0 = __shfl_sync(FULL, sw.x, last), w1 = __shfl_sync(FULL, sw.y, last);
                const uint32_t w2 = __shfl_sync(FULL, sw.z, last), w3 = __shfl_sync(FULL, sw.w, last);
                const uint32_t qe_l = w0 & 0xff, kind_l = (w0 >> 8) & 0xff;
                const uint32_t from_l = (w0 >> 16) & 0xff, to_l = w0 >> 24;
                const uint32_t dir_l = w1 & 0xff, avoid_l = (w1 >> 8) & 0xff;
                const int32_t label_l = (int32_t)(int16_t)(w1 >> 16);
                const uint32_t pred_l = w2 & 0xffff, succ_l = w2 >> 16, bv_l = w3 & 0xffff;
                // temporal bounds from edges bound above, then this lane's candidate
                const uint32_t others = ~(1u << qe_p);
                const uint32_t pe = ((pred_l & others) >> lane) & 1u, se = ((succ_l & others) >> lane) & 1u;
                uint32_t tl = __reduce_max_sync(FULL, pe ? g + 1 : 0u);
                uint32_t th = __reduce_min_sync(FULL, se ? g : 0xffffffffu);
                tl = max(tl, avoid_l ? av_lo : p.vis_lo);
                th = min(th, avoid_l ? av_hi : p.vis_hi);
                if ((pred_l >> qe_p) & 1u) tl = max(tl, rel_c + 1);
                if ((succ_l >> qe_p) & 1u) th = min(th, rel_c);
                const uint32_t f_from = __shfl_sync(FULL, f, from_l), f_to = __shfl_sync(FULL, f, to_l);
                const uint32_t fv = from_l == to_p ? nb_c : f_from;
                const uint32_t tv = to_l == to_p ? nb_c : f_to;
                const uint32_t L = p.L, b32 = p.base32;
                uint32_t beg = 0, end2 = 0, dsl = dir_l + 2, tg = 0;
                if (okc) {
                    if (kind_l == K_EXTEND) {
                        const uint32_t *o = p.offs[dir_l];
                        if (label_l >= 0) { beg = o[fv * L + label_l]; end2 = o[fv * L + label_l + 1]; }
                        else              { beg = o[fv * L];           end2 = o[fv * L + L]; }
                        if (label_l >= 0 && beg < end2) {
                            const uint32_t *sq = p.s32[dsl];
                            auto key = [&](uint32_t i) { return sq[i] - b32; };
                            uint32_t r1, r2;
                            lane_bounds2<true>(key, beg, end2, tl, max(tl, th), r1, r2);
                            beg = r1;
                            end2 = r2;
                        }
                    } else {
                        const uint32_t *oa = p.offs[dir_l], *ob = p.offs[dir_l ^ 1u];
                        uint32_t a0, a1, c0, c1;
                        if (label_l >= 0) {
                            a0 = oa[fv * L + label_l]; a1 = oa[fv * L + label_l + 1];
                            c0 = ob[tv * L + label_l]; c1 = ob[tv * L + label_l + 1];
                        } else {
                            a0 = oa[fv * L]; a1 = oa[fv * L + L];
                            c0 = ob[tv * L]; c1 = ob[tv * L + L];
                        }
                        if (a1 - a0 <= c1 - c0) { dsl = dir_l; tg = tv; beg = a0; end2 = a1; }
                        else                    { dsl = dir_l ^ 1u; tg = fv; beg = c0; end2 = c1; }
                        if (label_l >= 0 && beg < end2) {
                            const uint32_t *nbv = p.nbr[dsl];
                            auto keyn = [&](uint32_t i) { return nbv[i]; };
                            uint32_t lb, ub;
                            lane_bounds2<false>(keyn, beg, end2, tg, tg + 1, lb, ub);
                            const uint32_t *sq = p.s32[dsl];
                            auto key = [&](uint32_t i) { return sq[i] - b32; };
                            uint32_t r1, r2;
                            lane_bounds2<false>(key, lb, ub, tl, max(tl, th), r1, r2);
                            beg = r1;
                            end2 = r2;
                        }
                    }
                }
                uint32_t len = end2 > beg ? end2 - beg : 0u;
                // idle warps: hand them the large last-depth ranges, each as a
                // task at the last depth carrying its candidate's binding
                if (p.tasks) {
                    uint32_t idle = 0;
                    if (lane == 0) { idle = idle_seen; idle_seen = vload(&sc->idle.v); }
                    idle = __shfl_sync(FULL, idle, 0);
                    uint32_t big = idle ? __ballot_sync(FULL, len >= p.split_min) : 0u;
                    while (big && idle) {
                        const uint32_t b = __ffs(big) - 1;
                        big &= big - 1;
                        const uint32_t bb = __shfl_sync(FULL, beg, b), be = __shfl_sync(FULL, end2, b);
                        const uint32_t bn = __shfl_sync(FULL, nb_c, b), br = __shfl_sync(FULL, rel_c, b);
                        if (!push(last, bb, be, to_p, bn, qe_p, br)) break;
                        if ((uint32_t)lane == b) len = 0;
                        idle--;
                    }
                }
                uint32_t inc = len;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(FULL, inc, d);
                    if (lane >= d) inc += y;
                }
                const uint32_t total = __shfl_sync(FULL, inc, 31);
                const uint32_t exc = inc - len;
                w_binds += __popc(__ballot_sync(FULL, okc));
                for (uint32_t t0 = 0; t0 < total; t0 += 32) {
                    if (++iters > p.max_iters) {
                        if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
                        break;
                    }
                    const uint32_t t = t0 + (uint32_t)lane;
                    uint32_t o = 0;                  // first lane whose inclusive prefix exceeds t
#pragma unroll
                    for (uint32_t st = 16; st; st >>= 1) {
                        const uint32_t ip = __shfl_sync(FULL, inc, o + st - 1);
                        if (ip <= t) o += st;
                    }
                    const uint32_t obeg = __shfl_sync(FULL, beg, o), oexc = __shfl_sync(FULL, exc, o);
                    const uint32_t otl = __shfl_sync(FULL, tl, o), oth = __shfl_sync(FULL, th, o);
                    const uint32_t onb = __shfl_sync(FULL, nb_c, o), orel = __shfl_sync(FULL, rel_c, o);
                    const uint32_t otg = __shfl_sync(FULL, tg, o), odsl = __shfl_sync(FULL, dsl, o);
                    bool ok2 = false;
                    uint32_t nb2 = 0, rel2 = 0;
                    if (t < total) {
                        const uint32_t idx = obeg + (t - oexc);
                        nb2 = p.nbr[odsl][idx];
                        const uint32_t sv = p.s32[odsl][idx];
                        rel2 = sv - b32;
                        ok2 = rel2 >= otl && rel2 < oth;
                        if (ok2) ok2 = (debi[sv & p.cap_mask] >> qe_l) & 1u;
                        if (ok2 && avoid_l && p.batch_flag) ok2 = p.batch_flag[sv & p.cap_mask] == 0;
                        if (kind_l == K_CLOSE) ok2 = ok2 && nb2 == otg;
                    }
                    if (FILTER && ok2 && kind_l == K_EXTEND)
                        ok2 = (buq[to_l * p.W32 + (nb2 >> 5)] >> (nb2 & 31)) & 1u;
                    if (kind_l == K_EXTEND && iso) {
                        for (uint32_t bv = bv_l; bv; bv &= bv - 1) {
                            const uint32_t wv = __ffs(bv) - 1;
                            uint32_t fw = __shfl_sync(FULL, f, wv);
                            if (wv == to_p) fw = onb;
                            ok2 = ok2 && nb2 != fw;
                        }
                    }
                    w_scanned += min(32u, total - t0);
                    emit(ok2, kind_l == K_EXTEND ? to_l : 0xffu, nb2, qe_l, rel2, to_p, onb, qe_p, orel);
                }
            };

            open(lvl, kind == 2);
            // a seed whose predicted work is above the threshold (k_pick):
            // its first depth's candidates go to the task ring in up to
            // PRESPLIT_PIECES ranges right away, before any warp is idle
            if (presplit && p.tasks && lvl < last) {
                const uint32_t len = end > cur ? end - cur : 0u;
                const uint32_t pieces = min(len, (uint32_t)PRESPLIT_PIECES);
                if (pieces > 1) {
                    const uint32_t sz = (len + pieces - 1) / pieces;
                    uint32_t cut = end;
                    for (uint32_t b0 = cur + sz; b0 < end; b0 += sz) {
                        if (!push(lvl, b0, min(end, b0 + sz))) break;
                        if (cut == end) cut = b0;
                    }
                    end = cut;
                    if (lane == (int)lvl) Lend = cut;
                }
            }
            while (lvl >= root) {
                if (++iters > p.max_iters) {
                    if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
                    break;
                }
                if (mask == 0) {
                    if (cur >= end) {               // depth exhausted: backtrack
                        if (STAGE) sg_drain();
                        lvl--;
                        if (lvl >= root) restore(lvl);
                        continue;
                    }
                    // when some warp is idle, hand it work of the shallowest
                    // depth that has some left: half of a large unexplored
                    // range, else the upper half of the candidates still
                    // pending from the chunk in progress there (entries from
                    // the first of them on; the receiver tests them again)
                    if (p.tasks && (++poll & poll_mask) == 0) {
                        uint32_t idle = 0;
                        if (lane == 0) { idle = idle_seen; idle_seen = vload(&sc->idle.v); }
                        idle = __shfl_sync(FULL, idle, 0);
                        poll_mask = idle > many_idle ? 1u : 7u;
                        if (idle) {
                            // lanes root..lvl-1: chunk [Lcur - 32, Lcur) with
                            // pending bits Lmask, unexplored [Lcur, Lend) (Lend
                            // below Lcur after a split of pending bits); this
                            // depth keeps its next chunk
                            uint32_t rb = 0, re = 0, keep = 0;
                            if ((uint32_t)lane >= root && (uint32_t)lane < lvl) {
                                keep = Lmask;
                                if (Lend > Lcur && Lend - Lcur >= p.split_min) {
                                    rb = Lcur + (Lend - Lcur) / 2;
                                    re = Lend;
                                } else if (Lmask) {
                                    uint32_t give = Lmask;
                                    for (uint32_t k = __popc(Lmask) / 2; k; k--) give &= give - 1;
                                    const uint32_t b = __ffs(give) - 1;
                                    rb = Lcur - 32 + b;
                                    re = Lend;
                                    keep = Lmask & ((1u << b) - 1u);
                                }
                            }
                            if ((uint32_t)lane == lvl && end > cur + 32 && end - (cur + 32) >= p.split_min) {
                                rb = cur + 32 + (end - cur - 32) / 2;
                                re = end;
                            }
                            const bool can = (uint32_t)lane <= p.split_depth && re > rb;
                            const uint32_t big = __ballot_sync(FULL, can);
                            if (big) {
                                const uint32_t l = __ffs(big) - 1;
                                const uint32_t b0 = __shfl_sync(FULL, rb, l);
                                const uint32_t e0 = __shfl_sync(FULL, re, l);
                                if (push(l, b0, e0)) {
                                    // the donor's depth l now ends at b0 (a later
                                    // split there hands out entries below b0 only)
                                    if (lane == (int)l) {
                                        Lend = b0;
                                        if (l < lvl) Lmask = keep;
                                    }
                                    if (l == lvl) end = b0;
                                }
                            }
                        }
                    }
                    // a long range of the last two depths: open its windows
                    if (STAGE && !(sg_bits & 16u) && lvl + 1 >= last && end - cur >= p.stage_min) {
                        sg_ws0 = cur & ~3u;
                        sg_wlo = 0;
                        sg_bits |= 16u;
                        sg_issue(0);
                        sg_issue(1);
                    }
                    bool staged = false;
                    if (STAGE && (sg_bits & 16u)) {
                        // windows below the chunk are done: each buffer takes
                        // the window two ahead of the one it held
                        const uint32_t ka = (cur - sg_ws0) / SLICE_WIN;
                        while (sg_wlo < ka) {
                            sg_wait(sg_wlo & 1u);
                            sg_issue(sg_wlo + 2);
                            sg_wlo++;
                        }
                        const uint32_t kb = (min(cur + 32u, end) - 1u - sg_ws0) / SLICE_WIN;
                        sg_wait(ka & 1u);
                        if (kb != ka) sg_wait(kb & 1u);
                        staged = true;
                        w_staged += min(32u, end - cur);
                    }
                    // test the next 32 candidates, one per lane
                    const uint32_t idx = cur + (uint32_t)lane;
                    bool ok = false;
                    uint32_t nb = 0, rel = 0;
                    if (idx < end) {
                        uint32_t sv;
                        if (STAGE && staged) {
                            const uint32_t r = idx - sg_ws0;
                            const uint32_t b = (r / SLICE_WIN) & 1u;
                            nb = win[b][0][r % SLICE_WIN];
                            sv = win[b][1][r % SLICE_WIN];
                        } else {
                            nb = p.nbr[dsel][idx];
                            sv = p.s32[dsel][idx];
                        }
                        rel = sv - p.base32;
                        ok = rel >= tlo && rel < thi;
                        if (ok) ok = (debi[sv & p.cap_mask] >> qe) & 1u;
                        if (ok && avoid && p.batch_flag) ok = p.batch_flag[sv & p.cap_mask] == 0;
                        if (kind_s == K_CLOSE) ok = ok && nb == tgt;
                        if (FILTER && ok && kind_s == K_EXTEND)
                            ok = (buq[to * p.W32 + (nb >> 5)] >> (nb & 31)) & 1u;
                    }
                    if (kind_s == K_EXTEND && iso) {
                        for (uint32_t bv = bound_v; bv; bv &= bv - 1) {
                            const uint32_t fw = __shfl_sync(FULL, f, __ffs(bv) - 1);
                            ok = ok && nb != fw;
                        }
                    }
                    w_scanned += min(32u, end - cur);
                    cur += 32;
                    if (lvl == last) {
                        emit(ok, kind_s == K_EXTEND ? to : 0xffu, nb, qe, rel);
                        continue;
                    }
                    if (lvl + 1 == last) {           // candidates' last depths, all at once
                        expand_last(ok, nb, rel);
                        continue;
                    }
                    mask = __ballot_sync(FULL, ok);
                    continue;
                }
                // bind the next valid candidate of this depth and descend
                const uint32_t b = __ffs(mask) - 1;
                mask &= mask - 1;
                w_binds++;
                const uint32_t idx = cur - 32 + b;
                const uint32_t nb = p.nbr[dsel][idx];
                const uint32_t rel = p.s32[dsel][idx] - p.base32;
                if (lane == (int)qe) g = rel;
                if (kind_s == K_EXTEND && lane == (int)to) f = nb;
                if (lane == (int)lvl) { Lcur = cur; Lmask = mask; }
                lvl++;
                open(lvl, false);
            }
            if (STAGE) sg_drain();                   // a unit left early (work budget)
        }
        if (p.count_only && lane == 0 && warp_count)
            atomicAdd(&p.counts[q * 3 + sign], warp_count);
        if (lane == 0) {                             // measured SM cycles of this unit
            const unsigned long long cyc = (unsigned long long)(clock64() - t_unit);
            w_busy += cyc;
            unsigned long long *sw_log = set ? p.seed_work1 : p.seed_work;
            if (sw_log) atomicAdd(&sw_log[sid], cyc);
            if (p.q_cycles) {
                const unsigned long long sdw = (set ? p.seeds1 : p.seeds)[sid];
                atomicAdd(&p.q_cycles[q * MARGIN_SLOTS + ((uint32_t)(sdw >> SEED_MARGIN_SHIFT) & 15u)], cyc);
            }
        }
        if (lane == 0) {
            __threadfence();
            atomicSub(&sc->busy.v, 1u);
        }
        uint32_t stop = 0;
        if (lane == 0) stop = vload(p.status) & ST_TIMEOUT;
        if (__shfl_sync(FULL, stop, 0)) break;
    }
    flush();
    if (lane == 0 && p.work) {
        atomicAdd(&p.work[0], w_seeds);
        atomicAdd(&p.work[1], w_scanned);
        atomicAdd(&p.work[2], w_binds);
        atomicAdd(&p.work[3], w_records);
        atomicAdd(&p.work[4], w_busy);
        atomicAdd(&p.work[5], w_tasks);
        atomicAdd(&p.work[6], w_pruned);
        atomicAdd(&p.work[7], w_staged);
    }
}

// ------------------------------------------------------------------ expiry / deletion

// Expired edges (seq in [seq_lo, seq_lo + n)): clear their DEBI words
// (Sec. IV-A memory recycling) and take them off the degree counters.
__global__ void k_expire(uint64_t seq_lo, uint32_t n, uint32_t cap_mask, uint32_t L, uint32_t nq,
                         uint32_t *const *debi, const uint32_t *r_src, const uint32_t *r_dst,
                         const uint8_t *r_label, uint32_t *cnt0, uint32_t *cnt1,
                         const uint32_t *status)
{
    if (*status) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t slot = (uint32_t)(seq_lo + i) & cap_mask;
    for (uint32_t q = 0; q < nq; q++) debi[q][slot] = 0;
    const uint32_t lab = r_label[slot];
    atomicSub(&cnt0[r_src[slot] * L + lab], 1u);
    atomicSub(&cnt1[r_dst[slot] * L + lab], 1u);
}

// Validate an explicit deletion list: live, not yet deleted, no repeats.
// Marks the batch flag of each slot.
__global__ void k_delete_mark(const unsigned long long *seqs, uint32_t n, unsigned long long lo,
                              unsigned long long hi, uint32_t cap_mask, const uint8_t *r_dead,
                              uint8_t *batch_flag, uint32_t *status)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long s = seqs[i];
    if (s < lo || s >= hi) { atomicOr(status, ST_BAD_DELETE); return; }
    const uint32_t slot = (uint32_t)s & cap_mask;
    if (r_dead[slot]) { atomicOr(status, ST_BAD_DELETE); return; }
    unsigned int *w = reinterpret_cast<unsigned int *>(batch_flag + (slot & ~3u));
    const unsigned int bit = 1u << ((slot & 3u) * 8);
    const unsigned int old = atomicOr(w, bit);
    if (old & bit) atomicOr(status, ST_BAD_DELETE);
}

// Apply (or, on a validation error, only undo the marks of) a deletion list.
__global__ void k_delete_apply(const unsigned long long *seqs, uint32_t n, uint32_t cap_mask,
                               uint32_t nq, uint32_t *const *debi, uint8_t *r_dead,
                               uint8_t *batch_flag, const uint32_t *status)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t slot = (uint32_t)seqs[i] & cap_mask;
    batch_flag[slot] = 0;
    if (*status) return;
    r_dead[slot] = 1;
    for (uint32_t q = 0; q < nq; q++) debi[q][slot] = 0;
}

}  // namespace mn

// ------------------------------------------------------------------ sorted fetch

namespace mn {

// Lexicographic order of two result records: the vertex ids f(u_0..u_{nv-1})
// (u32), then the edge seqs (u64, at byte offset goff) -- the order of the
// rows (f..., seq...) a caller sorts by.
__device__ __forceinline__ bool rec_less(const uint8_t *recs, uint32_t rb, uint32_t nv, uint32_t ne,
                                         uint32_t goff, uint32_t a, uint32_t b)
{
    const uint32_t *va = reinterpret_cast<const uint32_t *>(recs + (size_t)a * rb);
    const uint32_t *vb = reinterpret_cast<const uint32_t *>(recs + (size_t)b * rb);
    for (uint32_t u = 0; u < nv; u++)
        if (va[u] != vb[u]) return va[u] < vb[u];
    const unsigned long long *ga = reinterpret_cast<const unsigned long long *>(recs + (size_t)a * rb + goff);
    const unsigned long long *gb = reinterpret_cast<const unsigned long long *>(recs + (size_t)b * rb + goff);
    for (uint32_t e = 0; e < ne; e++)
        if (ga[e] != gb[e]) return ga[e] < gb[e];
    return a < b;                 // equal records keep their order (stable)
}

// Runs of MERGE_ITEMS records sorted by one thread each (insertion sort of
// their indices): the first merge pass then starts at runs of MERGE_ITEMS, so
// that no thread's outputs straddle two merged pairs.
__global__ void k_rec_sort_runs(const uint8_t *recs, uint32_t rb, uint32_t nv, uint32_t ne, uint32_t goff,
                                uint32_t *idx, uint32_t n)
{
    const uint32_t o = (blockIdx.x * blockDim.x + threadIdx.x) * MERGE_ITEMS;
    if (o >= n) return;
    const uint32_t m = min((uint32_t)MERGE_ITEMS, n - o);
    uint32_t r[MERGE_ITEMS];
#pragma unroll
    for (int k = 0; k < MERGE_ITEMS; k++) r[k] = o + k;
    for (uint32_t k = 1; k < m; k++) {
        const uint32_t x = r[k];
        uint32_t j = k;
        while (j > 0 && rec_less(recs, rb, nv, ne, goff, x, r[j - 1])) { r[j] = r[j - 1]; j--; }
        r[j] = x;
    }
    for (uint32_t k = 0; k < m; k++) idx[o + k] = r[k];
}

// One pass of a bottom-up merge sort of record indices: neighbouring sorted
// runs of length R merged into runs of 2R (merge path, MERGE_ITEMS outputs
// per thread).
__global__ void k_rec_merge_pass(const uint8_t *recs, uint32_t rb, uint32_t nv, uint32_t ne, uint32_t goff,
                                 const uint32_t *src, uint32_t *dst, uint32_t n, uint32_t R)
{
    const uint32_t o = (blockIdx.x * blockDim.x + threadIdx.x) * MERGE_ITEMS;
    if (o >= n) return;
    const uint32_t pbase = o / (2 * R) * (2 * R);
    const uint32_t nA = min(R, n - pbase);
    const uint32_t nB = min(R, n - pbase - nA);
    const uint32_t *A = src + pbase, *Bv = A + nA;
    const uint32_t d = o - pbase;
    uint32_t lo = d > nB ? d - nB : 0, hi = min(d, nA);
    while (lo < hi) {                       // first i with B[d - 1 - i] < A[i]
        const uint32_t mid = (lo + hi) >> 1;
        if (!rec_less(recs, rb, nv, ne, goff, Bv[d - 1 - mid], A[mid])) lo = mid + 1;
        else hi = mid;
    }
    uint32_t i = lo, j = d - lo;
    for (int t = 0; t < MERGE_ITEMS && o + t < pbase + nA + nB; t++) {
        const bool takeA = j >= nB || (i < nA && !rec_less(recs, rb, nv, ne, goff, Bv[j], A[i]));
        dst[o + t] = takeA ? A[i++] : Bv[j++];
    }
}

// out[k] = record idx[k] (rb bytes each, a multiple of 8).  An index out of
// range (a broken permutation) reads nothing and sets *status.
__global__ void k_rec_gather(const uint8_t *recs, uint32_t rb, const uint32_t *idx, uint32_t n, uint8_t *out,
                             uint32_t *status)
{
    const uint32_t words = rb / 8;
    const size_t total = (size_t)n * words;
    for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        const size_t k = w / words, x = w % words;
        const uint32_t i = idx[k];
        if (i >= n) {
            atomicOr(status, 1u);
            reinterpret_cast<unsigned long long *>(out)[w] = 0;
            continue;
        }
        reinterpret_cast<unsigned long long *>(out)[w] =
            reinterpret_cast<const unsigned long long *>(recs + (size_t)i * rb)[x];
    }
}

}  // namespace mn

// ------------------------------------------------------------------ host spill

namespace mn {

// One spilled edge: the caller's record, its seq, and the DEBI word of every
// query at the time it left the window (Sec. IV-A, external memory: edges
// leaving the in-memory window are written out with their index entries).
struct SpillRec {
    mn_edge e;
    unsigned long long seq;
};

// Pack the edges at seqs [seq_lo, seq_lo + n) from the ring (SoA) into
// records and their DEBI words ([q][n]) for the copy to host memory.
__global__ void k_spill_pack(uint64_t seq_lo, uint32_t n, uint32_t cap_mask, const uint32_t *r_src,
                             const uint32_t *r_dst, const uint8_t *r_label, const int32_t *r_attr,
                             const int64_t *r_ts, uint32_t nq, uint32_t *const *debi, SpillRec *out,
                             uint32_t *words, const uint32_t *status)
{
    if (*status) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t slot = (uint32_t)(seq_lo + i) & cap_mask;
    SpillRec r;
    r.e.src = r_src[slot];
    r.e.dst = r_dst[slot];
    r.e.label = r_label[slot];
    r.e.attr = r_attr[slot];
    r.e.ts = r_ts[slot];
    r.seq = seq_lo + i;
    out[i] = r;
    for (uint32_t q = 0; q < nq; q++) words[(size_t)q * n + i] = debi[q][slot];
}

}  // namespace mn
