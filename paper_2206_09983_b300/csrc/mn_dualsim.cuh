// mn_dualsim.cuh -- dual simulation over the live window (Sec. III names it
// as a matching variant built on the same index; Sec. VII-C evaluates it per
// snapshot).
//
// The largest relation S between query vertices u and data vertices v such
// that v carries u's labels and, for every query edge e leaving (entering) u,
// some live data edge leaving (entering) v matches e -- its DEBI bit e is set
// -- and leads to (comes from) a data vertex related to e's other endpoint.
// One word per data vertex holds the query vertices related to it.  The
// refinement starts from all label-compatible pairs and removes violating
// pairs until a pass changes nothing; passes read the words in place (a
// removal seen early only removes what a later pass would), so the result is
// the same largest relation in any schedule.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "mnemonic.h"

namespace mn {

struct DualSimParams {
    uint32_t nv, ne, V, L, cap_mask;
    uint32_t base32, vis_lo, vis_hi;       // live seqs, relative to the adjacency base
    uint32_t qmask[MN_MAX_QV];             // query vertex label masks (subset test)
    uint32_t out_e[MN_MAX_QV];             // query edges leaving u (bit e)
    uint32_t in_e[MN_MAX_QV];              // query edges entering u
    uint8_t esrc[MN_MAX_QE], edst[MN_MAX_QE];
    const uint32_t *offs[2];               // (vertex, label) offsets: 0 out, 1 in
    const uint32_t *nbr[2];                // by-neighbour adjacency: 0 out, 1 in
    const uint32_t *s32[2];
    const uint32_t *debi;                  // this query's DEBI words
    const uint32_t *vmask;                 // data vertex label masks
    uint32_t *sim;                         // [V] bit u: (u, v) related
    uint32_t *flags;                       // [0] changed in this pass, [1] OR of all words
};

__global__ void k_dualsim_init(DualSimParams p)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= p.V) return;
    const uint32_t vm = p.vmask[v];
    uint32_t w = 0;
    for (uint32_t u = 0; u < p.nv; u++)
        if ((vm & p.qmask[u]) == p.qmask[u]) w |= 1u << u;
    p.sim[v] = w;
}

// One refinement pass, a thread per data vertex: which query edges its live
// out- and in-edges satisfy given the current words, then drop the query
// vertices whose edges are not all satisfied.
__global__ void k_dualsim_pass(DualSimParams p)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= p.V) return;
    const uint32_t cur = p.sim[v];
    if (!cur) return;
    uint32_t sat[2] = {0u, 0u};
    uint32_t need[2] = {0u, 0u};
    for (uint32_t m = cur; m; m &= m - 1) {
        const uint32_t u = __ffs(m) - 1;
        need[0] |= p.out_e[u];
        need[1] |= p.in_e[u];
    }
    for (int d = 0; d < 2; d++) {          // 0: edges (v, w); 1: edges (w, v)
        if (!need[d]) continue;
        const uint32_t b = p.offs[d][(uint64_t)v * p.L], e = p.offs[d][(uint64_t)v * p.L + p.L];
        for (uint32_t i = b; i < e && (sat[d] & need[d]) != need[d]; i++) {
            const uint32_t sv = p.s32[d][i];
            const uint32_t rel = sv - p.base32;
            if (rel < p.vis_lo || rel >= p.vis_hi) continue;
            const uint32_t word = p.debi[sv & p.cap_mask] & need[d] & ~sat[d];
            if (!word) continue;
            const uint32_t sw = p.sim[p.nbr[d][i]];
            for (uint32_t m = word; m; m &= m - 1) {
                const uint32_t qe = __ffs(m) - 1;
                const uint32_t other = d == 0 ? p.edst[qe] : p.esrc[qe];
                if ((sw >> other) & 1u) sat[d] |= 1u << qe;
            }
        }
    }
    uint32_t keep = cur;
    for (uint32_t m = cur; m; m &= m - 1) {
        const uint32_t u = __ffs(m) - 1;
        if ((p.out_e[u] & ~sat[0]) || (p.in_e[u] & ~sat[1])) keep &= ~(1u << u);
    }
    if (keep != cur) {
        p.sim[v] = keep;
        p.flags[0] = 1u;
    }
}

// OR of every word (which query vertices are related to some data vertex) and
// the number of related pairs.
__global__ void k_dualsim_summary(DualSimParams p, unsigned long long *pairs)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t w = v < p.V ? p.sim[v] : 0u;
    uint32_t o = w;
    unsigned long long c = __popc(w);
    for (int s = 16; s; s >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, s);
        c += __shfl_xor_sync(0xffffffffu, c, s);
    }
    if ((threadIdx.x & 31) == 0 && (o || c)) {
        atomicOr(&p.flags[1], o);
        atomicAdd(pairs, c);
    }
}

}  // namespace mn
